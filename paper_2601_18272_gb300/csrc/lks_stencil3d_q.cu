// D3Q15 LKS predictor (Sec. 2.2) and its exact transpose, row-streamed form for FP32 fields on
// grids periodic in y and z (open or periodic x): the form every 3D workload of the library takes.
// The general kernels of lks_stencil3d.cu serve every other case (walls in y or z, FP64 fields,
// nx not a multiple of 4 or below 64).
//
// Layout. A CTA of 16 warps owns a window of 64 input columns (x0 - 2 .. x0 + 61, two adjacent
// columns per lane) by 16 input rows (one row per warp) and marches over a chunk of z planes; it
// writes the 60 x 12 outputs of lanes 1..30 and warps 2..13. Each plane of the window arrives by
// one TMA box of 16 rows (cp.async.bulk.tensor over a 5D view of the state: x, field, y, z, slot;
// the first and last row tiles add a 2-row box for the rows wrapped across y = 0) into a ring of
// plane slots guarded by mbarriers, so the bytes in flight need no registers. One box per plane
// matters: boxes of one row each kept the copy engine at about half the HBM rate.
// Neighbours along z are the previous planes held in registers; along x they come by warp
// shuffles (one per value and direction, shared by the lane's two columns); along y through two
// small shared-memory exchanges per plane. All arithmetic is packed FP32x2 (one instruction for
// the lane's two columns).
//
// Forward, per plane zr: the velocity gradient is separable,
//   10 G_ab = D_b u_a + D_b S_c S_d u_a   ({b, c, d} = {x, y, z}; D f = f(+1) - f(-1), S f = f(+1) + f(-1)),
// so each lane forms S_z u, D_z u from its own planes, the y pass takes them (and u) from the rows
// above and below, and the x pass takes the y-combined values from the neighbouring lanes. The
// fifteen f_i^eq of the node then scatter into three rolling output planes (c_z = -1, 0, +1):
// c_y != 0 values through the second exchange, c_x != 0 values through shuffles.
// Transpose, per plane zr: the moments P, U, S of the adjoint gather
// fbar_c(y) = lam_p*(y + c) / 3 + c . lam_u*(y + c) with the same separable structure (z in
// registers, then y, then x), and the gradient transpose h_a = -sum_b D_b (1 + S S) S_ab scatters
// into three rolling output planes.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lks_kernels.h"
#include "lks_stencil_common.cuh"

namespace lks {

namespace {

constexpr int QW = 16;              // warps per CTA = input rows of a window
constexpr int QT = QW * 32;         // threads per CTA
constexpr int QOY = QW - 4;         // output rows per window
constexpr int QIX = 64;             // input columns per window (two per lane)
constexpr int QOX = 60;             // output columns per window
constexpr int QR = 5;               // plane slots in flight (transpose)
constexpr int QROWB = 4 * QIX * 4;  // bytes of one row of one plane: 4 fields x 64 columns
constexpr int QSTB = 3 * QIX * 4;   // bytes of one row of the state's velocity (transpose)
constexpr int QSR = QW + 2;         // rows of a plane slot: the 16-row box and a 2-row wrap box
constexpr unsigned kFull = 0xffffffffu;

// ---- packed FP32x2 arithmetic ------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }  // exact a - b
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Neighbours along x of two-column quantities (lane L holds columns 2L, 2L + 1 of the window; lane
// 0's left and lane 31's right neighbours are not in the window and come back wrong, which only the
// unused edge columns see). The combinations are formed by scalar operations straight into the
// result pair: a packed operation on a shifted value would first move it into a register pair.
// D_x v = v(x + 1) - v(x - 1), S_x v = v(x + 1) + v(x - 1):
__device__ __forceinline__ float2 dx2(float2 v) {
  const float pv = __shfl_up_sync(kFull, v.y, 1), nv = __shfl_down_sync(kFull, v.x, 1);
  return make_float2(v.y - pv, nv - v.x);
}
__device__ __forceinline__ float2 sx2(float2 v) {
  const float pv = __shfl_up_sync(kFull, v.y, 1), nv = __shfl_down_sync(kFull, v.x, 1);
  return make_float2(v.y + pv, nv + v.x);
}
// r(x + 1) + l(x - 1):
__device__ __forceinline__ float2 rl2(float2 r, float2 l) {
  const float nr = __shfl_down_sync(kFull, r.x, 1), pl = __shfl_up_sync(kFull, l.y, 1);
  return make_float2(r.y + pl, nr + l.x);
}
// r(x + 1) + l(x - 1) and r(x + 1) - l(x - 1):
__device__ __forceinline__ void rl2_sd(float2 r, float2 l, float2& sum, float2& diff) {
  const float nr = __shfl_down_sync(kFull, r.x, 1), pl = __shfl_up_sync(kFull, l.y, 1);
  sum = make_float2(r.y + pl, nr + l.x);
  diff = make_float2(r.y - pl, nr - l.x);
}

// ---- mbarrier and TMA (inline PTX) -------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// Shared-memory reads of a slot (generic proxy) happen before the next TMA write into it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of barrier b, for at most about a second; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(b, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}

// One tiled copy of a 5D box into shared memory, completing on barrier b. The tensor maps view the
// state as (x, field, y, z, slot), so a box of (columns, fields, rows) lands as [row][field][column].
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int x, int f, int y, int z, int s,
                                            unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(f), "r"(y), "r"(z), "r"(s), "r"(smem_u32(b))
      : "memory");
}

// ---- windows and chunks --------------------------------------------------------------------------
// Window i reads columns 60 i - 4 .. 60 i + 59 (a multiple of 4, as a TMA box start must be) and
// writes columns 60 i - 2 .. 60 i + 57 that lie on the grid.
__host__ __device__ __forceinline__ int q_windows(int nx) { return (nx + 2 + QOX - 1) / QOX; }
__host__ __device__ __forceinline__ int q_tiles_y(int ny) { return (ny + QOY - 1) / QOY; }

// Rows of a tile. Tile j writes rows y0 .. y0 + 11 with y0 = min(12 j, ny - 12) (the last tile
// ends at the grid's end and may repeat rows of the one before: the same values) and reads rows
// y0 - 2 .. y0 + 13, which one box of 16 rows starting at ys = clamp(y0 - 2, 0, ny - 16) holds
// except for at most two rows wrapped across y = 0 (first tile: ny - 2, ny - 1; last tile: 0, 1),
// which a 2-row box puts in slot rows 16, 17. slot_row: the slot row of tile row r.
struct QRows {
  int y0, ys, halo_y;  // halo_y: grid row of the 2-row box, or -1 if the tile needs none
  __device__ __forceinline__ QRows(int j, int ny) {
    y0 = min(QOY * j, ny - QOY);
    ys = min(max(y0 - 2, 0), ny - QW);
    halo_y = y0 - 2 < 0 ? ny - 2 : (y0 + QW - 2 > ny ? 0 : -1);
  }
  __device__ __forceinline__ int slot_row(int r, int ny) const {
    const int y = y0 - 2 + r;
    if (y < 0) return QW + (y + 2);
    if (y >= ny) return QW + (y - ny);
    return y - ys;
  }
};

// Columns of a window outside the grid take, per open x plane, the boundary node (the gradient's
// ghost rule; TMA fills zeros there) or, periodic in x, the wrapped node from a 4-column copy of
// the far end of the row. col_src: >= 0 a column of the window tile, <= -1 column (-1 - v) of the
// wrap copy, kNoSrc no value (zero).
// The transpose asks for zero (clamp = false): the adjoint of a node off the grid is zero.
constexpr int kNoSrc = -1000;
__device__ __forceinline__ int col_source(int xc, int xs, int nx, bool px, int gx0, bool clamp) {
  if (xc >= 0 && xc < nx) return xc - xs;
  if (!px) return clamp ? (xc < 0 ? 0 : nx - 1) - xs : kNoSrc;
  const int xw = xc < 0 ? xc + nx : xc - nx;
  const int k = xw - gx0;
  return (k >= 0 && k < 4) ? -1 - k : kNoSrc;
}

// Output planes [*za, *zb) of this CTA's chunk: chunks split nz evenly.
__device__ __forceinline__ void q_chunk(int nz, int* za, int* zb) {
  *za = (int)(((long long)blockIdx.z * nz) / gridDim.z);
  *zb = (int)(((long long)(blockIdx.z + 1) * nz) / gridDim.z);
}

// ---- forward ---------------------------------------------------------------------------------------
// Per plane zr, two block barriers: after the first the rows read exchange 1 (u, S_z u, D_z u of
// plane zr from the rows above and below) and rows 1..14 form the gradient and f^eq, writing the
// c_y != 0 values to exchange 2; after the second rows 2..13 gather those and complete output
// plane zr - 1. The ring holds QRF planes, so about QRF - 1 planes (16 KB each) are in flight per
// SM while the CTA computes: with one CTA per SM, fewer left the copies latency-bound.
constexpr int QRF = 7;
struct QFwdSmem {
  float ring[QRF][QSR][4][QIX];  // plane slots: per row p, u_x, u_y, u_z over the window's columns
  float ghost[QRF][QSR][4][4];   // periodic x: the 4 wrapped columns of each row
  float2 r1[9][QW][32];          // exchange 1: u, S_z u, D_z u of every row
  float2 r2[10][QW][32];         // exchange 2: f_3, f_4 and the eight corner values of every row
  unsigned long long bar[QRF];
};

// The tensor maps of a state (or adjoint) array for the row-streamed kernels: boxes of 64 or 4
// columns by 4 fields by 16 or 2 rows of one plane of one slot.
struct QMaps {
  CUtensorMap main, halo, gmain, ghalo;
};

// One forward step t = ctrl->t0 + di: state slot(t - 1) -> slot(t).
template <bool PX>
__global__ void __launch_bounds__(QT, 1)
    k_stencil3d_q(const __grid_constant__ QMaps tm, Geo g, Slots<float> S, Ctrl* ctrl, int di) {
  extern __shared__ __align__(128) unsigned char q_smem[];
  QFwdSmem& s = *reinterpret_cast<QFwdSmem*>(q_smem);  // shared-space addresses throughout
  if (smem_u32(q_smem) & 127u) {  // the copy engine needs 128-byte aligned slots
    if (threadIdx.x == 0) atomicOr(&ctrl->status, ST_SYNC_TIMEOUT);
    return;
  }
  if (ctrl->status & ST_SYNC_TIMEOUT) return;  // an earlier wait of this call timed out: results are void
  const bool skip_copy = (ctrl->sync_skip & 2) != 0;  // test hook: withhold the copy of plane 2
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int t = ctrl->t0 + di, base = ctrl->base;
  int sslot = (t - 1 - base) % S.nslots;
  if (sslot < 0) sslot += S.nslots;
  float* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int xs = QOX * (int)blockIdx.x - 4;  // first column of the window
  const QRows rows(blockIdx.y, ny);
  const int y0 = rows.y0;  // first output row (input rows y0 - 2 .. y0 + 13)
  const int srow = rows.slot_row(w, ny);
  int za, zb;
  q_chunk(nz, &za, &zb);
  const int nq = zb - za + 4;  // input planes za - 2 .. zb + 1, indexed 0 .. nq - 1
  const bool wrap_lo = PX && xs < 0, wrap_hi = PX && xs + QIX > nx, ghost = wrap_lo || wrap_hi;
  const int gx0 = wrap_lo ? nx - 4 : 0;
  const bool halo = rows.halo_y >= 0;
  const unsigned plane_bytes = (QW + (halo ? 2 : 0)) * (QROWB + (ghost ? 64 : 0));
  const int xc0 = xs + 2 * lane;  // this lane's columns xc0, xc0 + 1
  const bool edge = xc0 < 0 || xc0 + 1 >= nx;
  const int src0 = col_source(xc0, xs, nx, PX, gx0, true), src1 = col_source(xc0 + 1, xs, nx, PX, gx0, true);
  const bool inflow = g.bc[0] == BC_INFLOW_OUTFLOW;
  const float u_in = (float)g.u_in, dp = (float)g.dp;
  const float kA = g.A2 * 0.1f;  // 2A / 10 (the G below are ten times the gradient)
  const float2 kAw1 = f2(kA / 9.0f), kAw3 = f2(kA / 72.0f);
  const bool row_f = w >= 1 && w <= QW - 2, row_out = w >= 2 && w <= QW - 3;
  float* const out_row = dst + xc0 + (long long)nx * (y0 + w - 2);  // this lane's output row of plane 0
  const bool store_row = row_out && lane >= 1 && lane <= 30;

  auto issue = [&](int jq) {  // thread 0: plane za - 2 + jq into slot jq % QRF
    if (skip_copy && jq == 2) return;  // its wait runs out; no copy is left in flight
    const int sl = jq % QRF, zq = wrapi(za - 2 + jq, nz);
    mbar_expect_tx(&s.bar[sl], plane_bytes);
    tma_load_5d(&s.ring[sl][0][0][0], &tm.main, xs, 0, rows.ys, zq, sslot, &s.bar[sl]);
    if (halo) tma_load_5d(&s.ring[sl][QW][0][0], &tm.halo, xs, 0, rows.halo_y, zq, sslot, &s.bar[sl]);
    if (ghost) {
      tma_load_5d(&s.ghost[sl][0][0][0], &tm.gmain, gx0, 0, rows.ys, zq, sslot, &s.bar[sl]);
      if (halo) tma_load_5d(&s.ghost[sl][QW][0][0], &tm.ghalo, gx0, 0, rows.halo_y, zq, sslot, &s.bar[sl]);
    }
  };
  auto read_plane = [&](int jq, float2& p, float2 (&u)[3]) -> bool {  // this row's values of plane jq
    const int sl = jq % QRF;
    const bool ok = mbar_wait_bounded(&s.bar[sl], (unsigned)(jq / QRF) & 1u);
    if (!ok) atomicOr(&ctrl->status, ST_SYNC_TIMEOUT);
    const float* row = &s.ring[sl][srow][0][0];
    if (!edge) {
      p = *reinterpret_cast<const float2*>(row + 2 * lane);
#pragma unroll
      for (int a = 0; a < 3; ++a) u[a] = *reinterpret_cast<const float2*>(row + (1 + a) * QIX + 2 * lane);
    } else {
      const float* gh = &s.ghost[sl][srow][0][0];
      auto pick = [&](int c, int src) {
        return src >= 0 ? row[c * QIX + src] : (src == kNoSrc ? 0.0f : gh[c * 4 + (-1 - src)]);
      };
      p = make_float2(pick(0, src0), pick(0, src1));
#pragma unroll
      for (int a = 0; a < 3; ++a) u[a] = make_float2(pick(1 + a, src0), pick(1 + a, src1));
    }
    return ok;
  };

  // Step jq (2 .. nq - 1): plane jq (zr + 1) arrives into (P1, U1); Um, U0 hold planes zr - 1, zr
  // and P0 plane zr's p; Am, Ac, Ap are output planes zr - 1, zr, zr + 1. False if a copy's wait
  // timed out anywhere in the block.
  auto step = [&](int jq, float2 (&Am)[4], float2 (&Ac)[4], float2 (&Ap)[4], float2 (&Um)[3], float2 (&U0)[3],
                  float2 (&U1)[3], float2& P0, float2& P1) -> bool {
    const int zr = za + jq - 3;
    const bool fail = !read_plane(jq, P1, U1);
    float2 Dz[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Dz[a] = sub2(U1[a], Um[a]);
      s.r1[a][w][lane] = U0[a];
      s.r1[3 + a][w][lane] = add2(U1[a], Um[a]);
      s.r1[6 + a][w][lane] = Dz[a];
    }
    if (__syncthreads_or(fail)) return false;  // exchange 1 written; plane jq's slot consumed
    if (tid == 0 && jq + QRF < nq) {
      fence_proxy_async();
      issue(jq + QRF);
    }
    if (row_f) {
      float2 G[3][3];  // ten times d_b u_a at this node
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 Uu = s.r1[a][w + 1][lane], Ud = s.r1[a][w - 1][lane];
        const float2 Su = s.r1[3 + a][w + 1][lane], Sd = s.r1[3 + a][w - 1][lane];
        const float2 Du = s.r1[6 + a][w + 1][lane], Dd = s.r1[6 + a][w - 1][lane];
        const float2 X1v = add2(U0[a], add2(Su, Sd));
        const float2 dysz = sub2(Su, Sd), sydz = add2(Du, Dd);
        G[a][0] = dx2(X1v);
        G[a][1] = add2(sub2(Uu, Ud), sx2(dysz));
        G[a][2] = add2(Dz[a], sx2(sydz));
      }
      const float2 ux = U0[0], uy = U0[1], uz = U0[2];
      const float2 usq = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
      const float2 a0 = fma2(usq, f2(-1.5f), mul2(P0, f2(3.0f)));  // 3p - 3/2 |u|^2
      // axis vectors: w1 (a0 + Q_kk) +- 3 w1 u_k with Q_kk = 9/2 u_k^2 + 2A G_kk
      const float2 w1a0 = mul2(a0, f2(1.0f / 9.0f));
      const float2 tx = fma2(mul2(ux, ux), f2(0.5f), fma2(G[0][0], kAw1, w1a0));
      const float2 ty = fma2(mul2(uy, uy), f2(0.5f), fma2(G[1][1], kAw1, w1a0));
      const float2 tz = fma2(mul2(uz, uz), f2(0.5f), fma2(G[2][2], kAw1, w1a0));
      const float2 bx = mul2(ux, f2(1.0f / 3.0f)), by = mul2(uy, f2(1.0f / 3.0f)), bz = mul2(uz, f2(1.0f / 3.0f));
      // corners s: w3 (a0 + tr Q + 3 s.u + s_x s_y Q_xy + s_x s_z Q_xz + s_y s_z Q_yz),
      // a0 + tr Q = 3 (p + |u|^2) + 2A tr G, Q_ab = 9 u_a u_b + 2A (G_ab + G_ba)
      const float2 trG = add2(add2(G[0][0], G[1][1]), G[2][2]);
      const float2 al = fma2(trG, kAw3, mul2(add2(P0, usq), f2(3.0f / 72.0f)));
      const float2 Bx = mul2(ux, f2(3.0f / 72.0f)), By = mul2(uy, f2(3.0f / 72.0f)), Bz = mul2(uz, f2(3.0f / 72.0f));
      const float2 Qxy = fma2(add2(G[0][1], G[1][0]), kAw3, mul2(mul2(ux, uy), f2(9.0f / 72.0f)));
      const float2 Qxz = fma2(add2(G[0][2], G[2][0]), kAw3, mul2(mul2(ux, uz), f2(9.0f / 72.0f)));
      const float2 Qyz = fma2(add2(G[1][2], G[2][1]), kAw3, mul2(mul2(uy, uz), f2(9.0f / 72.0f)));
      s.r2[0][w][lane] = add2(ty, by);  // f_3 (c = +y), read by the row above
      s.r2[1][w][lane] = sub2(ty, by);  // f_4 (c = -y), read by the row below
#pragma unroll
      for (int iz = 0; iz < 2; ++iz) {  // s_z = +1, -1
        const float2 e = iz ? sub2(al, Bz) : add2(al, Bz);
        const float2 X = iz ? sub2(Bx, Qxz) : add2(Bx, Qxz), Y = iz ? sub2(By, Qyz) : add2(By, Qyz);
        const float2 t1 = add2(e, Qxy), t2 = sub2(e, Qxy), P = add2(X, Y), M = sub2(X, Y);
        // s_y = +1 values go to the row above, s_y = -1 values to the row below
        s.r2[2 + 2 * iz][w][lane] = add2(t1, P);  // (+, +)
        s.r2[3 + 2 * iz][w][lane] = sub2(t2, M);  // (-, +)
        s.r2[6 + 2 * iz][w][lane] = add2(t2, M);  // (+, -)
        s.r2[7 + 2 * iz][w][lane] = sub2(t1, P);  // (-, -)
      }
      if (row_out) {  // the node's own values along x (plane zr) and z (planes zr + 1, zr - 1)
        const float2 f0 = mul2(a0, f2(2.0f / 9.0f));
        float2 sx, dx;  // f_2 (c = -x) from x + 1 and f_1 (c = +x) from x - 1: sum and difference
        rl2_sd(sub2(tx, bx), add2(tx, bx), sx, dx);
        const float2 f5 = add2(tz, bz), f6 = sub2(tz, bz);
        Ac[0] = add2(Ac[0], add2(f0, sx));
        Ac[1] = sub2(Ac[1], dx);
        Ap[0] = add2(Ap[0], f5);
        Ap[3] = add2(Ap[3], f5);
        Am[0] = add2(Am[0], f6);
        Am[3] = sub2(Am[3], f6);
      }
    }
    __syncthreads();  // exchange 2 written
    if (row_out) {
      const float2 f3d = s.r2[0][w - 1][lane], f4u = s.r2[1][w + 1][lane];
      Ac[0] = add2(Ac[0], add2(f3d, f4u));
      Ac[2] = add2(Ac[2], sub2(f3d, f4u));
#pragma unroll
      for (int iz = 0; iz < 2; ++iz) {
        // (s_x, s_z) groups: from the row below (s_y = +1) and the row above (s_y = -1)
        const float2 dP = s.r2[2 + 2 * iz][w - 1][lane], dM = s.r2[3 + 2 * iz][w - 1][lane];
        const float2 uP = s.r2[6 + 2 * iz][w + 1][lane], uM = s.r2[7 + 2 * iz][w + 1][lane];
        // s_x = +1 values from x - 1, s_x = -1 values from x + 1
        float2 sA, mA;  // mA: the s_x = -1 values less the s_x = +1 ones
        rl2_sd(add2(dM, uM), add2(dP, uP), sA, mA);
        const float2 sB = rl2(sub2(dM, uM), sub2(dP, uP));
        if (iz == 0) {  // s_z = +1: output plane zr + 1
          Ap[0] = add2(Ap[0], sA);
          Ap[1] = sub2(Ap[1], mA);
          Ap[2] = add2(Ap[2], sB);
          Ap[3] = add2(Ap[3], sA);
        } else {  // s_z = -1: output plane zr - 1
          Am[0] = add2(Am[0], sA);
          Am[1] = sub2(Am[1], mA);
          Am[2] = add2(Am[2], sB);
          Am[3] = sub2(Am[3], sA);
        }
      }
      if (store_row && zr - 1 >= za) {  // output plane zr - 1 is complete
        float2 o[4] = {mul2(Am[0], f2(1.0f / 3.0f)), Am[1], Am[2], Am[3]};
        if (!PX) {  // open x planes: prescribed values from the inner node
          if (xc0 == 0) {
            o[0].x = inflow ? o[0].y : dp;
            o[1].x = inflow ? u_in : o[1].y;
            o[2].x = inflow ? 0.0f : o[2].y;
            o[3].x = inflow ? 0.0f : o[3].y;
          }
          if (xc0 + 1 == nx - 1) {
            o[0].y = 0.0f;
            o[1].y = o[1].x;
            o[2].y = o[2].x;
            o[3].y = o[3].x;
          }
        }
        float* op = out_row + (long long)(zr - 1) * nx * ny;
        if (!edge) {
#pragma unroll
          for (int c = 0; c < 4; ++c) *reinterpret_cast<float2*>(op + c * N) = o[c];
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (xc0 >= 0 && xc0 < nx) op[c * N] = o[c].x;
            if (xc0 + 1 >= 0 && xc0 + 1 < nx) op[c * N + 1] = o[c].y;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) Am[c] = f2(0.0f);  // becomes output plane zr + 2
    return true;
  };

  if (tid == 0) {
    for (int i = 0; i < QRF; ++i) mbar_init(&s.bar[i], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < QRF && j < nq; ++j) issue(j);
  // planes by index mod 3 (X: 0, 3, ...; Y: 1, 4, ...; Z: 2, 5, ...), outputs likewise (A, B, C)
  float2 pX, X[3], pY, Y[3], pZ, Z[3];
  bool fail0 = !read_plane(0, pX, X);
  fail0 = !read_plane(1, pY, Y) || fail0;
  bool ok = !__syncthreads_or(fail0);
  int drain_from = 0, issued = min(nq, QRF);
  if (tid == 0 && ok) {
    fence_proxy_async();
    for (int j = QRF; j < QRF + 2 && j < nq; ++j) issue(j);
  }
  float2 A[4], B[4], C[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) A[c] = B[c] = C[c] = f2(0.0f);
  for (int jq = 2; jq < nq && ok; jq += 3) {
    int j = jq;
    ok = step(j, A, B, C, X, Y, Z, pY, pZ);
    if (ok && ++j < nq) ok = step(j, B, C, A, Y, Z, X, pZ, pX);
    if (ok && ++j < nq) ok = step(j, C, A, B, Z, X, Y, pX, pY);
    if (!ok) {  // planes from j on may still be in flight
      drain_from = j;
      issued = min(nq, j - 1 + QRF + 1);
    }
  }
  // after a timed-out wait: wait (bounded) for the copies still in flight before the CTA exits
  if (tid == 0 && !ok)
    for (int k = drain_from; k < issued; ++k) (void)mbar_wait_bounded(&s.bar[k % QRF], (unsigned)(k / QRF) & 1u);
}

// ---- transpose -------------------------------------------------------------------------------------
struct QAdjSmem {
  float ring[QR][QSR][4][QIX];  // plane slots: per row lam_p*, lam_u* over the window's columns
  float st[QR][QOY][3][QIX];    // u(t-1) of the output rows
  float ghost[QR][QSR][4][4];   // periodic x: the 4 wrapped columns of each adjoint row
  float2 r1[10][QW][32];              // exchange 1: phi_{+y}, phi_{-y}, Gamma and Delta of every row
  float2 r2[6][QW][32];               // exchange 2: S_xx, S_yy, S_zz, S_xy, S_xz, S_yz of every row
  unsigned long long bar[QR];
  int abort;
};

// One reverse step t = ctrl->t0 - di: adjoint Lb[t & 1] -> Lb[(t - 1) & 1] at the state slot(t - 1).
// tl: the adjoint's maps; tu: boxes of 64 columns x 3 fields (u_x, u_y, u_z) x 12 rows of the state.
template <bool PX>
__global__ void __launch_bounds__(QT, 1)
    k_stencil3d_adj_q(const __grid_constant__ QMaps tl, const __grid_constant__ CUtensorMap tu, Geo g,
                      Slots<float> S, float* Lb, long long lstride, Ctrl* ctrl, int di) {
  extern __shared__ __align__(128) unsigned char q_smem[];
  QAdjSmem& s = *reinterpret_cast<QAdjSmem*>(q_smem);  // shared-space addresses throughout
  if (smem_u32(q_smem) & 127u) {  // the copy engine needs 128-byte aligned slots
    if (threadIdx.x == 0) atomicOr(&ctrl->status, ST_SYNC_TIMEOUT);
    return;
  }
  if (ctrl->status & ST_SYNC_TIMEOUT) return;  // an earlier wait of this call timed out: results are void
  const bool skip_copy = (ctrl->sync_skip & 2) != 0;  // test hook: withhold the copy of plane 2
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int t = ctrl->t0 - di, base = ctrl->base;
  int sslot = (t - 1 - base) % S.nslots;
  if (sslot < 0) sslot += S.nslots;
  const int lslot = t & 1;
  float* __restrict__ Lnext = Lb + (long long)((t - 1) & 1) * lstride;
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int xs = QOX * (int)blockIdx.x - 4;
  const QRows rows(blockIdx.y, ny);
  const int y0 = rows.y0;
  const int srow = rows.slot_row(w, ny);
  int za, zb;
  q_chunk(nz, &za, &zb);
  const int nq = zb - za + 4;
  const bool wrap_lo = PX && xs < 0, wrap_hi = PX && xs + QIX > nx, ghost = wrap_lo || wrap_hi;
  const int gx0 = wrap_lo ? nx - 4 : 0;
  const bool halo = rows.halo_y >= 0;
  const unsigned plane_bytes = (QW + (halo ? 2 : 0)) * (QROWB + (ghost ? 64 : 0)) + QOY * QSTB;
  const int xc0 = xs + 2 * lane;
  // lanes holding a column off the grid or a column of an open x plane (0, nx - 1)
  const bool edge = xc0 < 0 || xc0 + 1 >= nx || (!PX && (xc0 == 0 || xc0 + 1 == nx - 1));
  const int src0 = col_source(xc0, xs, nx, PX, gx0, false), src1 = col_source(xc0 + 1, xs, nx, PX, gx0, false);
  const bool on0 = PX || (xc0 >= 0 && xc0 < nx), on1 = PX || (xc0 + 1 >= 0 && xc0 + 1 < nx);
  const int bx = g.bc[0];

  auto issue = [&](int jq) {
    if (skip_copy && jq == 2) return;  // test hook: its wait runs out; no copy is left in flight
    const int sl = jq % QR, zq = wrapi(za - 2 + jq, nz);
    mbar_expect_tx(&s.bar[sl], plane_bytes);
    tma_load_5d(&s.ring[sl][0][0][0], &tl.main, xs, 0, rows.ys, zq, lslot, &s.bar[sl]);
    if (halo) tma_load_5d(&s.ring[sl][QW][0][0], &tl.halo, xs, 0, rows.halo_y, zq, lslot, &s.bar[sl]);
    if (ghost) {
      tma_load_5d(&s.ghost[sl][0][0][0], &tl.gmain, gx0, 0, rows.ys, zq, lslot, &s.bar[sl]);
      if (halo) tma_load_5d(&s.ghost[sl][QW][0][0], &tl.ghalo, gx0, 0, rows.halo_y, zq, lslot, &s.bar[sl]);
    }
    tma_load_5d(&s.st[sl][0][0][0], &tu, xs, 1, y0, zq, sslot, &s.bar[sl]);
  };
  // This row's a = lam_p* / 3 and b = lam_u* of plane jq, after the reverse of the open x planes'
  // rules: a boundary node's own entries are zero and the entries of the values it prescribed
  // from an inner node go to that node (inflow: p at 1 from 0; pressure: u at 1 from 0; outlet
  // and pressure outlet: u at nx - 2 from nx - 1). Also the state's u at the node (output rows).
  auto read_plane = [&](int jq, float2& a, float2 (&b)[3], float2 (&us)[3]) {
    const int sl = jq % QR;
    if (!mbar_wait_bounded(&s.bar[sl], (unsigned)(jq / QR) & 1u)) {
      atomicOr(&ctrl->status, ST_SYNC_TIMEOUT);
      s.abort = 1;
    }
    const float* row = &s.ring[sl][srow][0][0];
    float2 lp, lu[3];
    if (!edge) {
      lp = *reinterpret_cast<const float2*>(row + 2 * lane);
#pragma unroll
      for (int c = 0; c < 3; ++c) lu[c] = *reinterpret_cast<const float2*>(row + (1 + c) * QIX + 2 * lane);
    } else {
      const float* gh = &s.ghost[sl][srow][0][0];
      auto pick = [&](int c, int src) {
        return src >= 0 ? row[c * QIX + src] : (src == kNoSrc ? 0.0f : gh[c * 4 + (-1 - src)]);
      };
      lp = make_float2(pick(0, src0), pick(0, src1));
#pragma unroll
      for (int c = 0; c < 3; ++c) lu[c] = make_float2(pick(1 + c, src0), pick(1 + c, src1));
      if (!PX) {
        if (xc0 == 0) {  // columns 0 and 1
          if (bx == BC_INFLOW_OUTFLOW) lp.y += lp.x;
          else
#pragma unroll
            for (int c = 0; c < 3; ++c) lu[c].y += lu[c].x;
          lp.x = 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) lu[c].x = 0.0f;
        }
        if (xc0 + 1 == nx - 1) {  // columns nx - 2 and nx - 1
#pragma unroll
          for (int c = 0; c < 3; ++c) lu[c].x += lu[c].y;
          lp.y = 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) lu[c].y = 0.0f;
        }
      }
    }
    a = mul2(lp, f2(1.0f / 3.0f));
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c] = lu[c];
    if (w >= 2 && w < QW - 2) {
      const float* srow = &s.st[sl][w - 2][0][0];
#pragma unroll
      for (int c = 0; c < 3; ++c) us[c] = *reinterpret_cast<const float2*>(srow + c * QIX + 2 * lane);
    }
  };

  if (tid == 0) {
    for (int i = 0; i < QR; ++i) mbar_init(&s.bar[i], 1);
    mbar_init_fence();
    s.abort = 0;
  }
  __syncthreads();
  if (tid == 0)
    for (int j = 0; j < QR && j < nq; ++j) issue(j);
  float2 am_, a0_, bm_[3], b0_[3], us0[3], usd[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) us0[c] = usd[c] = f2(0.0f);
  read_plane(0, am_, bm_, usd);
  read_plane(1, a0_, b0_, us0);
  __syncthreads();
  const bool aborted0 = s.abort != 0;
  if (tid == 0 && !aborted0) {
    fence_proxy_async();
    for (int j = QR; j < QR + 2 && j < nq; ++j) issue(j);
  }
  float2 qm[4], qc[4], qp[4];  // output planes zr - 1, zr, zr + 1: lam_p, lam_u
#pragma unroll
  for (int c = 0; c < 4; ++c) qm[c] = qc[c] = qp[c] = f2(0.0f);
  const float2 kA = f2(g.A2 * 0.1f);  // 2A / 10
  const float2 w0 = f2(2.0f / 9.0f), w1 = f2(1.0f / 9.0f), w3 = f2(1.0f / 72.0f);
  const bool row_m = w >= 1 && w <= QW - 2, row_out = w >= 2 && w <= QW - 3;
  int jstop = aborted0 ? 0 : nq;

  for (int jq = 2; jq < nq && !aborted0; ++jq) {
    const int zr = za + jq - 3;  // plane of this step's moments (plane zr + 1 arrives)
    float2 ap_, bp_[3], us1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) us1[c] = f2(0.0f);
    read_plane(jq, ap_, bp_, us1);
    // z pass: S_z and D_z of a and b, then the corner combinations Gamma_{sx,sy} (moments P, U_x,
    // U_y, S_xy) and Delta_{sx,sy} (U_z, S_xz, S_yz) that the rows and columns around gather
    const float2 Szbx = add2(bp_[0], bm_[0]), Dzbx = sub2(bp_[0], bm_[0]);
    const float2 Szby = add2(bp_[1], bm_[1]), Dzby = sub2(bp_[1], bm_[1]);
    const float2 al = add2(add2(ap_, am_), sub2(bp_[2], bm_[2]));  // S_z a + D_z b_z
    const float2 be = add2(sub2(ap_, am_), add2(bp_[2], bm_[2]));  // D_z a + S_z b_z
    {
      const float2 g1 = add2(al, Szbx), g2 = sub2(al, Szbx), d1 = add2(be, Dzbx), d2 = sub2(be, Dzbx);
      s.r1[0][w][lane] = add2(a0_, b0_[1]);  // phi_{+y}, read by the row below
      s.r1[1][w][lane] = sub2(a0_, b0_[1]);  // phi_{-y}, read by the row above
      s.r1[2][w][lane] = add2(g1, Szby);     // Gamma_{+,+}
      s.r1[3][w][lane] = add2(g2, Szby);     // Gamma_{-,+}
      s.r1[4][w][lane] = add2(d1, Dzby);     // Delta_{+,+}
      s.r1[5][w][lane] = add2(d2, Dzby);     // Delta_{-,+}
      s.r1[6][w][lane] = sub2(g1, Szby);     // Gamma_{+,-}
      s.r1[7][w][lane] = sub2(g2, Szby);     // Gamma_{-,-}
      s.r1[8][w][lane] = sub2(d1, Dzby);     // Delta_{+,-}
      s.r1[9][w][lane] = sub2(d2, Dzby);     // Delta_{-,-}
    }
    __syncthreads();  // S1
    if (s.abort) {
      jstop = jq;
      break;
    }
    if (tid == 0 && jq + QR < nq) {
      fence_proxy_async();
      issue(jq + QR);
    }
    float2 P, U[3], Sm[6];  // moments at this node of plane zr (S: xx, yy, zz, xy, xz, yz)
    if (row_m) {
      // y pass: s_y = +1 values from the row above, s_y = -1 values from the row below
      const float2 Yp = s.r1[0][w + 1][lane], Ym = s.r1[1][w - 1][lane];
      const float2 gpp = s.r1[2][w + 1][lane], gmp = s.r1[3][w + 1][lane];
      const float2 dpp = s.r1[4][w + 1][lane], dmp = s.r1[5][w + 1][lane];
      const float2 gpm = s.r1[6][w - 1][lane], gmm = s.r1[7][w - 1][lane];
      const float2 dpm = s.r1[8][w - 1][lane], dmm = s.r1[9][w - 1][lane];
      // x pass: s_x = +1 values from x + 1, s_x = -1 values from x - 1
      float2 Pc, Uxc, Uyc, Sxyc, Uzc, Sxzc, sX, dX;
      rl2_sd(add2(gpp, gpm), add2(gmp, gmm), Pc, Uxc);
      rl2_sd(sub2(gpp, gpm), sub2(gmp, gmm), Uyc, Sxyc);
      rl2_sd(add2(dpp, dpm), add2(dmp, dmm), Uzc, Sxzc);
      const float2 Syzc = rl2(sub2(dpp, dpm), sub2(dmp, dmm));
      rl2_sd(add2(a0_, b0_[0]), sub2(a0_, b0_[0]), sX, dX);
      const float2 Zp = add2(ap_, bp_[2]), Zm = sub2(am_, bm_[2]);
      const float2 sY = add2(Yp, Ym), sZ = add2(Zp, Zm);
      P = fma2(w0, a0_, fma2(w1, add2(add2(sX, sY), sZ), mul2(w3, Pc)));
      U[0] = fma2(w1, dX, mul2(w3, Uxc));
      U[1] = fma2(w1, sub2(Yp, Ym), mul2(w3, Uyc));
      U[2] = fma2(w1, sub2(Zp, Zm), mul2(w3, Uzc));
      Sm[0] = fma2(w1, sX, mul2(w3, Pc));
      Sm[1] = fma2(w1, sY, mul2(w3, Pc));
      Sm[2] = fma2(w1, sZ, mul2(w3, Pc));
      Sm[3] = mul2(w3, Sxyc);
      Sm[4] = mul2(w3, Sxzc);
      Sm[5] = mul2(w3, Syzc);
      if (!on0 || !on1) {  // the moments are zero off the grid (open x)
        if (!on0) {
          P.x = 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) U[c].x = 0.0f;
#pragma unroll
          for (int c = 0; c < 6; ++c) Sm[c].x = 0.0f;
        }
        if (!on1) {
          P.y = 0.0f;
#pragma unroll
          for (int c = 0; c < 3; ++c) U[c].y = 0.0f;
#pragma unroll
          for (int c = 0; c < 6; ++c) Sm[c].y = 0.0f;
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) s.r2[c][w][lane] = Sm[c];
      if (row_out) {  // local part: lam_p = 3P, lam_u = 3U + 9 S u - 3 u P
        const float2 ux = us0[0], uy = us0[1], uz = us0[2];
        const float2 Sux = fma2(Sm[4], uz, fma2(Sm[3], uy, mul2(Sm[0], ux)));
        const float2 Suy = fma2(Sm[5], uz, fma2(Sm[1], uy, mul2(Sm[3], ux)));
        const float2 Suz = fma2(Sm[2], uz, fma2(Sm[5], uy, mul2(Sm[4], ux)));
        const float2 m3P = mul2(P, f2(-3.0f));
        qc[0] = fma2(P, f2(3.0f), qc[0]);
        qc[1] = add2(qc[1], fma2(U[0], f2(3.0f), fma2(Sux, f2(9.0f), mul2(ux, m3P))));
        qc[2] = add2(qc[2], fma2(U[1], f2(3.0f), fma2(Suy, f2(9.0f), mul2(uy, m3P))));
        qc[3] = add2(qc[3], fma2(U[2], f2(3.0f), fma2(Suz, f2(9.0f), mul2(uz, m3P))));
      }
    }
    __syncthreads();  // S2
    if (row_out) {
      // gradient transpose h_a = -sum_b D_b (1 + S S) S_ab, scattered over planes zr - 1, zr, zr + 1
      float2 Su[6], Sd[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        Su[c] = s.r2[c][w + 1][lane];
        Sd[c] = s.r2[c][w - 1][lane];
      }
      // (S_ax, S_ay, S_az) for a = x, y, z in the symmetric storage order xx, yy, zz, xy, xz, yz
      constexpr int IX[3] = {0, 3, 4}, IY[3] = {3, 1, 5}, IZ[3] = {4, 5, 2};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 sySax = add2(Su[IX[a]], Sd[IX[a]]);
        const float2 dySay = sub2(Su[IY[a]], Sd[IY[a]]);
        const float2 sySaz = add2(Su[IZ[a]], Sd[IZ[a]]);
        const float2 Sax = Sm[IX[a]], Saz = Sm[IZ[a]];
        // plane zr: -(D_x S_ax + D_y S_ay)
        const float2 h0 = sub2(f2(0.0f), add2(dx2(Sax), dySay));
        // planes zr +- 1: +-S_az - (D_x S_y S_ax + S_x D_y S_ay) +- S_x S_y S_az
        const float2 m = add2(sySax, dySay), n = sub2(dySay, sySax);
        const float2 hp = add2(Saz, rl2(sub2(sySaz, m), sub2(sySaz, n)));
        const float2 hm = sub2(f2(0.0f), add2(Saz, rl2(add2(m, sySaz), add2(n, sySaz))));
        qc[1 + a] = fma2(kA, h0, qc[1 + a]);
        qp[1 + a] = fma2(kA, hp, qp[1 + a]);
        qm[1 + a] = fma2(kA, hm, qm[1 + a]);
      }
      const int zo = zr - 1;
      const int y = y0 + w - 2;
      // open x planes: the gradient's ghost nodes -1 and nx copied nodes 0 and nx - 1, so what h
      // put on a ghost column belongs to the node it copied
      if (!PX && (xs < 0 || xs + QIX > nx)) {
#pragma unroll
        for (int c = 1; c < 4; ++c) {
          const float lo = __shfl_up_sync(kFull, qm[c].y, 1), hi = __shfl_down_sync(kFull, qm[c].x, 1);
          if (xc0 == 0) qm[c].x += lo;
          if (xc0 + 1 == nx - 1) qm[c].y += hi;
        }
      }
      if (zo >= za && lane >= 1 && lane <= 30) {
        const long long n = xc0 + (long long)nx * (y + (long long)ny * zo);
        if (xc0 >= 0 && xc0 + 1 < nx) {
#pragma unroll
          for (int c = 0; c < 4; ++c) *reinterpret_cast<float2*>(Lnext + c * N + n) = qm[c];
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if (xc0 >= 0 && xc0 < nx) Lnext[c * N + n] = qm[c].x;
            if (xc0 + 1 >= 0 && xc0 + 1 < nx) Lnext[c * N + n + 1] = qm[c].y;
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qm[c] = qc[c];
      qc[c] = qp[c];
      qp[c] = f2(0.0f);
    }
    am_ = a0_;
    a0_ = ap_;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bm_[c] = b0_[c];
      b0_[c] = bp_[c];
      us0[c] = us1[c];
    }
  }
  if (tid == 0 && jstop < nq) {
    const int issued = min(nq, (jstop < 2 ? 0 : jstop) + QR);
    for (int j = jstop; j < issued; ++j) (void)mbar_wait_bounded(&s.bar[j % QR], (unsigned)(j / QR) & 1u);
  }
}

// ---- host ---------------------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    cudaGetLastError();
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// A 5D view (x, field, y, z, slot) of nslots consecutive slots of 4 FP32 planes each, read in boxes
// of box_x columns x box_f fields x box_y rows of one plane.
bool encode_slots(CUtensorMap* m, const float* base, const Geo& g, long long slot_stride, int nslots, int box_x,
                  int box_f, int box_y) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[5] = {(cuuint64_t)g.n[0], 4, (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], (cuuint64_t)nslots};
  const cuuint64_t strides[4] = {(cuuint64_t)g.N * 4, (cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4,
                                 (cuuint64_t)slot_stride * 4};
  const cuuint32_t box[5] = {(cuuint32_t)box_x, (cuuint32_t)box_f, (cuuint32_t)box_y, 1, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_maps(QMaps* m, const float* base, const Geo& g, long long slot_stride, int nslots) {
  return encode_slots(&m->main, base, g, slot_stride, nslots, QIX, 4, QW) &&
         encode_slots(&m->halo, base, g, slot_stride, nslots, QIX, 4, 2) &&
         encode_slots(&m->gmain, base, g, slot_stride, nslots, 4, 4, QW) &&
         encode_slots(&m->ghalo, base, g, slot_stride, nslots, 4, 4, 2);
}

int device_sms() {
  static int sms = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 152;
    cudaGetLastError();
    return v;
  }();
  return sms;
}

// z chunks: the count that best fills whole waves of CTAs (one per SM) weighed against the three
// extra planes each chunk reads; every chunk holds at least four planes.
int q_chunks(const Geo& g) {
  const long long tiles = (long long)q_windows(g.n[0]) * q_tiles_y(g.n[1]);
  const int slots = device_sms();
  const int cmax = g.n[2] / 4 < 1 ? 1 : g.n[2] / 4;
  int best = 1;
  double best_eff = 0.0;
  for (int c = 1; c <= cmax; ++c) {
    const long long total = tiles * c;
    const long long waves = (total + slots - 1) / slots;
    const double planes = (double)g.n[2] / c;
    const double eff = (double)total / (double)(waves * slots) * planes / (planes + 3.0);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = c;
    }
  }
  return best;
}

constexpr size_t kFwdSmem = sizeof(QFwdSmem), kAdjSmem = sizeof(QAdjSmem);

}  // namespace

bool stencil3d_q_fits(const Geo& g) {
  return g.dim == 3 && g.bc[1] == BC_PERIODIC && g.bc[2] == BC_PERIODIC && g.bc[0] != BC_WALL && g.n[0] % 4 == 0 &&
         g.n[0] >= QIX && g.n[1] >= QW && tensor_map_encoder() != nullptr;
}

void prepare_stencil3d_q() {
  cudaFuncSetAttribute(k_stencil3d_q<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  cudaFuncSetAttribute(k_stencil3d_q<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  cudaFuncSetAttribute(k_stencil3d_adj_q<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
  cudaFuncSetAttribute(k_stencil3d_adj_q<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
}

bool launch_stencil3d_q_fwd(const Geo& g, const Slots<float>& S, const Ctrl* ctrl, int di, cudaStream_t st) {
  if (!stencil3d_q_fits(g)) return false;
  QMaps tm;
  if (!encode_maps(&tm, S.base, g, S.stride, S.nslots)) return false;
  const dim3 grid(q_windows(g.n[0]), q_tiles_y(g.n[1]), q_chunks(g));
  // the kernel writes ctrl->status only to report a timed-out wait
  Ctrl* c = const_cast<Ctrl*>(ctrl);
  if (g.bc[0] == BC_PERIODIC)
    launch(k_stencil3d_q<true>, grid, QT, kFwdSmem, st, tm, g, S, c, di);
  else
    launch(k_stencil3d_q<false>, grid, QT, kFwdSmem, st, tm, g, S, c, di);
  return true;
}

bool launch_stencil3d_q_adj(const Geo& g, const Slots<float>& S, float* Lb, long long lstride, const Ctrl* ctrl,
                            int di, cudaStream_t st) {
  if (!stencil3d_q_fits(g)) return false;
  QMaps tl;
  CUtensorMap tu;
  if (!encode_maps(&tl, Lb, g, lstride, 2) || !encode_slots(&tu, S.base, g, S.stride, S.nslots, QIX, 3, QOY))
    return false;
  const dim3 grid(q_windows(g.n[0]), q_tiles_y(g.n[1]), q_chunks(g));
  Ctrl* c = const_cast<Ctrl*>(ctrl);
  if (g.bc[0] == BC_PERIODIC)
    launch(k_stencil3d_adj_q<true>, grid, QT, kAdjSmem, st, tl, tu, g, S, Lb, lstride, c, di);
  else
    launch(k_stencil3d_adj_q<false>, grid, QT, kAdjSmem, st, tl, tu, g, S, Lb, lstride, c, di);
  return true;
}

}  // namespace lks
