// LKS predictor (Sec. 2.2) and its exact transpose on D3Q15.
//
// Velocities: rest (w = 2/9), the six axis vectors (w = 1/9) and the eight (+-1, +-1, +-1)
// (w = 1/72). With tau = 1, per cell x:
//   f_i^eq(y) = w_i (a + c.b + sum_ab c_a c_b Q_ab),  a = 3p - 3/2 |u|^2,  b = 3u,
//   Q_aa = 9/2 u_a^2 + 2A G_aa,  Q_ab = 9 u_a u_b + 2A (G_ab + G_ba)  (a < b),
//   G_ab = d_b u_a = sum_j c_jb u_a(y + c_j) / 10,
//   p*(x) = 1/3 sum_i f_i^eq(x - c_i),  u*(x) = sum_i c_i f_i^eq(x - c_i).
// Boundary values (Sec. 2.2), in this order: y walls for nodes with x and z interior (u = 0, p from
// the inner row), z walls for nodes with x interior (u = 0, p from the inner plane), then the open
// x planes (all rows). Gradient ghosts: open planes copy the boundary node, walls reflect u with a
// sign flip.
//
// GB300 form: one CTA of 512 threads per 32 x 16 column of cells marches over a chunk of z planes.
// Shared memory holds a ring of three input planes (halo 2 in x and y) and one plane of the 15
// f_i^eq values (halo 1); each plane's f values are scattered into three register accumulators
// (outputs at z - 1, z, z + 1). Each thread resolves its halo nodes' sources (the ghost rule along
// x and y) once for the whole march, and the next plane's global loads are issued into registers
// before the current plane is worked on, so their latency hides behind the f^eq arithmetic. Tiles
// whose outputs need no boundary phase write them straight from the accumulators. The number of z
// chunks is chosen to fill whole waves of resident CTAs. A z-wall plane is completed from its
// neighbour plane inside the same chunk (chunks hold at least four planes).
//
// Algorithmic traffic per cell: read p, u (4 values), write p*, u* (4 values): 32 B in FP32.
// Transpose: read the adjoint (4 values) and u(t-1) (3 values), write 4 values: 44 B in FP32.
#include "lks_kernels.h"
#include "lks_stencil_common.cuh"

namespace lks {

namespace {

constexpr int TX = kTileX, TY = kTileY3;
constexpr int NT = TX * TY;
constexpr int RX = TX + 4, RY = TY + 4;  // halo-2 input plane
constexpr int FX = TX + 2, FY = TY + 2;  // halo-1 plane of per-node values
constexpr int RPL = RX * RY, FPL = FX * FY;

template <typename T>
struct Fwd3Smem {
  T raw[3][4][RY][RX];  // ring of input planes: p, ux, uy, uz
  T f[15][FY][FX];      // f_i^eq of one plane
  T out[4][TY][TX];     // the plane being completed
  T out0[4][TY][TX];    // plane 0 of a z-wall, built from plane 1
  T prevp[TY][TX];      // p of the previous plane after the y-wall phase
};

template <typename T>
struct Adj3Smem {
  T raw[3][4][RY][RX];  // ring of adjoint planes with the boundary rules reversed
  T m[10][FY][FX];      // P, Ux, Uy, Uz, Sxx, Syy, Szz, Sxy, Sxz, Syz of one plane
};

__device__ __forceinline__ int ring(int z, int z0) { return (z - z0 + 3) % 3; }

// z range of this CTA's chunk: chunks split nz evenly (the host keeps each at >= 2 planes).
__device__ __forceinline__ void chunk_range(int nz, int* z0, int* z1) {
  *z0 = (int)(((long long)blockIdx.z * nz) / gridDim.z);
  *z1 = (int)(((long long)(blockIdx.z + 1) * nz) / gridDim.z);
}

// corner k = 0..7: (sx, sy, sz) = (+-1, +-1, +-1) with bit 0, 1, 2 selecting the minus sign
__device__ __forceinline__ constexpr int csx(int k) { return (k & 1) ? -1 : 1; }
__device__ __forceinline__ constexpr int csy(int k) { return (k & 2) ? -1 : 1; }
__device__ __forceinline__ constexpr int csz(int k) { return (k & 4) ? -1 : 1; }

constexpr int NLD = (RPL + NT - 1) / NT;  // halo-2 plane nodes per thread
constexpr int NFQ = (FPL + NT - 1) / NT;  // halo-1 plane nodes per thread

// This thread's nodes of the halo-2 input plane, resolved once for the whole z march: the source
// column x + nx y after the ghost rule along x and y, its sign for u, and the shared-memory slot.
struct PlaneSrc {
  long long off[NLD];
  int slot[NLD];  // lj * RX + li, or -1
  int sgn[NLD];   // 0: no source (beyond the ghost layer), else +-1
};

__device__ __forceinline__ PlaneSrc plane_src(const Geo& g, int x0, int y0) {
  PlaneSrc ps;
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    const int q = threadIdx.x + j * NT;
    ps.slot[j] = -1;
    ps.sgn[j] = 0;
    ps.off[j] = 0;
    if (q >= RPL) continue;
    const int li = q % RX, lj = q / RX;
    int gx = x0 - 2 + li, gy = y0 - 2 + lj, sgn = 1;
    ps.slot[j] = q;
    if (ghost_axis(g.bc[0], g.n[0], &gx, &sgn) && ghost_axis(g.bc[1], g.n[1], &gy, &sgn)) {
      ps.sgn[j] = sgn;
      ps.off[j] = gx + (long long)g.n[0] * gy;
    }
  }
  return ps;
}

// Read plane zr of the state (after the ghost rule along z) into registers.
template <typename T>
__device__ __forceinline__ void fetch_plane(const Geo& g, const T* __restrict__ src, const PlaneSrc& ps, int zr,
                                            T (&v)[NLD][4]) {
  int gz = zr, sz = 1;
  const bool okz = ghost_axis(g.bc[2], g.n[2], &gz, &sz);
  const long long N = g.N, zoff = (long long)gz * g.n[0] * g.n[1];
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    const bool ok = okz && ps.sgn[j] != 0;
    const long long n = ps.off[j] + zoff;
    const T sg = T(ps.sgn[j] * sz);
    v[j][0] = ok ? src[n] : T(0);
    v[j][1] = ok ? sg * src[N + n] : T(0);
    v[j][2] = ok ? sg * src[2 * N + n] : T(0);
    v[j][3] = ok ? sg * src[3 * N + n] : T(0);
  }
}

template <typename T>
__device__ __forceinline__ void store_plane(T (*dst)[RY][RX], const PlaneSrc& ps, const T (&v)[NLD][4]) {
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    if (ps.slot[j] < 0) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) (&dst[c][0][0])[ps.slot[j]] = v[j][c];
  }
}

// f_i^eq of one halo-1 node (ci, cj) of plane zr from the input planes zr - 1, zr, zr + 1.
// The velocity gradient sums the corner columns along z first. The eight corner values share
// their terms: with alpha = w3 (a + Qxx + Qyy + Qzz) and the w3-scaled b, Q, the corners of one z
// sign are (alpha +- Bz + Qxy) +- (X + Y) and (alpha +- Bz - Qxy) +- (X - Y), X = Bx +- Qxz,
// Y = By +- Qyz.
template <typename T>
__device__ __forceinline__ void feq_node(const Geo& g, Fwd3Smem<T>& s, int sm, int s0, int sp, int ci, int cj) {
  const int li = ci + 1, lj = cj + 1;
  const T A2 = two_a<T>(g), tenth = T(0.1);
  const T p = s.raw[s0][0][lj][li];
  T u[3], G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T(*U0)[RX] = s.raw[s0][1 + a];
    const T(*Um)[RX] = s.raw[sm][1 + a];
    const T(*Up)[RX] = s.raw[sp][1 + a];
    u[a] = U0[lj][li];
    const T pp = Up[lj + 1][li + 1], pm = Up[lj - 1][li + 1], mp = Up[lj + 1][li - 1], mm = Up[lj - 1][li - 1];
    const T qp = Um[lj + 1][li + 1], qm = Um[lj - 1][li + 1], np_ = Um[lj + 1][li - 1], nm = Um[lj - 1][li - 1];
    const T Spp = pp + qp, Spm = pm + qm, Smp = mp + np_, Smm = mm + nm;
    const T gx = (U0[lj][li + 1] - U0[lj][li - 1]) + (Spp + Spm) - (Smp + Smm);
    const T gy = (U0[lj + 1][li] - U0[lj - 1][li]) + (Spp + Smp) - (Spm + Smm);
    const T gz = (Up[lj][li] - Um[lj][li]) + ((pp - qp) + (pm - qm)) + ((mp - np_) + (mm - nm));
    G[a][0] = gx * tenth;
    G[a][1] = gy * tenth;
    G[a][2] = gz * tenth;
  }
  const T w0 = T(2.0 / 9.0), w1 = T(1.0 / 9.0), w3 = T(1.0 / 72.0);
  const T a0 = T(3) * p - T(1.5) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const T qxx = T(4.5) * u[0] * u[0] + A2 * G[0][0];
  const T qyy = T(4.5) * u[1] * u[1] + A2 * G[1][1];
  const T qzz = T(4.5) * u[2] * u[2] + A2 * G[2][2];
  const T qxy = T(9) * u[0] * u[1] + A2 * (G[0][1] + G[1][0]);
  const T qxz = T(9) * u[0] * u[2] + A2 * (G[0][2] + G[2][0]);
  const T qyz = T(9) * u[1] * u[2] + A2 * (G[1][2] + G[2][1]);
  s.f[0][cj][ci] = w0 * a0;
  const T bx1 = T(3) * w1 * u[0], by1 = T(3) * w1 * u[1], bz1 = T(3) * w1 * u[2];
  const T tx = w1 * (a0 + qxx), ty = w1 * (a0 + qyy), tz = w1 * (a0 + qzz);
  s.f[1][cj][ci] = tx + bx1;
  s.f[2][cj][ci] = tx - bx1;
  s.f[3][cj][ci] = ty + by1;
  s.f[4][cj][ci] = ty - by1;
  s.f[5][cj][ci] = tz + bz1;
  s.f[6][cj][ci] = tz - bz1;
  const T al = w3 * (a0 + qxx + qyy + qzz);
  const T Bx = T(3) * w3 * u[0], By = T(3) * w3 * u[1], Bz = T(3) * w3 * u[2];
  const T Qxy = w3 * qxy, Qxz = w3 * qxz, Qyz = w3 * qyz;
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // h = 0: c_z = +1 (k = 0..3), h = 1: c_z = -1 (k = 4..7)
    const T e = h ? al - Bz : al + Bz;
    const T X = h ? Bx - Qxz : Bx + Qxz, Y = h ? By - Qyz : By + Qyz;
    const T t1 = e + Qxy, t2 = e - Qxy, P = X + Y, M = X - Y;
    s.f[7 + 4 * h + 0][cj][ci] = t1 + P;  // (+, +)
    s.f[7 + 4 * h + 1][cj][ci] = t2 - M;  // (-, +)
    s.f[7 + 4 * h + 2][cj][ci] = t2 + M;  // (+, -)
    s.f[7 + 4 * h + 3][cj][ci] = t1 - P;  // (-, -)
  }
}

// Open x planes on one completed plane (rows of this tile).
template <typename T>
__device__ __forceinline__ void x_planes(const Geo& g, T (*O)[TY][TX], int gx, int tx, int ty) {
  const int nx = g.n[0];
  if (g.bc[0] == BC_PERIODIC || !(gx == 0 || gx == nx - 1)) return;
  const bool inlet = gx == 0;
  const int tin = inlet ? tx + 1 : tx - 1;
  if (g.bc[0] == BC_INFLOW_OUTFLOW) {
    if (inlet) {
      O[0][ty][tx] = O[0][ty][tin];
      O[1][ty][tx] = T(g.u_in);
      O[2][ty][tx] = T(0);
      O[3][ty][tx] = T(0);
    } else {
      O[0][ty][tx] = T(0);
      for (int c = 1; c < 4; ++c) O[c][ty][tx] = O[c][ty][tin];
    }
  } else {
    O[0][ty][tx] = inlet ? T(g.dp) : T(0);
    for (int c = 1; c < 4; ++c) O[c][ty][tx] = O[c][ty][tin];
  }
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_stencil3d(Geo g, Slots<T> S, const Ctrl* __restrict__ ctrl, int di) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  Fwd3Smem<T>& s = *reinterpret_cast<Fwd3Smem<T>*>(smem_bytes);
  const int t = ctrl->t0 + di, base = ctrl->base;
  const T* __restrict__ src = slot_ptr(S, t - 1, base);
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool ingrid = gx < nx && gy < ny;
  const bool zwall = g.bc[2] == BC_WALL;
  int z0, z1;
  chunk_range(nz, &z0, &z1);
  // a tile whose outputs need no boundary phase writes them straight from registers
  const bool plain = (g.bc[0] == BC_PERIODIC || (x0 >= 1 && x0 + TX <= nx - 1)) &&
                     (g.bc[1] != BC_WALL || (y0 >= 1 && y0 + TY <= ny - 1)) && (!zwall || (z0 >= 2 && z1 <= nz - 2));
  const int ci = tx + 1, cj = ty + 1;
  int fci[NFQ], fcj[NFQ];
#pragma unroll
  for (int j = 0; j < NFQ; ++j) {
    const int q = threadIdx.x + j * NT;
    fci[j] = q < FPL ? q % FX : -1;
    fcj[j] = q < FPL ? q / FX : -1;
  }
  const PlaneSrc ps = plane_src(g, x0, y0);
  // acc[d]: output plane zr - 1 + d, (sum f, sum c_x f, sum c_y f, sum c_z f)
  T acc[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[d][c] = T(0);

  T v[NLD][4];
  for (int zl = z0 - 2; zl <= z0; ++zl) {
    fetch_plane(g, src, ps, zl, v);
    store_plane(s.raw[ring(zl, z0)], ps, v);
  }
  fetch_plane(g, src, ps, z0 + 1, v);  // in flight while plane z0 - 1 is worked on
  for (int zr = z0 - 1; zr <= z1; ++zr) {
    __syncthreads();  // planes zr - 1 .. zr + 1 are in the ring; the previous f plane is consumed
    {
      const int sm = ring(zr - 1, z0), s0 = ring(zr, z0), sp = ring(zr + 1, z0);
#pragma unroll
      for (int j = 0; j < NFQ; ++j)
        if (fci[j] >= 0) feq_node(g, s, sm, s0, sp, fci[j], fcj[j]);
    }
    __syncthreads();
    if (zr + 2 <= z1 + 1) {
      store_plane(s.raw[ring(zr + 2, z0)], ps, v);  // replaces plane zr - 1, no longer read
      if (zr + 3 <= z1 + 1) fetch_plane(g, src, ps, zr + 3, v);
    }
    {
      // c_z = 0: rest and the four in-plane axis vectors -> output zr
      const T f0 = s.f[0][cj][ci], f1 = s.f[1][cj][ci - 1], f2 = s.f[2][cj][ci + 1];
      const T f3 = s.f[3][cj - 1][ci], f4 = s.f[4][cj + 1][ci];
      acc[1][0] += f0 + f1 + f2 + f3 + f4;
      acc[1][1] += f1 - f2;
      acc[1][2] += f3 - f4;
      // +z axis -> output zr + 1, -z axis -> output zr - 1
      const T f5 = s.f[5][cj][ci], f6 = s.f[6][cj][ci];
      acc[2][0] += f5;
      acc[2][3] += f5;
      acc[0][0] += f6;
      acc[0][3] -= f6;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int sx = csx(k), sy = csy(k), sz = csz(k);
        const T vv = s.f[7 + k][cj - sy][ci - sx];
        const int d = sz > 0 ? 2 : 0;
        acc[d][0] += vv;
        acc[d][1] += T(sx) * vv;
        acc[d][2] += T(sy) * vv;
        acc[d][3] += T(sz) * vv;
      }
    }
    const int zo = zr - 1;
    if (zo >= z0) {  // output plane zo is complete
      if (plain) {
        if (ingrid) {
          const long long n = gx + (long long)nx * (gy + (long long)ny * zo);
          dst[n] = acc[0][0] * T(1.0 / 3.0);
          dst[N + n] = acc[0][1];
          dst[2 * N + n] = acc[0][2];
          dst[3 * N + n] = acc[0][3];
        }
      } else {
        s.out[0][ty][tx] = acc[0][0] * T(1.0 / 3.0);
        s.out[1][ty][tx] = acc[0][1];
        s.out[2][ty][tx] = acc[0][2];
        s.out[3][ty][tx] = acc[0][3];
        __syncthreads();
        // y walls, for nodes with x and z interior
        if (ingrid && g.bc[1] == BC_WALL && (gy == 0 || gy == ny - 1) && interior_axis(g.bc[0], nx, gx) &&
            interior_axis(g.bc[2], nz, zo)) {
          const int tin = (gy == 0) ? ty + 1 : ty - 1;
          s.out[0][ty][tx] = s.out[0][tin][tx];
          s.out[1][ty][tx] = s.out[2][ty][tx] = s.out[3][ty][tx] = T(0);
        }
        __syncthreads();
        // z walls, for nodes with x interior (own column only)
        const T pp = s.out[0][ty][tx];
        if (zwall && interior_axis(g.bc[0], nx, gx)) {
          if (zo == nz - 1) {
            s.out[0][ty][tx] = s.prevp[ty][tx];
            s.out[1][ty][tx] = s.out[2][ty][tx] = s.out[3][ty][tx] = T(0);
          }
          if (zo == 1) {
            s.out0[0][ty][tx] = pp;
            s.out0[1][ty][tx] = s.out0[2][ty][tx] = s.out0[3][ty][tx] = T(0);
          }
        }
        s.prevp[ty][tx] = pp;
        __syncthreads();
        if (ingrid) {
          x_planes(g, s.out, gx, tx, ty);
          if (zwall && zo == 1) x_planes(g, s.out0, gx, tx, ty);
          const long long n = gx + (long long)nx * gy;
          if (!(zwall && zo == 0)) {
            const long long nz_off = (long long)zo * nx * ny;
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c * N + nz_off + n] = s.out[c][ty][tx];
          }
          if (zwall && zo == 1) {
#pragma unroll
            for (int c = 0; c < 4; ++c) dst[c * N + n] = s.out0[c][ty][tx];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[0][c] = acc[1][c];
      acc[1][c] = acc[2][c];
      acc[2][c] = T(0);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Transpose. The adjoint of (p*, u*) is first routed back through the boundary rules
// (lam_star3), giving zero on every non-interior node. Then with
// fbar_i(y) = 1/3 lam_p*(y + c_i) + c_i . lam_u*(y + c_i) and the moments
//   P = sum_i w_i fbar_i, U = sum_i w_i c_i fbar_i, S = sum_i w_i c_i c_i fbar_i,
//   lam_p(z) = 3P,  lam_u(z) = 3U + 9 S u - 3 u P + (2A/10) sum_{(y,j): nbr(y,c_j) = z} sgn S(y) c_j
// where the last sum is the transpose of the velocity-gradient stencil with its ghost rule.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ldl(const T* L, long long N, int c, int nx, int ny, int x, int y, int z) {
  return L[c * N + x + (long long)nx * (y + (long long)ny * z)];
}

// Adjoint of (p*, u*) seen by interior node (x, y, z) once the boundary rules are reversed: p is
// copied (through the y-wall, z-wall and inflow phases) into every node of the product of
// {x, inlet if x == 1} x {y, wall row if y is next to it} x {z, wall plane likewise}; u is copied
// only by the outflow / pressure planes from x = nx - 2 and (pressure) x = 1.
template <typename T>
__device__ __forceinline__ void lam_star3(const Geo& g, const T* L, int x, int y, int z, T* v) {
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  if (!interior_axis(g.bc[0], nx, x) || !interior_axis(g.bc[1], ny, y) || !interior_axis(g.bc[2], nz, z)) {
    v[0] = v[1] = v[2] = v[3] = T(0);
    return;
  }
  const int bx = g.bc[0];
  int xs[2] = {x, 0}, ys[2] = {y, 0}, zs[2] = {z, 0};
  const int nxs = (bx == BC_INFLOW_OUTFLOW && x == 1) ? 2 : 1;
  int nys = 1, nzs = 1;
  if (g.bc[1] == BC_WALL && (y == 1 || y == ny - 2)) {
    ys[1] = (y == 1) ? 0 : ny - 1;
    nys = 2;
  }
  if (g.bc[2] == BC_WALL && (z == 1 || z == nz - 2)) {
    zs[1] = (z == 1) ? 0 : nz - 1;
    nzs = 2;
  }
  T p = T(0);
  for (int c = 0; c < nzs; ++c)
    for (int b = 0; b < nys; ++b)
      for (int a = 0; a < nxs; ++a) p += ldl(L, N, 0, nx, ny, xs[a], ys[b], zs[c]);
  v[0] = p;
  for (int c = 1; c < 4; ++c) {
    T u = ldl(L, N, c, nx, ny, x, y, z);
    if ((bx == BC_INFLOW_OUTFLOW || bx == BC_PRESSURE) && x == nx - 2) u += ldl(L, N, c, nx, ny, nx - 1, y, z);
    if (bx == BC_PRESSURE && x == 1) u += ldl(L, N, c, nx, ny, 0, y, z);
    v[c] = u;
  }
}

// This thread's nodes of the adjoint's halo-2 input plane: the (wrapped) column and whether it is
// on the grid, resolved once for the whole z march.
struct AdjSrc {
  int gx[NLD], gy[NLD];
  int slot[NLD];  // lj * RX + li, or -1
  bool ok[NLD];
};

__device__ __forceinline__ AdjSrc adj_src(const Geo& g, int x0, int y0) {
  AdjSrc as;
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    const int q = threadIdx.x + j * NT;
    as.slot[j] = q < RPL ? q : -1;
    int gx = x0 - 2 + q % RX, gy = y0 - 2 + q / RX;
    bool ok = q < RPL;
    if (g.bc[0] == BC_PERIODIC) gx = wrapi(gx, g.n[0]);
    else if (gx < 0 || gx >= g.n[0]) ok = false;
    if (g.bc[1] == BC_PERIODIC) gy = wrapi(gy, g.n[1]);
    else if (gy < 0 || gy >= g.n[1]) ok = false;
    as.gx[j] = gx;
    as.gy[j] = gy;
    as.ok[j] = ok;
  }
  return as;
}

template <typename T>
__device__ __forceinline__ void store_raw(T (*dst)[RY][RX], const AdjSrc& as, const T (&v)[NLD][4]) {
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
    if (as.slot[j] < 0) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) (&dst[c][0][0])[as.slot[j]] = v[j][c];
  }
}

// Plane zr of the adjoint with the boundary rules reversed (lam_star3), into registers. In a
// column whose halo stays two nodes away from every non-periodic boundary (direct) and on a plane
// likewise, the rules are the identity and the values are read directly.
template <typename T>
__device__ __forceinline__ void fetch_adj_plane(const Geo& g, const T* __restrict__ L, const AdjSrc& as, bool direct,
                                                int zr, T (&v)[NLD][4]) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  int gz = zr;
  bool okz = true;
  if (g.bc[2] == BC_PERIODIC) gz = wrapi(gz, nz);
  else if (gz < 0 || gz >= nz) okz = false;
  const bool dz = g.bc[2] == BC_PERIODIC || (zr >= 2 && zr <= nz - 3);
  const long long N = g.N;
#pragma unroll
  for (int j = 0; j < NLD; ++j) {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[j][c] = T(0);
    if (!as.ok[j] || !okz) continue;
    if (direct && dz) {
      const long long n = as.gx[j] + (long long)nx * (as.gy[j] + (long long)ny * gz);
#pragma unroll
      for (int c = 0; c < 4; ++c) v[j][c] = L[c * N + n];
    } else {
      lam_star3(g, L, as.gx[j], as.gy[j], gz, v[j]);
    }
  }
}

// Moments of plane zr at the halo-1 node (ci, cj); zero on nodes off the grid (non-periodic axes),
// where the gradient-stencil transpose reads them as absent (off: the node is off the grid).
template <typename T>
__device__ __forceinline__ void moment_node(Adj3Smem<T>& s, int sm, int s0, int sp, int ci, int cj, bool off) {
  const T third = T(1.0 / 3.0), w0 = T(2.0 / 9.0), w1 = T(1.0 / 9.0), w3 = T(1.0 / 72.0);
  if (off) {
#pragma unroll
    for (int c = 0; c < 10; ++c) s.m[c][cj][ci] = T(0);
    return;
  }
  const int li = ci + 1, lj = cj + 1;
  const T(*P0)[RX] = s.raw[s0][0];
  const T fb0 = third * P0[lj][li];
  const T fpx = third * P0[lj][li + 1] + s.raw[s0][1][lj][li + 1];
  const T fmx = third * P0[lj][li - 1] - s.raw[s0][1][lj][li - 1];
  const T fpy = third * P0[lj + 1][li] + s.raw[s0][2][lj + 1][li];
  const T fmy = third * P0[lj - 1][li] - s.raw[s0][2][lj - 1][li];
  const T fpz = third * s.raw[sp][0][lj][li] + s.raw[sp][3][lj][li];
  const T fmz = third * s.raw[sm][0][lj][li] - s.raw[sm][3][lj][li];
  T cP = T(0), cX = T(0), cY = T(0), cZ = T(0), cXY = T(0), cXZ = T(0), cYZ = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int sx = csx(k), sy = csy(k), sz = csz(k);
    const int pl = sz > 0 ? sp : sm;
    const int yy = lj + sy, xx = li + sx;
    const T fb = third * s.raw[pl][0][yy][xx] + T(sx) * s.raw[pl][1][yy][xx] + T(sy) * s.raw[pl][2][yy][xx] +
                 T(sz) * s.raw[pl][3][yy][xx];
    cP += fb;
    cX += T(sx) * fb;
    cY += T(sy) * fb;
    cZ += T(sz) * fb;
    cXY += T(sx * sy) * fb;
    cXZ += T(sx * sz) * fb;
    cYZ += T(sy * sz) * fb;
  }
  s.m[0][cj][ci] = w0 * fb0 + w1 * (fpx + fmx + fpy + fmy + fpz + fmz) + w3 * cP;
  s.m[1][cj][ci] = w1 * (fpx - fmx) + w3 * cX;
  s.m[2][cj][ci] = w1 * (fpy - fmy) + w3 * cY;
  s.m[3][cj][ci] = w1 * (fpz - fmz) + w3 * cZ;
  s.m[4][cj][ci] = w1 * (fpx + fmx) + w3 * cP;
  s.m[5][cj][ci] = w1 * (fpy + fmy) + w3 * cP;
  s.m[6][cj][ci] = w1 * (fpz + fmz) + w3 * cP;
  s.m[7][cj][ci] = w3 * cXY;
  s.m[8][cj][ci] = w3 * cXZ;
  s.m[9][cj][ci] = w3 * cYZ;
}

// S_ab of the moment plane at (cj, ci), b-th column (symmetric).
template <typename T>
__device__ __forceinline__ T Sab(const Adj3Smem<T>& s, int a, int b, int cj, int ci) {
  const int idx = (a == b) ? 4 + a : (a + b == 1 ? 7 : (a + b == 2 ? 8 : 9));
  return s.m[idx][cj][ci];
}

// Moment S_ab at (cj, ci) of the moment plane, zero outside the plane's halo (those positions are
// off the grid whenever they are read).
template <typename T>
__device__ __forceinline__ T Sab_or0(const Adj3Smem<T>& s, int a, int b, int cj, int ci) {
  return (cj >= 0 && cj < FY && ci >= 0 && ci < FX) ? Sab(s, a, b, cj, ci) : T(0);
}

// h_a = sum_j c_j . S_a(z - c_j) at position (cj, ci) split by the plane offset of c_j:
// hv[0] (c_z = -1, output plane zr - 1), hv[1] (c_z = 0, plane zr), hv[2] (c_z = +1, plane zr + 1).
template <typename T, bool CHECK>
__device__ __forceinline__ void h_plane(const Adj3Smem<T>& s, int cj, int ci, T (&hv)[3][3]) {
  auto S = [&](int a, int b, int j, int i) { return CHECK ? Sab_or0(s, a, b, j, i) : Sab(s, a, b, j, i); };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T v1 = S(a, 0, cj, ci - 1) - S(a, 0, cj, ci + 1) + S(a, 1, cj - 1, ci) - S(a, 1, cj + 1, ci);
    T v2 = S(a, 2, cj, ci), v0 = -S(a, 2, cj, ci);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int sx = csx(k), sy = csy(k), sz = csz(k);
      const int yy = cj - sy, xx = ci - sx;
      const T h = T(sx) * S(a, 0, yy, xx) + T(sy) * S(a, 1, yy, xx) + T(sz) * S(a, 2, yy, xx);
      if (sz > 0) v2 += h;
      else v0 += h;
    }
    hv[0][a] = v0;
    hv[1][a] = v1;
    hv[2][a] = v2;
  }
}

// hv += sgn * h at a ghost position (cj, ci)
template <typename T>
__device__ __forceinline__ void h_add(const Adj3Smem<T>& s, int cj, int ci, T sgn, T (&hv)[3][3]) {
  T g[3][3];
  h_plane<T, true>(s, cj, ci, g);
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int a = 0; a < 3; ++a) hv[d][a] += sgn * g[d][a];
}

template <typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 2 : 1) k_stencil3d_adj(Geo g, Slots<T> S, T* Lb, long long lstride,
                                                      const Ctrl* __restrict__ ctrl, int di) {
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  Adj3Smem<T>& s = *reinterpret_cast<Adj3Smem<T>*>(smem_bytes);
  const int t = ctrl->t0 - di, base = ctrl->base;
  const T* __restrict__ Lcur = Lb + (long long)(t & 1) * lstride;
  T* __restrict__ Lnext = Lb + (long long)((t - 1) & 1) * lstride;
  const T* __restrict__ st = slot_ptr(S, t - 1, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool ingrid = gx < nx && gy < ny;
  int z0, z1;
  chunk_range(nz, &z0, &z1);
  const int ci = tx + 1, cj = ty + 1;
  const T kA = two_a<T>(g) * T(0.1);
  T acc[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[d][c] = T(0);

  int fci[NFQ], fcj[NFQ];
  bool foffxy[NFQ];
#pragma unroll
  for (int j = 0; j < NFQ; ++j) {
    const int q = threadIdx.x + j * NT;
    fci[j] = q < FPL ? q % FX : -1;
    fcj[j] = q < FPL ? q / FX : -1;
    const int x = x0 - 1 + fci[j], y = y0 - 1 + fcj[j];
    foffxy[j] = (g.bc[0] != BC_PERIODIC && (x < 0 || x >= nx)) || (g.bc[1] != BC_PERIODIC && (y < 0 || y >= ny));
  }
  const AdjSrc as = adj_src(g, x0, y0);
  // every halo node of the column two nodes clear of the non-periodic boundaries
  const bool direct = (g.bc[0] == BC_PERIODIC || (x0 >= 4 && x0 + TX + 4 <= nx)) &&
                      (g.bc[1] == BC_PERIODIC || (y0 >= 4 && y0 + TY + 4 <= ny));
  T v[NLD][4];
  for (int zl = z0 - 2; zl <= z0; ++zl) {
    fetch_adj_plane(g, Lcur, as, direct, zl, v);
    store_raw(s.raw[ring(zl, z0)], as, v);
  }
  fetch_adj_plane(g, Lcur, as, direct, z0 + 1, v);
  for (int zr = z0 - 1; zr <= z1; ++zr) {
    __syncthreads();  // planes zr - 1 .. zr + 1 are in the ring; the previous moment plane is consumed
    {
      const int sm = ring(zr - 1, z0), s0 = ring(zr, z0), sp = ring(zr + 1, z0);
      const bool zoff = g.bc[2] != BC_PERIODIC && (zr < 0 || zr >= nz);
#pragma unroll
      for (int j = 0; j < NFQ; ++j)
        if (fci[j] >= 0) moment_node(s, sm, s0, sp, fci[j], fcj[j], zoff || foffxy[j]);
    }
    __syncthreads();
    if (zr + 2 <= z1 + 1) {
      store_raw(s.raw[ring(zr + 2, z0)], as, v);  // replaces plane zr - 1, no longer read
      if (zr + 3 <= z1 + 1) fetch_adj_plane(g, Lcur, as, direct, zr + 3, v);
    }
    // local part of output zr
    if (ingrid && zr >= z0 && zr < z1) {
      const long long n = gx + (long long)nx * (gy + (long long)ny * zr);
      const T u[3] = {st[N + n], st[2 * N + n], st[3 * N + n]};
      const T P = s.m[0][cj][ci];
      acc[1][0] += T(3) * P;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T su = T(0);
#pragma unroll
        for (int b = 0; b < 3; ++b) su += Sab(s, a, b, cj, ci) * u[b];
        acc[1][1 + a] += T(3) * s.m[1 + a][cj][ci] + T(9) * su - T(3) * u[a] * P;
      }
    }
    // velocity-gradient transpose: moment plane zr feeds outputs zr - 1, zr, zr + 1 at this
    // node, plus the ghost positions that the gradient stencil mapped onto it (open x planes copy:
    // sign +1; walls reflect: sign -1). S is zero off the grid, so one formula serves all.
    if (ingrid) {
      T hv[3][3];
      h_plane<T, false>(s, cj, ci, hv);
      const bool gx_lo = g.bc[0] != BC_PERIODIC && gx == 0, gx_hi = g.bc[0] != BC_PERIODIC && gx == nx - 1;
      const bool gy_lo = g.bc[1] == BC_WALL && gy == 1, gy_hi = g.bc[1] == BC_WALL && gy == ny - 2;
      if (gx_lo || gx_hi || gy_lo || gy_hi) {
        // ghost offsets (in the moment plane) and signs along x and y
        const int ox = gx_lo ? -1 : (gx_hi ? 1 : 0);
        const int oy = gy_lo ? -2 : (gy_hi ? 2 : 0);
        if (ox != 0) h_add<T>(s, cj, ci + ox, T(1), hv);
        if (oy != 0) h_add<T>(s, cj + oy, ci, T(-1), hv);
        if (ox != 0 && oy != 0) h_add<T>(s, cj + oy, ci + ox, T(-1), hv);
      }
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[d][1 + a] += kA * hv[d][a];
    }
    // wall planes: ghost plane -1 (complete once moment plane 0 is in) reflects onto plane 1,
    // ghost plane nz (complete once moment plane nz - 1 is in) onto plane nz - 2
    if (g.bc[2] == BC_WALL && zr == 0) {
#pragma unroll
      for (int a = 1; a < 4; ++a) acc[2][a] -= acc[0][a];
    }
    if (g.bc[2] == BC_WALL && zr == nz - 1) {
#pragma unroll
      for (int a = 1; a < 4; ++a) acc[0][a] -= acc[2][a];
    }
    const int zo = zr - 1;
    if (ingrid && zo >= z0) {
      const long long n = gx + (long long)nx * (gy + (long long)ny * zo);
#pragma unroll
      for (int c = 0; c < 4; ++c) Lnext[c * N + n] = acc[0][c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[0][c] = acc[1][c];
      acc[1][c] = acc[2][c];
      acc[2][c] = T(0);
    }
  }
}

// Number of z chunks: the count that best fills whole waves of resident CTAs (ctas_per_sm on each
// of the 152 SMs) weighed against the two extra planes of f^eq each chunk computes; every chunk
// holds at least four planes.
int z_chunks(const Geo& g, int ctas_per_sm) {
  const int tiles = ((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY);
  const int slots = 152 * ctas_per_sm;
  const int cmax = g.n[2] / 4 < 1 ? 1 : g.n[2] / 4;
  int best = 1;
  double best_eff = 0.0;
  for (int c = 1; c <= cmax; ++c) {
    const long long total = (long long)tiles * c;
    const long long waves = (total + slots - 1) / slots;
    const double planes = (double)g.n[2] / c;
    const double eff = (double)total / (double)(waves * slots) * planes / (planes + 2.0);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = c;
    }
  }
  return best;
}

}  // namespace

template <typename T>
void prepare_stencil3d() {
  cudaFuncSetAttribute(k_stencil3d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Fwd3Smem<T>));
  cudaFuncSetAttribute(k_stencil3d_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Adj3Smem<T>));
  if (sizeof(T) == 4) prepare_stencil3d_q();
}

template <typename T>
void launch_stencil3d_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, int di, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (launch_stencil3d_q_fwd(g, S, ctrl, di, st)) return;
  }
  const dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, z_chunks(g, sizeof(T) == 4 ? 2 : 1));
  launch(k_stencil3d<T>, grid, NT, sizeof(Fwd3Smem<T>), st, g, S, ctrl, di);
}

template <typename T>
void launch_stencil3d_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, const Ctrl* ctrl, int di,
                          cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (launch_stencil3d_q_adj(g, S, Lb, lstride, ctrl, di, st)) return;
  }
  const dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, z_chunks(g, sizeof(T) == 4 ? 2 : 1));
  launch(k_stencil3d_adj<T>, grid, NT, sizeof(Adj3Smem<T>), st, g, S, Lb, lstride, ctrl, di);
}

template void prepare_stencil3d<float>();
template void prepare_stencil3d<double>();
template void launch_stencil3d_fwd<float>(const Geo&, const Slots<float>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil3d_fwd<double>(const Geo&, const Slots<double>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil3d_adj<float>(const Geo&, const Slots<float>&, float*, long long, const Ctrl*, int,
                                          cudaStream_t);
template void launch_stencil3d_adj<double>(const Geo&, const Slots<double>&, double*, long long, const Ctrl*, int,
                                           cudaStream_t);

}  // namespace lks
