// LKS predictor (Sec. 2.2) and its exact transpose on D2Q9.
//
// Forward, per cell x (tau = 1 so f_i* is f_i^eq streamed from x - c_i):
//   f_i^eq(y) = w_i (3p + 3c.u + 9/2 (c.u)^2 - 3/2 |u|^2 + 2A sum_ab G_ab c_a c_b),
//   G_ab = d_b u_a by the isotropic central stencil sum_j c_jb u_a(y + c_j) / 6,
//   p*(x) = 1/3 sum_i f_i^eq(x - c_i),  u*(x) = sum_i c_i f_i^eq(x - c_i).
// Boundary values are prescribed directly (Sec. 2.2): walls in y (u = 0, p from the inner row) for
// x-interior nodes, then open x planes (inflow u = u_in and p copied inward, outflow p = 0 and u
// copied inward; pressure-driven p = dp / 0 and u copied). Ghosts for the gradient: open planes
// copy the boundary node, walls reflect u with a sign flip.
//
// GB300 form: each warp streams a strip of rows through 64 consecutive columns, two per lane
// (lane L holds columns x0 - 2 + 2L and x0 - 1 + 2L, loaded as one vector where the pair is on the
// grid), and writes the W <= 60 columns of lanes 1 .. W/2. Neighbour columns come from warp
// shuffles (one per neighbouring lane and value, shared by the pair), so there is no shared
// memory and no block barrier. Per row the warp loads the state once, forms the velocity-gradient
// row sums, the nine f_i^eq of the row above the newest, and scatters them into three rolling row
// accumulators (outputs y-1, y, y+1).
//
// Algorithmic traffic per cell: read p, u (3 values), write p*, u* (3 values): 24 B in FP32;
// the transpose reads the adjoint (3) and u(t-1) (2) and writes 3 values: 32 B.
#include "lks_kernels.h"
#include "lks_stencil_common.cuh"

namespace lks {

namespace {

constexpr int SW = kStripWarps;  // warps per CTA (independent strips)

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ T shup(T v) {  // value of lane L - 1
  return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shdn(T v) {  // value of lane L + 1
  return __shfl_down_sync(0xffffffffu, v, 1);
}

// Asynchronous global -> shared copies (cp.async): each lane stages its own values of a row into
// a per-warp ring of shared-memory row slots, several rows ahead of their use, so the bytes in
// flight do not depend on registers. A copy with valid = false fills zeros.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_u32(sdst)), "l"(gsrc), "n"(BYTES),
               "r"(valid ? BYTES : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Rows staged ahead per warp and the shared memory they take per CTA.
template <typename T>
struct Ring {
  static constexpr int rows = sizeof(T) == 4 ? 8 : 4;
  static constexpr int bytes(int planes) { return SW * rows * planes * 64 * (int)sizeof(T); }
};

// This warp's strip: output columns [x0, x0 + W), rows [y0, y1). False if the warp has no strip.
struct Strip {
  int x0, y0, y1, lane, ca, cb;  // ca, cb = ca + 1: this lane's columns (unwrapped)
  bool out;                      // lane holds output columns
};
__device__ __forceinline__ bool strip_of(const Geo& g, const StripPlan& sp, Strip* st) {
  const int wid = blockIdx.x * SW + (threadIdx.x >> 5);
  if (wid >= sp.ntx * sp.nstrip) return false;
  const int tx = wid % sp.ntx, sy = wid / sp.ntx;
  st->lane = threadIdx.x & 31;
  st->x0 = tx * sp.W;
  st->y0 = (int)(((long long)sy * g.n[1]) / sp.nstrip);
  st->y1 = (int)(((long long)(sy + 1) * g.n[1]) / sp.nstrip);
  st->ca = st->x0 - 2 + 2 * st->lane;
  st->cb = st->ca + 1;
  st->out = st->lane >= 1 && st->lane <= sp.W / 2;
  return true;
}

// A column under the gradient ghost rule.
struct Col {
  int m, sg;
  bool ok;
};
__device__ __forceinline__ Col col_of(const Geo& g, int c) {
  Col k;
  k.m = c;
  k.sg = 1;
  k.ok = ghost_axis(g.bc[0], g.n[0], &k.m, &k.sg);
  return k;
}

__device__ __forceinline__ bool xint_of(const Geo& g, int c) {
  return c >= 0 && c < g.n[0] && interior_axis(g.bc[0], g.n[0], c);
}

// Two columns of three planes (p, u_x, u_y, or the adjoint of those).
template <typename T>
struct Pair3 {
  T pa, pb, xa, xb, ya, yb;
  __device__ __forceinline__ void zero() { pa = pb = xa = xb = ya = yb = T(0); }
};

template <typename T>
__device__ __forceinline__ void ld_pair(const T* base, long long off, T& a, T& b) {
  const typename Vec2<T>::type v = *reinterpret_cast<const typename Vec2<T>::type*>(base + off);
  a = v.x;
  b = v.y;
}
template <typename T>
__device__ __forceinline__ void st_pair(T* base, long long off, T a, T b) {
  typename Vec2<T>::type v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename Vec2<T>::type*>(base + off) = v;
}

// Nine f_i^eq at one node from its state and the gradient row sums (dxu = u(x+1) - u(x-1) summed
// over rows r-2 .. r; sxu = u(x-1) + u(x) + u(x+1) of rows r and r-2), per velocity component.
template <typename T>
struct F9 {
  T f0, f1, f2, f3, f4, f5, f6, f7, f8;
};
template <typename T>
__device__ __forceinline__ F9<T> feq9(T p, T ux, T uy, T dxux, T dxuy, T sxux_up, T sxux_dn, T sxuy_up, T sxuy_dn,
                                      T K) {
  // K = 2A/6 multiplies the raw row sums (the gradient's 1/6 folded in); with ux2 = ux^2 etc.:
  //   a = 3p - 3/2 (ux2 + uy2),  f0 = 4/9 a,
  //   f1,3 = 1/9 (a + 9/2 ux2 + K Gxx) +- ux/3,  f2,4 = 1/9 (a + 9/2 uy2 + K Gyy) +- uy/3,
  //   f5..8 = 1/36 (d +- qxy) + (+-ux +-uy)/12 with d = 3p + 3 (ux2 + uy2) + K (Gxx + Gyy),
  //   qxy = 9 ux uy + K (Gxy + Gyx)
  const T ux2 = ux * ux, uy2 = uy * uy, s2 = ux2 + uy2, p3 = T(3) * p;
  const T kxx = K * dxux, kyy = K * (sxuy_up - sxuy_dn);
  const T kxy = K * ((sxux_up - sxux_dn) + dxuy);
  const T a = fma(T(-1.5), s2, p3);
  const T h1 = T(1.0 / 9.0) * (fma(T(4.5), ux2, a) + kxx), v1 = T(1.0 / 3.0) * ux;
  const T h2 = T(1.0 / 9.0) * (fma(T(4.5), uy2, a) + kyy), v2 = T(1.0 / 3.0) * uy;
  const T d36 = T(1.0 / 36.0) * (fma(T(3), s2, p3) + kxx + kyy);
  const T q36 = T(1.0 / 36.0) * fma(T(9) * ux, uy, kxy);
  const T bx = T(1.0 / 12.0) * ux, by = T(1.0 / 12.0) * uy;
  const T e1 = d36 + q36, e2 = d36 - q36, s1 = bx + by, sm = bx - by;
  F9<T> f;
  f.f0 = T(4.0 / 9.0) * a;
  f.f1 = h1 + v1;
  f.f3 = h1 - v1;
  f.f2 = h2 + v2;
  f.f4 = h2 - v2;
  f.f5 = e1 + s1;
  f.f7 = e1 - s1;
  f.f6 = e2 - sm;
  f.f8 = e2 + sm;
  return f;
}

// Running sums of one output row for the two columns: 3 p*, u*_x, u*_y.
template <typename T>
struct Acc2 {
  T pa, xa, ya, pb, xb, yb;
  __device__ __forceinline__ void zero() { pa = xa = ya = pb = xb = yb = T(0); }
};

// A strip whose 64 columns and rows y0-2 .. y1+1 all lie on the grid, clear of every boundary node
// and of any wrap: it needs neither the ghost rule nor a boundary phase (most strips of a large grid).
__device__ __forceinline__ bool interior_strip(const Geo& g, const StripPlan& sp, const Strip& st) {
  return st.x0 - 2 >= 0 && st.x0 + 62 <= g.n[0] && st.y0 - 2 >= 0 && st.y1 + 1 <= g.n[1] - 1;
}

// One warp's strip of the predictor. LEAN: the strip is interior (interior_strip), so every load
// and store is a vector on the grid and the boundary code is compiled out.
template <typename T, bool VEC, bool LEAN>
__device__ __forceinline__ void fwd_strip(const Geo& g, const Slots<T>& S, const Ctrl* __restrict__ ctrl, int di,
                                          const StripPlan& sp, const Strip& st) {
  const int t = ctrl->t0 + di, base = ctrl->base;
  const T* __restrict__ src = slot_ptr(S, t - 1, base);
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  const Col ka = col_of(g, st.ca), kb = col_of(g, st.cb);
  const bool pairv = LEAN || (VEC && st.ca >= 0 && st.cb < nx);  // the pair is on the grid: one vector
  const bool xia = xint_of(g, st.ca), xib = xint_of(g, st.cb);
  const bool has_xb = !LEAN && g.bc[0] != BC_PERIODIC && (st.x0 == 0 || st.x0 + sp.W >= nx - 1);
  const bool wall_y = !LEAN && g.bc[1] == BC_WALL;
  const T K = two_a<T>(g) * T(1.0 / 6.0);

  // Row r of the state at this lane's two columns, staged through the warp's shared ring.
  constexpr int D = Ring<T>::rows;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * (D * 3 * 64);
  const int ring_r0 = st.y0 - 2;  // first row of the strip's pipeline
  auto slot = [&](int r) { return ring + ((unsigned)(r - ring_r0) % D) * (3 * 64); };
  auto issue = [&](int r) {  // start the copies of row r (nothing past the strip) and close a group
    if (r <= st.y1 + 1) {
      int my = r, sgy = 1;
      const bool rok = LEAN || ghost_axis(g.bc[1], ny, &my, &sgy);
      const long long rb = (long long)nx * (rok ? my : 0);
      T* sl = slot(r) + 2 * st.lane;
      if (pairv) {
#pragma unroll
        for (int c = 0; c < 3; ++c) cp_async<2 * sizeof(T)>(sl + c * 64, src + c * N + rb + st.ca, rok);
      } else {
        const long long na = rb + (ka.ok ? ka.m : 0), nb = rb + (kb.ok ? kb.m : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cp_async<sizeof(T)>(sl + c * 64, src + c * N + na, rok && ka.ok);
          cp_async<sizeof(T)>(sl + c * 64 + 1, src + c * N + nb, rok && kb.ok);
        }
      }
    }
    cp_commit();
  };
  auto load = [&](int r, Pair3<T>& R) {  // the oldest staged row, then refill its slot
    cp_wait<D - 1>();
    int my = r, sgy = 1;
    if (!LEAN) ghost_axis(g.bc[1], ny, &my, &sgy);
    const T* sl = slot(r) + 2 * st.lane;
    const T sa = T(pairv ? sgy : ka.sg * sgy), sb = T(pairv ? sgy : kb.sg * sgy);
    R.pa = sl[0];
    R.pb = sl[1];
    R.xa = sa * sl[64];
    R.xb = sb * sl[65];
    R.ya = sa * sl[128];
    R.yb = sb * sl[129];
  };
  auto refill = [&](int r) { issue(r + D); };  // row r's values are in registers and used
  // gradient row sums of one row for both columns
  struct RowG {
    T dxa, dya, sxa, sya, dxb, dyb, sxb, syb;
  };
  auto rowg = [&](const Pair3<T>& R) {
    const T xl = shup(R.xb), yl = shup(R.yb);  // column ca - 1
    const T xr = shdn(R.xa), yr = shdn(R.ya);  // column cb + 1
    RowG G;
    G.dxa = R.xb - xl;
    G.dya = R.yb - yl;
    G.sxa = xl + R.xa + R.xb;
    G.sya = yl + R.ya + R.yb;
    G.dxb = xr - R.xa;
    G.dyb = yr - R.ya;
    G.sxb = R.xa + R.xb + xr;
    G.syb = R.ya + R.yb + yr;
    return G;
  };

  // One row step for newest row r: prefetch row r+1 into X, form the gradient sums gC of row r
  // (state cC), the f_i^eq of the centre row q = r - 1 (state cB, sums gA gB gC), scatter them
  // into output rows q-1 (oA), q (oB) and q+1 (oC, started here), and emit row r - 2 from oA. The
  // caller rotates the roles of three register sets, so the rolling buffers cost no copies.
  T prevpa = T(0), prevpb = T(0);
  auto step = [&](int r, Acc2<T>& oA, Acc2<T>& oB, Acc2<T>& oC, const RowG& gA, const RowG& gB, RowG& gC,
                  const Pair3<T>& cB, const Pair3<T>& cC, Pair3<T>& X) {
    gC = rowg(cC);
    refill(r);  // row r is in registers and used
    if (r + 1 <= st.y1 + 1) load(r + 1, X);
    {
      const F9<T> A = feq9(cB.pa, cB.xa, cB.ya, gA.dxa + gB.dxa + gC.dxa, gA.dya + gB.dya + gC.dya, gC.sxa, gA.sxa,
                           gC.sya, gA.sya, K);
      const F9<T> B = feq9(cB.pb, cB.xb, cB.yb, gA.dxb + gB.dxb + gC.dxb, gA.dyb + gB.dyb + gC.dyb, gC.sxb, gA.sxb,
                           gC.syb, gA.syb, K);
      // c_x = +1 directions reach the next column, c_x = -1 the previous one
      const T l1 = shup(B.f1), l5 = shup(B.f5), l8 = shup(B.f8);  // from column ca - 1
      const T r3 = shdn(A.f3), r6 = shdn(A.f6), r7 = shdn(A.f7);  // from column cb + 1
      // column ca: left neighbour (l*), right neighbour = column cb (B)
      const T a2 = A.f2 + l5 + B.f6, a0 = A.f4 + l8 + B.f7;
      oC.pa = a2;
      oC.xa = l5 - B.f6;
      oC.ya = a2;
      oB.pa += A.f0 + l1 + B.f3;
      oB.xa += l1 - B.f3;
      oA.pa += a0;
      oA.xa += l8 - B.f7;
      oA.ya -= a0;
      // column cb: left neighbour = column ca (A), right neighbour (r*)
      const T b2 = B.f2 + A.f5 + r6, b0 = B.f4 + A.f8 + r7;
      oC.pb = b2;
      oC.xb = A.f5 - r6;
      oC.yb = b2;
      oB.pb += B.f0 + A.f1 + r3;
      oB.xb += A.f1 - r3;
      oA.pb += b0;
      oA.xb += A.f8 - r7;
      oA.yb -= b0;
    }
    const int y = r - 2;  // output row oA is complete
    if (y < st.y0) return;
    Pair3<T> O;
    O.pa = oA.pa * T(1.0 / 3.0);
    O.pb = oA.pb * T(1.0 / 3.0);
    O.xa = oA.xa;
    O.xb = oA.xb;
    O.ya = oA.ya;
    O.yb = oA.yb;
    // y walls, for x-interior nodes (row 0 is built from row 1 below)
    if (wall_y && y == ny - 1) {
      if (xia) {
        O.pa = prevpa;
        O.xa = O.ya = T(0);
      }
      if (xib) {
        O.pb = prevpb;
        O.xb = O.yb = T(0);
      }
    }
    prevpa = O.pa;
    prevpb = O.pb;
    const bool row0 = wall_y && y == 1;  // emit row 0 too: p from row 1, u = 0
    Pair3<T> Z;
    Z.zero();
    Z.pa = O.pa;
    Z.pb = O.pb;
    if (has_xb) {
      // open x planes, after the wall phase. Column 0 is always a lane's ca (its inner
      // neighbour is cb of the same lane); column nx-1 is a cb (inner neighbour ca) or a ca
      // (inner neighbour: cb of the previous lane).
      const T xl = shup(O.xb), yl = shup(O.yb);
      if (g.bc[0] == BC_INFLOW_OUTFLOW) {
        if (st.ca == 0) {
          O.pa = O.pb;
          O.xa = T(g.u_in);
          O.ya = T(0);
          Z.pa = Z.pb;
          Z.xa = T(g.u_in);
        }
        if (st.cb == nx - 1) {
          O.pb = T(0);
          O.xb = O.xa;
          O.yb = O.ya;
          Z.pb = T(0);
        }
        if (st.ca == nx - 1) {
          O.pa = T(0);
          O.xa = xl;
          O.ya = yl;
          Z.pa = T(0);
        }
      } else {
        if (st.ca == 0) {
          O.pa = T(g.dp);
          O.xa = O.xb;
          O.ya = O.yb;
          Z.pa = T(g.dp);
        }
        if (st.cb == nx - 1) {
          O.pb = T(0);
          O.xb = O.xa;
          O.yb = O.ya;
          Z.pb = T(0);
        }
        if (st.ca == nx - 1) {
          O.pa = T(0);
          O.xa = xl;
          O.ya = yl;
          Z.pa = T(0);
        }
      }
    }
    if (st.out && y < st.y1) {
      const long long rb = (long long)nx * y;
      if (!(wall_y && y == 0)) {
        if (pairv) {
          st_pair(dst, rb + st.ca, O.pa, O.pb);
          st_pair(dst + N, rb + st.ca, O.xa, O.xb);
          st_pair(dst + 2 * N, rb + st.ca, O.ya, O.yb);
        } else {
          if (st.ca < nx) {
            dst[rb + st.ca] = O.pa;
            dst[N + rb + st.ca] = O.xa;
            dst[2 * N + rb + st.ca] = O.ya;
          }
          if (st.cb < nx) {
            dst[rb + st.cb] = O.pb;
            dst[N + rb + st.cb] = O.xb;
            dst[2 * N + rb + st.cb] = O.yb;
          }
        }
      }
      if (row0) {
        if (st.ca < nx) {
          dst[st.ca] = Z.pa;
          dst[N + st.ca] = Z.xa;
          dst[2 * N + st.ca] = Z.ya;
        }
        if (st.cb < nx) {
          dst[st.cb] = Z.pb;
          dst[N + st.cb] = Z.xb;
          dst[2 * N + st.cb] = Z.yb;
        }
      }
    }
  };

  Pair3<T> c0, c1, c2;  // state rows in rotation: centre, newest, prefetched
  RowG g0, g1, g2;      // gradient sums in rotation
  Acc2<T> o0, o1, o2;   // output rows in rotation
  for (int i = 0; i < D; ++i) issue(ring_r0 + i);
  load(st.y0 - 2, c2);
  g0 = rowg(c2);
  refill(st.y0 - 2);
  load(st.y0 - 1, c0);
  g1 = rowg(c0);
  refill(st.y0 - 1);
  load(st.y0, c1);
  o0.zero();
  o1.zero();
  o2.zero();
  for (int r = st.y0; r <= st.y1 + 1; r += 3) {
    step(r, o0, o1, o2, g0, g1, g2, c0, c1, c2);
    if (r + 1 > st.y1 + 1) break;
    step(r + 1, o1, o2, o0, g1, g2, g0, c1, c2, c0);
    if (r + 2 > st.y1 + 1) break;
    step(r + 2, o2, o0, o1, g2, g0, g1, c2, c0, c1);
  }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(SW * 32) k_stencil2d(Geo g, Slots<T> S, const Ctrl* __restrict__ ctrl, int di,
                                                       StripPlan sp) {
  Strip st;
  if (!strip_of(g, sp, &st)) return;  // uniform per warp
  if (VEC && interior_strip(g, sp, st))
    fwd_strip<T, VEC, true>(g, S, ctrl, di, sp, st);
  else
    fwd_strip<T, VEC, false>(g, S, ctrl, di, sp, st);
}

// ---------------------------------------------------------------------------------------------
// Transpose. The adjoint of (p*, u*) is first routed back through the boundary rules
// (lam_star2), which leaves zero on every non-interior node. With
// fbar_i(y) = 1/3 lam_p*(y + c_i) + c_i . lam_u*(y + c_i) and the moments
//   P = sum_i w_i fbar_i, U = sum_i w_i c_i fbar_i, S = sum_i w_i c_i c_i fbar_i,
//   lam_p(z) = 3P,  lam_u(z) = 3U + 9 S u - 3 u P + (2A/6) h(z),  h_a(z) = sum_j c_j . S_a(z - c_j)
// for interior z. Near a non-periodic boundary the gradient stencil read ghost nodes: its
// transpose is h evaluated on the ghost layer as well (S taken as zero off the grid) and folded
// back onto the node each ghost copied (open planes, sign +1) or reflected (walls, sign -1).
// Each warp streams rows as in the forward kernel: the adjoint row is scattered into three
// rolling moment rows, each completed moment row into three rolling output rows.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld_lam(const T* L, long long N, int plane, int x, int y, int nx) {
  return L[plane * N + x + (long long)nx * y];
}

// Adjoint of (p*, u*) seen by interior node (x, y) once the boundary rules are reversed.
template <typename T>
__device__ __forceinline__ void lam_star2(const Geo& g, const T* L, int x, int y, T* lp, T* lux, T* luy) {
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  if (!interior_axis(g.bc[0], nx, x) || !interior_axis(g.bc[1], ny, y)) {
    *lp = *lux = *luy = T(0);
    return;
  }
  T p = ld_lam(L, N, 0, x, y, nx);
  T ux = ld_lam(L, N, 1, x, y, nx);
  T uy = ld_lam(L, N, 2, x, y, nx);
  const int bx = g.bc[0];
  const bool inl = bx == BC_INFLOW_OUTFLOW && x == 1;
  if (inl) p += ld_lam(L, N, 0, 0, y, nx);
  if (g.bc[1] == BC_WALL && (y == 1 || y == ny - 2)) {
    const int yw = (y == 1) ? 0 : ny - 1;
    p += ld_lam(L, N, 0, x, yw, nx);
    if (inl) p += ld_lam(L, N, 0, 0, yw, nx);
  }
  if ((bx == BC_INFLOW_OUTFLOW || bx == BC_PRESSURE) && x == nx - 2) {
    ux += ld_lam(L, N, 1, nx - 1, y, nx);
    uy += ld_lam(L, N, 2, nx - 1, y, nx);
  }
  if (bx == BC_PRESSURE && x == 1) {
    ux += ld_lam(L, N, 1, 0, y, nx);
    uy += ld_lam(L, N, 2, 0, y, nx);
  }
  *lp = p;
  *lux = ux;
  *luy = uy;
}

// Running moment sums of one row and column: P, Ux, Uy, Sxx, Syy, Sxy.
template <typename T>
struct Mom {
  T P, Ux, Uy, Sxx, Syy, Sxy;
  __device__ __forceinline__ void zero() { P = Ux = Uy = Sxx = Syy = Sxy = T(0); }
};

// fbar contributions of one node: g_i = 1/3 lam_p + c_i . lam_u, grouped by c_x.
template <typename T>
struct G9 {
  T g0, g2, g4, g1, g5, g8, g3, g6, g7;
};
template <typename T>
__device__ __forceinline__ G9<T> gbar(T lp, T lx, T ly) {
  const T tp = T(1.0 / 3.0) * lp;
  G9<T> q;
  q.g0 = tp;
  q.g2 = tp + ly;
  q.g4 = tp - ly;
  q.g1 = tp + lx;
  q.g5 = q.g1 + ly;
  q.g8 = q.g1 - ly;
  q.g3 = tp - lx;
  q.g6 = q.g3 + ly;
  q.g7 = q.g3 - ly;
  return q;
}

// Moment rows r-1 (m0), r (m1), r+1 (m2) of one column receive the adjoint row r: its own node
// (o*), the next column's c_x = +1 terms (R*) and the previous column's c_x = -1 terms (L*).
template <typename T>
__device__ __forceinline__ void mom_add(Mom<T>& m0, Mom<T>& m1, Mom<T>& m2, T o0, T o2, T o4, T R1, T R5, T R8,
                                        T L3, T L6, T L7) {
  const T w0 = T(4.0 / 9.0), w1 = T(1.0 / 9.0), w5 = T(1.0 / 36.0);
  m1.P += w0 * o0 + w1 * (R1 + L3);
  m1.Ux += w1 * (R1 - L3);
  m1.Sxx += w1 * (R1 + L3);
  const T s0 = w5 * (R5 + L6), d0 = w5 * (R5 - L6), e0 = w1 * o2 + s0;
  m0.P += e0;
  m0.Ux += d0;
  m0.Uy += e0;
  m0.Sxx += s0;
  m0.Syy += e0;
  m0.Sxy += d0;
  const T s2 = w5 * (R8 + L7), d2 = w5 * (R8 - L7), e2 = w1 * o4 + s2;
  m2.P += e2;
  m2.Ux += d2;
  m2.Uy -= e2;
  m2.Sxx += s2;
  m2.Syy += e2;
  m2.Sxy -= d2;
}

// Output rows q-1 (a0), q (a1), q+1 (a2) of one column receive h from moment row q: own S (o*),
// previous column's (l*) and next column's (r*).
template <typename T>
__device__ __forceinline__ void h_add2(T& a0x, T& a0y, T& a1x, T& a1y, T& a2x, T& a2y, T oxy, T oyy, T lxx, T lxy,
                                       T lyy, T rxx, T rxy, T ryy, T kA) {
  a1x += kA * (lxx - rxx);
  a1y += kA * (lxy - rxy);
  a2x += kA * (oxy + lxx + lxy - rxx + rxy);
  a2y += kA * (oyy + lxy + lyy - rxy + ryy);
  a0x += kA * (-oxy + lxx - lxy - rxx - rxy);
  a0y += kA * (-oyy + lxy - lyy - rxy - ryy);
}

// Boundary routing of the adjoint of (p*, u*) at node (x, y) given its raw values: zero on
// non-interior nodes, plus the terms the boundary phases copied from it (see lam_star2).
template <typename T>
__device__ __forceinline__ void lam_route(const Geo& g, const T* L, int x, int y, T* lp, T* lux, T* luy) {
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  if (!interior_axis(g.bc[0], nx, x) || !interior_axis(g.bc[1], ny, y)) {
    *lp = *lux = *luy = T(0);
    return;
  }
  const int bx = g.bc[0];
  const bool inl = bx == BC_INFLOW_OUTFLOW && x == 1;
  if (inl) *lp += ld_lam(L, N, 0, 0, y, nx);
  if (g.bc[1] == BC_WALL && (y == 1 || y == ny - 2)) {
    const int yw = (y == 1) ? 0 : ny - 1;
    *lp += ld_lam(L, N, 0, x, yw, nx);
    if (inl) *lp += ld_lam(L, N, 0, 0, yw, nx);
  }
  if ((bx == BC_INFLOW_OUTFLOW || bx == BC_PRESSURE) && x == nx - 2) {
    *lux += ld_lam(L, N, 1, nx - 1, y, nx);
    *luy += ld_lam(L, N, 2, nx - 1, y, nx);
  }
  if (bx == BC_PRESSURE && x == 1) {
    *lux += ld_lam(L, N, 1, 0, y, nx);
    *luy += ld_lam(L, N, 2, 0, y, nx);
  }
}

// A strip of the transpose that touches no node within two of a non-periodic boundary (so no
// boundary routing, ghost fold or off-grid node) and no wrap.
__device__ __forceinline__ bool interior_strip_adj(const Geo& g, const Strip& st) {
  const int mx = g.bc[0] == BC_PERIODIC ? 0 : 2, my = g.bc[1] == BC_PERIODIC ? 0 : 2;
  return st.x0 - 2 >= mx && st.x0 + 62 <= g.n[0] - mx && st.y0 - 2 >= my && st.y1 + 1 <= g.n[1] - 1 - my;
}

// One warp's strip of the transpose (LEAN as in fwd_strip, with interior_strip_adj).
template <typename T, bool VEC, bool LEAN>
__device__ __forceinline__ void adj_strip(const Geo& g, const Slots<T>& S, T* Lb, long long lstride,
                                          const Ctrl* __restrict__ ctrl, int di, const StripPlan& sp,
                                          const Strip& st) {
  const int t = ctrl->t0 - di, base = ctrl->base;
  const T* __restrict__ Lcur = Lb + (long long)(t & 1) * lstride;
  T* __restrict__ Lnext = Lb + (long long)((t - 1) & 1) * lstride;
  const T* __restrict__ su = slot_ptr(S, t - 1, base);
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  const bool perx = g.bc[0] == BC_PERIODIC, pery = g.bc[1] == BC_PERIODIC;
  // this lane's columns on the grid (wrapped), or off the grid
  int gxa = st.ca, gxb = st.cb;
  bool cga = true, cgb = true;
  if (!LEAN) {
    if (perx) {
      gxa = wrapi(gxa, nx);
      gxb = wrapi(gxb, nx);
    } else {
      cga = gxa >= 0 && gxa < nx;
      cgb = gxb >= 0 && gxb < nx;
    }
  }
  const bool pairv = LEAN || (VEC && st.ca >= 0 && st.cb < nx);
  const bool has_xb = !LEAN && !perx && (st.x0 == 0 || st.x0 + sp.W >= nx - 1);
  const bool wall_y = !LEAN && g.bc[1] == BC_WALL;
  const T kA = two_a<T>(g) * T(1.0 / 6.0);

  auto row_grid = [&](int r, int* ry) {
    if (LEAN) {
      *ry = r;
      return true;
    }
    if (pery) {
      *ry = wrapi(r, ny);
      return true;
    }
    *ry = r;
    return r >= 0 && r < ny;
  };

  // Rows of the adjoint (3 planes) and of u(t-1) (2 planes) staged through the warp's shared
  // ring; row r's slot is refilled once the next step has read its u.
  constexpr int D = Ring<T>::rows;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * (D * 5 * 64);
  const int ring_r0 = st.y0 - 2;
  auto slot = [&](int r) { return ring + ((unsigned)(r - ring_r0) % D) * (5 * 64) + 2 * st.lane; };
  auto issue = [&](int r) {
    int ry;
    if (r <= st.y1 + 1 && row_grid(r, &ry)) {
      const long long rb = (long long)nx * ry;
      T* sl = slot(r);
      if (pairv) {
#pragma unroll
        for (int c = 0; c < 3; ++c) cp_async<2 * sizeof(T)>(sl + c * 64, Lcur + c * N + rb + st.ca, true);
#pragma unroll
        for (int c = 1; c < 3; ++c) cp_async<2 * sizeof(T)>(sl + (2 + c) * 64, su + c * N + rb + st.ca, true);
      } else {
        const long long na = rb + (cga ? gxa : 0), nb = rb + (cgb ? gxb : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cp_async<sizeof(T)>(sl + c * 64, Lcur + c * N + na, cga);
          cp_async<sizeof(T)>(sl + c * 64 + 1, Lcur + c * N + nb, cgb);
        }
#pragma unroll
        for (int c = 1; c < 3; ++c) {
          cp_async<sizeof(T)>(sl + (2 + c) * 64, su + c * N + na, cga);
          cp_async<sizeof(T)>(sl + (2 + c) * 64 + 1, su + c * N + nb, cgb);
        }
      }
    } else if (r <= st.y1 + 1) {
      T* sl = slot(r);  // off the grid: zeros
#pragma unroll
      for (int c = 0; c < 5; ++c) sl[c * 64] = sl[c * 64 + 1] = T(0);
    }
    cp_commit();
  };
  auto load = [&](int r, Pair3<T>& R) {  // adjoint row r, routed through the boundary rules
    cp_wait<D - 2>();
    const T* sl = slot(r);
    R.pa = sl[0];
    R.pb = sl[1];
    R.xa = sl[64];
    R.xb = sl[65];
    R.ya = sl[128];
    R.yb = sl[129];
    if (!LEAN) {
      int ry;
      if (!row_grid(r, &ry)) {
        R.zero();
      } else {
        if (cga) lam_route(g, Lcur, gxa, ry, &R.pa, &R.xa, &R.ya);
        else R.pa = R.xa = R.ya = T(0);
        if (cgb) lam_route(g, Lcur, gxb, ry, &R.pb, &R.xb, &R.yb);
        else R.pb = R.xb = R.yb = T(0);
      }
    }
  };

  // Moments of a column pair for one row.
  struct Mom2 {
    Mom<T> a, b;
  };
  // One row step for adjoint row r: scatter its fbar terms into moment rows r-1 (mA, completed
  // here), r (mB) and r+1 (mC, started here); then moment row q = r - 1 gives the local part of
  // output row q (oB) and h to output rows q-1 (oA, completed and emitted here), q (oB) and q+1
  // (oC, started here). The caller rotates the roles of three register sets.
  auto step = [&](int r, Mom2& mA, Mom2& mB, Mom2& mC, Acc2<T>& oA, Acc2<T>& oB, Acc2<T>& oC) {
    Pair3<T> R;
    load(r, R);
    {
      const G9<T> A = gbar(R.pa, R.xa, R.ya), B = gbar(R.pb, R.xb, R.yb);
      const T n1 = shdn(A.g1), n5 = shdn(A.g5), n8 = shdn(A.g8);  // column cb + 1, c_x = +1
      const T p3 = shup(B.g3), p6 = shup(B.g6), p7 = shup(B.g7);  // column ca - 1, c_x = -1
      mC.a.zero();
      mC.b.zero();
      mom_add(mA.a, mB.a, mC.a, A.g0, A.g2, A.g4, B.g1, B.g5, B.g8, p3, p6, p7);
      mom_add(mA.b, mB.b, mC.b, B.g0, B.g2, B.g4, n1, n5, n8, A.g3, A.g6, A.g7);
    }
    // moment row q = r - 1 is complete
    const int q = r - 1;
    int qy;
    const bool qrow = row_grid(q, &qy);
    Mom<T>& ma = mA.a;
    Mom<T>& mb = mA.b;
    if (!LEAN) {
      if (!(qrow && cga)) ma.zero();  // S is zero off the grid
      if (!(qrow && cgb)) mb.zero();
    }
    oC.zero();
    // local part of output row q (u(t-1) of row q from its ring slot), then refill that slot
    if (q >= ring_r0) {
      const T* sl = slot(q);
      const T uxa = sl[3 * 64], uxb = sl[3 * 64 + 1], uya = sl[4 * 64], uyb = sl[4 * 64 + 1];
      oB.pa += T(3) * ma.P;
      oB.xa += T(3) * ma.Ux + T(9) * (ma.Sxx * uxa + ma.Sxy * uya) - T(3) * uxa * ma.P;
      oB.ya += T(3) * ma.Uy + T(9) * (ma.Sxy * uxa + ma.Syy * uya) - T(3) * uya * ma.P;
      oB.pb += T(3) * mb.P;
      oB.xb += T(3) * mb.Ux + T(9) * (mb.Sxx * uxb + mb.Sxy * uyb) - T(3) * uxb * mb.P;
      oB.yb += T(3) * mb.Uy + T(9) * (mb.Sxy * uxb + mb.Syy * uyb) - T(3) * uyb * mb.P;
      issue(q + D);
    }
    // h: moment row q feeds output rows q-1, q, q+1
    const T lxx = shup(mb.Sxx), lxy = shup(mb.Sxy), lyy = shup(mb.Syy);  // column ca - 1
    const T rxx = shdn(ma.Sxx), rxy = shdn(ma.Sxy), ryy = shdn(ma.Syy);  // column cb + 1
    h_add2(oA.xa, oA.ya, oB.xa, oB.ya, oC.xa, oC.ya, ma.Sxy, ma.Syy, lxx, lxy, lyy, mb.Sxx, mb.Sxy, mb.Syy, kA);
    h_add2(oA.xb, oA.yb, oB.xb, oB.yb, oC.xb, oC.yb, mb.Sxy, mb.Syy, ma.Sxx, ma.Sxy, ma.Syy, rxx, rxy, ryy, kA);
    // wall ghost rows: row -1 (complete once moment row 0 is in) reflects onto row 1, row ny
    // (complete once moment row ny - 1 is in) onto row ny - 2
    if (wall_y && q == 0) {
      oC.xa -= oA.xa;
      oC.ya -= oA.ya;
      oC.xb -= oA.xb;
      oC.yb -= oA.yb;
    }
    if (wall_y && q == ny - 1) {
      oA.xa -= oC.xa;
      oA.ya -= oC.ya;
      oA.xb -= oC.xb;
      oA.yb -= oC.yb;
    }
    const int y = q - 1;  // output row oA is complete
    if (y < st.y0) return;
    Acc2<T> O = oA;
    if (has_xb) {
      // the x axis is open: ghost columns -1 and nx copied columns 0 and nx-1, so their h folds
      // back there with sign +1. Column -1 is the previous lane's cb; column nx is the next
      // lane's ca (when nx-1 is a cb) or this lane's cb (when nx-1 is a ca).
      const T gxl = shup(O.xb), gyl = shup(O.yb), gxr = shdn(O.xa), gyr = shdn(O.ya);
      if (st.ca == 0) {
        O.xa += gxl;
        O.ya += gyl;
      }
      if (st.cb == nx - 1) {
        O.xb += gxr;
        O.yb += gyr;
      }
      if (st.ca == nx - 1) {
        O.xa += O.xb;
        O.ya += O.yb;
      }
    }
    if (st.out && y < st.y1) {
      const long long rb = (long long)nx * y;
      if (pairv) {
        st_pair(Lnext, rb + st.ca, O.pa, O.pb);
        st_pair(Lnext + N, rb + st.ca, O.xa, O.xb);
        st_pair(Lnext + 2 * N, rb + st.ca, O.ya, O.yb);
      } else {
        if (st.ca < nx) {
          Lnext[rb + st.ca] = O.pa;
          Lnext[N + rb + st.ca] = O.xa;
          Lnext[2 * N + rb + st.ca] = O.ya;
        }
        if (st.cb < nx) {
          Lnext[rb + st.cb] = O.pb;
          Lnext[N + rb + st.cb] = O.xb;
          Lnext[2 * N + rb + st.cb] = O.yb;
        }
      }
    }
  };

  Mom2 m0, m1, m2;     // moment rows in rotation
  Acc2<T> o0, o1, o2;  // output rows in rotation (p: lam_p, x/y: lam_u)
  m0.a.zero();
  m0.b.zero();
  m1.a.zero();
  m1.b.zero();
  o0.zero();
  o1.zero();
  for (int i = 0; i < D; ++i) issue(ring_r0 + i);
  for (int r = st.y0 - 2; r <= st.y1 + 1; r += 3) {
    step(r, m0, m1, m2, o0, o1, o2);
    if (r + 1 > st.y1 + 1) break;
    step(r + 1, m1, m2, m0, o1, o2, o0);
    if (r + 2 > st.y1 + 1) break;
    step(r + 2, m2, m0, m1, o2, o0, o1);
  }
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(SW * 32) k_stencil2d_adj(Geo g, Slots<T> S, T* Lb, long long lstride,
                                                           const Ctrl* __restrict__ ctrl, int di, StripPlan sp) {
  Strip st;
  if (!strip_of(g, sp, &st)) return;  // uniform per warp
  if (VEC && interior_strip_adj(g, st))
    adj_strip<T, VEC, true>(g, S, Lb, lstride, ctrl, di, sp, st);
  else
    adj_strip<T, VEC, false>(g, S, Lb, lstride, ctrl, di, sp, st);
}

// Column tiles and row strips: W output columns per warp (60, or a little less so that the
// columns nx-2 and nx-1 of a non-periodic x axis share a warp; always even so column pairs start
// on an even column), strips of rows sized so the grid has about 32 warps per SM scheduler (short
// strips recompute two halo rows each, but more warps hide the shuffle and shared-memory
// latencies; measured on 8192x4096, predictor / transpose in % of HBM: 8 warps 59 / 50, 16 warps
// 71 / 65, 32 warps 76 / 72, 48 warps 74 / 73). Small grids are capped by the two-row minimum.
StripPlan plan_strips(const Geo& g) {
  StripPlan sp;
  sp.W = 60;
  if (g.bc[0] != BC_PERIODIC)
    while ((g.n[0] - 1) % sp.W == 0) sp.W -= 2;
  sp.ntx = (g.n[0] + sp.W - 1) / sp.W;
  const int want = 32 * 152 * 4;  // warps
  int ns = (want + sp.ntx - 1) / sp.ntx;
  const int maxs = g.n[1] / 2;  // at least two rows per strip (a wall row is built from the next)
  if (ns > maxs) ns = maxs;
  sp.nstrip = ns < 1 ? 1 : ns;
  return sp;
}

// Vector loads need every row to start on an even element (even nx; slots and planes then start
// on even elements too, the buffers being 256-byte aligned).
bool vec_ok(const Geo& g) { return g.n[0] % 2 == 0; }

}  // namespace

template <typename T>
void launch_stencil_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, int di, cudaStream_t st) {
  if (g.dim == 2) {
    const StripPlan sp = plan_strips(g);
    const int warps = sp.ntx * sp.nstrip;
    const size_t smem = Ring<T>::bytes(3);
    if (vec_ok(g))
      launch(k_stencil2d<T, true>, (warps + SW - 1) / SW, SW * 32, smem, st, g, S, ctrl, di, sp);
    else
      launch(k_stencil2d<T, false>, (warps + SW - 1) / SW, SW * 32, smem, st, g, S, ctrl, di, sp);
  } else {
    launch_stencil3d_fwd<T>(g, S, ctrl, di, st);
  }
}

template <typename T>
void launch_stencil_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, const Ctrl* ctrl, int di,
                        cudaStream_t st) {
  if (g.dim == 2) {
    const StripPlan sp = plan_strips(g);
    const int warps = sp.ntx * sp.nstrip;
    const size_t smem = Ring<T>::bytes(5);
    if (vec_ok(g))
      launch(k_stencil2d_adj<T, true>, (warps + SW - 1) / SW, SW * 32, smem, st, g, S, Lb, lstride, ctrl, di, sp);
    else
      launch(k_stencil2d_adj<T, false>, (warps + SW - 1) / SW, SW * 32, smem, st, g, S, Lb, lstride, ctrl, di, sp);
  } else {
    launch_stencil3d_adj<T>(g, S, Lb, lstride, ctrl, di, st);
  }
}

template void launch_stencil_fwd<float>(const Geo&, const Slots<float>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil_fwd<double>(const Geo&, const Slots<double>&, const Ctrl*, int, cudaStream_t);
template void launch_stencil_adj<float>(const Geo&, const Slots<float>&, float*, long long, const Ctrl*, int,
                                        cudaStream_t);
template void launch_stencil_adj<double>(const Geo&, const Slots<double>&, double*, long long, const Ctrl*, int,
                                         cudaStream_t);

}  // namespace lks
