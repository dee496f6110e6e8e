// The paper's adjoint, ALKS (Sec. 2.5, Appendix A), beside the exact discrete adjoint (single
// rotation axis). Variables: the moments p~, u~, s~ of the adjoint distribution (one slot holds
// p~, u~[D] and the D(D+1)/2 distinct entries of the symmetric s~) and the body multipliers x~G,
// u~G, theta~, omega~ (the paper's sign: the multipliers of the residuals).
//
// Reverse step t, with the converged DOFs s(t) and the state u(t) recomputed from the checkpoints:
//   k_alks_spread   box cells: kappa_n, u^S_n (Eqs. kappa_mapping, us_mapping at s(t)) and the
//                   omega~ source of Eq. au, sum_m kappa_m W (e x l_m)
//   k_alks_design   design points: the coupling sums of Eqs. axg, aug, atheta, aomega over each
//                   point's support window. Eq. au makes the fluid multiplier affine in the body
//                   multipliers, u~ = a + e u~G + f omega~ with a = u~*/(1+kappa), e = kappa/(3(1+kappa)),
//                   f = source/(3(1+kappa)), so every sum splits into a constant part and the
//                   coefficients of u~G and omega~; per point also the coefficients of the step's
//                   term of Eq. design_sensitivity
//   k_alks_finish   one CTA: the partial sums, then Algorithm 1's N_itr fixed-point iterations of
//                   the printed equations (each iteration is the affine map above applied to the
//                   previous iterate), in FP64
//   k_alks_write    box cells: u~(t) of Eq. au with u~G, omega~ of iteration N_itr - 1
//   k_alks_sens     design points: the step's term of Eq. design_sensitivity into dJ/dkappa^ref
//   k_alks_z        3D, all nodes: Z = u~ + 3 s~ u - p~ u - (A/3) sum_b d_b (s~ + s~^T), so that the
//                   adjoint equilibrium is f~eq_i = p~ + 3 c_i . Z
//   k_alks_gather   3D, all nodes: the star moments at t - 1 (Eqs. ap_tmp, au_tmp, as_tmp),
//                   p~* = sum_i w_i f~eq_i(x + c_i) and its first and second moments, with the boundary
//                   values prescribed: a quantity the forward fixes has a zero multiplier, one it
//                   copies from the inward neighbour copies the neighbour's, except u~ on the
//                   outlet plane, which follows the outflow condition of the convective adjoint,
//                   (u . n) u~ + nu du~/dn = 0: u~ = nu / (nu + max(u_x, 0)) u~(inward); s~ is copied.
//   k_alks_tile2d   2D: the two passes above in one tiled kernel (Z kept in shared memory).
// The terminal multipliers (x~G = -dJ/dxG, M u~G = -dJ/duG, theta~ = -dJ/dtheta, I omega~ = -dJ/domega)
// belong to a step N_t + 1; the fluid multipliers start at zero.
#include "lks_body_common.cuh"

namespace lks {

namespace {

// Velocity sets (rest, axis directions, diagonals; the sums below run over whole classes, so the
// order within a class does not matter) and weights (Sec. 2.2).
__constant__ int c_cv2[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
__constant__ int c_cv3[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                 {0, 0, 1},  {0, 0, -1}, {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},
                                 {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

template <int D>
struct Lat;
template <>
struct Lat<2> {
  static constexpr int Q = 9;
  static constexpr int NS = 3;  // distinct entries of s~: xx, yy, xy
  __device__ static int c(int i, int a) { return a < 2 ? c_cv2[i][a] : 0; }
  __device__ static double w(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
  static constexpr double cn = 6.0;  // sum_j c_jb^2
};
template <>
struct Lat<3> {
  static constexpr int Q = 15;
  static constexpr int NS = 6;  // xx, yy, zz, xy, xz, yz
  __device__ static int c(int i, int a) { return c_cv3[i][a]; }
  __device__ static double w(int i) { return i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0); }
  static constexpr double cn = 10.0;
};

// Plane of s~_ab in a moment slot (after p~ and u~[D]).
template <int D>
__host__ __device__ constexpr int sym(int a, int b) {
  return a == b ? a : (D == 2 ? 2 : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)));
}
template <int D>
__host__ __device__ constexpr int nplanes() {
  return 1 + D + Lat<D>::NS;
}

// Layout of the design-point partial sums (see k_alks_design): the coefficients of the affine maps.
template <int D>
struct NvA {
  static constexpr int r0X = 0, rGX = D, rWX = D + D * D, r0U = rWX + D, rGU = r0U + D, rWU = rGU + 1, r0T = rWU + D,
                       rGT = r0T + 1, rWT = rGT + D, r0O = rWT + 1, rGO = r0O + 1, rWO = rGO + D, GX = rWO + 1,
                       HX = GX + D * D, K0 = HX + D, LU = K0 + 1, GT = LU + D, HT = GT + D, PO = HT + 1, LO = PO + D,
                       N = LO + 1;
  static constexpr int NSENS = 3 + 2 * D;  // per design point: s0, sG[D], sW, Dm[D], lD
};

template <int AX>
__device__ __forceinline__ float cross_ax(const float* a, const float* b) {
  constexpr int B = Axes<AX>::B, C = Axes<AX>::C;
  return a[B] * b[C] - a[C] * b[B];
}
template <int AX>
__device__ __forceinline__ double cross_ax(const double* a, const double* b) {
  constexpr int B = Axes<AX>::B, C = Axes<AX>::C;
  return a[B] * b[C] - a[C] * b[B];
}

// Block sum of NV per-thread values into out[0..NV) (global, FP64), written by threads < NV. FP32:
// a shuffle tree in FP32 within each warp, then the warps' totals summed in FP64 by NV threads (the
// double-float tree of the exact reverse costs a dependent chain per value, too long for the 36 to
// 56 values here); FP64: the fixed-order FP64 tree. smem: 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void alks_block_sum(float (&v)[NV], double* out, double* smem) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = (double)v[i];
  __syncthreads();
  if (tid < NV) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += smem[w * NV + tid];
    out[tid] = acc;
  }
}
template <int NV>
__device__ __forceinline__ void alks_block_sum(double (&v)[NV], double* out, double* smem) {
  block_sum<NV>(v, smem);
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = v[i];
}

// u~G, omega~ of iterations N_itr - 1 (k = 0) and N_itr (k = 1) in the field type.
template <typename T>
__device__ __forceinline__ T al_it(const Ctrl* ctrl, int i);
template <>
__device__ __forceinline__ float al_it<float>(const Ctrl* ctrl, int i) { return ctrl->al_itf[i]; }
template <>
__device__ __forceinline__ double al_it<double>(const Ctrl* ctrl, int i) { return ctrl->al_it[i]; }

// ---- spread at s(t) -------------------------------------------------------------------------
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, BoxCta<D>::min_blocks) k_alks_spread(Geo g, const Ctrl* ctrl, const Dof* it,
                                                                 const T* __restrict__ kref, T* __restrict__ abox,
                                                                 int di) {
  const int t = ctrl->t0 - di, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[K];
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  const CellSlot cc = cell_slot<D>(g);
  const int px = lo[0] + cc.j0, py = lo[1] + cc.j1, pz = lo[2] + cc.j2;
  long long n = 0;
  const bool ing = cell_index<D>(g, px, py, pz, n);
  const DofView<T> V(sk);
  const T d[3] = {V.rel(0, px), V.rel(1, py), D == 3 ? V.rel(2, pz) : T(0)};
  Acc<T> A;
  T rotv[3], L[3];
  gather_cell<T, D, AX>(g, kref, sk, V, d, cc.lane, cc.active && ing, A, rotv, L);
  if (!cc.active || cc.lane != 0) return;
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
  T tq[3] = {T(0), T(0), T(0)};  // e x L, L = sum_m W kappa_m l_m
  tq[b] = -L[c];
  tq[c] = L[b];
  const long long BC = g.box_cells, bl = cc.j0 + (long long)g.B[0] * (cc.j1 + (long long)g.B[1] * cc.j2);
  abox[bl] = ing ? A.kap : T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    abox[(1 + a) * BC + bl] = ing ? V.ug[a] * A.phi + rotv[a] : T(0);
    abox[(1 + D + a) * BC + bl] = ing ? tq[a] : T(0);
  }
}

// ---- coupling sums over the design points' support windows -----------------------------------
// Per window node n of design point m (W = W(x_n, x^ref_m), dW = dW/dx^ref, p_m = dx^ref/dtheta,
// v_n = u_n - uS_n, q_n = -3 kappa_m v_n + 3 kappa_n uS,ref_m), with u~_n = a_n + e_n u~G + f_n omega~:
//   Eq. axg:    dW_al (q_n . u~_n) + kappa_m dW_al (u~G . u_n) + omega~ kappa_m dW_al (l_m x u_n)
//   Eq. aug:    3 kappa_n W u~_n,al
//   Eq. atheta: ((dW . p_m) q_n + 3 kappa_n W duS,ref_m/dtheta) . u~_n + kappa_m (dW . p_m)(u~G . u_n
//               + omega~ (l_m x u_n))
//   Eq. aomega: 3 kappa_n W p_m . u~_n
// and per point: -u~G kappa_m, -omega~ kappa_m (l_m x e_al) (Eq. aug), -kappa_m u~G . duS,ref/dtheta,
// omega~ kappa_m ((p_m x D_m) - (l_m x duS,ref/dtheta)) with D_m = u^ref_m - uS,ref_m (Eq. atheta),
// -kappa_m u~G . p_m, -omega~ kappa_m (l_m x p_m) (Eq. aomega). Cross products are along the axis.
// Four lanes per point split the window (rows in 2D, planes in 3D) as in the exact reverse.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(kDesignBlock) k_alks_design(Geo g, Slots<T> S, Ctrl* ctrl, const Dof* it,
                                                              const T* __restrict__ kref, const T* __restrict__ abox,
                                                              const T* __restrict__ Ab, long long astride,
                                                              T* __restrict__ sstore, void* partials, int di) {
  using NV = NvA<D>;
  __shared__ double red[32 * NV::N];
  const int t = ctrl->t0 - di, K = g.K, base = ctrl->base;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[K];
  const T* __restrict__ st = slot_ptr(S, t, base);
  const T* __restrict__ am = Ab + (long long)(t & 1) * astride;
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  const int lane = threadIdx.x % LN;
  T v[NV::N];
#pragma unroll
  for (int i = 0; i < NV::N; ++i) v[i] = T(0);
  bool inside = true;
  // chunks of kDesignPointsPerCta points, grid-strided (design_ctas caps the grid)
  for (int m0 = blockIdx.x * kDesignPointsPerCta; m0 < g.ND; m0 += gridDim.x * kDesignPointsPerCta) {
  const int m = m0 + threadIdx.x / LN;
  const bool valid_m = m < g.ND;
  const int mm = valid_m ? m : 0;
  const int ix = mm % g.nd[0], iy = (mm / g.nd[0]) % g.nd[1], iz = mm / (g.nd[0] * g.nd[1]);
  const bool valid = valid_m && dsq(ix, g.nd[0]) + dsq(iy, g.nd[1]) + dsq(iz, g.nd[2]) <= g.rad4;
  const T r[3] = {(T)ix - pivot<T>(g, 0), (T)iy - pivot<T>(g, 1), D == 3 ? (T)iz - pivot<T>(g, 2) : T(0)};
  const DofView<T> V(sk);
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
  T l[3], p[3];
  rot<AX>(V.cs, V.sn, r, l);
  drot<AX>(V.cs, V.sn, r, p);
  T usr[3] = {T(0), T(0), T(0)}, dus[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) usr[a] = V.ug[a] + V.om * p[a];
  dus[b] = -V.om * l[b];
  dus[c] = -V.om * l[c];
  const T km = valid ? kref[mm] : T(0);
  int f[3] = {0, 0, 0};
  T fr[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) V.split(a, l[a], &f[a], &fr[a]);
  const int S2 = 2 * g.s;
  constexpr int E = (D == 3) ? 2 : 1;  // the window axis split across the lanes
  T wv[3][4], dwv[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      wv[a][q] = (a < D) ? T(0) : T(1);
      dwv[a][q] = T(0);
    }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == E) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T rr = (T)(q - g.s + 1) - fr[a];  // x_n - x^ref along a
      if (q < S2 && fabs(rr) < (T)g.s) {
        wv[a][q] = wfun(g.wk, rr);
        dwv[a][q] = dwfun(g.wk, rr);
      }
    }
  }
  T we = T(0), dwe = T(0);
  {
    const T rr = (T)(lane - g.s + 1) - fr[E];
    if (lane < S2 && fabs(rr) < (T)g.s) {
      we = wfun(g.wk, rr);
      dwe = dwfun(g.wk, rr);
    }
  }
  T uref[3] = {T(0), T(0), T(0)}, sG[3] = {T(0), T(0), T(0)}, sa = T(0), sW = T(0);
  const long long N = g.N, BC = g.box_cells;
  const int B0 = g.B[0], B1 = g.B[1], B2 = (D == 3) ? g.B[2] : 1;
#pragma unroll
  for (int uu = 0; uu < (D == 3 ? 4 : 1); ++uu)
#pragma unroll
    for (int q0 = 0; q0 < 4; ++q0) {
      const int q1 = (D == 3) ? uu : lane, q2 = (D == 3) ? lane : 0;
      if (!valid || q0 >= S2 || q1 >= S2 || (D == 3 && q2 >= S2)) continue;
      const T w0 = wv[0][q0];
      const T w1 = (E == 1) ? we : wv[1][uu], dw1 = (E == 1) ? dwe : dwv[1][uu];
      const T w2 = (E == 2) ? we : T(1), dw2 = (E == 2) ? dwe : T(0);
      const T W = w0 * w1 * w2;
      // dW/dx^ref_e = -w'(x_e - x^ref_e) prod_{a != e} w
      const T dW[3] = {-dwv[0][q0] * w1 * w2, -w0 * dw1 * w2, -w0 * w1 * dw2};
      if (W == T(0) && dW[0] == T(0) && dW[1] == T(0) && dW[2] == T(0)) continue;
      const int gx = f[0] - g.s + 1 + q0, gy = f[1] - g.s + 1 + q1, gz = (D == 3) ? f[2] - g.s + 1 + q2 : 0;
      const int p0 = gx - lo[0], p1 = gy - lo[1], p2 = (D == 3) ? gz - lo[2] : 0;
      long long n = 0;
      if (p0 < 0 || p0 >= B0 || p1 < 0 || p1 >= B1 || p2 < 0 || p2 >= B2 || !cell_index<D>(g, gx, gy, gz, n)) {
        inside = false;
        continue;
      }
      const long long bl = p0 + (long long)B0 * (p1 + (long long)B1 * p2);
      const T kn = abox[bl];
      const T inv = T(1) / (T(1) + kn), en = kn * inv * T(1.0 / 3.0);
      T un[3] = {T(0), T(0), T(0)}, an[3] = {T(0), T(0), T(0)}, fn[3] = {T(0), T(0), T(0)};
      T vn[3] = {T(0), T(0), T(0)}, q[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        un[a] = st[(1 + a) * N + n];
        an[a] = am[(1 + a) * N + n] * inv;
        fn[a] = abox[(1 + D + a) * BC + bl] * inv * T(1.0 / 3.0);
        vn[a] = un[a] - abox[(1 + a) * BC + bl];
        q[a] = T(-3) * km * vn[a] + T(3) * kn * usr[a];
      }
      T qa = T(0), qf = T(0), dWp = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        qa += q[a] * an[a];
        qf += q[a] * fn[a];
        dWp += dW[a] * p[a];
      }
      const T t3 = T(3) * kn * W;
      const T lu = cross_ax<AX>(l, un);
      T cT[3], cTa = T(0), cTf = T(0), pa = T(0), pf = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        cT[a] = dWp * q[a] + t3 * dus[a];
        cTa += cT[a] * an[a];
        cTf += cT[a] * fn[a];
        pa += p[a] * an[a];
        pf += p[a] * fn[a];
      }
#pragma unroll
      for (int al = 0; al < D; ++al) {
        v[NV::r0X + al] += dW[al] * qa;
        v[NV::rWX + al] += dW[al] * qf;
#pragma unroll
        for (int be = 0; be < D; ++be) {
          v[NV::rGX + al * D + be] += dW[al] * q[be] * en;
          v[NV::GX + al * D + be] += km * dW[al] * un[be];
        }
        v[NV::HX + al] += km * lu * dW[al];
        v[NV::r0U + al] += t3 * an[al];
        v[NV::rWU + al] += t3 * fn[al];
        v[NV::rGT + al] += cT[al] * en;
        v[NV::rGO + al] += t3 * p[al] * en;
        v[NV::GT + al] += km * un[al] * dWp;
      }
      v[NV::rGU] += t3 * en;
      v[NV::r0T] += cTa;
      v[NV::rWT] += cTf;
      v[NV::r0O] += t3 * pa;
      v[NV::rWO] += t3 * pf;
      v[NV::HT] += km * lu * dWp;
      // the step's design sensitivity: sum_n 3 W v_n . u~_n
      const T w3 = T(3) * W;
      T va = T(0), vf = T(0);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uref[a] += W * un[a];
        va += vn[a] * an[a];
        vf += vn[a] * fn[a];
        sG[a] += w3 * vn[a] * en;
      }
      sa += w3 * va;
      sW += w3 * vf;
    }
#pragma unroll
  for (int off = 1; off < LN; off <<= 1) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      uref[a] += __shfl_xor_sync(0xffffffffu, uref[a], off);
      sG[a] += __shfl_xor_sync(0xffffffffu, sG[a], off);
    }
    sa += __shfl_xor_sync(0xffffffffu, sa, off);
    sW += __shfl_xor_sync(0xffffffffu, sW, off);
    inside = __shfl_xor_sync(0xffffffffu, (int)inside, off) && inside;
  }
  if (valid && lane == 0) {
    T Dm[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) Dm[a] = uref[a] - usr[a];
    v[NV::K0] += km;
#pragma unroll
    for (int al = 0; al < D; ++al) {
      const T lxe = (al == b) ? -l[c] : (al == c ? l[b] : T(0));  // (l x e_al) along the axis
      v[NV::LU + al] += km * lxe;
      v[NV::GT + al] -= km * dus[al];
      v[NV::PO + al] += km * p[al];
    }
    v[NV::HT] += km * (cross_ax<AX>(p, Dm) - cross_ax<AX>(l, dus));
    v[NV::LO] += km * cross_ax<AX>(l, p);
    T* sm = sstore + (long long)m * NV::NSENS;
    sm[0] = sa;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      sm[1 + a] = sG[a];
      sm[2 + D + a] = Dm[a];
    }
    sm[1 + D] = sW;
    sm[2 + 2 * D] = cross_ax<AX>(l, Dm);
  }
  }
  if (!inside && lane == 0) atomicOr(&ctrl->status, ST_BOX_OVERFLOW);
  alks_block_sum<NV::N>(v, static_cast<double*>(partials) + blockIdx.x * NV::N, red);
}

// ---- Algorithm 1's adjoint fixed-point iterations on the reduced sums (one CTA) ----------------
template <typename T, int D>
__global__ void __launch_bounds__(kFinishThreads) k_alks_finish(Geo g, Ctrl* ctrl, const double* partials, int nparts) {
  using NV = NvA<D>;
  __shared__ double red[kFinishThreads];
  __shared__ double Sm[NV::N];
  // the partials [nparts][NV], column-parallel: thread (i, j) sums value i over rows j, j + G, ...
  // (G groups of NV threads), then thread i sums its column's G results; fixed order, FP64
  constexpr int G = kFinishThreads / NV::N;
  const int tid = threadIdx.x, col = tid % NV::N, grp = tid / NV::N;
  if (grp < G) {
    double acc = 0.0;
    for (int q = grp; q < nparts; q += G) acc += __ldcg(&partials[(long long)q * NV::N + col]);
    red[grp * NV::N + col] = acc;
  }
  __syncthreads();
  if (tid < NV::N) {
    double acc = 0.0;
    for (int j = 0; j < G; ++j) acc += red[j * NV::N + tid];
    Sm[tid] = acc;
  }
  __syncthreads();
  if (tid != 0) return;
  const int mask = g.dof_mask, K = g.K;
  double nxt[8], cur[8], k1[4];
  for (int i = 0; i < 8; ++i) nxt[i] = cur[i] = ctrl->al_b[i];
  for (int a = 0; a < 3; ++a) k1[a] = cur[3 + a];
  k1[3] = cur[7];
  for (int k = 1; k <= K; ++k) {
    double nw[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int al = 0; al < D; ++al) {
      if (!(mask & (1 << al))) continue;
      double X = Sm[NV::r0X + al] + (Sm[NV::rWX + al] + Sm[NV::HX + al]) * cur[7];
      for (int be = 0; be < D; ++be) X += (Sm[NV::rGX + al * D + be] + Sm[NV::GX + al * D + be]) * cur[3 + be];
      nw[al] = nxt[al] + X;  // Eq. axg
      const double U = Sm[NV::r0U + al] + (Sm[NV::rGU] - Sm[NV::K0]) * cur[3 + al] +
                       (Sm[NV::rWU + al] - Sm[NV::LU + al]) * cur[7];
      nw[3 + al] = nxt[3 + al] + (nw[al] + U) * g.inv_mass;  // Eq. aug
    }
    if (mask & DOF_ROT) {
      double Th = Sm[NV::r0T] + (Sm[NV::rWT] + Sm[NV::HT]) * cur[7];
      double Om = Sm[NV::r0O] + (Sm[NV::rWO] - Sm[NV::LO]) * cur[7];
      for (int be = 0; be < D; ++be) {
        Th += (Sm[NV::rGT + be] + Sm[NV::GT + be]) * cur[3 + be];
        Om += (Sm[NV::rGO + be] - Sm[NV::PO + be]) * cur[3 + be];
      }
      nw[6] = nxt[6] + Th;                                 // Eq. atheta
      nw[7] = nxt[7] + (nw[6] + Om) * g.inv_inertia;       // Eq. aomega
    }
    if (k == K - 1) {
      for (int a = 0; a < 3; ++a) k1[a] = nw[3 + a];
      k1[3] = nw[7];
    }
    for (int i = 0; i < 8; ++i) cur[i] = nw[i];
  }
  for (int i = 0; i < 8; ++i) ctrl->al_b[i] = cur[i];
  const double itv[8] = {k1[0], k1[1], k1[2], k1[3], cur[3], cur[4], cur[5], cur[7]};
  for (int i = 0; i < 8; ++i) {
    ctrl->al_it[i] = itv[i];
    ctrl->al_itf[i] = (float)itv[i];
  }
}

// ---- u~(t) in the box (Eq. au with u~G, omega~ of iteration N_itr - 1) ---------------------------
template <typename T, int D>
__global__ void k_alks_write(Geo g, const Ctrl* ctrl, const Dof* it, const T* __restrict__ abox, T* Ab,
                             long long astride, int di) {
  const int t = ctrl->t0 - di, K = g.K;
  const Dof s0 = it[(long long)(t - 1) * (K + 1)];
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  T* am = Ab + (long long)(t & 1) * astride;
  const T ug[3] = {al_it<T>(ctrl, 0), al_it<T>(ctrl, 1), al_it<T>(ctrl, 2)}, om = al_it<T>(ctrl, 3);
  const long long BC = g.box_cells, N = g.N;
  for (long long bl = blockIdx.x * (long long)blockDim.x + threadIdx.x; bl < BC; bl += (long long)gridDim.x * blockDim.x) {
    const T kn = abox[bl];
    if (kn == T(0)) continue;  // no body here: u~ = u~*
    const int j0 = (int)(bl % g.B[0]), j1 = (int)((bl / g.B[0]) % g.B[1]), j2 = (int)(bl / ((long long)g.B[0] * g.B[1]));
    long long n = 0;
    if (!cell_index<D>(g, lo[0] + j0, lo[1] + j1, lo[2] + j2, n)) continue;
    const T inv = T(1) / (T(1) + kn);
#pragma unroll
    for (int a = 0; a < D; ++a)
      am[(1 + a) * N + n] = (am[(1 + a) * N + n] + (kn * ug[a] + om * abox[(1 + D + a) * BC + bl]) * T(1.0 / 3.0)) * inv;
  }
}

// ---- the step's term of Eq. design_sensitivity ---------------------------------------------------
template <typename T, int D>
__global__ void k_alks_sens(Geo g, const Ctrl* ctrl, const T* __restrict__ sstore, double* __restrict__ dkref) {
  using NV = NvA<D>;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.ND) return;
  const int ix = m % g.nd[0], iy = (m / g.nd[0]) % g.nd[1], iz = m / (g.nd[0] * g.nd[1]);
  if (dsq(ix, g.nd[0]) + dsq(iy, g.nd[1]) + dsq(iz, g.nd[2]) > g.rad4) return;
  const T* sm = sstore + (long long)m * NV::NSENS;
  T s = sm[0] + sm[1 + D] * al_it<T>(ctrl, 3) - sm[2 + 2 * D] * al_it<T>(ctrl, 7);
#pragma unroll
  for (int a = 0; a < D; ++a) s += sm[1 + a] * al_it<T>(ctrl, a) - sm[2 + D + a] * al_it<T>(ctrl, 4 + a);
  dkref[m] += (double)s;
}

// ---- the adjoint equilibrium at t and its star moments at t - 1 --------------------------------
// Neighbour of node x along c: wrapped on periodic axes, clamped (the ghost copies the boundary
// node) on the others.
template <int D>
__device__ __forceinline__ long long alks_nbr(const Geo& g, const int (&x)[3], int j) {
  int y[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int v = x[a] + Lat<D>::c(j, a);
    if (g.bc[a] == BC_PERIODIC)
      v = wrapi(v, g.n[a]);
    else
      v = min(max(v, 0), g.n[a] - 1);
    y[a] = v;
  }
  return (long long)y[0] + (long long)g.n[0] * ((long long)y[1] + (long long)g.n[1] * y[2]);
}

// D3Q15 vector components as compile-time values, in the order of c_cv3: rest, +-x, +-y, +-z,
// then the corners with s_x alternating, s_y in pairs and s_z in fours.
__host__ __device__ constexpr int cv3(int i, int a) {
  return i == 0 ? 0 : (i < 7 ? ((i - 1) / 2 == a ? ((i & 1) ? 1 : -1) : 0) : ((((i - 7) >> a) & 1) ? -1 : 1));
}
constexpr int kCv3Order[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1}, {1, 1, 1},  {-1, 1, 1},  {1, -1, 1},
                                  {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
constexpr bool cv3_in_order() {
  for (int i = 0; i < 15; ++i)
    for (int a = 0; a < 3; ++a)
      if (cv3(i, a) != kCv3Order[i][a]) return false;
  return true;
}
static_assert(cv3_in_order(), "cv3 must list the D3Q15 vectors in the order of c_cv3");

// The node indices alks_nbr gives for the D3Q15 vectors of node x, with the wrap or clamp done
// once per axis and coordinate (components are -1, 0 or +1) instead of once per vector and axis:
// o[a][k] is coordinate x_a + k - 1, wrapped or clamped, times the stride of axis a. Call with a
// compile-time vector index (unrolled loops), so o stays in registers.
struct NodeNbrs3 {
  long long o[3][3];
  __device__ __forceinline__ NodeNbrs3(const Geo& g, const int (&x)[3]) {
    long long stride = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        int v = x[a] + k - 1;
        if (g.bc[a] == BC_PERIODIC)
          v = v < 0 ? v + g.n[a] : (v >= g.n[a] ? v - g.n[a] : v);
        else
          v = min(max(v, 0), g.n[a] - 1);
        o[a][k] = (long long)v * stride;
      }
      stride *= g.n[a];
    }
  }
  __device__ __forceinline__ long long operator()(int j) const {
    return o[0][cv3(j, 0) + 1] + o[1][cv3(j, 1) + 1] + o[2][cv3(j, 2) + 1];
  }
};

template <int D>
__device__ __forceinline__ void node_coords(const Geo& g, long long n, int (&x)[3]) {
  if (n <= 0x7fffffffLL) {  // 32-bit division where the index allows it
    const unsigned u = (unsigned)n, r = u / (unsigned)g.n[0];
    x[0] = (int)(u - r * (unsigned)g.n[0]);
    x[1] = (int)(r % (unsigned)g.n[1]);
    x[2] = (D == 3) ? (int)(r / (unsigned)g.n[1]) : 0;
    return;
  }
  x[0] = (int)(n % g.n[0]);
  x[1] = (int)((n / g.n[0]) % g.n[1]);
  x[2] = (D == 3) ? (int)(n / ((long long)g.n[0] * g.n[1])) : 0;
}

template <typename T, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 0) k_alks_z(Geo g, const Ctrl* ctrl, Slots<T> S, const T* __restrict__ Ab,
                                                long long astride, T* __restrict__ zb, int di) {
  constexpr int NS = Lat<D>::NS;
  const int t = ctrl->t0 - di;
  const T* __restrict__ st = slot_ptr(S, t, ctrl->base);
  const T* __restrict__ am = Ab + (long long)(t & 1) * astride;
  const long long N = g.N;
  const T cA = (T)(2.0 * g.A / (3.0 * Lat<D>::cn));  // (A/3) * 2 / sum_j c_jb^2
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    int x[3];
    node_coords<D>(g, n, x);
    T gs[D][D];  // sum_j c_jb s~_ab(x + c_j)
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) gs[a][bb] = T(0);
    static_assert(D == 3, "the node kernels through Z are the 3D form");
    const NodeNbrs3 nb(g, x);
#pragma unroll
    for (int j = 1; j < Lat<D>::Q; ++j) {
      const long long m = nb(j);
      T sv[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) sv[k] = am[(1 + D + k) * N + m];
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) {
          const int cb = Lat<D>::c(j, bb);
          if (cb != 0) gs[a][bb] += (T)cb * sv[sym<D>(a, bb)];
        }
    }
    const T pt = am[n];
    T u[D];
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = st[(1 + a) * N + n];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      T Z = am[(1 + a) * N + n] - pt * u[a];
#pragma unroll
      for (int bb = 0; bb < D; ++bb) Z += T(3) * am[(1 + D + sym<D>(a, bb)) * N + n] * u[bb] - cA * gs[a][bb];
      zb[a * N + n] = Z;
    }
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 0) k_alks_gather(Geo g, const Ctrl* ctrl, Slots<T> S, T* Ab, long long astride,
                                                     const T* __restrict__ zb, T nu, int di) {
  constexpr int NS = Lat<D>::NS;
  const int t = ctrl->t0 - di;
  const T* __restrict__ st = slot_ptr(S, t, ctrl->base);
  const T* __restrict__ am = Ab + (long long)(t & 1) * astride;
  T* __restrict__ out = Ab + (long long)((t - 1) & 1) * astride;
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    int x[3];
    node_coords<D>(g, n, x);
    // boundary node: the value of its inward neighbour (through every boundary axis), with a zero
    // multiplier for what the forward prescribes there and the outflow factor for u~ on the outlet
    bool zp = false, zu = false;
    T fu = T(1);
    if (g.bc[0] != BC_PERIODIC) {
      if (x[0] == 0) {
        x[0] = 1;
        if (g.bc[0] == BC_INFLOW_OUTFLOW)
          zu = true;
        else
          zp = true;
      } else if (x[0] == g.n[0] - 1) {
        x[0] = g.n[0] - 2;
        zp = true;
        fu = nu / (nu + fmax(st[N + n], T(0)));  // u_x of the state on the outlet node
      }
    }
#pragma unroll
    for (int a = 1; a < D; ++a)
      if (g.bc[a] == BC_WALL && (x[a] == 0 || x[a] == g.n[a] - 1)) {
        x[a] = (x[a] == 0) ? 1 : g.n[a] - 2;
        zu = true;
      }
    T P = T(0), U[D], Sv[NS];
#pragma unroll
    for (int a = 0; a < D; ++a) U[a] = T(0);
#pragma unroll
    for (int k = 0; k < NS; ++k) Sv[k] = T(0);
    static_assert(D == 3, "the node kernels through Z are the 3D form");
    const NodeNbrs3 nb(g, x);  // x is interior on non-periodic axes: no clamping
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) {
      const long long m = nb(i);
      T F = am[m];
#pragma unroll
      for (int a = 0; a < D; ++a) F += T(3) * (T)Lat<D>::c(i, a) * zb[a * N + m];
      const T wF = (T)Lat<D>::w(i) * F;
      P += wF;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T cw = (T)Lat<D>::c(i, a) * wF;
        U[a] += cw;
#pragma unroll
        for (int bb = a; bb < D; ++bb) Sv[sym<D>(a, bb)] += (T)Lat<D>::c(i, bb) * cw;
      }
    }
    out[n] = zp ? T(0) : P;
#pragma unroll
    for (int a = 0; a < D; ++a) out[(1 + a) * N + n] = zu ? T(0) : fu * U[a];
#pragma unroll
    for (int k = 0; k < NS; ++k) out[(1 + D + k) * N + n] = Sv[k];
  }
}

// Terminal body multipliers (step N_t + 1) for J = seed * sum_d w_d s_d(N_t).
__global__ void k_alks_init(Geo g, Ctrl* ctrl, const double* objw, double seed) {
  double bv[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int a = 0; a < g.dim; ++a) {
    if (!(g.dof_mask & (1 << a))) continue;
    bv[a] = -seed * objw[a];
    bv[3 + a] = -seed * objw[3 + a] * g.inv_mass;
  }
  if (g.dof_mask & DOF_ROT) {
    bv[6] = -seed * objw[6];
    bv[7] = -seed * objw[7] * g.inv_inertia;
  }
  for (int i = 0; i < 8; ++i) ctrl->al_b[i] = bv[i];
}

// 2D: the two node kernels in one pass. A 32 x TY tile with a halo of three holds p~, u~, s~ and u
// (each read once, with the derivative's ghost rule applied on load: wrapped on periodic axes,
// clamped on the others, so the tile holds what the derivative reads); Z is formed on the halo-2
// region in shared memory, and the tile's star moments are gathered from it with the boundary
// values prescribed as in k_alks_gather (a boundary node's source is its inward neighbour, at most
// one node outside the tile). TY = 16 in FP32, 8 in FP64 (static shared memory below 48 KB).
constexpr int kAlksTileX = 32;
template <typename T>
__host__ __device__ constexpr int alks_tile_y() { return sizeof(T) == 4 ? 16 : 8; }

template <typename T>
__global__ void __launch_bounds__(kAlksTileX * alks_tile_y<T>()) k_alks_tile2d(Geo g, const Ctrl* ctrl, Slots<T> S,
                                                                               T* Ab, long long astride, T nu, int di) {
  constexpr int TY = alks_tile_y<T>(), NTH = kAlksTileX * TY;
  constexpr int IX = kAlksTileX + 6, IY = TY + 6, ZX = kAlksTileX + 4, ZY = TY + 4;
  __shared__ T in[8][IY][IX];  // p~, u~x, u~y, s~xx, s~yy, s~xy, ux, uy
  __shared__ T zs[2][ZY][ZX];  // Z on the halo-2 region
  const int t = ctrl->t0 - di;
  const T* __restrict__ st = slot_ptr(S, t, ctrl->base);
  const T* __restrict__ am = Ab + (long long)(t & 1) * astride;
  T* __restrict__ out = Ab + (long long)((t - 1) & 1) * astride;
  const long long N = g.N;
  const int nx = g.n[0], ny = g.n[1];
  const int x0 = blockIdx.x * kAlksTileX, y0 = blockIdx.y * TY;
  for (int q = threadIdx.x; q < IX * IY; q += NTH) {
    const int li = q % IX, lj = q / IX;
    int gx = x0 - 3 + li, gy = y0 - 3 + lj;
    gx = (g.bc[0] == BC_PERIODIC) ? wrapi(gx, nx) : min(max(gx, 0), nx - 1);
    gy = (g.bc[1] == BC_PERIODIC) ? wrapi(gy, ny) : min(max(gy, 0), ny - 1);
    const long long n = gx + (long long)nx * gy;
#pragma unroll
    for (int k = 0; k < 6; ++k) in[k][lj][li] = am[k * N + n];
    in[6][lj][li] = st[N + n];
    in[7][lj][li] = st[2 * N + n];
  }
  __syncthreads();
  const T cA = (T)(2.0 * g.A / 18.0);  // (A/3) * 2 / sum_j c_jb^2
  for (int q = threadIdx.x; q < ZX * ZY; q += NTH) {
    const int zi = q % ZX, zj = q / ZX, i = zi + 1, j = zj + 1;
    T d[3][2];  // sum_j c_jb s~(y + c_j) for the planes xx, yy, xy and b = x, y
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T(*s)[IX] = in[3 + k];
      d[k][0] = (s[j][i + 1] - s[j][i - 1]) + (s[j + 1][i + 1] - s[j + 1][i - 1]) + (s[j - 1][i + 1] - s[j - 1][i - 1]);
      d[k][1] = (s[j + 1][i] - s[j - 1][i]) + (s[j + 1][i + 1] - s[j - 1][i + 1]) + (s[j + 1][i - 1] - s[j - 1][i - 1]);
    }
    const T p = in[0][j][i], ux = in[6][j][i], uy = in[7][j][i];
    const T sxx = in[3][j][i], syy = in[4][j][i], sxy = in[5][j][i];
    zs[0][zj][zi] = in[1][j][i] + T(3) * (sxx * ux + sxy * uy) - p * ux - cA * (d[0][0] + d[2][1]);
    zs[1][zj][zi] = in[2][j][i] + T(3) * (sxy * ux + syy * uy) - p * uy - cA * (d[2][0] + d[1][1]);
  }
  __syncthreads();
  const int tx = threadIdx.x % kAlksTileX, ty = threadIdx.x / kAlksTileX;
  const int gx = x0 + tx, gy = y0 + ty;
  if (gx >= nx || gy >= ny) return;
  const long long n = gx + (long long)nx * gy;
  int sx = gx, sy = gy;
  bool zp = false, zu = false;
  T fu = T(1);
  if (g.bc[0] != BC_PERIODIC) {
    if (gx == 0) {
      sx = 1;
      if (g.bc[0] == BC_INFLOW_OUTFLOW)
        zu = true;
      else
        zp = true;
    } else if (gx == nx - 1) {
      sx = nx - 2;
      zp = true;
      fu = nu / (nu + fmax(st[N + n], T(0)));
    }
  }
  if (g.bc[1] == BC_WALL && (gy == 0 || gy == ny - 1)) {
    sy = (gy == 0) ? 1 : ny - 2;
    zu = true;
  }
  const int zi = sx - x0 + 2, zj = sy - y0 + 2;
  T P = T(0), Ux = T(0), Uy = T(0), Sxx = T(0), Syy = T(0), Sxy = T(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cx = Lat<2>::c(i, 0), cy = Lat<2>::c(i, 1);
    const int yi = zi + cx, yj = zj + cy;
    const T F = in[0][yj + 1][yi + 1] + T(3) * ((T)cx * zs[0][yj][yi] + (T)cy * zs[1][yj][yi]);
    const T wF = (T)Lat<2>::w(i) * F;
    P += wF;
    Ux += (T)cx * wF;
    Uy += (T)cy * wF;
    Sxx += (T)(cx * cx) * wF;
    Syy += (T)(cy * cy) * wF;
    Sxy += (T)(cx * cy) * wF;
  }
  out[n] = zp ? T(0) : P;
  out[N + n] = zu ? T(0) : fu * Ux;
  out[2 * N + n] = zu ? T(0) : fu * Uy;
  out[3 * N + n] = Sxx;
  out[4 * N + n] = Syy;
  out[5 * N + n] = Sxy;
}

unsigned node_blocks(const Geo& g) {
  const long long nb = (g.N + 255) / 256;
  return (unsigned)(nb < (1 << 20) ? nb : (1 << 20));
}

}  // namespace

// Dispatch on the dimension and the single rotation axis.
#define ALKS_DISPATCH(KERNEL, GRID, BLOCK, ...)                   \
  do {                                                            \
    if (g.dim == 2)                                               \
      launch(KERNEL<T, 2, 2>, GRID, BLOCK, 0, st, __VA_ARGS__);   \
    else if (g.ax == 0)                                           \
      launch(KERNEL<T, 3, 0>, GRID, BLOCK, 0, st, __VA_ARGS__);   \
    else if (g.ax == 1)                                           \
      launch(KERNEL<T, 3, 1>, GRID, BLOCK, 0, st, __VA_ARGS__);   \
    else                                                          \
      launch(KERNEL<T, 3, 2>, GRID, BLOCK, 0, st, __VA_ARGS__);   \
  } while (0)

int alks_partial_values(int dim) { return dim == 2 ? NvA<2>::N : NvA<3>::N; }
int alks_sens_values(int dim) { return dim == 2 ? NvA<2>::NSENS : NvA<3>::NSENS; }
int alks_planes(int dim) { return dim == 2 ? nplanes<2>() : nplanes<3>(); }
int alks_stencil_kernels(int dim) { return dim == 2 ? 1 : 2; }

void launch_alks_init(const Geo& g, Ctrl* ctrl, const double* objw, double seed, double* dkref, cudaStream_t st) {
  cudaMemsetAsync(dkref, 0, sizeof(double) * (size_t)g.ND, st);
  launch(k_alks_init, 1, 1, 0, st, g, ctrl, objw, seed);
}

template <typename T>
void launch_alks_body(const Geo& g, const Slots<T>& S, Ctrl* ctrl, const Dof* it, const T* kref, T* abox, T* Ab,
                      long long astride, T* sstore, void* partials, double* dkref, int di, cudaStream_t st) {
  ALKS_DISPATCH(k_alks_spread, box_grid(g), box_threads(g), g, ctrl, it, kref, abox, di);
  const unsigned nb = (unsigned)design_ctas(g);
  ALKS_DISPATCH(k_alks_design, nb, kDesignBlock, g, S, ctrl, it, kref, (const T*)abox, (const T*)Ab, astride, sstore,
                partials, di);
  const long long wb = (g.box_cells + 255) / 256;
  const unsigned sb = (unsigned)((g.ND + 255) / 256);
  if (g.dim == 2) {
    launch(k_alks_finish<T, 2>, 1, kFinishThreads, 0, st, g, ctrl, (const double*)partials, (int)nb);
    launch(k_alks_write<T, 2>, (unsigned)(wb < 4096 ? wb : 4096), 256, 0, st, g, (const Ctrl*)ctrl, it,
           (const T*)abox, Ab, astride, di);
    launch(k_alks_sens<T, 2>, sb, 256, 0, st, g, (const Ctrl*)ctrl, (const T*)sstore, dkref);
  } else {
    launch(k_alks_finish<T, 3>, 1, kFinishThreads, 0, st, g, ctrl, (const double*)partials, (int)nb);
    launch(k_alks_write<T, 3>, (unsigned)(wb < 4096 ? wb : 4096), 256, 0, st, g, (const Ctrl*)ctrl, it,
           (const T*)abox, Ab, astride, di);
    launch(k_alks_sens<T, 3>, sb, 256, 0, st, g, (const Ctrl*)ctrl, (const T*)sstore, dkref);
  }
}

template <typename T>
void launch_alks_stencil(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, T* Ab, long long astride, T* zb, int di,
                         cudaStream_t st) {
  const T nu = (T)(1.0 / 6.0 - 2.0 * g.A / 9.0);  // nu = 1/6 - 2A/9 (Sec. 2.2)
  if (g.dim == 2) {
    const dim3 grid((g.n[0] + kAlksTileX - 1) / kAlksTileX, (g.n[1] + alks_tile_y<T>() - 1) / alks_tile_y<T>());
    launch(k_alks_tile2d<T>, grid, kAlksTileX * alks_tile_y<T>(), 0, st, g, ctrl, S, Ab, astride, nu, di);
  } else {
    launch(k_alks_z<T, 3>, node_blocks(g), 256, 0, st, g, ctrl, S, (const T*)Ab, astride, zb, di);
    launch(k_alks_gather<T, 3>, node_blocks(g), 256, 0, st, g, ctrl, S, Ab, astride, (const T*)zb, nu, di);
  }
}

#define LKS_ALKS_INST(T)                                                                                          \
  template void launch_alks_body<T>(const Geo&, const Slots<T>&, Ctrl*, const Dof*, const T*, T*, T*, long long, T*, \
                                    void*, double*, int, cudaStream_t);                                           \
  template void launch_alks_stencil<T>(const Geo&, const Slots<T>&, const Ctrl*, T*, long long, T*, int,          \
                                       cudaStream_t);

LKS_ALKS_INST(float)
LKS_ALKS_INST(double)

}  // namespace lks
