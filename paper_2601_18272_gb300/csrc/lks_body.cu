// Grid separation, Brinkman coupling and rigid-body EOM (Sec. 2.2-2.4, 3.1) and their reverse.
//
// Forward coupling iteration k of step t, one thread per cell of the body box:
//   gather the design points within the kernel support of the cell under s^(k-1)
//     kappa_n = sum_m W kappa_m,  u^S_n = sum_m W u^S,ref_m = u^G phi_n + omega R' (sum_m W r_m)
//   Brinkman update u_n = (u*_n + kappa_n u^S_n) / (1 + kappa_n)                       (Eq. u)
//   force and torque on the body (Sec. 2.4) as
//     F = sum_n kappa_n u_n - sum_m kappa_m u^S,ref_m,
//     T = sum_n (L_n x u_n) . e - sum_m kappa_m (R r_m x u^S,ref_m) . e,  L_n = sum_m W kappa_m R r_m,
//   which equals the design-grid sum sum_m kappa_m (u^ref_m - u^S,ref_m) of Sec. 2.4 up to the
//   order of summation, because the interpolation (Eq. u_mapping) uses the same weights as the
//   spread; the design-side sums are closed forms in (u^G, omega) over precomputed moments.
//   Per-block FP64 partials, then the last block sums them in block order and applies the
//   explicit Euler EOM (Sec. 2.4) in FP64.
//
// Reverse of iteration k: a cell-side kernel (Brinkman and interpolation reverse, accumulation of
// dJ/du*) and a design-side kernel, one thread per design point, that gathers its axis-aligned
// support window of cells for the spread / interpolation / transform reverse (the dW/dx^ref
// terms), accumulates dJ/dkappa^ref without atomics and reduces dJ/ds^(k-1).
#include "lks_kernels.h"

namespace lks {

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ int block_linear() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }
__device__ __forceinline__ int thread_linear() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }

template <typename T>
__global__ void __launch_bounds__(256) k_prep(Geo g, const double* __restrict__ gamma, double kmax, double q,
                                               T* __restrict__ kref, Moments* mom, double* partials, Ctrl* ctrl) {
  __shared__ double red[32 * 5];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double v[5] = {0, 0, 0, 0, 0};
  if (m < g.ND) {
    const double gm = gamma[m];
    const T k = (T)(kmax * q * gm / ((1.0 - gm) + q));  // Eq. brinkman_coefficient
    kref[m] = k;
    const double kd = (double)k;
    int i[3] = {m % g.nd[0], (m / g.nd[0]) % g.nd[1], m / (g.nd[0] * g.nd[1])};
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = (a < g.dim) ? i[a] - g.xic[a] : 0.0;
    v[0] = kd;
    v[1] = kd * r[0];
    v[2] = kd * r[1];
    v[3] = kd * r[2];
    v[4] = kd * (r[g.axb] * r[g.axb] + r[g.axc] * r[g.axc]);
  }
  block_sum<5>(v, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 5; ++a) partials[blockIdx.x * 5 + a] = v[a];
  if (last_block_done(&ctrl->count[CNT_PREP]) && threadIdx.x == 0) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < (int)gridDim.x; ++b)
      for (int a = 0; a < 5; ++a) s[a] += __ldcg(&partials[b * 5 + a]);
    mom->K0 = s[0];
    mom->K1[0] = s[1];
    mom->K1[1] = s[2];
    mom->K1[2] = s[3];
    mom->K2p = s[4];
    ctrl->count[CNT_PREP] = 0;
  }
}

template <typename T, int D, int AX>
__global__ void __launch_bounds__(BX* BY) k_couple(Geo g, Slots<T> S, Ctrl* ctrl, Dof* it, const T* __restrict__ kref,
                                                    const Moments* __restrict__ mom, double* partials, int k,
                                                    T* __restrict__ boxstore, int nbox) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
  __shared__ double red[32 * 4];
  const int t = ctrl->t, base = ctrl->base, K = g.K;
  Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[k - 1];
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  int lx, ly, lz;
  box_origin<D>(g, s0, lx, ly, lz);
  const int j0 = blockIdx.x * BX + threadIdx.x, j1 = blockIdx.y * BY + threadIdx.y, j2 = blockIdx.z;
  double v[4] = {0, 0, 0, 0};
  if (j0 < g.B[0] && j1 < g.B[1]) {
    const int px = lx + j0, py = ly + j1, pz = lz + j2;
    long long n = 0;
    const bool ing = cell_index<D>(g, px, py, pz, n);
    const T d[3] = {(T)((double)px - sk.s[0]), (T)((double)py - sk.s[1]), D == 3 ? (T)((double)pz - sk.s[2]) : T(0)};
    const T cs = (T)sk.cs, sn = (T)sk.sn;
    Acc<T> A;
    gather<T, D, AX>(g, kref, d, cs, sn, A);
    if (A.phi > T(0) && (!ing || forbidden<D>(g, px, py, pz))) atomicOr(&ctrl->status, ST_BODY_OUTSIDE);
    if (ing) {
      T dwr[3], L[3], u[3] = {T(0), T(0), T(0)};
      drot<AX>(cs, sn, A.wr, dwr);
      rot<AX>(cs, sn, A.kr, L);
      const T om = (T)sk.s[7];
      const T inv = T(1) / (T(1) + A.kap);
      const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
      T* bs = boxstore ? boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D : nullptr;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T us = (T)sk.s[3 + a] * A.phi + om * dwr[a];
        const T ustar = dst[(a + 1) * N + n];
        u[a] = (ustar + A.kap * us) * inv;
        v[a] = (double)(A.kap * u[a]);
        if (k == K) {
          if (bs) bs[a * g.box_cells + bl] = ustar;
          dst[(a + 1) * N + n] = u[a];
        }
      }
      v[D] = (double)(L[b] * u[c] - L[c] * u[b]);  // torque about AX
    }
  }
  block_sum<4>(v, red);
  const int tid = thread_linear();
  if (tid == 0)
    for (int a = 0; a < 4; ++a) partials[block_linear() * 4 + a] = v[a];
  if (last_block_done(&ctrl->count[CNT_COUPLE]) && tid == 0) {
    double s[4] = {0, 0, 0, 0};
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    for (int q = 0; q < nb; ++q)
      for (int a = 0; a < 4; ++a) s[a] += __ldcg(&partials[q * 4 + a]);
    const double cs = sk.cs, sn = sk.sn, om = sk.s[7];
    const double K1[3] = {mom->K1[0], mom->K1[1], mom->K1[2]};
    double K1r[3], K1d[3];
    rot<AX>(cs, sn, K1, K1r);
    drot<AX>(cs, sn, K1, K1d);
    const double ug[3] = {sk.s[3], sk.s[4], sk.s[5]};
    double F[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) F[a] = s[a] - (mom->K0 * ug[a] + om * K1d[a]);
    const double Tq = s[D] - (K1r[b] * ug[c] - K1r[c] * ug[b]) - om * mom->K2p;
    bool finite = isfinite(Tq);
    for (int a = 0; a < D; ++a) finite = finite && isfinite(F[a]);
    if (!finite) ctrl->status |= ST_NONFINITE;
    Dof nx;
    eom_update(g, s0, F, Tq, &nx);
    for (int a = 0; a < D; ++a)
      if (fabs(nx.s[a] - s0.s[a]) > (double)g.margin) ctrl->status |= ST_BOX_OVERFLOW;
    row[k] = nx;
    if (k == K) {
      it[(long long)t * (K + 1)] = nx;
      ctrl->t = t + 1;
    }
    ctrl->count[CNT_COUPLE] = 0;
  }
}

// Recompute of one step's Brinkman update from the stored iterate s^(K-1).
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BX* BY) k_apply(Geo g, Slots<T> S, Ctrl* ctrl, const Dof* it,
                                                   const T* __restrict__ kref, T* __restrict__ boxstore, int nbox) {
  const int t = ctrl->t, base = ctrl->base, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[K - 1];
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  int lx, ly, lz;
  box_origin<D>(g, s0, lx, ly, lz);
  const int j0 = blockIdx.x * BX + threadIdx.x, j1 = blockIdx.y * BY + threadIdx.y, j2 = blockIdx.z;
  if (j0 < g.B[0] && j1 < g.B[1]) {
    const int px = lx + j0, py = ly + j1, pz = lz + j2;
    long long n = 0;
    if (cell_index<D>(g, px, py, pz, n)) {
      const T d[3] = {(T)((double)px - sk.s[0]), (T)((double)py - sk.s[1]), D == 3 ? (T)((double)pz - sk.s[2]) : T(0)};
      const T cs = (T)sk.cs, sn = (T)sk.sn;
      Acc<T> A;
      gather<T, D, AX>(g, kref, d, cs, sn, A);
      T dwr[3];
      drot<AX>(cs, sn, A.wr, dwr);
      const T om = (T)sk.s[7];
      const T inv = T(1) / (T(1) + A.kap);
      const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
      T* bs = boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T us = (T)sk.s[3 + a] * A.phi + om * dwr[a];
        const T ustar = dst[(a + 1) * N + n];
        bs[a * g.box_cells + bl] = ustar;
        dst[(a + 1) * N + n] = (ustar + A.kap * us) * inv;
      }
    }
  }
  if (last_block_done(&ctrl->count[CNT_APPLY]) && thread_linear() == 0) {
    ctrl->t = t + 1;
    ctrl->count[CNT_APPLY] = 0;
  }
}

// Reverse of coupling iteration k, cell side. Scratch planes per box cell:
//   [0, D): u^(k);  D: dJ/dkappa_n;  [D+1, 2D+1): dJ/du^S_n.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BX* BY) k_adj_cell(Geo g, Ctrl* ctrl, const Dof* it, const T* __restrict__ kref,
                                                      const T* __restrict__ boxstore, int nbox, T* Lb,
                                                      long long lstride, T* __restrict__ acc, T* __restrict__ scratch,
                                                      int k) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
  const int t = ctrl->t, base = ctrl->base, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[k - 1];
  const double lF[3] = {ctrl->lam_F[0], ctrl->lam_F[1], ctrl->lam_F[2]};
  const double lT = ctrl->lam_T;
  T* Lcur = Lb + (long long)(t & 1) * lstride;
  const long long N = g.N, BC = g.box_cells;
  int lx, ly, lz;
  box_origin<D>(g, s0, lx, ly, lz);
  const int j0 = blockIdx.x * BX + threadIdx.x, j1 = blockIdx.y * BY + threadIdx.y, j2 = blockIdx.z;
  if (j0 >= g.B[0] || j1 >= g.B[1]) return;
  const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
  const int px = lx + j0, py = ly + j1, pz = lz + j2;
  long long n = 0;
  if (!cell_index<D>(g, px, py, pz, n)) {
    for (int q = 0; q < 2 * D + 1; ++q) scratch[q * BC + bl] = T(0);
    return;
  }
  const T* bs = boxstore + (long long)((t - base - 1) % nbox) * BC * D;
  const T d[3] = {(T)((double)px - sk.s[0]), (T)((double)py - sk.s[1]), D == 3 ? (T)((double)pz - sk.s[2]) : T(0)};
  const T cs = (T)sk.cs, sn = (T)sk.sn;
  Acc<T> A;
  gather<T, D, AX>(g, kref, d, cs, sn, A);
  T dwr[3], L[3];
  drot<AX>(cs, sn, A.wr, dwr);
  rot<AX>(cs, sn, A.kr, L);
  const T om = (T)sk.s[7];
  const T inv = T(1) / (T(1) + A.kap);
  // sum_m W dJ/du^ref_m = kappa_n lam_F + lam_T (e x L_n), in the rotation plane
  T extra[3] = {T(0), T(0), T(0)};
  extra[b] = -(T)lT * L[c];
  extra[c] = (T)lT * L[b];
  T lkap = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T us = (T)sk.s[3 + a] * A.phi + om * dwr[a];
    const T uk = (bs[a * BC + bl] + A.kap * us) * inv;
    T lu = A.kap * (T)lF[a] + extra[a];
    if (k == K) lu += Lcur[(a + 1) * N + n];
    const T accv = (k == K ? T(0) : acc[a * BC + bl]) + lu * inv;
    if (k == 1)
      Lcur[(a + 1) * N + n] = accv;
    else
      acc[a * BC + bl] = accv;
    lkap += lu * (us - uk) * inv;
    scratch[a * BC + bl] = uk;
    scratch[(D + 1 + a) * BC + bl] = lu * A.kap * inv;
  }
  scratch[D * BC + bl] = lkap;
}

// Reverse of coupling iteration k, design side (one thread per design point m).
template <typename T, int D, int AX>
__global__ void __launch_bounds__(256) k_adj_design(Geo g, Ctrl* ctrl, const Dof* it, const T* __restrict__ kref,
                                                     const T* __restrict__ scratch, double* __restrict__ dkref,
                                                     double* partials, int k) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, ax = Axes<AX>::A;
  __shared__ double red[32 * 8];
  const int t = ctrl->t, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[k - 1];
  const double lF[3] = {ctrl->lam_F[0], ctrl->lam_F[1], ctrl->lam_F[2]};
  const double lT = ctrl->lam_T;
  const long long BC = g.box_cells;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (m < g.ND) {
    int lx, ly, lz;
    box_origin<D>(g, s0, lx, ly, lz);
    const int ix = m % g.nd[0], iy = (m / g.nd[0]) % g.nd[1], iz = m / (g.nd[0] * g.nd[1]);
    const T r[3] = {(T)(ix - g.xic[0]), (T)(iy - g.xic[1]), D == 3 ? (T)(iz - g.xic[2]) : T(0)};
    const T cs = (T)sk.cs, sn = (T)sk.sn, om = (T)sk.s[7];
    T l[3], dl[3];
    rot<AX>(cs, sn, r, l);
    drot<AX>(cs, sn, r, dl);
    const T km = kref[m];
    T usr[3] = {T(0), T(0), T(0)}, luref[3] = {T(0), T(0), T(0)}, rotl[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) usr[a] = (T)sk.s[3 + a] + om * dl[a];
    rotl[b] = -(T)lT * l[c];
    rotl[c] = (T)lT * l[b];
#pragma unroll
    for (int a = 0; a < D; ++a) luref[a] = km * ((T)lF[a] + rotl[a]);
    // window of analysis cells around x^ref_m: 2s cells per axis from floor(x^ref) - s + 1
    int f[3] = {0, 0, 0};
    T fr[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double xr = sk.s[a] + (double)l[a];
      const double fl = floor(xr);
      f[a] = (int)fl;
      fr[a] = (T)(xr - fl);
    }
    const int S2 = 2 * g.s;
    T wv[3][4], dwv[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        wv[a][q] = (a < D) ? T(0) : T(1);
        dwv[a][q] = T(0);
      }
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T rr = (T)(q - g.s + 1) - fr[a];  // x_n - x^ref along a
        if (q < S2 && fabs(rr) < (T)g.s) {
          wv[a][q] = wfun(g.wk, rr);
          dwv[a][q] = dwfun(g.wk, rr);
        }
      }
    T uref[3] = {T(0), T(0), T(0)}, slus[3] = {T(0), T(0), T(0)}, lxr[3] = {T(0), T(0), T(0)};
    T slk = T(0);
    bool over = false;
    const int B0 = g.B[0], B1 = g.B[1], B2 = (D == 3) ? g.B[2] : 1;
#pragma unroll
    for (int q2 = 0; q2 < (D == 3 ? 4 : 1); ++q2)
#pragma unroll
      for (int q1 = 0; q1 < 4; ++q1)
#pragma unroll
        for (int q0 = 0; q0 < 4; ++q0) {
          if (q0 >= S2 || q1 >= S2 || (D == 3 && q2 >= S2)) continue;
          const T w0 = wv[0][q0], w1 = wv[1][q1], w2 = wv[2][q2];
          const T W = w0 * w1 * w2;
          const T dW0 = dwv[0][q0] * w1 * w2, dW1 = w0 * dwv[1][q1] * w2, dW2 = w0 * w1 * dwv[2][q2];
          if (W == T(0) && dW0 == T(0) && dW1 == T(0) && dW2 == T(0)) continue;
          const int p0 = f[0] - g.s + 1 + q0 - lx, p1 = f[1] - g.s + 1 + q1 - ly;
          const int p2 = (D == 3) ? f[2] - g.s + 1 + q2 - lz : 0;
          if (p0 < 0 || p0 >= B0 || p1 < 0 || p1 >= B1 || p2 < 0 || p2 >= B2) {
            over = true;
            continue;
          }
          const long long bl = p0 + (long long)B0 * (p1 + (long long)B1 * p2);
          T uk[3] = {T(0), T(0), T(0)}, lus[3] = {T(0), T(0), T(0)};
#pragma unroll
          for (int a = 0; a < D; ++a) {
            uk[a] = scratch[a * BC + bl];
            lus[a] = scratch[(D + 1 + a) * BC + bl];
          }
          const T lk = scratch[D * BC + bl];
          T qv = km * lk;
#pragma unroll
          for (int a = 0; a < D; ++a) {
            uref[a] += W * uk[a];
            slus[a] += W * lus[a];
            qv += luref[a] * uk[a] + usr[a] * lus[a];
          }
          slk += W * lk;
          // dW/dx^ref_e = -w'(x_e - x^ref_e) prod_{a != e} w
          lxr[0] -= dW0 * qv;
          lxr[1] -= dW1 * qv;
          lxr[2] -= dW2 * qv;
        }
    if (over) atomicOr(&ctrl->status, ST_BOX_OVERFLOW);
    T Dl[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) Dl[a] = uref[a] - usr[a];
    double dk = (double)slk + lT * (double)(l[b] * Dl[c] - l[c] * Dl[b]);
#pragma unroll
    for (int a = 0; a < D; ++a) dk += lF[a] * (double)Dl[a];
    dkref[m] += dk;
    T lusr[3] = {T(0), T(0), T(0)}, ll[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < D; ++a) lusr[a] = -luref[a] + slus[a];
    ll[b] = (T)lT * km * Dl[c];
    ll[c] = -(T)lT * km * Dl[b];
    double lth = 0.0, lom = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T ddl = (a == ax) ? T(0) : -l[a];  // R'' r
      lth += (double)((lxr[a] + ll[a]) * dl[a] + om * lusr[a] * ddl);
      lom += (double)(lusr[a] * dl[a]);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      v[a] = (double)lxr[a];
      v[3 + a] = (double)lusr[a];
    }
    v[6] = lth;
    v[7] = lom;
  }
  block_sum<8>(v, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < 8; ++a) partials[blockIdx.x * 8 + a] = v[a];
  if (last_block_done(&ctrl->count[CNT_DESIGN]) && threadIdx.x == 0) {
    double ls[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < (int)gridDim.x; ++q)
      for (int a = 0; a < 8; ++a) ls[a] += __ldcg(&partials[q * 8 + a]);
    double lp[8];
    for (int a = 0; a < 8; ++a) lp[a] = ctrl->lam_prev[a];
    double nF[3], nT;
    if (k > 1) {
      eom_reverse(g, ls, nF, &nT, lp);
    } else {
      double lsm1[8];
      for (int a = 0; a < 8; ++a) {
        lsm1[a] = lp[a] + ls[a];
        ctrl->lam_s0[a] = lsm1[a];
        lp[a] = 0.0;
      }
      eom_reverse(g, lsm1, nF, &nT, lp);
    }
    for (int a = 0; a < 8; ++a) ctrl->lam_prev[a] = lp[a];
    for (int a = 0; a < 3; ++a) ctrl->lam_F[a] = nF[a];
    ctrl->lam_T = nT;
    ctrl->count[CNT_DESIGN] = 0;
  }
}

template <typename T>
__global__ void k_init_forward(Geo g, Slots<T> S, const double* __restrict__ p0, const double* __restrict__ u0,
                               const double* __restrict__ s0, Dof* it, Ctrl* ctrl) {
  const long long N = g.N;
  T* dst = S.base;  // slot of step 0
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    dst[n] = (T)p0[n];
    for (int a = 0; a < g.dim; ++a) dst[(a + 1) * N + n] = (T)u0[a * N + n];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Dof d;
    for (int a = 0; a < 8; ++a) d.s[a] = s0[a];
    d.cs = cos(d.s[6]);
    d.sn = sin(d.s[6]);
    it[0] = d;
    ctrl->t = 1;
    ctrl->base = 0;
    ctrl->status = 0;
  }
}

__global__ void k_set_step(Ctrl* ctrl, int t, int base) {
  ctrl->t = t;
  ctrl->base = base;
}

__global__ void k_adj_init(Geo g, Ctrl* ctrl, const double* objw, double seed) {
  double ls[8], lp[8], nF[3], nT;
  for (int a = 0; a < 8; ++a) {
    ls[a] = seed * objw[a];
    lp[a] = 0.0;
  }
  eom_reverse(g, ls, nF, &nT, lp);
  for (int a = 0; a < 8; ++a) ctrl->lam_prev[a] = lp[a];
  for (int a = 0; a < 3; ++a) ctrl->lam_F[a] = nF[a];
  ctrl->lam_T = nT;
}

__global__ void k_sensitivity(int nd, const double* __restrict__ gamma, const double* __restrict__ dkref, double kmax,
                              double q, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nd) return;
  const double den = (1.0 - gamma[m]) + q;
  out[m] = dkref[m] * kmax * q * (1.0 + q) / (den * den);
}

template <typename T>
__global__ void k_ckpt_pack(Geo g, Slots<T> S, T* ckpt, long long cstride, int every, const Ctrl* ctrl) {
  const int tn = ctrl->t - 1;
  const T* src = slot_ptr(S, tn, ctrl->base);
  T* dst = ckpt + (long long)(tn / every) * cstride;
  const long long M = (long long)(g.dim + 1) * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

inline dim3 box_grid(const Geo& g) { return dim3((g.B[0] + BX - 1) / BX, (g.B[1] + BY - 1) / BY, g.dim == 3 ? g.B[2] : 1); }

}  // namespace

template <typename T>
void launch_prep(const Geo& g, const double* gamma, double kappa_max, double q, T* kref, Moments* mom,
                 double* partials, Ctrl* ctrl, cudaStream_t st) {
  k_prep<T><<<(g.ND + 255) / 256, 256, 0, st>>>(g, gamma, kappa_max, q, kref, mom, partials, ctrl);
}

// Dispatch on the dimension and the (runtime) rotation axis to the compile-time instantiation.
#define LKS_BOX_DISPATCH(KERNEL, GRID, BLOCK, ...)                                   \
  do {                                                                               \
    if (g.dim == 2)                                                                  \
      KERNEL<T, 2, 2><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__);                          \
    else if (g.ax == 0)                                                              \
      KERNEL<T, 3, 0><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__);                          \
    else if (g.ax == 1)                                                              \
      KERNEL<T, 3, 1><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__);                          \
    else                                                                             \
      KERNEL<T, 3, 2><<<GRID, BLOCK, 0, st>>>(__VA_ARGS__);                          \
  } while (0)

template <typename T>
void launch_couple(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                   double* partials, int k, T* boxstore, int nbox, cudaStream_t st) {
  LKS_BOX_DISPATCH(k_couple, box_grid(g), dim3(BX, BY), g, S, ctrl, it, kref, mom, partials, k, boxstore, nbox);
}

template <typename T>
void launch_apply(const Geo& g, const Slots<T>& S, Ctrl* ctrl, const Dof* it, const T* kref, T* boxstore, int nbox,
                  cudaStream_t st) {
  LKS_BOX_DISPATCH(k_apply, box_grid(g), dim3(BX, BY), g, S, ctrl, it, kref, boxstore, nbox);
}

template <typename T>
void launch_adj_cell(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, int k, cudaStream_t st) {
  LKS_BOX_DISPATCH(k_adj_cell, box_grid(g), dim3(BX, BY), g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc,
                   scratch, k);
}

template <typename T>
void launch_adj_design(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* scratch, double* dkref,
                       double* partials, int k, cudaStream_t st) {
  const unsigned nb = (unsigned)((g.ND + 255) / 256);
  LKS_BOX_DISPATCH(k_adj_design, nb, 256, g, ctrl, it, kref, scratch, dkref, partials, k);
}

template <typename T>
void launch_init_forward(const Geo& g, const Slots<T>& S, const double* p0, const double* u0, const double* s0dev,
                         Dof* it, Ctrl* ctrl, cudaStream_t st) {
  const long long nb = (g.N + 255) / 256;
  k_init_forward<T><<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(g, S, p0, u0, s0dev, it, ctrl);
}

void launch_set_step(Ctrl* ctrl, int t, int base, cudaStream_t st) { k_set_step<<<1, 1, 0, st>>>(ctrl, t, base); }

void launch_adj_init(const Geo& g, Ctrl* ctrl, const double* objw, double seed, double* dkref, int nd,
                     cudaStream_t st) {
  cudaMemsetAsync(dkref, 0, sizeof(double) * (size_t)nd, st);
  k_adj_init<<<1, 1, 0, st>>>(g, ctrl, objw, seed);
}

void launch_sensitivity(const Geo& g, const double* gamma, const double* dkref, double kappa_max, double q,
                        double* out, cudaStream_t st) {
  k_sensitivity<<<(g.ND + 255) / 256, 256, 0, st>>>(g.ND, gamma, dkref, kappa_max, q, out);
}

template <typename T>
void launch_ckpt_pack(const Geo& g, const Slots<T>& S, T* ckpt, long long cstride, int every, const Ctrl* ctrl,
                      cudaStream_t st) {
  const long long M = (long long)(g.dim + 1) * g.N;
  const long long nb = (M + 255) / 256;
  k_ckpt_pack<T><<<(unsigned)(nb < 8192 ? nb : 8192), 256, 0, st>>>(g, S, ckpt, cstride, every, ctrl);
}

#define LKS_INST(T)                                                                                              \
  template void launch_prep<T>(const Geo&, const double*, double, double, T*, Moments*, double*, Ctrl*,           \
                               cudaStream_t);                                                                    \
  template void launch_couple<T>(const Geo&, const Slots<T>&, Ctrl*, Dof*, const T*, const Moments*, double*, int, \
                                 T*, int, cudaStream_t);                                                         \
  template void launch_apply<T>(const Geo&, const Slots<T>&, Ctrl*, const Dof*, const T*, T*, int, cudaStream_t); \
  template void launch_adj_cell<T>(const Geo&, Ctrl*, const Dof*, const T*, const T*, int, T*, long long, T*, T*, \
                                   int, cudaStream_t);                                                           \
  template void launch_adj_design<T>(const Geo&, Ctrl*, const Dof*, const T*, const T*, double*, double*, int,    \
                                     cudaStream_t);                                                              \
  template void launch_init_forward<T>(const Geo&, const Slots<T>&, const double*, const double*, const double*,  \
                                       Dof*, Ctrl*, cudaStream_t);                                               \
  template void launch_ckpt_pack<T>(const Geo&, const Slots<T>&, T*, long long, int, const Ctrl*, cudaStream_t);

LKS_INST(float)
LKS_INST(double)

}  // namespace lks
