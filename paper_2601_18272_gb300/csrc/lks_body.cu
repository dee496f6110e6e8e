// Grid separation, Brinkman coupling and rigid-body EOM (Sec. 2.2-2.4, 3.1) and their reverse.
//
// Forward coupling iteration k of step t, per cell n of the body box:
//   gather the design points within the kernel support of the cell under s^(k-1)
//     kappa_n = sum_m W kappa_m,  u^S_n = sum_m W u^S,ref_m = u^G phi_n + omega R' (sum_m W r_m)
//   Brinkman update u_n = (u*_n + kappa_n u^S_n) / (1 + kappa_n)                       (Eq. u)
//   force and torque on the body (Sec. 2.4) as
//     F = sum_n kappa_n u_n - sum_m kappa_m u^S,ref_m,
//     T = sum_n (L_n x u_n) . e - sum_m kappa_m (R r_m x u^S,ref_m) . e,  L_n = sum_m W kappa_m R r_m,
//   which equals the design-grid sum sum_m kappa_m (u^ref_m - u^S,ref_m) of Sec. 2.4 up to the
//   order of summation, because the interpolation (Eq. u_mapping) uses the same weights as the
//   spread; the design-side sums are closed forms in (u^G, omega) over precomputed moments.
//   FP64 partial sums, then the explicit Euler EOM (Sec. 2.4) in FP64.
//
// Reverse of iteration k: a cell phase (Brinkman and interpolation reverse, accumulation of
// dJ/du*) and a design-point phase that gathers each point's axis-aligned support window of cells
// for the spread / interpolation / transform reverse (the dW/dx^ref terms), accumulates
// dJ/dkappa^ref without atomics and reduces dJ/ds^(k-1).
//
// Free rotation (AX = AX_FREE): R is a full rotation matrix and omega a vector; the solid velocity
// is u^G phi_n + omega x (R sum_m W r_m), the torque a vector sum_n L_n x u_n - sum_m kappa_m
// (R r_m) x u^S,ref_m whose design-side part is (R K1) x u^G + K2s omega - R K2 R^T omega with
// K2s = sum kappa_m |r_m|^2, K2 = sum kappa_m r_m r_m^T.
//
// Each iteration's global reduction is split into a kernel over all SMs that writes one FP64
// partial per CTA (double-float pairs in the FP32 form) and a finish that sums the partials in a
// fixed order and applies the (reverse) EOM: the kernel boundary orders the partials, so no
// GPU-scope fence or counter is needed, and the sums are deterministic. In the forward the next
// coupling kernel does the finish in every CTA (one launch per iteration) while the grid has at
// most kFusedFinishMaxParts CTAs, and a one-CTA k_couple_pre does it once above that; in the
// reverse the one-CTA k_design_finish does it after the design-point kernel, whose grid is capped
// (design_ctas) so that it sums few partials.
#include <climits>

#include "lks_body_common.cuh"

namespace lks {

namespace {


// Partial sums per CTA: the coupling reduces force and torque (one torque component about the
// axis, or the torque vector with free rotation); the design-point reverse reduces dJ/ds^(k-1)
// through the transform: (xG, uG, theta, omega), or (xG, uG, omega[3], R[9]) with free rotation.
template <int AX>
__host__ __device__ constexpr int nv_couple() { return AX == AX_FREE ? 6 : 4; }
template <int AX>
__host__ __device__ constexpr int nv_design() { return AX == AX_FREE ? 18 : 8; }

// dJ/dF and dJ/dT of the iteration being reversed, in the field type (dJ/dT about the axis in [0]).
template <typename T>
__device__ __forceinline__ void lam_load(const Ctrl* ctrl, T (&lF)[3], T (&lT)[3]);
template <>
__device__ __forceinline__ void lam_load<float>(const Ctrl* ctrl, float (&lF)[3], float (&lT)[3]) {
  for (int a = 0; a < 3; ++a) {
    lF[a] = ctrl->lam_Ff[a];
    lT[a] = ctrl->lam_Tf[a];
  }
}
template <>
__device__ __forceinline__ void lam_load<double>(const Ctrl* ctrl, double (&lF)[3], double (&lT)[3]) {
  for (int a = 0; a < 3; ++a) {
    lF[a] = ctrl->lam_F[a];
    lT[a] = ctrl->lam_T[a];
  }
}

__device__ __forceinline__ void lam_store(Ctrl* ctrl, const double* lF, const double* lT) {
  for (int a = 0; a < 3; ++a) {
    ctrl->lam_F[a] = lF[a];
    ctrl->lam_Ff[a] = (float)lF[a];
    ctrl->lam_T[a] = lT[a];
    ctrl->lam_Tf[a] = (float)lT[a];
  }
}

// Forward coupling work for box cell (j0, j1, j2), called by all LN lanes of the cell (every
// thread of the warp must call it: the gather combines lanes with shuffles); lane 0 adds
// kappa_n u_n and the torque density to v. On the last iteration lane 0 writes u(t) into dst and,
// if bs is set, the predictor u* into the box store.
template <typename T, int D, int AX>
__device__ __forceinline__ void couple_cell(const Geo& g, const T* __restrict__ kref, const Dof& sk, const int (&lo)[3],
                                            const CellSlot& cc, T* __restrict__ dst, T* __restrict__ bs, bool last,
                                            int* status, T* v) {
  const long long N = g.N;
  const int j0 = cc.j0, j1 = cc.j1, j2 = cc.j2;
  const int px = lo[0] + j0, py = lo[1] + j1, pz = lo[2] + j2;
  long long n = 0;
  const bool ing = cell_index<D>(g, px, py, pz, n);
  const DofView<T> V(sk);
  const T d[3] = {V.rel(0, px), V.rel(1, py), D == 3 ? V.rel(2, pz) : T(0)};
  Acc<T> A;
  T rotv[3], L[3], u[3] = {T(0), T(0), T(0)};
  gather_cell<T, D, AX>(g, kref, sk, V, d, cc.lane, cc.active, A, rotv, L);
  if (!cc.active || cc.lane != 0) return;
  if (A.phi > T(0) && (!ing || forbidden<D>(g, px, py, pz))) atomicOr(status, ST_BODY_OUTSIDE);
  if (!ing) return;
  const T inv = T(1) / (T(1) + A.kap);
  const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T us = V.ug[a] * A.phi + rotv[a];
    const T ustar = dst[(a + 1) * N + n];
    u[a] = (ustar + A.kap * us) * inv;
    v[a] += A.kap * u[a];
    if (last) {
      if (bs) bs[a * g.box_cells + bl] = ustar;
      dst[(a + 1) * N + n] = u[a];
    }
  }
  if constexpr (AX == AX_FREE) {  // torque density vector L_n x u_n
    T tq[3];
    cross3(L, u, tq);
    v[3] += tq[0];
    v[4] += tq[1];
    v[5] += tq[2];
  } else {  // about AX
    constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
    v[D] += L[b] * u[c] - L[c] * u[b];
  }
}

// Closed-form design-side terms and the EOM update of iteration k from the cell sums s[0..D].
template <int D, int AX>
__device__ __forceinline__ void couple_finish(const Geo& g, const Moments* mom, const Dof& s0, const Dof& sk,
                                              const double* s, Dof* nx, int* status) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
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
  if (!finite) *status |= ST_NONFINITE;
  eom_update<D>(g, s0, F, Tq, nx);
  for (int a = 0; a < D; ++a)
    if (fabs(nx->s[a] - s0.s[a]) > (double)g.margin) *status |= ST_BOX_OVERFLOW;
}

// couple_finish on the lanes of one warp (one rotation axis): lane a < 3 the force, velocity,
// position and FP32 views of axis a, lane 3 the torque, angular velocity, angle and cos/sin, lane 4
// the unused DOF entries, so the FP64 chain on the critical path is the rotation's alone. Each
// quantity is computed by the same operations in the same order as couple_finish, so the iterate is
// the same to the bit. Every lane of the warp calls it; s (the cell sums) is taken from lane 0; the
// status bits are returned to every lane.
template <int D, int AX>
__device__ __forceinline__ int couple_finish_lanes(const Geo& g, const Moments& mom, const Dof& s0, const Dof& sk,
                                                   const double* s_in, Dof* nx, int lane) {
  constexpr int NS = D + 1;
  double s[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) s[i] = __shfl_sync(0xffffffffu, s_in[i], 0);
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
  const double cs = sk.cs, sn = sk.sn, om = sk.s[7];
  const double K1[3] = {mom.K1[0], mom.K1[1], mom.K1[2]};
  const double ug[3] = {sk.s[3], sk.s[4], sk.s[5]};
  int st = 0;
  if (lane < 3) {
    const int a = lane;
    double x = s0.s[a], u = s0.s[3 + a];
    if (a < D) {
      double K1d[3];
      drot<AX>(cs, sn, K1, K1d);
      const double F = s[a] - (mom.K0 * ug[a] + om * K1d[a]);
      if (!isfinite(F)) st |= ST_NONFINITE;
      if (g.dof_mask & (1 << a)) {
        u = s0.s[3 + a] + F * g.inv_mass;
        x = s0.s[a] + u;
      }
      if (fabs(x - s0.s[a]) > (double)g.margin) st |= ST_BOX_OVERFLOW;
    }
    nx->s[a] = x;
    nx->s[3 + a] = u;
    const double fl = floor(x);
    nx->xi[a] = (int)fl;
    nx->xf[a] = (float)(x - fl);
    nx->ug[a] = (float)u;
  } else if (lane == 3) {
    double K1r[3];
    rot<AX>(cs, sn, K1, K1r);
    const double Tq = s[D] - (K1r[b] * ug[c] - K1r[c] * ug[b]) - om * mom.K2p;
    if (!isfinite(Tq)) st |= ST_NONFINITE;
    double w = s0.s[7], th = s0.s[6];
    if (g.dof_mask & DOF_ROT) {
      w = s0.s[7] + Tq * g.inv_inertia;
      th = s0.s[6] + w;
    }
    nx->s[6] = th;
    nx->s[7] = w;
    double ncs, nsn;
    rotate_angle(s0, th - s0.s[6], &ncs, &nsn);
    nx->cs = ncs;
    nx->sn = nsn;
    nx->om = (float)w;
    nx->csf = (float)ncs;
    nx->snf = (float)nsn;
  } else if (lane == 4) {
#pragma unroll
    for (int a = kNdofAxis; a < kNdofFree; ++a) nx->s[a] = 0.0;
  }
  return __reduce_or_sync(0xffffffffu, st);
}

// The one-block finish kernels' part (one rotation axis): stage s0 = base[0] and sk = base[kprev]
// in shared memory, sum the partials, run couple_finish_lanes on warp 0 and store the new iterate
// to out (and to out2 if not null). All threads of the block call it.
template <int D, int AX, typename PT, int NV>
__device__ __forceinline__ void finish_lanes_to(const Geo& g, Ctrl* ctrl, const Moments* __restrict__ mom,
                                                const Dof* base, int kprev, const PT* pin, int nparts, double* red,
                                                Dof (&sdd)[3], Dof* out, Dof* out2) {
  constexpr int DW = sizeof(Dof) / sizeof(double);
  const int tid = threadIdx.x;
  double* sdw = reinterpret_cast<double*>(sdd);
  if (tid < DW) {
    sdw[tid] = reinterpret_cast<const double*>(base)[tid];
    sdw[DW + tid] = reinterpret_cast<const double*>(base + kprev)[tid];
  }
  Moments m;
  if (tid < 32) m = *mom;
  double sm[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) sm[a] = 0.0;
  block_sum_partials<NV>(pin, nparts, sm, red);  // its barriers order the staging copies
  if (tid < 32) {
    const int st = couple_finish_lanes<D, AX>(g, m, sdd[0], sdd[1], sm, &sdd[2], tid);
    if (tid == 0 && st) ctrl->status |= st;
  }
  __syncthreads();
  if (tid < DW) {
    reinterpret_cast<double*>(out)[tid] = sdw[2 * DW + tid];
    if (out2) reinterpret_cast<double*>(out2)[tid] = sdw[2 * DW + tid];
  }
}

// The same with free rotation from the cell sums s[0..5] = (F_cell, T_cell).
__device__ __forceinline__ void couple_finish_free(const Geo& g, const Moments* mom, const Dof& s0, const Dof& sk,
                                                   const double* s, Dof* nx, int* status) {
  const double* R = sk.s + S_R;
  const double* om = sk.s + S_OM;
  const double ug[3] = {sk.s[3], sk.s[4], sk.s[5]};
  double K1r[3], oxk[3], kxu[3], K2o[3], v1[3];
  matvec3(R, mom->K1, K1r);
  cross3(om, K1r, oxk);
  cross3(K1r, ug, kxu);
  // R K2 R^T omega
  const double K2[9] = {mom->K2[0], mom->K2[3], mom->K2[4], mom->K2[3], mom->K2[1],
                        mom->K2[5], mom->K2[4], mom->K2[5], mom->K2[2]};
  matTvec3(R, om, v1);
  double v2[3];
  matvec3(K2, v1, v2);
  matvec3(R, v2, K2o);
  double F[3], Tv[3];
  bool finite = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    F[a] = s[a] - (mom->K0 * ug[a] + oxk[a]);
    Tv[a] = s[3 + a] - (kxu[a] + mom->K2s * om[a] - K2o[a]);
    finite = finite && isfinite(F[a]) && isfinite(Tv[a]);
  }
  if (!finite) *status |= ST_NONFINITE;
  eom_update_free(g, s0, F, Tv, nx);
  for (int a = 0; a < 3; ++a)
    if (fabs(nx->s[a] - s0.s[a]) > (double)g.margin) *status |= ST_BOX_OVERFLOW;
}

template <int D, int AX>
__device__ __forceinline__ void couple_finish_any(const Geo& g, const Moments* mom, const Dof& s0, const Dof& sk,
                                                  const double* s, Dof* nx, int* status) {
  if constexpr (AX == AX_FREE)
    couple_finish_free(g, mom, s0, sk, s, nx, status);
  else
    couple_finish<D, AX>(g, mom, s0, sk, s, nx, status);
}

// Reverse of coupling iteration k for box cell (j0, j1, j2). Scratch planes per box cell:
//   [0, D): u^(k);  D: dJ/dkappa_n;  [D+1, 2D+1): dJ/du^S_n.  acc accumulates dJ/du*.
// Called by all LN lanes of the cell (see couple_cell); lane 0 does the per-cell work.
template <typename T, int D, int AX>
__device__ __forceinline__ void adj_cell_work(const Geo& g, const T* __restrict__ kref, const Dof& sk,
                                              const int (&lo)[3], const CellSlot& cc, const T* __restrict__ bs,
                                              T* Lcur, T* __restrict__ acc, T* __restrict__ scratch, int k, int K,
                                              const T (&lF)[3], const T (&lT)[3]) {
  const long long N = g.N, BC = g.box_cells;
  const int j0 = cc.j0, j1 = cc.j1, j2 = cc.j2;
  const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
  const int px = lo[0] + j0, py = lo[1] + j1, pz = lo[2] + j2;
  long long n = 0;
  const bool ing = cell_index<D>(g, px, py, pz, n);
  const DofView<T> V(sk);
  const T d[3] = {V.rel(0, px), V.rel(1, py), D == 3 ? V.rel(2, pz) : T(0)};
  Acc<T> A;
  T rotv[3], L[3];
  gather_cell<T, D, AX>(g, kref, sk, V, d, cc.lane, cc.active && ing, A, rotv, L);
  if (!cc.active || cc.lane != 0) return;
  if (!ing) {
    for (int q = 0; q < 2 * D + 1; ++q) scratch[q * BC + bl] = T(0);
    return;
  }
  const T inv = T(1) / (T(1) + A.kap);
  // sum_m W dJ/du^ref_m = kappa_n lam_F + lam_T x L_n (lam_T along the axis for one axis)
  T extra[3] = {T(0), T(0), T(0)};
  if constexpr (AX == AX_FREE) {
    cross3(lT, L, extra);
  } else {
    constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
    extra[b] = -lT[0] * L[c];
    extra[c] = lT[0] * L[b];
  }
  T lkap = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T us = V.ug[a] * A.phi + rotv[a];
    const T uk = (bs[a * BC + bl] + A.kap * us) * inv;
    T lu = A.kap * lF[a] + extra[a];
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

// Reverse of coupling iteration k for design point m: dJ/dkappa^ref_m += ..., and the point's
// contribution to dJ/ds^(k-1) added to v: (xG[3], uG[3], theta, omega) about one axis, or
// (xG[3], uG[3], omega[3], R[9]) with free rotation. Called by all LN lanes of the point (each
// takes one row, or in 3D one plane, of the support window; every thread of the warp must call it);
// lane 0 finishes the point. Design points outside the design domain do nothing. Returns false if
// the support window left the body box.
template <typename T, int D, int AX, bool COHERENT>
__device__ __forceinline__ bool adj_design_point(const Geo& g, const T* __restrict__ kref, const T* scratch,
                                                 const Dof& sk, const int (&lo)[3], int m, bool valid_m, int lane,
                                                 const T (&lF)[3], const T (&lT)[3], double* __restrict__ dkref,
                                                 T* v) {
  const long long BC = g.box_cells;
  const int mm = valid_m ? m : 0;
  const int ix = mm % g.nd[0], iy = (mm / g.nd[0]) % g.nd[1], iz = mm / (g.nd[0] * g.nd[1]);
  const bool valid = valid_m && dsq(ix, g.nd[0]) + dsq(iy, g.nd[1]) + dsq(iz, g.nd[2]) <= g.rad4;
  const T r[3] = {(T)ix - pivot<T>(g, 0), (T)iy - pivot<T>(g, 1), D == 3 ? (T)iz - pivot<T>(g, 2) : T(0)};
  const DofView<T> V(sk);
  T l[3], dl[3] = {T(0), T(0), T(0)}, om3[3] = {T(0), T(0), T(0)};
  const T km = kref[mm];
  T usr[3] = {T(0), T(0), T(0)}, luref[3] = {T(0), T(0), T(0)}, rotl[3] = {T(0), T(0), T(0)};
  if constexpr (AX == AX_FREE) {
    const FreeView<T> FV(sk);
    matvec3(FV.R, r, l);
    T oxl[3];
    cross3(FV.om, l, oxl);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      om3[a] = FV.om[a];
      usr[a] = V.ug[a] + oxl[a];
    }
    cross3(lT, l, rotl);
  } else {
    constexpr int b = Axes<AX>::B, c = Axes<AX>::C;
    rot<AX>(V.cs, V.sn, r, l);
    drot<AX>(V.cs, V.sn, r, dl);
#pragma unroll
    for (int a = 0; a < D; ++a) usr[a] = V.ug[a] + V.om * dl[a];
    rotl[b] = -lT[0] * l[c];
    rotl[c] = lT[0] * l[b];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) luref[a] = km * (lF[a] + rotl[a]);
  // support window: 2s cells per axis from floor(x^ref) - s + 1
  int f[3] = {0, 0, 0};
  T fr[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) V.split(a, l[a], &f[a], &fr[a]);
  const int S2 = 2 * g.s;
  // kernel weights along each axis of the window; the axis E split across the lanes only needs
  // this lane's entry (q = lane)
  constexpr int E = (D == 3) ? 2 : 1;
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
  T uref[3] = {T(0), T(0), T(0)}, slus[3] = {T(0), T(0), T(0)}, lxr[3] = {T(0), T(0), T(0)};
  T slk = T(0);
  bool inside = true;
  const int B0 = g.B[0], B1 = g.B[1], B2 = (D == 3) ? g.B[2] : 1;
  // this lane's part of the window: row q1 = lane (2D) or plane q2 = lane (3D)
#pragma unroll
  for (int u = 0; u < (D == 3 ? 4 : 1); ++u)
#pragma unroll
    for (int q0 = 0; q0 < 4; ++q0) {
      const int q1 = (D == 3) ? u : lane, q2 = (D == 3) ? lane : 0;
      if (!valid || q0 >= S2 || q1 >= S2 || (D == 3 && q2 >= S2)) continue;
      const T w0 = wv[0][q0];
      const T w1 = (E == 1) ? we : wv[1][u], dw1 = (E == 1) ? dwe : dwv[1][u];
      const T w2 = (E == 2) ? we : T(1), dw2 = (E == 2) ? dwe : T(0);
      const T W = w0 * w1 * w2;
      const T dW0 = dwv[0][q0] * w1 * w2, dW1 = w0 * dw1 * w2, dW2 = w0 * w1 * dw2;
      if (W == T(0) && dW0 == T(0) && dW1 == T(0) && dW2 == T(0)) continue;
      const int p0 = f[0] - g.s + 1 + q0 - lo[0], p1 = f[1] - g.s + 1 + q1 - lo[1];
      const int p2 = (D == 3) ? f[2] - g.s + 1 + q2 - lo[2] : 0;
      if (p0 < 0 || p0 >= B0 || p1 < 0 || p1 >= B1 || p2 < 0 || p2 >= B2) {
        inside = false;
        continue;
      }
      const long long bl = p0 + (long long)B0 * (p1 + (long long)B1 * p2);
      // scratch is read-only in a kernel of its own (neighbouring points share most of their
      // windows, so through L1); the persistent kernel rewrites it between its barriers (L2 only)
      auto ld = [&](long long i) { return COHERENT ? __ldcg(&scratch[i]) : __ldg(&scratch[i]); };
      T uk[3] = {T(0), T(0), T(0)}, lus[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int a = 0; a < D; ++a) {
        uk[a] = ld(a * BC + bl);
        lus[a] = ld((D + 1 + a) * BC + bl);
      }
      const T lk = ld(D * BC + bl);
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
  // combine the LN lanes of this point (consecutive lanes of one warp)
#pragma unroll
  for (int off = 1; off < LN; off <<= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      uref[a] += __shfl_xor_sync(0xffffffffu, uref[a], off);
      slus[a] += __shfl_xor_sync(0xffffffffu, slus[a], off);
      lxr[a] += __shfl_xor_sync(0xffffffffu, lxr[a], off);
    }
    slk += __shfl_xor_sync(0xffffffffu, slk, off);
    inside = __shfl_xor_sync(0xffffffffu, (int)inside, off) && inside;
  }
  if (!valid || lane != 0) return true;
  T Dl[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) Dl[a] = uref[a] - usr[a];
  if constexpr (AX == AX_FREE) {
    T lxD[3], DxT[3], lusr[3], lxu[3], uxo[3];
    cross3(l, Dl, lxD);
    cross3(Dl, lT, DxT);
    T dk = slk;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dk += lF[a] * Dl[a] + lT[a] * lxD[a];
      lusr[a] = -luref[a] + slus[a];
    }
    dkref[m] += (double)dk;
    cross3(l, lusr, lxu);   // lusr . (omega x l) = omega . (l x lusr)
    cross3(lusr, om3, uxo);  //                   = l . (lusr x omega)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v[i] += lxr[i];
      v[3 + i] += lusr[i];
      v[6 + i] += lxu[i];
      const T gl = lxr[i] + km * DxT[i] + uxo[i];  // dJ/d(R r_m): transform, torque lever, solid velocity
#pragma unroll
      for (int j = 0; j < 3; ++j) v[9 + 3 * i + j] += gl * r[j];
    }
    return inside;
  } else {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, ax = Axes<AX>::A;
  T dk = slk + lT[0] * (l[b] * Dl[c] - l[c] * Dl[b]);
#pragma unroll
  for (int a = 0; a < D; ++a) dk += lF[a] * Dl[a];
  dkref[m] += (double)dk;
  T lusr[3] = {T(0), T(0), T(0)}, ll[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int a = 0; a < D; ++a) lusr[a] = -luref[a] + slus[a];
  ll[b] = lT[0] * km * Dl[c];
  ll[c] = -lT[0] * km * Dl[b];
  T lth = T(0), lom = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T ddl = (a == ax) ? T(0) : -l[a];  // R'' r
    lth += (lxr[a] + ll[a]) * dl[a] + V.om * lusr[a] * ddl;
    lom += lusr[a] * dl[a];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    v[a] += lxr[a];
    v[3 + a] += lusr[a];
  }
  v[6] += lth;
  v[7] += lom;
  return inside;
  }
}

// From the transform part ls = dJ/ds^(k-1) (design-point sums): the EOM reverse of iteration
// k - 1, or for k = 1 the completed dJ/ds(t-1) and the EOM reverse of iteration N_itr of step t-1.
__device__ __forceinline__ void adj_finish(const Geo& g, int k, const double* ls, double* lam_prev, double* lamF,
                                           double* lamT, double* lam_s0) {
  if (k > 1) {
    eom_reverse(g, ls, lamF, lamT, lam_prev);
  } else {
    double lsm1[kNdofAxis];
    for (int a = 0; a < kNdofAxis; ++a) {
      lsm1[a] = lam_prev[a] + ls[a];
      lam_s0[a] = lsm1[a];
      lam_prev[a] = 0.0;
    }
    eom_reverse(g, lsm1, lamF, lamT, lam_prev);
  }
}

// adj_finish with free rotation. ls = (xG[3], uG[3], omega[3], R[9]) from the design points; the
// EOM being reversed maps e0 = s(t'-1) to ek = s^(k') (iteration k - 1 of step t, or N_itr of step
// t - 1); has_eom is false before step 1.
__device__ __forceinline__ void adj_finish_free(const Geo& g, int k, const double* ls, double* lam_prev,
                                                double* lamF, double* lamT, double* lam_s0, const Dof& e0,
                                                const Dof& ek, bool has_eom) {
  double lsf[kNdofFree];
#pragma unroll
  for (int a = 0; a < 6; ++a) lsf[a] = ls[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lsf[S_H + a] = 0.0;
    lsf[S_OM + a] = ls[6 + a];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) lsf[S_R + i] = ls[9 + i];
  if (k == 1) {
#pragma unroll
    for (int a = 0; a < kNdofFree; ++a) {
      lsf[a] += lam_prev[a];
      lam_s0[a] = lsf[a];
      lam_prev[a] = 0.0;
    }
  }
  if (has_eom) {
    eom_reverse_free(g, e0, ek, lsf, lamF, lamT, lam_prev);
  } else {
    for (int a = 0; a < 3; ++a) lamF[a] = lamT[a] = 0.0;
  }
}

// kappa^ref (Eq. brinkman_coefficient; zero outside the design domain) and the design-grid
// moments of kappa^ref.
template <typename T>
__global__ void __launch_bounds__(256) k_prep(Geo g, const double* __restrict__ gamma, double kmax, double q,
                                               T* __restrict__ kref, Moments* mom, double* partials, Ctrl* ctrl) {
  constexpr int NM = 12;  // K0, K1[3], K2p, K2s, K2[6]
  __shared__ double red[32 * NM];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  double v[NM];
#pragma unroll
  for (int a = 0; a < NM; ++a) v[a] = 0.0;
  if (m < g.ND) {
    const int i[3] = {m % g.nd[0], (m / g.nd[0]) % g.nd[1], m / (g.nd[0] * g.nd[1])};
    const bool dom = dsq(i[0], g.nd[0]) + dsq(i[1], g.nd[1]) + dsq(i[2], g.nd[2]) <= g.rad4;
    const double gm = gamma[m];
    // a non-finite design value is reported through the status word and enters the march as void
    const bool fin = isfinite(gm);
    if (!fin) atomicOr(&ctrl->prep_status, ST_NONFINITE);
    const T k = (dom && fin) ? (T)(kmax * q * gm / ((1.0 - gm) + q)) : T(0);
    kref[m] = k;
    const double kd = (double)k;
    double r[3];
    for (int a = 0; a < 3; ++a) r[a] = (a < g.dim) ? i[a] - g.xic[a] : 0.0;
    v[0] = kd;
    v[1] = kd * r[0];
    v[2] = kd * r[1];
    v[3] = kd * r[2];
    v[4] = kd * (r[g.axb] * r[g.axb] + r[g.axc] * r[g.axc]);
    v[5] = kd * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    v[6] = kd * r[0] * r[0];
    v[7] = kd * r[1] * r[1];
    v[8] = kd * r[2] * r[2];
    v[9] = kd * r[0] * r[1];
    v[10] = kd * r[0] * r[2];
    v[11] = kd * r[1] * r[2];
  }
  block_sum<NM>(v, red);
  if (threadIdx.x == 0)
    for (int a = 0; a < NM; ++a) partials[blockIdx.x * NM + a] = v[a];
  if (!last_block_done(&ctrl->count[CNT_PREP])) return;
  double s[NM];
  sum_partials<NM>(partials, gridDim.x, s, red);
  if (threadIdx.x == 0) {
    mom->K0 = s[0];
    mom->K1[0] = s[1];
    mom->K1[1] = s[2];
    mom->K1[2] = s[3];
    mom->K2p = s[4];
    mom->K2s = s[5];
    for (int a = 0; a < 6; ++a) mom->K2[a] = s[6 + a];
    ctrl->count[CNT_PREP] = 0;
  }
}

// ---- grid form ----------------------------------------------------------------------------

// Coupling iteration k of step t. The EOM of the previous iteration (k-1 of step t, or N_itr of
// step t-1) is folded into this kernel: every CTA sums that iteration's partials (double-buffered
// by the parity of the iteration index) and runs the same deterministic FP64 EOM, and CTA 0 records
// the iterate. This removes a launch and a dependent round trip per iteration; the EOM of the run's
// last iteration is k_couple_last.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, BoxCta<D>::min_blocks) k_couple(Geo g, Slots<T> S, Ctrl* ctrl, Dof* it,
                                                          const T* __restrict__ kref, const Moments* __restrict__ mom,
                                                          void* partials, long long pstride, int nparts, int k,
                                                          T* __restrict__ boxstore, int nbox, int pre, int di) {
  using PT = typename Partial<T>::type;
  constexpr int NV = nv_couple<AX>();
  constexpr int DW = (int)(sizeof(Dof) / sizeof(double));  // the iterate in 8-byte words
  static_assert(sizeof(Dof) % sizeof(double) == 0, "iterate copies by 8-byte words");
  __shared__ double red[32 * NV];
  __shared__ Dof sd[3];  // s(t-1), s^(k-1), and the previous iteration's transform iterate
  const int t = ctrl->t0 + di, base = ctrl->base, K = g.K;
  Dof* row = it + (long long)(t - 1) * (K + 1);
  const long long idx = (long long)(t - 1) * K + (k - 1);  // iteration index in the run
  PT* pin = static_cast<PT*>(partials) + ((idx - 1) & 1) * pstride;
  PT* pout = static_cast<PT*>(partials) + (idx & 1) * pstride;
  double* sdw = reinterpret_cast<double*>(sd);
  const int tid = threadIdx.x;
  if (idx > 0 && pre) {
    // k_couple_pre has finished the previous iteration into the iterate rows
    const double* g0 = reinterpret_cast<const double*>(row);
    const double* gk = reinterpret_cast<const double*>(row + (k - 1));
    if (tid < DW) {
      sdw[tid] = g0[tid];
      sdw[DW + tid] = gk[tid];
    }
  } else if (idx > 0) {
    // previous iteration kp of step tp: its EOM starts from prow[0] with the transform of
    // prow[kp - 1]; both are staged in shared memory by the block (thread 0 then reads only the
    // fields it needs, keeping its FP64 chain in registers)
    Dof* prow = (k > 1) ? row : row - (K + 1);
    const int kp = (k > 1) ? k - 1 : K;
    const double* g0 = reinterpret_cast<const double*>(prow);
    const double* gk = reinterpret_cast<const double*>(prow + (kp - 1));
    if (tid < DW) {
      sdw[tid] = g0[tid];
      sdw[2 * DW + tid] = gk[tid];
    }
    Moments m;
    if (tid < 32) m = *mom;
    double sm[NV];
    block_sum_partials<NV>(pin, nparts, sm, red);  // its barriers order the staging copies
    int st = 0;
    if constexpr (AX == AX_FREE) {
      if (tid == 0) couple_finish_any<D, AX>(g, &m, sd[0], sd[2], sm, &sd[1], &st);
    } else {
      if (tid < 32) st = couple_finish_lanes<D, AX>(g, m, sd[0], sd[2], sm, &sd[1], tid);
    }
    __syncthreads();
    if (k == 1 && tid < DW) sdw[tid] = sdw[DW + tid];  // s(t-1) is the new iterate
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
      if (tid == 0 && st) ctrl->status |= st;
      double* o1 = reinterpret_cast<double*>(prow + kp);
      double* o2 = reinterpret_cast<double*>(row);
      if (tid < DW) {
        o1[tid] = sdw[DW + tid];
        if (kp == K) o2[tid] = sdw[DW + tid];
      }
    }
  } else if (tid < DW) {
    const double* g0 = reinterpret_cast<const double*>(row);
    sdw[tid] = g0[tid];
    sdw[DW + tid] = g0[tid];
  }
  __syncthreads();
  const Dof s0 = sd[0], sk = sd[1];
  T* __restrict__ dst = slot_ptr(S, t, base);
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  T* bs = (boxstore && k == K) ? boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D : nullptr;
  const CellSlot cc = cell_slot<D>(g);
  T v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = T(0);
  couple_cell<T, D, AX>(g, kref, sk, lo, cc, dst, bs, k == K, &ctrl->status, v);
  block_sum_partial<NV, LN>(v, pout + block_linear() * NV, red);
}

// The previous iteration's finish (sum of its partials and the EOM) for coupling iteration k of
// step t, once, for grids whose CTA count makes the fused per-CTA form of k_couple (every CTA sums
// all partials: loads quadratic in the CTA count) the larger cost. Same thread count and summation
// order as the fused form, so the iterates are the same to the bit.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads) k_couple_pre(Geo g, Ctrl* ctrl, Dof* it, const Moments* __restrict__ mom,
                                                             const void* __restrict__ partials, long long pstride,
                                                             int nparts, int k, int di) {
  using PT = typename Partial<T>::type;
  constexpr int NV = nv_couple<AX>();
  __shared__ double red[32 * NV];
  const int t = ctrl->t0 + di, K = g.K;
  Dof* row = it + (long long)(t - 1) * (K + 1);
  const long long idx = (long long)(t - 1) * K + (k - 1);
  if (idx == 0) return;
  Dof* prow = (k > 1) ? row : row - (K + 1);
  const int kp = (k > 1) ? k - 1 : K;
  const PT* pin = static_cast<const PT*>(partials) + ((idx - 1) & 1) * pstride;
  if constexpr (AX == AX_FREE) {
    Dof s0, sk;
    Moments m;
    if (threadIdx.x == 0) {
      s0 = prow[0];
      sk = prow[kp - 1];
      m = *mom;
    }
    double sm[NV];
    block_sum_partials<NV>(pin, nparts, sm, red);
    if (threadIdx.x == 0) {
      Dof nx;
      int st = 0;
      couple_finish_any<D, AX>(g, &m, s0, sk, sm, &nx, &st);
      if (st) ctrl->status |= st;
      prow[kp] = nx;
      if (kp == K) row[0] = nx;
    }
  } else {
    __shared__ Dof sdd[3];  // s0, s^(kp-1), the new iterate
    finish_lanes_to<D, AX, PT, NV>(g, ctrl, mom, prow, kp - 1, pin, nparts, red, sdd, prow + kp, kp == K ? row : nullptr);
  }
}

// EOM of the last coupling iteration of the run (step t_last, iteration N_itr).
template <typename T, int D, int AX>
__global__ void __launch_bounds__(kFinishThreads, 1) k_couple_last(Geo g, Ctrl* ctrl, Dof* it,
                                                                 const Moments* __restrict__ mom,
                                                                 const void* __restrict__ partials,
                                                                 long long pstride, int nparts, int t_last) {
  using PT = typename Partial<T>::type;
  constexpr int NV = nv_couple<AX>();
  __shared__ double red[32 * NV];
  const int K = g.K;
  Dof* row = it + (long long)(t_last - 1) * (K + 1);
  const long long idx = (long long)(t_last - 1) * K + (K - 1);
  const PT* pin = static_cast<const PT*>(partials) + (idx & 1) * pstride;
  if constexpr (AX == AX_FREE) {
    Dof s0, sk;
    Moments m;
    if (threadIdx.x == 0) {
      s0 = row[0];
      sk = row[K - 1];
      m = *mom;
    }
    double sm[NV];
    block_sum_partials<NV>(pin, nparts, sm, red);
    if (threadIdx.x == 0) {
      Dof nx;
      int st = 0;
      couple_finish_any<D, AX>(g, &m, s0, sk, sm, &nx, &st);
      if (st) ctrl->status |= st;
      row[K] = nx;
      it[(long long)t_last * (K + 1)] = nx;
    }
  } else {
    __shared__ Dof sdd[3];
    finish_lanes_to<D, AX, PT, NV>(g, ctrl, mom, row, K - 1, pin, nparts, red, sdd, row + K, it + (long long)t_last * (K + 1));
  }
}

// Recompute of one step's Brinkman update from the stored iterate s^(K-1).
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, BoxCta<D>::min_blocks) k_apply(Geo g, Slots<T> S, const Ctrl* ctrl, const Dof* it,
                                                   const T* __restrict__ kref, T* __restrict__ boxstore, int nbox,
                                                   int di) {
  const int t = ctrl->t0 + di, base = ctrl->base, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[K - 1];
  T* __restrict__ dst = slot_ptr(S, t, base);
  const long long N = g.N;
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  const CellSlot cc = cell_slot<D>(g);
  const int j0 = cc.j0, j1 = cc.j1, j2 = cc.j2;
  const int px = lo[0] + j0, py = lo[1] + j1, pz = lo[2] + j2;
  long long n = 0;
  const bool ing = cell_index<D>(g, px, py, pz, n);
  const DofView<T> V(sk);
  const T d[3] = {V.rel(0, px), V.rel(1, py), D == 3 ? V.rel(2, pz) : T(0)};
  Acc<T> A;
  T rotv[3], L[3];
  gather_cell<T, D, AX>(g, kref, sk, V, d, cc.lane, cc.active && ing, A, rotv, L);
  if (!cc.active || !ing || cc.lane != 0) return;
  const T inv = T(1) / (T(1) + A.kap);
  const long long bl = j0 + (long long)g.B[0] * (j1 + (long long)g.B[1] * j2);
  T* bs = boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T us = V.ug[a] * A.phi + rotv[a];
    const T ustar = dst[(a + 1) * N + n];
    bs[a * g.box_cells + bl] = ustar;
    dst[(a + 1) * N + n] = (ustar + A.kap * us) * inv;
  }
}

template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, BoxCta<D>::min_blocks) k_adj_cell(Geo g, const Ctrl* ctrl, const Dof* it, const T* __restrict__ kref,
                                                      const T* __restrict__ boxstore, int nbox, T* Lb,
                                                      long long lstride, T* __restrict__ acc, T* __restrict__ scratch,
                                                      int k, int di) {
  const int t = ctrl->t0 - di, base = ctrl->base, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[k - 1];
  T lF[3], lT[3];
  lam_load<T>(ctrl, lF, lT);
  T* Lcur = Lb + (long long)(t & 1) * lstride;
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  const CellSlot cc = cell_slot<D>(g);
  const T* bs = boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D;
  adj_cell_work<T, D, AX>(g, kref, sk, lo, cc, bs, Lcur, acc, scratch, k, K, lF, lT);
}

template <typename T, int D, int AX>
__global__ void __launch_bounds__(kDesignBlock) k_adj_design(Geo g, Ctrl* ctrl, const Dof* it,
                                                              const T* __restrict__ kref,
                                                              const T* __restrict__ scratch,
                                                              double* __restrict__ dkref, void* partials, int k,
                                                              int di) {
  constexpr int NV = nv_design<AX>();
  __shared__ double red[32 * NV];
  const int t = ctrl->t0 - di, K = g.K;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const Dof s0 = row[0], sk = row[k - 1];
  T lF[3], lT[3];
  lam_load<T>(ctrl, lF, lT);
  int lo[3];
  box_origin<D>(g, s0, lo[0], lo[1], lo[2]);
  const int lane = threadIdx.x % LN;
  T v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = T(0);
  bool inside = true;
  // chunks of kDesignPointsPerCta points, grid-strided (the grid is capped: see design_ctas)
  for (int m0 = blockIdx.x * kDesignPointsPerCta; m0 < g.ND; m0 += gridDim.x * kDesignPointsPerCta) {
    const int m = m0 + threadIdx.x / LN;
    inside = adj_design_point<T, D, AX, false>(g, kref, scratch, sk, lo, m, m < g.ND, lane, lF, lT, dkref, v) && inside;
  }
  if (!inside) atomicOr(&ctrl->status, ST_BOX_OVERFLOW);
  block_sum_partial<NV, LN>(v, static_cast<typename Partial<T>::type*>(partials) + blockIdx.x * NV, red);
}

// Sum of the design-point partials and the EOM reverse (adj_finish, or adj_finish_free with the
// iterates of the EOM being reversed).
template <typename T, bool FREE>
__global__ void __launch_bounds__(kFinishThreads) k_design_finish(Geo g, Ctrl* ctrl, const Dof* it,
                                                                  const void* __restrict__ partials, int nparts,
                                                                  int k, int di) {
  constexpr int NV = FREE ? nv_design<AX_FREE>() : nv_design<0>();
  constexpr int NS = FREE ? kNdofFree : kNdofAxis;
  __shared__ double red[32 * NV];
  double lp[NS];  // thread 0 fetches the carried adjoint (and the EOM's iterates) before the reduction
  Dof e0, ek;
  bool has_eom = true;
  if (threadIdx.x == 0) {
    for (int a = 0; a < NS; ++a) lp[a] = ctrl->lam_prev[a];
    if (FREE) {
      const int t = ctrl->t0 - di, K = g.K;
      const int te = (k > 1) ? t : t - 1, ke = (k > 1) ? k - 1 : K;
      has_eom = te >= 1;
      if (has_eom) {
        const Dof* row = it + (long long)(te - 1) * (K + 1);
        e0 = row[0];
        ek = row[ke];
      }
    }
  }
  double ls[NV];
  block_sum_partials<NV>(static_cast<const typename Partial<T>::type*>(partials), nparts, ls, red);
  if (threadIdx.x == 0) {
    double nF[3], nT[3];
    if constexpr (FREE)
      adj_finish_free(g, k, ls, lp, nF, nT, ctrl->lam_s0, e0, ek, has_eom);
    else
      adj_finish(g, k, ls, lp, nF, nT, ctrl->lam_s0);
    for (int a = 0; a < NS; ++a) ctrl->lam_prev[a] = lp[a];
    lam_store(ctrl, nF, nT);
  }
}

// ---- small kernels ------------------------------------------------------------------------

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
    const bool free_rot = g.ax == AX_FREE;
    for (int a = 0; a < kNdofFree; ++a) d.s[a] = (a < g.ns) ? s0[a] : 0.0;
    d.cs = free_rot ? 1.0 : cos(d.s[6]);
    d.sn = free_rot ? 0.0 : sin(d.s[6]);
    dof_views(&d, free_rot);
    it[0] = d;
    ctrl->t0 = 1;
    ctrl->base = 0;
    ctrl->status = 0;
  }
}

__global__ void k_set_step(Ctrl* ctrl, int t0, int base) {
  ctrl->t0 = t0;
  ctrl->base = base;
}

// Seed of the reverse sweep: dJ/ds(N_t) = seed * w, then the EOM reverse of iteration N_itr of
// step N_t (free rotation: from the iterates it[N_t - 1][0] and it[N_t - 1][N_itr]).
__global__ void k_adj_init(Geo g, Ctrl* ctrl, const Dof* it, int nt, const double* objw, double seed,
                           const double* term_s) {
  double ls[kNdofFree], lp[kNdofFree], nF[3], nT[3];
  for (int a = 0; a < kNdofFree; ++a) {
    ls[a] = (a < g.ns) ? seed * objw[a] + (term_s ? term_s[a] : 0.0) : 0.0;
    lp[a] = 0.0;
  }
  if (g.ax == AX_FREE) {
    const Dof* row = it + (long long)(nt - 1) * (g.K + 1);
    eom_reverse_free(g, row[0], row[g.K], ls, nF, nT, lp);
  } else {
    eom_reverse(g, ls, nF, nT, lp);
  }
  for (int a = 0; a < kNdofFree; ++a) ctrl->lam_prev[a] = lp[a];
  lam_store(ctrl, nF, nT);
}

__global__ void k_sensitivity(int nd, const double* __restrict__ gamma, const double* __restrict__ dkref, double kmax,
                              double q, double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nd) return;
  const double den = (1.0 - gamma[m]) + q;
  out[m] = dkref[m] * kmax * q * (1.0 + q) / (den * den);
}

template <typename T>
__global__ void k_ckpt_pack(Geo g, Slots<T> S, T* ckpt, long long cstride, int every, const Ctrl* ctrl, int di) {
  const int tn = ctrl->t0 + di;
  const T* src = slot_ptr(S, tn, ctrl->base);
  T* dst = ckpt + (long long)(tn / every) * cstride;
  const long long M = (long long)(g.dim + 1) * g.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// ---- persistent (cooperative) coupling ---------------------------------------------------------
//
// One launch per time step runs all N_itr coupling iterations (forward) or their reverse. Its CTAs
// are co-resident (cooperative launch) and stride over the box tiles in a fixed assignment, so
// every cell is handled by the same thread in every iteration; they meet at a grid barrier after
// each iteration's per-CTA partial sums, after which every CTA sums the partials in the same fixed
// order and runs the same FP64 EOM (or its reverse) on thread 0, so all CTAs hold the same iterate
// without a second barrier. The partials are double-buffered by the parity of the iteration: a
// buffer is rewritten only two barriers after it was read.

constexpr unsigned long long kSyncTimeoutNs = 1000000000ull;  // one second

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on one 32-bit word, sense-reversing: CTA 0 adds 2^31 - (G - 1) and every other CTA
// adds 1, so the top bit flips exactly when the last of the G CTAs arrives and the low bits are
// zero again for the next barrier. Each waiting CTA polls with acquire loads; the fence before the
// arrival publishes the CTA's writes (ordered before it by the block barrier). Every wait is
// bounded: after kSyncTimeoutNs, or as soon as another CTA has given up, the CTA sets
// ST_SYNC_TIMEOUT and the call returns false, on which the kernel must return. skip (a test hook)
// makes CTA 0 not arrive, so that the other CTAs' waits run out.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* status, bool skip) {
  __shared__ int sync_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned G = gridDim.x * gridDim.y * gridDim.z;
    const bool first = block_linear() == 0;
    const unsigned inc = first ? 0x80000000u - (G - 1u) : 1u;
    __threadfence();
    const unsigned old = (first && skip) ? ld_acquire_gpu(bar) : atomicAdd(bar, inc);
    const unsigned long long t0 = globaltimer_ns();
    int ok = 1;
    while (((ld_acquire_gpu(bar) ^ old) & 0x80000000u) == 0u) {
      if (*(volatile int*)status & ST_SYNC_TIMEOUT) {
        ok = 0;
        break;
      }
      if (globaltimer_ns() - t0 > kSyncTimeoutNs) {
        atomicOr(status, ST_SYNC_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
    sync_ok = ok;
  }
  __syncthreads();
  return sync_ok != 0;
}

// Forward: the N_itr coupling iterations of step t and the EOM of the last one.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, BoxCta<D>::min_blocks)
    k_couple_coop(Geo g, Slots<T> S, Ctrl* ctrl, Dof* it, const T* __restrict__ kref, const Moments* __restrict__ mom,
                  void* partials, long long pstride, T* __restrict__ boxstore, int nbox, int di) {
  using PT = typename Partial<T>::type;
  constexpr int NV = nv_couple<AX>();
  constexpr int DW = (int)(sizeof(Dof) / sizeof(double));
  __shared__ double red[32 * NV];
  __shared__ Dof sd[3];  // s(t-1), the current iterate s^(k-1), the next iterate
  if (*(volatile int*)&ctrl->status & ST_SYNC_TIMEOUT) return;  // an earlier launch gave up
  const int t = ctrl->t0 + di, base = ctrl->base, K = g.K;
  const bool skip = (ctrl->sync_skip & 1) != 0;
  Dof* row = it + (long long)(t - 1) * (K + 1);
  double* sdw = reinterpret_cast<double*>(sd);
  const int tid = threadIdx.x;
  if (tid < DW) {
    const double* g0 = reinterpret_cast<const double*>(row);
    sdw[tid] = g0[tid];
    sdw[DW + tid] = g0[tid];
  }
  __syncthreads();
  T* __restrict__ dst = slot_ptr(S, t, base);
  int lo[3];
  box_origin<D>(g, sd[0], lo[0], lo[1], lo[2]);
  T* bs = boxstore ? boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D : nullptr;
  const dim3 bg = box_grid(g);
  const int ntiles = (int)(bg.x * bg.y * bg.z);
  const int G = (int)gridDim.x;
  for (int k = 1; k <= K; ++k) {
    const Dof sk = sd[1];
    T v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = T(0);
    for (int tile = blockIdx.x; tile < ntiles; tile += G) {
      const CellSlot cc = cell_slot_tile<D>(g, tile, bg.x, bg.y);
      couple_cell<T, D, AX>(g, kref, sk, lo, cc, dst, k == K ? bs : nullptr, k == K, &ctrl->status, v);
    }
    PT* part = static_cast<PT*>(partials) + (k & 1) * pstride;
    block_sum_partial<NV, LN>(v, part + blockIdx.x * NV, red);
    if (!grid_sync(&ctrl->sync_bar, &ctrl->status, skip)) return;
    if (k == K && blockIdx.x != 0) return;  // the last EOM is needed only for the DOF history
    Moments m;
    if (tid < 32) m = *mom;
    double sm[NV];
    block_sum_partials<NV>(part, G, sm, red);
    if constexpr (AX == AX_FREE) {
      if (tid == 0) {
        int st = 0;
        couple_finish_any<D, AX>(g, &m, sd[0], sd[1], sm, &sd[2], &st);
        if (st && blockIdx.x == 0) atomicOr(&ctrl->status, st);
      }
    } else if (tid < 32) {
      const int st = couple_finish_lanes<D, AX>(g, m, sd[0], sd[1], sm, &sd[2], tid);
      if (tid == 0 && st && blockIdx.x == 0) atomicOr(&ctrl->status, st);
    }
    __syncthreads();
    if (tid < DW) {
      sdw[DW + tid] = sdw[2 * DW + tid];
      if (blockIdx.x == 0) {
        reinterpret_cast<double*>(row + k)[tid] = sdw[2 * DW + tid];
        if (k == K) reinterpret_cast<double*>(row + K + 1)[tid] = sdw[2 * DW + tid];  // s(t): the next step's row 0
      }
    }
    __syncthreads();
  }
}

// Reverse: for k = N_itr..1 the cell phase (Brinkman and interpolation reverse), a barrier, the
// design-point phase (spread and transform reverse, dJ/dkappa^ref, per-CTA partials of dJ/ds^(k-1)),
// a barrier, then in every CTA the sum of the partials and the EOM reverse of the previous iteration
// (adj_finish), whose dJ/dF, dJ/dT the next cell phase uses. CTA 0 stores the carried adjoint.
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads, 1)
    k_adj_coop(Geo g, Ctrl* ctrl, const Dof* it, const T* __restrict__ kref, const T* __restrict__ boxstore, int nbox,
               T* Lb, long long lstride, T* __restrict__ acc, T* __restrict__ scratch, double* __restrict__ dkref,
               void* partials, long long pstride, int di) {
  using PT = typename Partial<T>::type;
  constexpr bool FREE = AX == AX_FREE;
  constexpr int NV = nv_design<AX>();
  constexpr int NS = FREE ? kNdofFree : kNdofAxis;
  constexpr int PPC = BoxCta<D>::threads / LN;  // design points per CTA pass
  __shared__ double red[32 * NV];
  // thread 0's FP64 finish works in shared memory (kept out of every thread's registers): the
  // carried adjoint dJ/ds(t-1), dJ/ds(0) at step 1, dJ/dF and dJ/dT of the iteration to reverse
  // next, and with free rotation the two iterates of the EOM being reversed
  __shared__ double s_lp[NS], s_ls0[NS], slam[6];
  __shared__ Dof s_e[FREE ? 2 : 1];
  if (*(volatile int*)&ctrl->status & ST_SYNC_TIMEOUT) return;
  const int t = ctrl->t0 - di, base = ctrl->base, K = g.K;
  const bool skip = (ctrl->sync_skip & 1) != 0;
  const Dof* row = it + (long long)(t - 1) * (K + 1);
  const int tid = threadIdx.x, lane = tid % LN;
  T lF[3], lT[3];
  lam_load<T>(ctrl, lF, lT);
  if (tid < NS) {
    s_lp[tid] = ctrl->lam_prev[tid];
    s_ls0[tid] = 0.0;
  }
  if (tid < 6) slam[tid] = 0.0;
  T* Lcur = Lb + (long long)(t & 1) * lstride;
  int lo[3];
  box_origin<D>(g, row[0], lo[0], lo[1], lo[2]);
  const T* bs = boxstore + (long long)((t - base - 1) % nbox) * g.box_cells * D;
  const dim3 bg = box_grid(g);
  const int ntiles = (int)(bg.x * bg.y * bg.z);
  const int G = (int)gridDim.x;
  for (int k = K; k >= 1; --k) {
    const Dof sk = row[k - 1];
    for (int tile = blockIdx.x; tile < ntiles; tile += G) {
      const CellSlot cc = cell_slot_tile<D>(g, tile, bg.x, bg.y);
      adj_cell_work<T, D, AX>(g, kref, sk, lo, cc, bs, Lcur, acc, scratch, k, K, lF, lT);
    }
    if (!grid_sync(&ctrl->sync_bar, &ctrl->status, skip)) return;
    T v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = T(0);
    bool inside = true;
    // each CTA an equal contiguous share of the design points, PPC at a time
    const int share = (g.ND + G - 1) / G, mb = blockIdx.x * share, me = min(g.ND, mb + share);
    for (int m0 = mb; m0 < me; m0 += PPC) {
      const int m = m0 + tid / LN;
      inside = adj_design_point<T, D, AX, true>(g, kref, scratch, sk, lo, m, m < me, lane, lF, lT, dkref, v) && inside;
    }
    if (!inside) atomicOr(&ctrl->status, ST_BOX_OVERFLOW);
    PT* part = static_cast<PT*>(partials) + (k & 1) * pstride;
    block_sum_partial<NV, LN>(v, part + blockIdx.x * NV, red);
    if (!grid_sync(&ctrl->sync_bar, &ctrl->status, skip)) return;
    const int te = (k > 1) ? t : t - 1, ke = (k > 1) ? k - 1 : K;
    if constexpr (FREE) {
      constexpr int DW = (int)(sizeof(Dof) / sizeof(double));
      if (te >= 1 && tid < DW) {  // the EOM being reversed maps s(te - 1) to iterate ke of step te
        const Dof* erow = it + (long long)(te - 1) * (K + 1);
        reinterpret_cast<double*>(&s_e[0])[tid] = reinterpret_cast<const double*>(erow)[tid];
        reinterpret_cast<double*>(&s_e[1])[tid] = reinterpret_cast<const double*>(erow + ke)[tid];
      }
    }
    double ls[NV];
    block_sum_partials<NV>(static_cast<const PT*>(part), G, ls, red);  // its barriers order the staging
    if (tid == 0) {
      if constexpr (FREE)
        adj_finish_free(g, k, ls, s_lp, slam, slam + 3, s_ls0, s_e[0], s_e[FREE ? 1 : 0], te >= 1);
      else
        adj_finish(g, k, ls, s_lp, slam, slam + 3, s_ls0);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lF[a] = (T)slam[a];
      lT[a] = (T)slam[3 + a];
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    for (int a = 0; a < NS; ++a) {
      ctrl->lam_prev[a] = s_lp[a];
      ctrl->lam_s0[a] = s_ls0[a];
    }
    lam_store(ctrl, slam, slam + 3);
  }
}

// ---- index sets of the spread (test export) -------------------------------------------------

// Per box cell: the number of design points the gather accepts, the least and largest of their
// linear indices, and the sums of the indices and of their squares.
struct SetStats {
  long long c, lo, hi, s1, s2;
};
struct StatVisit {
  SetStats* st;
  __device__ __forceinline__ void operator()(int m) const {
    st->c += 1;
    st->lo = min(st->lo, (long long)m);
    st->hi = max(st->hi, (long long)m);
    st->s1 += m;
    st->s2 += (long long)m * m;
  }
};

// The box of the iterate s (the box a step starting from s would use), gathered as the coupling
// gathers it, recording the accepted index sets into out[box cell][5].
template <typename T, int D, int AX>
__global__ void __launch_bounds__(BoxCta<D>::threads) k_support_sets(Geo g, Dof s, const T* __restrict__ kref,
                                                                     long long* __restrict__ out) {
  int lo[3];
  box_origin<D>(g, s, lo[0], lo[1], lo[2]);
  const CellSlot cc = cell_slot<D>(g);
  const int px = lo[0] + cc.j0, py = lo[1] + cc.j1, pz = lo[2] + cc.j2;
  const DofView<T> V(s);
  const T d[3] = {V.rel(0, px), V.rel(1, py), D == 3 ? V.rel(2, pz) : T(0)};
  SetStats st{0, LLONG_MAX, -1, 0, 0};
  Acc<T> A;
  if constexpr (AX == AX_FREE) {
    const FreeView<T> FV(s);
    gather_free_lanes<T, LN>(g, kref, d, FV.R, cc.lane, cc.active, A, StatVisit{&st});
  } else {
    gather_lanes<T, D, AX, LN>(g, kref, d, V.cs, V.sn, cc.lane, cc.active, A, StatVisit{&st});
  }
#pragma unroll
  for (int off = 1; off < LN; off <<= 1) {
    st.c += __shfl_xor_sync(0xffffffffu, st.c, off);
    st.lo = min(st.lo, __shfl_xor_sync(0xffffffffu, st.lo, off));
    st.hi = max(st.hi, __shfl_xor_sync(0xffffffffu, st.hi, off));
    st.s1 += __shfl_xor_sync(0xffffffffu, st.s1, off);
    st.s2 += __shfl_xor_sync(0xffffffffu, st.s2, off);
  }
  if (!cc.active || cc.lane != 0) return;
  const long long bl = cc.j0 + (long long)g.B[0] * (cc.j1 + (long long)g.B[1] * cc.j2);
  out[5 * bl + 0] = st.c;
  out[5 * bl + 1] = st.c ? st.lo : -1;
  out[5 * bl + 2] = st.hi;
  out[5 * bl + 3] = st.s1;
  out[5 * bl + 4] = st.s2;
}

}  // namespace

template <typename T>
void launch_couple_coop(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                        void* partials, long long pstride, T* boxstore, int nbox, int di, cudaStream_t st) {
  const dim3 grid((unsigned)g.coop_fwd), block((unsigned)box_threads(g));
  if (g.dim == 2)
    launch_coop(k_couple_coop<T, 2, 2>, grid, block, 0, st, g, S, ctrl, it, kref, mom, partials, pstride, boxstore,
                nbox, di);
  else if (g.ax == 0)
    launch_coop(k_couple_coop<T, 3, 0>, grid, block, 0, st, g, S, ctrl, it, kref, mom, partials, pstride, boxstore,
                nbox, di);
  else if (g.ax == 1)
    launch_coop(k_couple_coop<T, 3, 1>, grid, block, 0, st, g, S, ctrl, it, kref, mom, partials, pstride, boxstore,
                nbox, di);
  else if (g.ax == 2)
    launch_coop(k_couple_coop<T, 3, 2>, grid, block, 0, st, g, S, ctrl, it, kref, mom, partials, pstride, boxstore,
                nbox, di);
  else
    launch_coop(k_couple_coop<T, 3, AX_FREE>, grid, block, 0, st, g, S, ctrl, it, kref, mom, partials, pstride,
                boxstore, nbox, di);
}

template <typename T>
void launch_adj_coop(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, double* dkref, void* partials, long long pstride, int di,
                     cudaStream_t st) {
  const dim3 grid((unsigned)g.coop_adj), block((unsigned)box_threads(g));
  if (g.dim == 2)
    launch_coop(k_adj_coop<T, 2, 2>, grid, block, 0, st, g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc, scratch,
                dkref, partials, pstride, di);
  else if (g.ax == 0)
    launch_coop(k_adj_coop<T, 3, 0>, grid, block, 0, st, g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc, scratch,
                dkref, partials, pstride, di);
  else if (g.ax == 1)
    launch_coop(k_adj_coop<T, 3, 1>, grid, block, 0, st, g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc, scratch,
                dkref, partials, pstride, di);
  else if (g.ax == 2)
    launch_coop(k_adj_coop<T, 3, 2>, grid, block, 0, st, g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc, scratch,
                dkref, partials, pstride, di);
  else
    launch_coop(k_adj_coop<T, 3, AX_FREE>, grid, block, 0, st, g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc,
                scratch, dkref, partials, pstride, di);
}

namespace {
// CTAs of a persistent kernel: the box tiles, at most as many as the device holds at once (0 if
// the query fails or none fits).
template <typename K>
int coop_ctas(const Geo& g, K kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, box_threads(g), 0) != cudaSuccess) return 0;
  const dim3 bg = box_grid(g);
  const long long ntiles = (long long)bg.x * bg.y * bg.z;
  const long long cap = (long long)per_sm * sms;
  return (int)(ntiles < cap ? ntiles : cap);
}
template <typename T, int D, int AX>
void coop_setup(Geo* g) {
  g->coop_fwd = coop_ctas(*g, k_couple_coop<T, D, AX>);
  g->coop_adj = coop_ctas(*g, k_adj_coop<T, D, AX>);
}
template <typename T>
void coop_setup_any(Geo* g) {
  if (g->dim == 2) coop_setup<T, 2, 2>(g);
  else if (g->ax == 0) coop_setup<T, 3, 0>(g);
  else if (g->ax == 1) coop_setup<T, 3, 1>(g);
  else if (g->ax == 2) coop_setup<T, 3, 2>(g);
  else coop_setup<T, 3, AX_FREE>(g);
}
}  // namespace

void setup_coop(Geo* g, bool fp64) {
  if (fp64)
    coop_setup_any<double>(g);
  else
    coop_setup_any<float>(g);
  cudaGetLastError();  // an occupancy query that failed leaves the per-iteration kernels in use
}

template <typename T>
void launch_support_sets(const Geo& g, const Dof& s, const T* kref, long long* out, cudaStream_t st) {
  LKS_BOX_DISPATCH(k_support_sets, box_grid(g), box_threads(g), g, s, kref, out);
}

template <typename T>
void launch_prep(const Geo& g, const double* gamma, double kappa_max, double q, T* kref, Moments* mom,
                 double* partials, Ctrl* ctrl, cudaStream_t st) {
  launch(k_prep<T>, (g.ND + 255) / 256, 256, 0, st, g, gamma, kappa_max, q, kref, mom, partials, ctrl);
}

template <typename T>
void launch_couple(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                   void* partials, long long pstride, int k, T* boxstore, int nbox, int di, cudaStream_t st) {
  const dim3 grid = box_grid(g);
  const int nparts = (int)(grid.x * grid.y * grid.z);
  const int pre = nparts > kFusedFinishMaxParts ? 1 : 0;
  if (pre)
    LKS_BOX_DISPATCH(k_couple_pre, 1, box_threads(g), g, ctrl, it, mom, (const void*)partials, pstride, nparts, k, di);
  LKS_BOX_DISPATCH(k_couple, grid, box_threads(g), g, S, ctrl, it, kref, mom, partials, pstride, nparts, k, boxstore,
                   nbox, pre, di);
}

int couple_kernels(const Geo& g) {
  const dim3 grid = box_grid(g);
  return (int)(grid.x * grid.y * grid.z) > kFusedFinishMaxParts ? 2 : 1;
}

template <typename T>
void launch_couple_last(const Geo& g, Ctrl* ctrl, Dof* it, const Moments* mom, const void* partials,
                        long long pstride, int t_last, cudaStream_t st) {
  const dim3 grid = box_grid(g);
  const int nparts = (int)(grid.x * grid.y * grid.z);
  LKS_BOX_DISPATCH(k_couple_last, 1, kFinishThreads, g, ctrl, it, mom, partials, pstride, nparts, t_last);
}

template <typename T>
void launch_apply(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, const Dof* it, const T* kref, T* boxstore,
                  int nbox, int di, cudaStream_t st) {
  LKS_BOX_DISPATCH(k_apply, box_grid(g), box_threads(g), g, S, ctrl, it, kref, boxstore, nbox, di);
}

template <typename T>
void launch_adj_cell(const Geo& g, const Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, int k, int di, cudaStream_t st) {
  LKS_BOX_DISPATCH(k_adj_cell, box_grid(g), box_threads(g), g, ctrl, it, kref, boxstore, nbox, Lb, lstride, acc,
                   scratch, k, di);
}

template <typename T>
void launch_adj_design(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* scratch, double* dkref,
                       void* partials, int k, int di, cudaStream_t st) {
  const unsigned nb = (unsigned)design_ctas(g);
  LKS_BOX_DISPATCH(k_adj_design, nb, kDesignBlock, g, ctrl, it, kref, scratch, dkref, partials, k, di);
  if (g.ax == AX_FREE)
    launch(k_design_finish<T, true>, 1, kFinishThreads, 0, st, g, ctrl, it, (const void*)partials, (int)nb, k, di);
  else
    launch(k_design_finish<T, false>, 1, kFinishThreads, 0, st, g, ctrl, it, (const void*)partials, (int)nb, k, di);
}

template <typename T>
void launch_init_forward(const Geo& g, const Slots<T>& S, const double* p0, const double* u0, const double* s0dev,
                         Dof* it, Ctrl* ctrl, cudaStream_t st) {
  const long long nb = (g.N + 255) / 256;
  launch(k_init_forward<T>, (unsigned)(nb < 4096 ? nb : 4096), 256, 0, st, g, S, p0, u0, s0dev, it, ctrl);
}

void launch_set_step(Ctrl* ctrl, int t0, int base, cudaStream_t st) { launch(k_set_step, 1, 1, 0, st, ctrl, t0, base); }

void launch_adj_init(const Geo& g, Ctrl* ctrl, const Dof* it, int nt, const double* objw, double seed,
                     const double* term_s, double* dkref, int nd, cudaStream_t st) {
  cudaMemsetAsync(dkref, 0, sizeof(double) * (size_t)nd, st);
  launch(k_adj_init, 1, 1, 0, st, g, ctrl, it, nt, objw, seed, term_s);
}

void launch_sensitivity(const Geo& g, const double* gamma, const double* dkref, double kappa_max, double q,
                        double* out, cudaStream_t st) {
  launch(k_sensitivity, (g.ND + 255) / 256, 256, 0, st, g.ND, gamma, dkref, kappa_max, q, out);
}

template <typename T>
void launch_ckpt_pack(const Geo& g, const Slots<T>& S, T* ckpt, long long cstride, int every, const Ctrl* ctrl, int di,
                      cudaStream_t st) {
  const long long M = (long long)(g.dim + 1) * g.N;
  const long long nb = (M + 255) / 256;
  launch(k_ckpt_pack<T>, (unsigned)(nb < 8192 ? nb : 8192), 256, 0, st, g, S, ckpt, cstride, every, ctrl, di);
}

#define LKS_INST(T)                                                                                                 \
  template void launch_prep<T>(const Geo&, const double*, double, double, T*, Moments*, double*, Ctrl*,              \
                               cudaStream_t);                                                                       \
  template void launch_couple<T>(const Geo&, const Slots<T>&, Ctrl*, Dof*, const T*, const Moments*, void*,          \
                                 long long, int, T*, int, int, cudaStream_t);                                       \
  template void launch_couple_last<T>(const Geo&, Ctrl*, Dof*, const Moments*, const void*, long long, int,          \
                                      cudaStream_t);                                                                \
  template void launch_apply<T>(const Geo&, const Slots<T>&, const Ctrl*, const Dof*, const T*, T*, int, int,        \
                                cudaStream_t);                                                                      \
  template void launch_adj_cell<T>(const Geo&, const Ctrl*, const Dof*, const T*, const T*, int, T*, long long, T*, \
                                   T*, int, int, cudaStream_t);                                                     \
  template void launch_adj_design<T>(const Geo&, Ctrl*, const Dof*, const T*, const T*, double*, void*, int, int,    \
                                     cudaStream_t);                                                                 \
  template void launch_init_forward<T>(const Geo&, const Slots<T>&, const double*, const double*, const double*,     \
                                       Dof*, Ctrl*, cudaStream_t);                                                  \
  template void launch_ckpt_pack<T>(const Geo&, const Slots<T>&, T*, long long, int, const Ctrl*, int, cudaStream_t); \
  template void launch_support_sets<T>(const Geo&, const Dof&, const T*, long long*, cudaStream_t);             \
  template void launch_couple_coop<T>(const Geo&, const Slots<T>&, Ctrl*, Dof*, const T*, const Moments*, void*,     \
                                      long long, T*, int, int, cudaStream_t);                                       \
  template void launch_adj_coop<T>(const Geo&, Ctrl*, const Dof*, const T*, const T*, int, T*, long long, T*, T*,    \
                                   double*, void*, long long, int, cudaStream_t);

LKS_INST(float)
LKS_INST(double)

}  // namespace lks
