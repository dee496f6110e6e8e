// Device-side types and helpers shared by the LKS kernels (sm_103a).
//
// Data layout in HBM
//   state slot   : (dim + 1) planes of N = nx*ny*nz values of T (p, u_x, u_y[, u_z]), x fastest
//   slot ring    : slot(t) = base_ptr + ((t - base) mod nslots) * slot_stride; ping-pong (2 slots)
//                  for the checkpointed forward, a segment of k+1 slots for recompute, N_t+1
//                  slots for the store-all form
//   body box     : the cells a body can touch during one step, a box of B[0]*B[1]*B[2] cells
//                  placed from x^G(t-1) (unwrapped coordinates, wrapped on periodic axes)
//   DOF iterates : Dof it[(t-1)*(K+1) + k], k = 0..K, s^(0) = s(t-1), s^(K) = s(t)  (FP64)
//   DOF vector   : (xG[3], uG[3], theta, omega) about one axis, or with free rotation
//                  (xG[3], uG[3], h[3], omega[3], R[9] row-major)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lks {

enum { BC_PERIODIC = 0, BC_INFLOW_OUTFLOW = 1, BC_WALL = 2, BC_PRESSURE = 3 };
enum { W_COS4 = 0, W_BILINEAR = 1 };
enum { DOF_TX = 1, DOF_TY = 2, DOF_TZ = 4, DOF_ROT = 8 };
enum { CKQ_BF16 = 1, CKQ_FP16 = 2 };  // reduced-precision checkpoint formats
enum { ST_BODY_OUTSIDE = 1, ST_NONFINITE = 2, ST_BOX_OVERFLOW = 4, ST_SYNC_TIMEOUT = 8 };
enum { CNT_COUPLE = 0, CNT_APPLY = 1, CNT_DESIGN = 2, CNT_ADJ_STENCIL = 3, CNT_PREP = 4, CNT_CKPT = 5, CNT_N = 8 };
// Rotation modes (the AX template argument of the body kernels): 0, 1, 2 = one axis; free rotation.
constexpr int AX_FREE = 3;
constexpr int kNdofAxis = 8, kNdofFree = 21;
// DOF-vector offsets with free rotation
constexpr int S_H = 6, S_OM = 9, S_R = 12;

// One DOF iterate: s plus cos/sin theta, and FP32 views of what the per-cell kernels need
// (written once per iterate by dof_views, so that FP32 kernels do no FP64 arithmetic: GB300 issues
// FP64 at a small fraction of the FP32 rate). With free rotation Rf and omf view R and omega.
struct Dof {
  double s[kNdofFree];
  double cs, sn;
  int xi[3];    // floor(x^G)
  float xf[3];  // x^G - floor(x^G)
  float ug[3];  // u^G
  float om, csf, snf;
  float Rf[9], omf[3];
};

__host__ __device__ inline void dof_views(Dof* d, bool free_rot) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double fl = floor(d->s[a]);
    d->xi[a] = (int)fl;
    d->xf[a] = (float)(d->s[a] - fl);
    d->ug[a] = (float)d->s[3 + a];
  }
  d->om = (float)d->s[7];
  d->csf = (float)d->cs;
  d->snf = (float)d->sn;
  if (free_rot) {
#pragma unroll
    for (int i = 0; i < 9; ++i) d->Rf[i] = (float)d->s[S_R + i];
#pragma unroll
    for (int a = 0; a < 3; ++a) d->omf[a] = (float)d->s[S_OM + a];
  }
}

// Per-thread view of an iterate in the field type T: FP32 fields read the FP32 views, FP64 fields
// the FP64 values.
template <typename T>
struct DofView;
template <>
struct DofView<float> {
  float cs, sn, om, ug[3], xf[3];
  int xi[3];
  __device__ __forceinline__ explicit DofView(const Dof& d) : cs(d.csf), sn(d.snf), om(d.om) {
    for (int a = 0; a < 3; ++a) {
      ug[a] = d.ug[a];
      xf[a] = d.xf[a];
      xi[a] = d.xi[a];
    }
  }
  // x_a - x^G_a for integer position p
  __device__ __forceinline__ float rel(int a, int p) const { return (float)(p - xi[a]) - xf[a]; }
  // x^G_a + off split as (integer cell, fraction in [0, 1))
  __device__ __forceinline__ void split(int a, float off, int* cell, float* frac) const {
    const float v = xf[a] + off, fl = floorf(v);
    *cell = xi[a] + (int)fl;
    *frac = v - fl;
  }
};
template <>
struct DofView<double> {
  double cs, sn, om, ug[3], x[3];
  __device__ __forceinline__ explicit DofView(const Dof& d) : cs(d.cs), sn(d.sn), om(d.s[7]) {
    for (int a = 0; a < 3; ++a) {
      ug[a] = d.s[3 + a];
      x[a] = d.s[a];
    }
  }
  __device__ __forceinline__ double rel(int a, int p) const { return (double)p - x[a]; }
  __device__ __forceinline__ void split(int a, double off, int* cell, double* frac) const {
    const double v = x[a] + off, fl = floor(v);
    *cell = (int)fl;
    *frac = v - fl;
  }
};

// Device control block (one per handle). The step a kernel works on is t0 + di (forward) or
// t0 - di (adjoint), with di baked into each captured launch, so one graph serves every chunk.
struct Ctrl {
  int t0;                 // forward: first step of the chunk; adjoint: last step of the chunk
  int base;               // step held in slot 0 of the resident segment
  int status;             // ST_* bits
  int prep_status;        // ST_NONFINITE if the design field held a NaN or an infinity (k_prep)
  unsigned sync_bar;      // grid barrier word of the cooperative coupling kernels (grid_sync)
  int sync_skip;          // test hooks: bit 0 makes CTA 0 skip its grid-barrier arrivals, bit 1 makes the
                          // row-streamed 3D stencils withhold one plane's copy (the waits time out)
  unsigned count[CNT_N];  // last-block counters, one per kernel family
  double lam_prev[kNdofFree];  // adjoint: direct EOM part of dJ/ds(t-1)
  double lam_F[3];        // adjoint: dJ/dF of the iteration being reversed
  double lam_T[3];        // adjoint: dJ/dT (about the axis in [0], or the vector with free rotation)
  double lam_s0[kNdofFree];  // adjoint: dJ/ds(0) after the sweep
  float lam_Ff[3], lam_Tf[3];  // FP32 copies of lam_F, lam_T
  // the paper-form adjoint (ALKS): body multipliers (x~G[3], u~G[3], theta~, omega~) of the step
  // last finished, and its u~G[3], omega~ of fixed-point iterations N_itr - 1 and N_itr
  double al_b[8];
  double al_it[8];
  float al_itf[8];  // FP32 copies of al_it
};

// Design-grid moments used by the closed-form design-side force and torque terms.
struct Moments {
  double K0;        // sum kappa_m
  double K1[3];     // sum kappa_m r_m
  double K2p;       // sum kappa_m |r_m perp|^2 (perpendicular to the rotation axis)
  double K2s;       // sum kappa_m |r_m|^2
  double K2[6];     // sum kappa_m r_m r_m^T: xx, yy, zz, xy, xz, yz
};

// Problem constants passed by value to every kernel.
struct Geo {
  int dim;
  int n[3];
  long long N;
  int bc[3];
  int nd[3];
  int ND;
  double xic[3];  // design pivot xi^G
  float xicf[3];  // FP32 copy of the pivot
  int ax, axb, axc;  // rotation axis and its plane; ax = AX_FREE with free rotation
  int ns;            // DOF vector length
  int rad4;          // design domain: 4|r_m|^2 <= rad4 (an integer test; INT_MAX for the whole grid)
  double Jinv[9];    // free rotation: I_b^-1
  double frad, pbeta, peta;  // design chain: filter radius, projection steepness and threshold
  int cyc;           // design chain: cyclic expansion order (1: none)
  int dof_mask;
  int wk, s;      // weight kind, support half-width (2 for cos4, 1 for bilinear)
  int K;          // N_itr
  double A, u_in, dp, mass, inertia;
  double inv_mass, inv_inertia;  // 1/M, 1/I (the EOM multiplies: FP64 division is a long sequence)
  float A2;       // 2A, for FP32 kernels
  int B[3];       // body box extent in cells
  int hb[3];      // box half extent (ceil of the body's half extent)
  int margin;     // cells of drift allowed within one step
  long long box_cells;
  int coop_fwd, coop_adj;  // CTAs of the cooperative coupling kernels (0: the per-iteration kernels)
};

// State slots.
template <typename T>
struct Slots {
  T* base;
  long long stride;  // elements per slot
  int nslots;
};

template <typename T>
__device__ __forceinline__ T* slot_ptr(const Slots<T>& S, int t, int base) {
  int i = t - base;
  i %= S.nslots;
  if (i < 0) i += S.nslots;
  return S.base + (long long)i * S.stride;
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Grid-separation weight w(r) (Sec. 2.3, Eq. weight_function read as (1 + cos(pi r / 2)) / 4 on
// |r| < 2), or bilinear 1 - |r| on |r| < 1; both evaluated only inside the support.
// FP32 uses the SFU intrinsics (absolute error about 4e-7 on (-pi, pi)); FP64 uses cospi / sinpi.
__device__ __forceinline__ float wfun(int wk, float r) {
  if (wk == W_BILINEAR) return 1.0f - fabsf(r);
  return 0.25f * (1.0f + __cosf(1.57079632679f * r));
}
__device__ __forceinline__ double wfun(int wk, double r) {
  if (wk == W_BILINEAR) return 1.0 - fabs(r);
  return 0.25 * (1.0 + cospi(0.5 * r));
}
// dw/dr inside the support; the bilinear kink at r = 0 takes the r >= 0 branch.
__device__ __forceinline__ float dwfun(int wk, float r) {
  if (wk == W_BILINEAR) return r >= 0.0f ? -1.0f : 1.0f;
  return -0.392699081699f * __sinf(1.57079632679f * r);
}
__device__ __forceinline__ double dwfun(int wk, double r) {
  if (wk == W_BILINEAR) return r >= 0.0 ? -1.0 : 1.0;
  return -0.125 * 3.141592653589793 * sinpi(0.5 * r);
}

// Design pivot component in the arithmetic type.
template <typename F>
__device__ __forceinline__ F pivot(const Geo& g, int a);
template <>
__device__ __forceinline__ float pivot<float>(const Geo& g, int a) { return g.xicf[a]; }
template <>
__device__ __forceinline__ double pivot<double>(const Geo& g, int a) { return g.xic[a]; }

// Rotation axis AX (compile time) and its in-plane axes, right-handed: (B, C) = (AX+1, AX+2) mod 3.
template <int AX>
struct Axes {
  static constexpr int A = AX, B = (AX + 1) % 3, C = (AX + 2) % 3;
};

// Box origin (unwrapped coordinates) for the step that starts from s(t-1).
template <int D>
__device__ __forceinline__ void box_origin(const Geo& g, const Dof& s0, int& lx, int& ly, int& lz) {
  lx = s0.xi[0] - g.hb[0] - g.s - g.margin;
  ly = s0.xi[1] - g.hb[1] - g.s - g.margin;
  lz = (D == 3) ? s0.xi[2] - g.hb[2] - g.s - g.margin : 0;
}

// Wrapped grid index of the unwrapped position (px, py, pz); false if it lies outside the grid on
// a non-periodic axis.
template <int D>
__device__ __forceinline__ bool cell_index(const Geo& g, int px, int py, int pz, long long& n) {
  int qx = px, qy = py, qz = 0;
  if (g.bc[0] == BC_PERIODIC) {
    qx = wrapi(px, g.n[0]);
  } else if (px < 0 || px >= g.n[0]) {
    return false;
  }
  if (g.bc[1] == BC_PERIODIC) {
    qy = wrapi(py, g.n[1]);
  } else if (py < 0 || py >= g.n[1]) {
    return false;
  }
  if (D == 3) {
    qz = pz;
    if (g.bc[2] == BC_PERIODIC) {
      qz = wrapi(pz, g.n[2]);
    } else if (pz < 0 || pz >= g.n[2]) {
      return false;
    }
  }
  n = (long long)qx + (long long)g.n[0] * ((long long)qy + (long long)g.n[1] * (long long)qz);
  return true;
}

// Cells within two of a non-periodic boundary plane may not be touched by the body.
template <int D>
__device__ __forceinline__ bool forbidden(const Geo& g, int px, int py, int pz) {
  if (g.bc[0] != BC_PERIODIC && (px < 2 || px > g.n[0] - 3)) return true;
  if (g.bc[1] != BC_PERIODIC && (py < 2 || py > g.n[1] - 3)) return true;
  if (D == 3 && g.bc[2] != BC_PERIODIC && (pz < 2 || pz > g.n[2] - 3)) return true;
  return false;
}

// Sums over the design points m within the kernel support of one analysis cell:
//   phi = sum W, kap = sum W kappa_m, wr = sum W r_m, kr = sum W kappa_m r_m   (r in design frame)
template <typename F>
struct Acc {
  F phi, kap;
  F wr[3], kr[3];
};

// Design-domain test on the doubled offset 2 r_m = 2 i - (nd - 1), exact in integers:
// 4 |r_m|^2 <= rad4.
__device__ __forceinline__ int dsq(int i, int nd) {
  const int e = 2 * i - (nd - 1);
  return e * e;
}

// Visitor of the design points a gather accepts (their linear indices); the default does nothing,
// a test export records the accepted index sets.
struct NoVisit {
  __device__ __forceinline__ void operator()(int) const {}
};

// Gather (Eqs. kappa_mapping, us_mapping) for the cell at d = x_n - x^G under rotation (cs, sn)
// about AX, split over LANES consecutive threads of a warp. Candidates: the design points of the
// design domain whose rotated position lies in the axis-aligned support square of the cell; in the
// design frame they lie within s (|cos| + |sin|) of the cell's image. Lane j takes candidate rows
// ib0 + j, ib0 + j + LANES, ...; the sums are combined with shuffles so every lane ends with the
// cell's totals.
template <typename F, int D, int AX, int LANES, typename Visit = NoVisit>
__device__ __forceinline__ void gather_lanes(const Geo& g, const F* __restrict__ kref, const F (&d)[3], F cs, F sn,
                                             int lane, bool active, Acc<F>& o, Visit visit = Visit()) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, ax = Axes<AX>::A;
  const F S = (F)g.s;
  const F xib = cs * d[b] + sn * d[c] + pivot<F>(g, b);
  const F xic = -sn * d[b] + cs * d[c] + pivot<F>(g, c);
  const F h = S * (fabs(cs) + fabs(sn));
  int ib0 = max(0, (int)ceil(xib - h)), ib1 = min(g.nd[b] - 1, (int)floor(xib + h));
  const int ic0 = max(0, (int)ceil(xic - h)), ic1 = min(g.nd[c] - 1, (int)floor(xic + h));
  if (!active) ib1 = ib0 - 1;
  int ia0 = 0, ia1 = 0;
  F xia = F(0);
  // 3D: the axial factor of W, its offset and the axial domain term depend only on ia, at most 2s of
  // them per cell: computed once here, not once per in-plane candidate
  F wa[4] = {F(0), F(0), F(0), F(0)}, ra[4] = {F(0), F(0), F(0), F(0)};
  int qa[4] = {0, 0, 0, 0};
  bool va[4] = {false, false, false, false};
  if (D == 3) {
    xia = d[ax] + pivot<F>(g, ax);
    const int fa = (int)floor(xia);
    ia0 = max(0, fa - g.s + 1);
    ia1 = min(g.nd[ax] - 1, fa + g.s);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int ia = ia0 + q;
      const F oa = (F)ia - xia;
      va[q] = ia <= ia1 && fabs(oa) < S;
      if (va[q]) {
        wa[q] = wfun(g.wk, oa);
        ra[q] = (F)ia - pivot<F>(g, ax);
        qa[q] = dsq(ia, g.nd[ax]);
      }
    }
  }
  o.phi = o.kap = F(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) o.wr[a] = o.kr[a] = F(0);
  const int sx = 1, sy = g.nd[0], sz = g.nd[0] * g.nd[1];
  const int sb = (b == 0) ? sx : (b == 1 ? sy : sz);
  const int sc = (c == 0) ? sx : (c == 1 ? sy : sz);
  const int sa = (ax == 0) ? sx : (ax == 1 ? sy : sz);
  const F tiny = F(1e-6), pad = F(1e-3);
  const F ics = fabs(cs) > tiny ? F(1) / cs : F(0), isn = fabs(sn) > tiny ? F(1) / sn : F(0);
  for (int ib = ib0 + lane; ib <= ib1; ib += LANES) {
    const F eb = (F)ib - xib;
    F elo = -F(1e30), ehi = F(1e30);
    if (isn != F(0)) {
      const F e1 = (cs * eb - S) * isn, e2 = (cs * eb + S) * isn;
      elo = fmax(elo, fmin(e1, e2));
      ehi = fmin(ehi, fmax(e1, e2));
    } else if (fabs(cs * eb) >= S + pad) {
      continue;
    }
    if (ics != F(0)) {
      const F e1 = (-S - sn * eb) * ics, e2 = (S - sn * eb) * ics;
      elo = fmax(elo, fmin(e1, e2));
      ehi = fmin(ehi, fmax(e1, e2));
    } else if (fabs(sn * eb) >= S + pad) {
      continue;
    }
    elo = fmax(elo, F(-1e6));
    ehi = fmin(ehi, F(1e6));
    const int jc0 = max(ic0, (int)ceil(xic + elo - pad)), jc1 = min(ic1, (int)floor(xic + ehi + pad));
    const F rb = (F)ib - pivot<F>(g, b);
    const int qb = dsq(ib, g.nd[b]);
    for (int ic = jc0; ic <= jc1; ++ic) {
      const F ec = (F)ic - xic;
      const F ob = cs * eb - sn * ec;
      const F oc = sn * eb + cs * ec;
      if (fabs(ob) >= S || fabs(oc) >= S) continue;
      const int qbc = qb + dsq(ic, g.nd[c]);
      if (D == 2 && qbc > g.rad4) continue;
      const F w2 = wfun(g.wk, ob) * wfun(g.wk, oc);
      const F rc = (F)ic - pivot<F>(g, c);
      const int m2 = ib * sb + ic * sc;
      if (D == 2) {
        visit(m2);
        const F wkap = w2 * kref[m2];
        o.phi += w2;
        o.kap += wkap;
        o.wr[b] += w2 * rb;
        o.wr[c] += w2 * rc;
        o.kr[b] += wkap * rb;
        o.kr[c] += wkap * rc;
      } else {
        // sums over this candidate's axial column, then the in-plane weight once
        F s1 = F(0), s0 = F(0), s2 = F(0), s3 = F(0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (!va[q] || qbc + qa[q] > g.rad4) continue;
          visit(m2 + (ia0 + q) * sa);
          const F wk = wa[q] * kref[m2 + (ia0 + q) * sa];
          s1 += wa[q];
          s0 += wk;
          s2 += wa[q] * ra[q];
          s3 += wk * ra[q];
        }
        const F w1 = w2 * s1, wk0 = w2 * s0;
        o.phi += w1;
        o.kap += wk0;
        o.wr[b] += w1 * rb;
        o.wr[c] += w1 * rc;
        o.wr[ax] += w2 * s2;
        o.kr[b] += wk0 * rb;
        o.kr[c] += wk0 * rc;
        o.kr[ax] += w2 * s3;
      }
    }
  }
#pragma unroll
  for (int off = 1; off < LANES; off <<= 1) {
    o.phi += __shfl_xor_sync(0xffffffffu, o.phi, off);
    o.kap += __shfl_xor_sync(0xffffffffu, o.kap, off);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (D == 2 && a == ax) continue;
      o.wr[a] += __shfl_xor_sync(0xffffffffu, o.wr[a], off);
      o.kr[a] += __shfl_xor_sync(0xffffffffu, o.kr[a], off);
    }
  }
}

// Gather with free rotation: R (row-major, FP32 or FP64 like the cell) maps design offsets to the
// world. The support cube |x^ref_m - x_n|_a < s of the cell, pulled back to the design frame, is the
// cube R^T [-s, s]^3 around the cell's image xi = R^T d + xi^G; its bounding box has half extents
// s sum_a |R_ab|. Rows (iy, iz) of that box are split over the lanes; within a row the three world
// offsets are linear in ix, which bounds ix to the interval where all three lie in (-s, s)
// (widened slightly; the exact test decides).
template <typename F, int LANES, typename Visit = NoVisit>
__device__ __forceinline__ void gather_free_lanes(const Geo& g, const F* __restrict__ kref, const F (&d)[3],
                                                  const F (&R)[9], int lane, bool active, Acc<F>& o,
                                                  Visit visit = Visit()) {
  const F S = (F)g.s;
  F xi[3];
  int lo[3], hi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    xi[b] = R[b] * d[0] + R[3 + b] * d[1] + R[6 + b] * d[2] + pivot<F>(g, b);
    const F h = S * (fabs(R[b]) + fabs(R[3 + b]) + fabs(R[6 + b]));
    lo[b] = max(0, (int)ceil(xi[b] - h));
    hi[b] = min(g.nd[b] - 1, (int)floor(xi[b] + h));
  }
  o.phi = o.kap = F(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) o.wr[a] = o.kr[a] = F(0);
  const int nyr = hi[1] - lo[1] + 1, nzr = hi[2] - lo[2] + 1;
  const int nrows = (active && nyr > 0 && nzr > 0) ? nyr * nzr : 0;
  const F tiny = F(1e-6), pad = F(1e-3);
  F inv[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) inv[a] = fabs(R[3 * a]) > tiny ? F(1) / R[3 * a] : F(0);
  const int sy = g.nd[0], sz = g.nd[0] * g.nd[1];
  for (int q = lane; q < nrows; q += LANES) {
    const int iy = lo[1] + q % nyr, iz = lo[2] + q / nyr;
    const int qyz = dsq(iy, g.nd[1]) + dsq(iz, g.nd[2]);
    if (qyz > g.rad4) continue;
    const F ey = (F)iy - xi[1], ez = (F)iz - xi[2];
    F cw[3];  // world offset of the row at ix = xi_x
    F elo = -F(1e30), ehi = F(1e30);
    bool empty = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cw[a] = R[3 * a + 1] * ey + R[3 * a + 2] * ez;
      if (inv[a] != F(0)) {
        const F e1 = (-S - cw[a]) * inv[a], e2 = (S - cw[a]) * inv[a];
        elo = fmax(elo, fmin(e1, e2));
        ehi = fmin(ehi, fmax(e1, e2));
      } else if (fabs(cw[a]) >= S + pad) {
        empty = true;
      }
    }
    if (empty) continue;
    elo = fmax(elo, F(-1e6));
    ehi = fmin(ehi, F(1e6));
    const int jx0 = max(lo[0], (int)ceil(xi[0] + elo - pad)), jx1 = min(hi[0], (int)floor(xi[0] + ehi + pad));
    const F ry = (F)iy - pivot<F>(g, 1), rz = (F)iz - pivot<F>(g, 2);
    const int mrow = iy * sy + iz * sz;
    for (int ix = jx0; ix <= jx1; ++ix) {
      const F ex = (F)ix - xi[0];
      const F o0 = R[0] * ex + cw[0], o1 = R[3] * ex + cw[1], o2 = R[6] * ex + cw[2];
      if (fabs(o0) >= S || fabs(o1) >= S || fabs(o2) >= S || qyz + dsq(ix, g.nd[0]) > g.rad4) continue;
      visit(mrow + ix);
      const F W = wfun(g.wk, o0) * wfun(g.wk, o1) * wfun(g.wk, o2);
      const F wkap = W * kref[mrow + ix];
      const F rx = (F)ix - pivot<F>(g, 0);
      o.phi += W;
      o.kap += wkap;
      o.wr[0] += W * rx;
      o.wr[1] += W * ry;
      o.wr[2] += W * rz;
      o.kr[0] += wkap * rx;
      o.kr[1] += wkap * ry;
      o.kr[2] += wkap * rz;
    }
  }
#pragma unroll
  for (int off = 1; off < LANES; off <<= 1) {
    o.phi += __shfl_xor_sync(0xffffffffu, o.phi, off);
    o.kap += __shfl_xor_sync(0xffffffffu, o.kap, off);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      o.wr[a] += __shfl_xor_sync(0xffffffffu, o.wr[a], off);
      o.kr[a] += __shfl_xor_sync(0xffffffffu, o.kr[a], off);
    }
  }
}

// Small 3-vector / 3x3 helpers (row-major matrices).
template <typename F>
__device__ __forceinline__ void cross3(const F* a, const F* b, F* out) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}
template <typename F>
__device__ __forceinline__ void matvec3(const F* M, const F* v, F* out) {
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
}
template <typename F>
__device__ __forceinline__ void matTvec3(const F* M, const F* v, F* out) {
#pragma unroll
  for (int j = 0; j < 3; ++j) out[j] = M[j] * v[0] + M[3 + j] * v[1] + M[6 + j] * v[2];
}

// R r and R' r = d(R r)/d theta for the rotation about AX.
template <int AX, typename F>
__device__ __forceinline__ void rot(F cs, F sn, const F (&r)[3], F (&out)[3]) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, a = Axes<AX>::A;
  out[b] = cs * r[b] - sn * r[c];
  out[c] = sn * r[b] + cs * r[c];
  out[a] = r[a];
}
template <int AX, typename F>
__device__ __forceinline__ void drot(F cs, F sn, const F (&r)[3], F (&out)[3]) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, a = Axes<AX>::A;
  out[b] = -sn * r[b] - cs * r[c];
  out[c] = cs * r[b] - sn * r[c];
  out[a] = F(0);
}

// Deterministic block sum of NV doubles (fixed shuffle tree, fixed warp order). Result in
// thread 0. Requires blockDim a multiple of 32 and <= 1024; smem >= 32 * NV doubles. STRIDE: only
// lanes whose index is a multiple of STRIDE hold values (the others zeros), so the warp tree skips
// the levels that would only add zeros.
template <int NV, int STRIDE = 1>
__device__ __forceinline__ void block_sum(double* v, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off >= STRIDE; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  const int warp = tid >> 5, lane = tid & 31, nw = nthreads >> 5;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) smem[warp * NV + i] = v[i];
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < NV; ++i) {
      double acc = 0.0;
      for (int w = 0; w < nw; ++w) acc += smem[w * NV + i];
      v[i] = acc;
    }
  }
  __syncthreads();
}

// Last-block election after thread 0 of every block has published the block's partial: true in
// exactly one block, which then sees all partials (read them with __ldcg). Only thread 0 fences
// and counts; no block waits on another.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
  __shared__ bool is_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    const unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == total - 1);
    if (is_last) __threadfence();
  }
  __syncthreads();
  return is_last;
}

// Double-float (two-sum) accumulation: (hi, lo) represents hi + lo exactly enough for FP64-grade
// sums while issuing only FP32 instructions (Knuth's two-sum; Dekker's renormalisation).
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  float e = (hi - (s - bb)) + (bh - bb);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

// In the elected last block: sum the per-CTA partials [nblocks][NV] with every thread (each
// thread a fixed strided subset, then the fixed block tree), so the order is deterministic and
// the L2 loads are issued in parallel. Result in thread 0. All threads of the block must call it.
template <int NV>
__device__ __forceinline__ void sum_partials(const double* partials, int nblocks, double* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  double v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = 0.0;
  for (int q = tid; q < nblocks; q += nthreads)
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] += __ldcg(&partials[q * NV + a]);
  block_sum<NV>(v, smem);
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = v[a];
}

// Per-CTA partial sums of NV values. FP32 kernels store double-float pairs (hi, lo), so neither
// they nor the one-warp finish kernels issue FP64 arithmetic; FP64 kernels store doubles.
template <typename T>
struct Partial;
template <>
struct Partial<float> {
  using type = float2;
};
template <>
struct Partial<double> {
  using type = double;
};

// Fixed-order shuffle tree of NV double-float pairs within a warp over the lanes whose index is a
// multiple of STRIDE (the other lanes hold zeros: the levels below STRIDE would only add zeros);
// lane 0 ends with the warp's total.
template <int NV, int STRIDE>
__device__ __forceinline__ void warp_df_tree(float (&hi)[NV], float (&lo)[NV]) {
#pragma unroll
  for (int off = 16; off >= STRIDE; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float bh = __shfl_xor_sync(0xffffffffu, hi[i], off), bl = __shfl_xor_sync(0xffffffffu, lo[i], off);
      df_add(hi[i], lo[i], bh, bl);
    }
}

// Fixed-order block tree of NV double-float pairs (shuffles within warps, then warp 0 over the
// warps' results); the total is in thread 0's (hi, lo). Requires blockDim a multiple of 32 and
// smem >= 32 * NV doubles. All threads of the block must call it. STRIDE as in warp_df_tree.
template <int NV, int STRIDE = 1>
__device__ __forceinline__ void block_df_tree(float (&hi)[NV], float (&lo)[NV], double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  warp_df_tree<NV, STRIDE>(hi, lo);
  float2* s2 = reinterpret_cast<float2*>(smem);
  const int warp = tid >> 5, lane = tid & 31, nw = nthreads >> 5;
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) s2[warp * NV + i] = make_float2(hi[i], lo[i]);
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      hi[i] = 0.0f;
      lo[i] = 0.0f;
      if (lane < nw) {
        hi[i] = s2[lane * NV + i].x;
        lo[i] = s2[lane * NV + i].y;
      }
    }
    warp_df_tree<NV, 1>(hi, lo);
  }
}

// Block sum of NV per-thread FP32 values as double-float pairs, written by thread 0 to out[0..NV).
// STRIDE: only lanes whose index is a multiple of STRIDE hold values (the body kernels, where one
// of the LN threads of a cell or design point does the accumulation).
template <int NV, int STRIDE = 1>
__device__ __forceinline__ void block_sum_partial(float (&v)[NV], float2* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  float hi[NV], lo[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    hi[i] = v[i];
    lo[i] = 0.0f;
  }
  block_df_tree<NV, STRIDE>(hi, lo, smem);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = make_float2(hi[i], lo[i]);
}
template <int NV, int STRIDE = 1>
__device__ __forceinline__ void block_sum_partial(double (&v)[NV], double* out, double* smem) {
  block_sum<NV, STRIDE>(v, smem);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = v[i];
}

// The block sums the partials [nblocks][NV] in a fixed order; the FP64 result is in thread 0.
// Only as many warps as one partial per lane needs take part (the partial sums are short; a
// tree over every thread of a large block costs more issue slots than the loads): warp w, lane l
// sums partials w * 32 + l + 32 W j in order, then its lanes by the shuffle tree, then warp 0 the
// W warps' totals. Double-float pairs are summed with FP32 instructions only. All threads of the
// block must call it; it starts with a block barrier (which also orders the callers' shared-memory
// staging before thread 0 reads it).
template <int NV>
__device__ __forceinline__ void block_sum_partials(const float2* partials, int nblocks, double* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int warp = tid >> 5, lane = tid & 31, nw = nthreads >> 5;
  const int W = min(nw, max(1, (nblocks + 31) / 32));
  float hi[NV], lo[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) hi[a] = lo[a] = 0.0f;
  __syncthreads();
  if (warp < W) {
#pragma unroll 4
    for (int q = warp * 32 + lane; q < nblocks; q += W * 32)
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        const float2 p = __ldcg(&partials[q * NV + a]);
        df_add(hi[a], lo[a], p.x, p.y);
      }
    warp_df_tree<NV, 1>(hi, lo);
  }
  if (W > 1) {
    float2* s2 = reinterpret_cast<float2*>(smem);
    if (warp < W && lane == 0)
#pragma unroll
      for (int a = 0; a < NV; ++a) s2[warp * NV + a] = make_float2(hi[a], lo[a]);
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        hi[a] = lane < W ? s2[lane * NV + a].x : 0.0f;
        lo[a] = lane < W ? s2[lane * NV + a].y : 0.0f;
      }
      warp_df_tree<NV, 1>(hi, lo);
    }
  }
  if (tid == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) out[a] = (double)hi[a] + (double)lo[a];
}
template <int NV>
__device__ __forceinline__ void block_sum_partials(const double* partials, int nblocks, double* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int warp = tid >> 5, lane = tid & 31, nw = nthreads >> 5;
  const int W = min(nw, max(1, (nblocks + 31) / 32));
  double v[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) v[a] = 0.0;
  __syncthreads();
  if (warp < W) {
    for (int q = warp * 32 + lane; q < nblocks; q += W * 32)
#pragma unroll
      for (int a = 0; a < NV; ++a) v[a] += __ldcg(&partials[q * NV + a]);
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], off);
  }
  if (W > 1) {
    if (warp < W && lane == 0)
#pragma unroll
      for (int a = 0; a < NV; ++a) smem[warp * NV + a] = v[a];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        v[a] = lane < W ? smem[lane * NV + a] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[a] += __shfl_xor_sync(0xffffffffu, v[a], off);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) out[a] = v[a];
}

// cos/sin of theta0 + dth from those of theta0 by the angle-addition formulas; the increment is
// one step's rotation, so a short Taylor series gives cos/sin(dth) to FP64 rounding: terms up to
// dth^8 for |dth| <= 1/64 (remainder below 1e-25), up to dth^16 for |dth| <= 1/4 (below 1e-27);
// larger increments fall back to sincos. The Horner coefficients 1/((2k-1)2k) and 1/(2k(2k+1))
// are compile-time constants, so the series is a chain of FP64 FMAs without divisions.
__device__ __forceinline__ void rotate_angle(const Dof& s0, double dth, double* cs, double* sn) {
  if (dth == 0.0) {
    *cs = s0.cs;
    *sn = s0.sn;
    return;
  }
  double c, s;
  const double adth = fabs(dth);
  if (adth <= 0.25) {
    const double x2 = dth * dth;
    // cos x = sum (-1)^k x^2k / (2k)!,  sin x = x sum (-1)^k x^2k / (2k+1)!   (Horner)
    constexpr double cc[9] = {0.0, 1.0 / 2.0, 1.0 / 12.0, 1.0 / 30.0, 1.0 / 56.0,
                              1.0 / 90.0, 1.0 / 132.0, 1.0 / 182.0, 1.0 / 240.0};
    constexpr double sc[9] = {0.0, 1.0 / 6.0, 1.0 / 20.0, 1.0 / 42.0, 1.0 / 72.0,
                              1.0 / 110.0, 1.0 / 156.0, 1.0 / 210.0, 1.0 / 272.0};
    double pc = 1.0, ps = 1.0;
    if (adth > 1.0 / 64.0) {
#pragma unroll
      for (int k = 8; k >= 5; --k) {
        pc = fma(-x2 * cc[k], pc, 1.0);
        ps = fma(-x2 * sc[k], ps, 1.0);
      }
    }
#pragma unroll
    for (int k = 4; k >= 1; --k) {
      pc = fma(-x2 * cc[k], pc, 1.0);
      ps = fma(-x2 * sc[k], ps, 1.0);
    }
    c = pc;
    s = dth * ps;
  } else {
    sincos(dth, &s, &c);
  }
  *cs = s0.cs * c - s0.sn * s;
  *sn = s0.sn * c + s0.cs * s;
}

// Explicit Euler equations of motion, velocity first (Sec. 2.4), masked by the free DOFs. All
// loops have compile-time bounds so the iterates stay in registers (a local-memory round trip
// would sit inside this single-thread FP64 chain).
template <int D>
__device__ __forceinline__ void eom_update(const Geo& g, const Dof& s0, const double* F, double T, Dof* out) {
#pragma unroll
  for (int a = 0; a < kNdofAxis; ++a) out->s[a] = s0.s[a];
#pragma unroll
  for (int a = kNdofAxis; a < kNdofFree; ++a) out->s[a] = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (!(g.dof_mask & (1 << a))) continue;
    out->s[3 + a] = s0.s[3 + a] + F[a] * g.inv_mass;
    out->s[a] = s0.s[a] + out->s[3 + a];
  }
  if (g.dof_mask & DOF_ROT) {
    out->s[7] = s0.s[7] + T * g.inv_inertia;
    out->s[6] = s0.s[6] + out->s[7];
  }
  rotate_angle(s0, out->s[6] - s0.s[6], &out->cs, &out->sn);
  dof_views(out, false);
}

// Reverse of the translational EOM: from dJ/ds^(k) give dJ/dF and add the direct part to dJ/ds(t-1).
__device__ __forceinline__ void eom_reverse_translation(const Geo& g, const double* lam_sk, double* lamF,
                                                        double* lam_prev) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool fr = (a < g.dim) && (g.dof_mask & (1 << a));
    if (fr) {
      const double lug = lam_sk[3 + a] + lam_sk[a];
      lamF[a] = lug * g.inv_mass;
      lam_prev[a] += lam_sk[a];
      lam_prev[3 + a] += lug;
    } else {
      lamF[a] = 0.0;
      lam_prev[a] += lam_sk[a];
      lam_prev[3 + a] += lam_sk[3 + a];
    }
  }
}

// Reverse of eom_update: from dJ/ds^(k) give dJ/dF, dJ/dT (about the axis, in lamT[0]) and add the
// direct part to dJ/ds(t-1).
__device__ __forceinline__ void eom_reverse(const Geo& g, const double* lam_sk, double* lamF, double* lamT,
                                            double* lam_prev) {
  eom_reverse_translation(g, lam_sk, lamF, lam_prev);
  lamT[1] = lamT[2] = 0.0;
  if (g.dof_mask & DOF_ROT) {
    const double lom = lam_sk[7] + lam_sk[6];
    lamT[0] = lom * g.inv_inertia;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lom;
  } else {
    lamT[0] = 0.0;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lam_sk[7];
  }
}

// Rodrigues' formula exp([w]x) = I + a [w]x + b [w]x^2 with a = sin t / t, b = (1 - cos t) / t^2,
// t = |w|, and the derivatives da/dx, db/dx with respect to x = t^2. For t <= 1/4 from the power
// series in x (a = sum (-x)^k / (2k+1)!, b = sum (-x)^k / (2k+2)!, terms to x^8, remainder below
// 1e-26); otherwise from the closed forms.
__device__ __forceinline__ void rod_coeffs(double x, double* a, double* b, double* da, double* db) {
  if (x <= 1.0 / 16.0) {
    // (-1)^k / (2k+1)! and (-1)^k / (2k+2)!, k = 0..8
    constexpr double ca[9] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0,
                              1.0 / 6227020800.0, -1.0 / 1307674368000.0, 1.0 / 355687428096000.0};
    constexpr double cb[9] = {1.0 / 2.0, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0,
                              -1.0 / 479001600.0, 1.0 / 87178291200.0, -1.0 / 20922789888000.0,
                              1.0 / 6402373705728000.0};
    double pa = ca[8], pb = cb[8], qa = 8.0 * ca[8], qb = 8.0 * cb[8];
#pragma unroll
    for (int k = 7; k >= 1; --k) {
      pa = fma(pa, x, ca[k]);
      pb = fma(pb, x, cb[k]);
      qa = fma(qa, x, k * ca[k]);
      qb = fma(qb, x, k * cb[k]);
    }
    *a = fma(pa, x, ca[0]);
    *b = fma(pb, x, cb[0]);
    *da = qa;
    *db = qb;
  } else {
    const double t = sqrt(x);
    double sn, cs;
    sincos(t, &sn, &cs);
    *a = sn / t;
    *b = (1.0 - cs) / x;
    *da = (t * cs - sn) / (2.0 * x * t);
    *db = (t * sn - 2.0 * (1.0 - cs)) / (2.0 * x * x);
  }
}

__device__ __forceinline__ void rod_matrix(const double* w, double a, double b, double* Q) {
  const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
  const double x = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)  // [w]x^2 = w w^T - x I
      Q[3 * i + j] = (i == j ? 1.0 : 0.0) + a * K[3 * i + j] + b * (w[i] * w[j] - (i == j ? x : 0.0));
}

// Explicit Euler EOM with free rotation (velocity first): u^G, x^G as eom_update;
// h = h(t-1) + T, omega = R0 I_b^-1 R0^T h, R = exp([omega]x) R0 with R0 = R(t-1).
__device__ __forceinline__ void eom_update_free(const Geo& g, const Dof& s0, const double* F, const double* T,
                                                Dof* out) {
#pragma unroll
  for (int a = 0; a < kNdofFree; ++a) out->s[a] = s0.s[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(g.dof_mask & (1 << a))) continue;
    out->s[3 + a] = s0.s[3 + a] + F[a] * g.inv_mass;
    out->s[a] = s0.s[a] + out->s[3 + a];
  }
  if (g.dof_mask & DOF_ROT) {
    const double* R0 = s0.s + S_R;
    double h[3], v1[3], v2[3], w[3], Q[9], a, b, da, db;
#pragma unroll
    for (int i = 0; i < 3; ++i) h[i] = s0.s[S_H + i] + T[i];
    matTvec3(R0, h, v1);
    matvec3(g.Jinv, v1, v2);
    matvec3(R0, v2, w);
    rod_coeffs(w[0] * w[0] + w[1] * w[1] + w[2] * w[2], &a, &b, &da, &db);
    rod_matrix(w, a, b, Q);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      out->s[S_H + i] = h[i];
      out->s[S_OM + i] = w[i];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        out->s[S_R + 3 * i + j] = Q[3 * i] * R0[j] + Q[3 * i + 1] * R0[3 + j] + Q[3 * i + 2] * R0[6 + j];
    }
  }
  out->cs = 1.0;
  out->sn = 0.0;
  dof_views(out, true);
}

// Reverse of eom_update_free from s0 = s(t-1) and the iterate sk = s^(k) it produced: dJ/dF,
// dJ/dT (vector) and the direct part of dJ/ds(t-1). With G = (dJ/dR) R0^T the rotation term
// phi(w) = <G, exp([w]x)> has gradient
//   2 a'(x) (w.v) w + a v + 2 b'(x) (w^T G w - x tr G) w + b ((G + G^T) w - 2 tr G w),
// v = (G21 - G12, G02 - G20, G10 - G01), x = |w|^2 (a', b' with respect to x).
__device__ __forceinline__ void eom_reverse_free(const Geo& g, const Dof& s0, const Dof& sk, const double* lam_sk,
                                                 double* lamF, double* lamT, double* lam_prev) {
  eom_reverse_translation(g, lam_sk, lamF, lam_prev);
  if (!(g.dof_mask & DOF_ROT)) {
#pragma unroll
    for (int a = S_H; a < kNdofFree; ++a) lam_prev[a] += lam_sk[a];
    lamT[0] = lamT[1] = lamT[2] = 0.0;
    return;
  }
  const double* R0 = s0.s + S_R;
  const double* h = sk.s + S_H;
  const double* w = sk.s + S_OM;
  const double* LR = lam_sk + S_R;
  const double x = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  double a, b, da, db, Q[9], G[9];
  rod_coeffs(x, &a, &b, &da, &db);
  rod_matrix(w, a, b, Q);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // R = Q R0:  dJ/dR0 += Q^T LR,  G = LR R0^T
      lam_prev[S_R + 3 * i + j] += Q[i] * LR[j] + Q[3 + i] * LR[3 + j] + Q[6 + i] * LR[6 + j];
      G[3 * i + j] = LR[3 * i] * R0[3 * j] + LR[3 * i + 1] * R0[3 * j + 1] + LR[3 * i + 2] * R0[3 * j + 2];
    }
  const double v[3] = {G[7] - G[5], G[2] - G[6], G[3] - G[1]};
  const double trG = G[0] + G[4] + G[8];
  double Gw[3], GTw[3];
  matvec3(G, w, Gw);
  matTvec3(G, w, GTw);
  const double wv = w[0] * v[0] + w[1] * v[1] + w[2] * v[2];
  const double wGw = w[0] * Gw[0] + w[1] * Gw[1] + w[2] * Gw[2];
  const double c1 = 2.0 * da * wv + 2.0 * db * (wGw - x * trG) - 2.0 * b * trG;
  double lw[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) lw[i] = lam_sk[S_OM + i] + c1 * w[i] + a * v[i] + b * (Gw[i] + GTw[i]);
  // w = R0 I_b^-1 R0^T h:  dJ/dh += R0 I_b^-1 R0^T lw,  dJ/dR0 += (lw h^T + h lw^T) R0 I_b^-1
  double p1[3], p2[3], lh[3], RJ[9];
  matTvec3(R0, lw, p1);
  matvec3(g.Jinv, p1, p2);
  matvec3(R0, p2, lh);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      RJ[3 * i + j] = R0[3 * i] * g.Jinv[j] + R0[3 * i + 1] * g.Jinv[3 + j] + R0[3 * i + 2] * g.Jinv[6 + j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int l = 0; l < 3; ++l) acc += (lw[i] * h[l] + h[i] * lw[l]) * RJ[3 * l + j];
      lam_prev[S_R + 3 * i + j] += acc;
    }
  // h = h(t-1) + T
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double lhi = lam_sk[S_H + i] + lh[i];
    lamT[i] = lhi;
    lam_prev[S_H + i] += lhi;
  }
}

}  // namespace lks
