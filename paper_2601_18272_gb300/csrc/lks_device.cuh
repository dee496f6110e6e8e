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
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lks {

enum { BC_PERIODIC = 0, BC_INFLOW_OUTFLOW = 1, BC_WALL = 2, BC_PRESSURE = 3 };
enum { W_COS4 = 0, W_BILINEAR = 1 };
enum { DOF_TX = 1, DOF_TY = 2, DOF_TZ = 4, DOF_ROT = 8 };
enum { CKQ_BF16 = 1, CKQ_FP16 = 2 };  // reduced-precision checkpoint formats
enum { ST_BODY_OUTSIDE = 1, ST_NONFINITE = 2, ST_BOX_OVERFLOW = 4 };
enum { CNT_COUPLE = 0, CNT_APPLY = 1, CNT_DESIGN = 2, CNT_ADJ_STENCIL = 3, CNT_PREP = 4, CNT_CKPT = 5, CNT_N = 8 };

// One DOF iterate: s = (xG[3], uG[3], theta, omega) plus cos/sin theta, and FP32 views of what the
// per-cell kernels need (written once per iterate by dof_views, so that FP32 kernels do no FP64
// arithmetic: GB300 issues FP64 at a small fraction of the FP32 rate).
struct Dof {
  double s[8];
  double cs, sn;
  int xi[3];    // floor(x^G)
  float xf[3];  // x^G - floor(x^G)
  float ug[3];  // u^G
  float om, csf, snf;
};

__host__ __device__ inline void dof_views(Dof* d) {
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
  int pad;
  unsigned count[CNT_N];  // last-block counters, one per kernel family
  double lam_prev[8];     // adjoint: direct EOM part of dJ/ds(t-1)
  double lam_F[3];        // adjoint: dJ/dF of the iteration being reversed
  double lam_T;           // adjoint: dJ/dT
  double lam_s0[8];       // adjoint: dJ/ds(0) after the sweep
  float lam_Ff[3], lam_Tf;  // FP32 copies of lam_F, lam_T
};

// Design-grid moments used by the closed-form design-side force and torque terms.
struct Moments {
  double K0;        // sum kappa_m
  double K1[3];     // sum kappa_m r_m
  double K2p;       // sum kappa_m |r_m perp|^2 (perpendicular to the rotation axis)
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
  int ax, axb, axc;
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

// Gather (Eqs. kappa_mapping, us_mapping) for the cell at d = x_n - x^G under rotation (cs, sn)
// about AX. Candidates: the design points whose rotated position lies in the axis-aligned support
// square of the cell; in the design frame they lie within s (|cos| + |sin|) of the cell's image.
template <typename F, int D, int AX>
__device__ __forceinline__ void gather(const Geo& g, const F* __restrict__ kref, const F (&d)[3], F cs, F sn,
                                       Acc<F>& o) {
  constexpr int b = Axes<AX>::B, c = Axes<AX>::C, ax = Axes<AX>::A;
  const F S = (F)g.s;
  const F xib = cs * d[b] + sn * d[c] + pivot<F>(g, b);
  const F xic = -sn * d[b] + cs * d[c] + pivot<F>(g, c);
  const F h = S * (fabs(cs) + fabs(sn));
  const int ib0 = max(0, (int)ceil(xib - h)), ib1 = min(g.nd[b] - 1, (int)floor(xib + h));
  const int ic0 = max(0, (int)ceil(xic - h)), ic1 = min(g.nd[c] - 1, (int)floor(xic + h));
  int ia0 = 0, ia1 = 0;
  F xia = F(0);
  if (D == 3) {
    xia = d[ax] + pivot<F>(g, ax);
    const int fa = (int)floor(xia);
    ia0 = max(0, fa - g.s + 1);
    ia1 = min(g.nd[ax] - 1, fa + g.s);
  }
  o.phi = o.kap = F(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) o.wr[a] = o.kr[a] = F(0);
  const int sx = 1, sy = g.nd[0], sz = g.nd[0] * g.nd[1];
  const int sb = (b == 0) ? sx : (b == 1 ? sy : sz);
  const int sc = (c == 0) ? sx : (c == 1 ? sy : sz);
  const int sa = (ax == 0) ? sx : (ax == 1 ? sy : sz);
  // For a candidate row ib, both rotated offsets are linear in ec = ic - xic:
  //   x^ref - x_n along b: cs eb - sn ec,  along c: sn eb + cs ec.
  // Bound the column loop by the interval where both lie in (-S, S), widened slightly; the exact
  // acceptance test below still decides.
  const F tiny = F(1e-6), pad = F(1e-3);
  const F ics = fabs(cs) > tiny ? F(1) / cs : F(0), isn = fabs(sn) > tiny ? F(1) / sn : F(0);
  for (int ib = ib0; ib <= ib1; ++ib) {
    const F eb = (F)ib - xib;
    F elo = -F(1e30), ehi = F(1e30);
    if (isn != F(0)) {  // |cs eb - sn ec| < S
      const F e1 = (cs * eb - S) * isn, e2 = (cs * eb + S) * isn;
      elo = fmax(elo, fmin(e1, e2));
      ehi = fmin(ehi, fmax(e1, e2));
    } else if (fabs(cs * eb) >= S + pad) {
      continue;
    }
    if (ics != F(0)) {  // |sn eb + cs ec| < S
      const F e1 = (-S - sn * eb) * ics, e2 = (S - sn * eb) * ics;
      elo = fmax(elo, fmin(e1, e2));
      ehi = fmin(ehi, fmax(e1, e2));
    } else if (fabs(sn * eb) >= S + pad) {
      continue;
    }
    elo = fmax(elo, F(-1e6));
    ehi = fmin(ehi, F(1e6));
    const int jc0 = max(ic0, (int)ceil(xic + elo - pad)), jc1 = min(ic1, (int)floor(xic + ehi + pad));
    for (int ic = jc0; ic <= jc1; ++ic) {
      const F ec = (F)ic - xic;
      const F ob = cs * eb - sn * ec;  // x^ref_m - x_n along b
      const F oc = sn * eb + cs * ec;
      if (fabs(ob) >= S || fabs(oc) >= S) continue;
      const F w2 = wfun(g.wk, ob) * wfun(g.wk, oc);
      const F rb = (F)ib - pivot<F>(g, b), rc = (F)ic - pivot<F>(g, c);
      const int m2 = ib * sb + ic * sc;
      if (D == 2) {
        const F wkap = w2 * kref[m2];
        o.phi += w2;
        o.kap += wkap;
        o.wr[b] += w2 * rb;
        o.wr[c] += w2 * rc;
        o.kr[b] += wkap * rb;
        o.kr[c] += wkap * rc;
      } else {
        for (int ia = ia0; ia <= ia1; ++ia) {
          const F oa = (F)ia - xia;
          if (fabs(oa) >= S) continue;
          const F W = w2 * wfun(g.wk, oa);
          const F wkap = W * kref[m2 + ia * sa];
          const F ra = (F)ia - pivot<F>(g, ax);
          o.phi += W;
          o.kap += wkap;
          o.wr[b] += W * rb;
          o.wr[c] += W * rc;
          o.wr[ax] += W * ra;
          o.kr[b] += wkap * rb;
          o.kr[c] += wkap * rc;
          o.kr[ax] += wkap * ra;
        }
      }
    }
  }
}

// The same gather split over LANES consecutive threads of a warp: lane j takes candidate rows
// ib0 + j, ib0 + j + LANES, ...; the sums are combined with shuffles so every lane ends with the
// cell's totals.
template <typename F, int D, int AX, int LANES>
__device__ __forceinline__ void gather_lanes(const Geo& g, const F* __restrict__ kref, const F (&d)[3], F cs, F sn,
                                             int lane, bool active, Acc<F>& o) {
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
  if (D == 3) {
    xia = d[ax] + pivot<F>(g, ax);
    const int fa = (int)floor(xia);
    ia0 = max(0, fa - g.s + 1);
    ia1 = min(g.nd[ax] - 1, fa + g.s);
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
    for (int ic = jc0; ic <= jc1; ++ic) {
      const F ec = (F)ic - xic;
      const F ob = cs * eb - sn * ec;
      const F oc = sn * eb + cs * ec;
      if (fabs(ob) >= S || fabs(oc) >= S) continue;
      const F w2 = wfun(g.wk, ob) * wfun(g.wk, oc);
      const F rc = (F)ic - pivot<F>(g, c);
      const int m2 = ib * sb + ic * sc;
      if (D == 2) {
        const F wkap = w2 * kref[m2];
        o.phi += w2;
        o.kap += wkap;
        o.wr[b] += w2 * rb;
        o.wr[c] += w2 * rc;
        o.kr[b] += wkap * rb;
        o.kr[c] += wkap * rc;
      } else {
        for (int ia = ia0; ia <= ia1; ++ia) {
          const F oa = (F)ia - xia;
          if (fabs(oa) >= S) continue;
          const F W = w2 * wfun(g.wk, oa);
          const F wkap = W * kref[m2 + ia * sa];
          const F ra = (F)ia - pivot<F>(g, ax);
          o.phi += W;
          o.kap += wkap;
          o.wr[b] += W * rb;
          o.wr[c] += W * rc;
          o.wr[ax] += W * ra;
          o.kr[b] += wkap * rb;
          o.kr[c] += wkap * rc;
          o.kr[ax] += wkap * ra;
        }
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
// thread 0. Requires blockDim a multiple of 32 and <= 1024; smem >= 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double* v, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
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

// Fixed-order block tree of NV double-float pairs (shuffles within warps, then warp 0 over the
// warps' results); the total is in thread 0's (hi, lo). Requires blockDim a multiple of 32 and
// smem >= 32 * NV doubles. All threads of the block must call it.
template <int NV>
__device__ __forceinline__ void block_df_tree(float (&hi)[NV], float (&lo)[NV], double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float bh = __shfl_xor_sync(0xffffffffu, hi[i], off), bl = __shfl_xor_sync(0xffffffffu, lo[i], off);
      df_add(hi[i], lo[i], bh, bl);
    }
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
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const float bh = __shfl_xor_sync(0xffffffffu, hi[i], off), bl = __shfl_xor_sync(0xffffffffu, lo[i], off);
        df_add(hi[i], lo[i], bh, bl);
      }
  }
}

// Block sum of NV per-thread FP32 values as double-float pairs, written by thread 0 to out[0..NV).
template <int NV>
__device__ __forceinline__ void block_sum_partial(float (&v)[NV], float2* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  float hi[NV], lo[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    hi[i] = v[i];
    lo[i] = 0.0f;
  }
  block_df_tree<NV>(hi, lo, smem);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = make_float2(hi[i], lo[i]);
}
template <int NV>
__device__ __forceinline__ void block_sum_partial(double (&v)[NV], double* out, double* smem) {
  block_sum<NV>(v, smem);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) out[i] = v[i];
}

// The block sums the partials [nblocks][NV] in a fixed order (thread-strided, then the fixed
// block tree); the FP64 result is in thread 0. Double-float pairs are summed with FP32
// instructions only.
template <int NV>
__device__ __forceinline__ void block_sum_partials(const float2* partials, int nblocks, double* out, double* smem) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  float hi[NV], lo[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) hi[a] = lo[a] = 0.0f;
#pragma unroll 4
  for (int q = tid; q < nblocks; q += nthreads)
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      const float2 p = __ldcg(&partials[q * NV + a]);
      df_add(hi[a], lo[a], p.x, p.y);
    }
  block_df_tree<NV>(hi, lo, smem);
  if (tid == 0)
#pragma unroll
    for (int a = 0; a < NV; ++a) out[a] = (double)hi[a] + (double)lo[a];
}
template <int NV>
__device__ __forceinline__ void block_sum_partials(const double* partials, int nblocks, double* out, double* smem) {
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
  for (int a = 0; a < 8; ++a) out->s[a] = s0.s[a];
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
  dof_views(out);
}

// Reverse of eom_update: from dJ/ds^(k) give dJ/dF, dJ/dT and add the direct part to dJ/ds(t-1).
__device__ __forceinline__ void eom_reverse(const Geo& g, const double* lam_sk, double* lamF, double* lamT,
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
  if (g.dof_mask & DOF_ROT) {
    const double lom = lam_sk[7] + lam_sk[6];
    *lamT = lom * g.inv_inertia;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lom;
  } else {
    *lamT = 0.0;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lam_sk[7];
  }
}

}  // namespace lks
