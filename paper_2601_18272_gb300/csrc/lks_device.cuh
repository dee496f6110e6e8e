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
enum { ST_BODY_OUTSIDE = 1, ST_NONFINITE = 2, ST_BOX_OVERFLOW = 4 };
enum { CNT_COUPLE = 0, CNT_APPLY = 1, CNT_DESIGN = 2, CNT_ADJ_STENCIL = 3, CNT_PREP = 4, CNT_CKPT = 5, CNT_N = 8 };

// One DOF iterate: s = (xG[3], uG[3], theta, omega) plus cos/sin theta.
struct Dof {
  double s[8];
  double cs, sn;
};

// Device control block (one per handle).
struct Ctrl {
  int t;                  // forward: step being computed; adjoint: step being reversed
  int base;               // step held in slot 0 of the resident segment
  int status;             // ST_* bits
  int pad;
  unsigned count[CNT_N];  // last-block counters, one per kernel family
  double lam_prev[8];     // adjoint: direct EOM part of dJ/ds(t-1)
  double lam_F[3];        // adjoint: dJ/dF of the iteration being reversed
  double lam_T;           // adjoint: dJ/dT
  double lam_s0[8];       // adjoint: dJ/ds(0) after the sweep
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
  int ax, axb, axc;
  int dof_mask;
  int wk, s;      // weight kind, support half-width (2 for cos4, 1 for bilinear)
  int K;          // N_itr
  double A, u_in, dp, mass, inertia;
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
__device__ __forceinline__ float wfun(int wk, float r) {
  if (wk == W_BILINEAR) return 1.0f - fabsf(r);
  return 0.25f * (1.0f + cospif(0.5f * r));
}
__device__ __forceinline__ double wfun(int wk, double r) {
  if (wk == W_BILINEAR) return 1.0 - fabs(r);
  return 0.25 * (1.0 + cospi(0.5 * r));
}
// dw/dr inside the support; the bilinear kink at r = 0 takes the r >= 0 branch.
__device__ __forceinline__ float dwfun(int wk, float r) {
  if (wk == W_BILINEAR) return r >= 0.0f ? -1.0f : 1.0f;
  return -0.125f * 3.14159265358979f * sinpif(0.5f * r);
}
__device__ __forceinline__ double dwfun(int wk, double r) {
  if (wk == W_BILINEAR) return r >= 0.0 ? -1.0 : 1.0;
  return -0.125 * 3.141592653589793 * sinpi(0.5 * r);
}

// Rotation axis AX (compile time) and its in-plane axes, right-handed: (B, C) = (AX+1, AX+2) mod 3.
template <int AX>
struct Axes {
  static constexpr int A = AX, B = (AX + 1) % 3, C = (AX + 2) % 3;
};

// Box origin (unwrapped coordinates) for the step that starts from s(t-1).
template <int D>
__device__ __forceinline__ void box_origin(const Geo& g, const Dof& s0, int& lx, int& ly, int& lz) {
  lx = (int)floor(s0.s[0]) - g.hb[0] - g.s - g.margin;
  ly = (int)floor(s0.s[1]) - g.hb[1] - g.s - g.margin;
  lz = (D == 3) ? (int)floor(s0.s[2]) - g.hb[2] - g.s - g.margin : 0;
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
  const F xib = cs * d[b] + sn * d[c] + (F)g.xic[b];
  const F xic = -sn * d[b] + cs * d[c] + (F)g.xic[c];
  const F h = S * (fabs(cs) + fabs(sn));
  const int ib0 = max(0, (int)ceil(xib - h)), ib1 = min(g.nd[b] - 1, (int)floor(xib + h));
  const int ic0 = max(0, (int)ceil(xic - h)), ic1 = min(g.nd[c] - 1, (int)floor(xic + h));
  int ia0 = 0, ia1 = 0;
  F xia = F(0);
  if (D == 3) {
    xia = d[ax] + (F)g.xic[ax];
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
  for (int ib = ib0; ib <= ib1; ++ib) {
    const F eb = (F)ib - xib;
    for (int ic = ic0; ic <= ic1; ++ic) {
      const F ec = (F)ic - xic;
      const F ob = cs * eb - sn * ec;  // x^ref_m - x_n along b
      const F oc = sn * eb + cs * ec;
      if (fabs(ob) >= S || fabs(oc) >= S) continue;
      const F w2 = wfun(g.wk, ob) * wfun(g.wk, oc);
      const F rb = (F)ib - (F)g.xic[b], rc = (F)ic - (F)g.xic[c];
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
          const F ra = (F)ia - (F)g.xic[ax];
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

// Last-block election after every block has published its partial: true in exactly one block,
// which then sees all partials (read them with __ldcg). No block waits on another.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
  __shared__ bool is_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned total = gridDim.x * gridDim.y * gridDim.z;
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == total - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Explicit Euler equations of motion, velocity first (Sec. 2.4), masked by the free DOFs.
__device__ __forceinline__ void eom_update(const Geo& g, const Dof& s0, const double* F, double T, Dof* out) {
  for (int a = 0; a < 8; ++a) out->s[a] = s0.s[a];
  for (int a = 0; a < g.dim; ++a) {
    if (!(g.dof_mask & (1 << a))) continue;
    out->s[3 + a] = s0.s[3 + a] + F[a] / g.mass;
    out->s[a] = s0.s[a] + out->s[3 + a];
  }
  if (g.dof_mask & DOF_ROT) {
    out->s[7] = s0.s[7] + T / g.inertia;
    out->s[6] = s0.s[6] + out->s[7];
  }
  out->cs = cos(out->s[6]);
  out->sn = sin(out->s[6]);
}

// Reverse of eom_update: from dJ/ds^(k) give dJ/dF, dJ/dT and add the direct part to dJ/ds(t-1).
__device__ __forceinline__ void eom_reverse(const Geo& g, const double* lam_sk, double* lamF, double* lamT,
                                            double* lam_prev) {
  for (int a = 0; a < 3; ++a) {
    const bool fr = (a < g.dim) && (g.dof_mask & (1 << a));
    if (fr) {
      const double lug = lam_sk[3 + a] + lam_sk[a];
      lamF[a] = lug / g.mass;
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
    *lamT = lom / g.inertia;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lom;
  } else {
    *lamT = 0.0;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lam_sk[7];
  }
}

}  // namespace lks
