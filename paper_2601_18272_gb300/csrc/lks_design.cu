// Design chain (Sec. 3.2, Eqs. filter and projection; Sec. 4.2, cyclic periodic mapping) and its
// transpose, on the design grid in FP64.
//
//   gamma --(cyclic expansion)--> g1 --(density filter)--> gtil --(Heaviside projection)--> gbar
//
// Cyclic expansion (order 2 or 4): every design point takes the value of its orbit's
// representative, the smallest index among its images under rotations by 360/order degrees about
// the design-grid centre in the plane normal to the rotation axis. Filter: gtil_i = sum_j w_ij g1_j
// / W_i with w_ij = (R - |x_i - x_j|) / R for |x_i - x_j| <= R and W_i = sum_j w_ij, both points in
// the design domain. Projection: gbar = (tanh(beta eta) + tanh(beta (gtil - eta))) /
// (tanh(beta eta) + tanh(beta (1 - eta))). gbar feeds the Brinkman coefficient and the volume
// constraint G = sum_dom gbar / (V_min N_dom) - 1 (Eq. constraint).
//
// Transpose: v3 = dJ/dgbar -> v2 = v3 dgbar/dgtil -> v1_j = sum_i w_ij v2_i / W_i (the weights are
// symmetric, so this is the same gather as the filter applied to v2 / W) -> out_m = sum of v1 over
// m's orbit when m is its own representative, else 0. Every output is one thread's fixed-order sum.
#include "lks_kernels.h"

namespace lks {

namespace {

constexpr int kDB = 256;

__device__ __forceinline__ void design_ijk(const Geo& g, int m, int* i) {
  i[0] = m % g.nd[0];
  i[1] = (m / g.nd[0]) % g.nd[1];
  i[2] = m / (g.nd[0] * g.nd[1]);
}
__device__ __forceinline__ int design_index(const Geo& g, const int* i) { return i[0] + g.nd[0] * (i[1] + g.nd[1] * i[2]); }

__device__ __forceinline__ bool in_domain(const Geo& g, const int* i) {
  return dsq(i[0], g.nd[0]) + dsq(i[1], g.nd[1]) + dsq(i[2], g.nd[2]) <= g.rad4;
}

// The images of design point m under the cyclic rotations (img[0] = m); returns their number.
__device__ __forceinline__ int orbit(const Geo& g, int m, int* img) {
  img[0] = m;
  if (g.cyc <= 1) return 1;
  const int b = g.axb, c = g.axc;
  int i[3];
  design_ijk(g, m, i);
  for (int k = 1; k < g.cyc; ++k) {
    int j[3] = {i[0], i[1], i[2]};
    if (g.cyc == 4) {
      j[b] = g.nd[c] - 1 - i[c];
      j[c] = i[b];
    } else {
      j[b] = g.nd[b] - 1 - i[b];
      j[c] = g.nd[c] - 1 - i[c];
    }
    i[0] = j[0];
    i[1] = j[1];
    i[2] = j[2];
    img[k] = design_index(g, i);
  }
  return g.cyc;
}

__global__ void __launch_bounds__(kDB) k_expand(Geo g, const double* __restrict__ gamma, double* __restrict__ g1) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int img[4];
  const int n = orbit(g, m, img);
  int rep = img[0];
  for (int k = 1; k < n; ++k) rep = min(rep, img[k]);
  g1[m] = gamma[rep];
}

// Sum of w_ij src_j over the filter disc of i (points of the design domain); W = sum of w_ij.
__device__ __forceinline__ void filter_sum(const Geo& g, const double* __restrict__ src, const int* i, double* acc,
                                           double* W) {
  const double R = g.frad;
  const int rr = (int)floor(R);
  const int ez = (g.dim == 3) ? rr : 0;
  double a = 0.0, w = 0.0;
  for (int dz = -ez; dz <= ez; ++dz)
    for (int dy = -rr; dy <= rr; ++dy)
      for (int dx = -rr; dx <= rr; ++dx) {
        const int j[3] = {i[0] + dx, i[1] + dy, i[2] + dz};
        if (j[0] < 0 || j[0] >= g.nd[0] || j[1] < 0 || j[1] >= g.nd[1] || j[2] < 0 || j[2] >= g.nd[2]) continue;
        const double dist = sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (dist > R || !in_domain(g, j)) continue;
        const double wij = (R - dist) / R;
        a += wij * src[design_index(g, j)];
        w += wij;
      }
  *acc = a;
  *W = w;
}

__global__ void __launch_bounds__(kDB) k_filter_project(Geo g, const double* __restrict__ g1, double* __restrict__ gtil,
                                                        double* __restrict__ gbar, double* __restrict__ W) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int i[3];
  design_ijk(g, m, i);
  if (!in_domain(g, i)) {
    gtil[m] = gbar[m] = 0.0;
    W[m] = 1.0;
    return;
  }
  double gt = g1[m], w = 1.0;
  if (g.frad > 0.0) {
    double a;
    filter_sum(g, g1, i, &a, &w);
    gt = a / w;
  }
  gtil[m] = gt;
  W[m] = w;
  if (g.pbeta > 0.0) {
    const double te = tanh(g.pbeta * g.peta);
    gbar[m] = (te + tanh(g.pbeta * (gt - g.peta))) / (te + tanh(g.pbeta * (1.0 - g.peta)));
  } else {
    gbar[m] = gt;
  }
}

// v <- v dgbar/dgtil / W (in place), zero outside the domain
__global__ void __launch_bounds__(kDB) k_project_T(Geo g, const double* __restrict__ gtil, const double* __restrict__ W,
                                                   double* __restrict__ v) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int i[3];
  design_ijk(g, m, i);
  if (!in_domain(g, i)) {
    v[m] = 0.0;
    return;
  }
  double d = 1.0;
  if (g.pbeta > 0.0) {
    const double th = tanh(g.pbeta * (gtil[m] - g.peta));
    d = g.pbeta * (1.0 - th * th) / (tanh(g.pbeta * g.peta) + tanh(g.pbeta * (1.0 - g.peta)));
  }
  v[m] = v[m] * d / W[m];
}

__global__ void __launch_bounds__(kDB) k_filter_T(Geo g, const double* __restrict__ v, double* __restrict__ out) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int i[3];
  design_ijk(g, m, i);
  if (!in_domain(g, i)) {
    out[m] = 0.0;
    return;
  }
  if (g.frad > 0.0) {
    double a, w;
    filter_sum(g, v, i, &a, &w);
    out[m] = a;
  } else {
    out[m] = v[m];
  }
}

__global__ void __launch_bounds__(kDB) k_orbit_sum(Geo g, const double* __restrict__ v, double* __restrict__ out) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int img[4];
  const int n = orbit(g, m, img);
  bool rep = true;
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    rep = rep && img[k] >= m;
    bool seen = false;  // a point the rotation fixes appears more than once among the images
    for (int q = 0; q < k; ++q) seen = seen || img[q] == img[k];
    if (!seen) s += v[img[k]];
  }
  out[m] = rep ? s : 0.0;
}

// One CTA: sum of gbar over the design domain in a fixed order, and the domain's point count.
__global__ void __launch_bounds__(1024) k_volume(Geo g, const double* __restrict__ gbar, double* __restrict__ out) {
  __shared__ double red[32 * 2];
  double v[2] = {0.0, 0.0};
  for (int m = threadIdx.x; m < g.ND; m += blockDim.x) {
    int i[3];
    design_ijk(g, m, i);
    if (in_domain(g, i)) {
      v[0] += gbar[m];
      v[1] += 1.0;
    }
  }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
  }
}

__global__ void __launch_bounds__(kDB) k_fill_domain(Geo g, double value, double* __restrict__ out) {
  const int m = blockIdx.x * kDB + threadIdx.x;
  if (m >= g.ND) return;
  int i[3];
  design_ijk(g, m, i);
  out[m] = in_domain(g, i) ? value : 0.0;
}

inline unsigned nblk(const Geo& g) { return (unsigned)((g.ND + kDB - 1) / kDB); }

}  // namespace

bool design_chain_active(const Geo& g) { return g.cyc > 1 || g.frad > 0.0 || g.pbeta > 0.0; }

void launch_design_chain(const Geo& g, const double* gamma, double* g1, double* gtil, double* gbar, double* W,
                         cudaStream_t st) {
  launch(k_expand, nblk(g), kDB, 0, st, g, gamma, g1);
  launch(k_filter_project, nblk(g), kDB, 0, st, g, (const double*)g1, gtil, gbar, W);
}

void launch_design_chain_T(const Geo& g, const double* gtil, const double* W, double* v, double* tmp, double* out,
                           cudaStream_t st) {
  launch(k_project_T, nblk(g), kDB, 0, st, g, gtil, W, v);
  launch(k_filter_T, nblk(g), kDB, 0, st, g, (const double*)v, tmp);
  launch(k_orbit_sum, nblk(g), kDB, 0, st, g, (const double*)tmp, out);
}

void launch_volume(const Geo& g, const double* gbar, double* out2, cudaStream_t st) {
  launch(k_volume, 1, 1024, 0, st, g, gbar, out2);
}

void launch_fill_domain(const Geo& g, double value, double* out, cudaStream_t st) {
  launch(k_fill_domain, nblk(g), kDB, 0, st, g, value, out);
}

}  // namespace lks
