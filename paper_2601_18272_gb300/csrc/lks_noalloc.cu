// One time step of the coupled LKS / rigid-body march that allocates no device memory.
//
// Who needs this: lks_create allocates a workspace with cudaMalloc, and some callers cannot let a
// library do that -- code running inside a relaxed-mode CUDA graph capture on its own stream,
// real-time loops whose device memory must be fixed before they start, and host frameworks that
// own every device allocation and forbid libraries from making their own. For them,
// lks_step_noalloc keeps all of its scratch (kappa^ref, the design moments, the DOF iterates, the
// control block and the per-CTA partial sums of the force/torque reduction) in one fixed array
// of device memory declared below. The caller still passes the design field and the state.
//
// Costs and rules:
//   - every GPU that loads this library holds the array (kScratchBytes, about 0.7 MB) until the
//     process exits;
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress) with
//     that device current and caches it; make that first call before any stream capture;
//   - all calls share the one array, which keeps the last call's contents: each call clears the
//     part that must start at zero, and calls that overlap on the GPU (two streams, two host
//     threads) race on it -- serialise them;
//   - sizes beyond the array's limits are rejected with LKS_ERR_BUDGET.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lks.h"
#include "lks_kernels.h"

using namespace lks;

namespace {

constexpr int kMaxDesign = 65536;  // design points (kappa^ref entries)
constexpr int kMaxItr = 16;        // N_itr
constexpr int kMaxBlocks = 4096;   // CTAs of one reduction (partials)
constexpr int kMaxDevices = 64;

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t align256(size_t b) { return ((b + 255) / 256) * 256; }
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffMom = kOffCtrl + align256(sizeof(Ctrl));
constexpr size_t kOffIt = kOffMom + align256(sizeof(Moments));
constexpr size_t kItBytes = align256(sizeof(Dof) * (kMaxItr + 2));
constexpr size_t kOffKref = kOffIt + kItBytes;
constexpr size_t kOffPartials = kOffKref + sizeof(double) * kMaxDesign;
constexpr size_t kScratchBytes = kOffPartials + sizeof(double) * 8 * kMaxBlocks;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once per device).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LKS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LKS_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = (unsigned char*)g_scratch_addr[dev];
  return LKS_OK;
}

__global__ void k_noalloc_seed(Ctrl* ctrl, Dof* it, Dof s0, int base) {
  ctrl->t0 = 1;
  ctrl->base = base;
  ctrl->status = 0;
  it[0] = s0;
}

// Problem constants for one step (2D, FP64 fields), the same as the handle-based path computes.
int make_geo(const lks_problem* P, Geo* g) {
  if (!P) return LKS_ERR_ARG;
  if (P->dim != 2 || P->velocity_set != LKS_D2Q9 || P->nz != 1 || P->ndz != 1 || P->rot_axis != 2)
    return P->dim == 3 ? LKS_ERR_UNSUPPORTED : LKS_ERR_ARG;
  if (P->field_precision != LKS_FP64) return LKS_ERR_UNSUPPORTED;
  if (P->nx < 4 || P->ny < 4 || P->ndx < 1 || P->ndy < 1) return LKS_ERR_ARG;
  if (P->bc[0] != LKS_BC_PERIODIC && P->bc[0] != LKS_BC_INFLOW_OUTFLOW && P->bc[0] != LKS_BC_PRESSURE) return LKS_ERR_ARG;
  if (P->bc[1] != LKS_BC_PERIODIC && P->bc[1] != LKS_BC_WALL) return LKS_ERR_ARG;
  if (!(P->nu > 0.0)) return LKS_ERR_UNSTABLE;
  if (P->n_itr < 1 || !(P->mass > 0.0) || !(P->inertia > 0.0)) return LKS_ERR_ARG;
  if (P->weight_kind != LKS_W_COS4 && P->weight_kind != LKS_W_BILINEAR) return LKS_ERR_ARG;
  if (P->design_radius != 0.0) return LKS_ERR_UNSUPPORTED;
  std::memset(g, 0, sizeof(Geo));
  g->dim = 2;
  g->n[0] = P->nx;
  g->n[1] = P->ny;
  g->n[2] = 1;
  g->N = (long long)P->nx * P->ny;
  g->bc[0] = P->bc[0];
  g->bc[1] = P->bc[1];
  g->bc[2] = LKS_BC_PERIODIC;
  g->nd[0] = P->ndx;
  g->nd[1] = P->ndy;
  g->nd[2] = 1;
  g->ND = P->ndx * P->ndy;
  g->xic[0] = (P->ndx - 1) / 2.0;
  g->xic[1] = (P->ndy - 1) / 2.0;
  g->xicf[0] = (float)g->xic[0];
  g->xicf[1] = (float)g->xic[1];
  g->ax = 2;
  g->axb = 0;
  g->axc = 1;
  g->ns = kNdofAxis;
  g->rad4 = INT_MAX;  // the whole design grid
  g->dof_mask = (int)P->dof_mask;
  g->wk = P->weight_kind;
  g->s = (P->weight_kind == LKS_W_BILINEAR) ? 1 : 2;
  g->K = P->n_itr;
  g->A = 4.5 * (1.0 / 6.0 - P->nu);
  g->A2 = (float)(2.0 * g->A);
  g->u_in = P->u_in;
  g->dp = P->dp;
  g->mass = P->mass;
  g->inertia = P->inertia;
  g->inv_mass = 1.0 / P->mass;
  g->inv_inertia = 1.0 / P->inertia;
  // body box placed from x^G(t-1): circumscribed in the plane (the body may rotate)
  const double hx = (P->ndx - 1) / 2.0, hy = (P->ndy - 1) / 2.0;
  const int hb = (int)std::ceil(std::sqrt(hx * hx + hy * hy) - 1e-12);
  g->margin = 1;
  for (int a = 0; a < 2; ++a) {
    g->hb[a] = hb;
    g->B[a] = 2 * hb + 2 * g->s + 2 * g->margin + 2;
    if (g->bc[a] == LKS_BC_PERIODIC && g->B[a] > g->n[a]) return LKS_ERR_UNSUPPORTED;
  }
  g->hb[2] = 0;
  g->B[2] = 1;
  g->box_cells = (long long)g->B[0] * g->B[1];
  return LKS_OK;
}

}  // namespace

extern "C" int lks_step_noalloc(const lks_problem* problem, const double* gamma_dev, double* state_dev, int t,
                                double* s_host, void* stream) {
  if (!problem || !gamma_dev || !state_dev || !s_host || t < 1) return LKS_ERR_ARG;
  Geo g;
  int r = make_geo(problem, &g);
  if (r != LKS_OK) return r;
  const long long box_blocks = (long long)((g.B[0] + kBoxCtaCellsX - 1) / kBoxCtaCellsX) * ((g.B[1] + kBoxCtaCellsY - 1) / kBoxCtaCellsY);
  const long long design_blocks = ((long long)g.ND * 4 + 255) / 256;
  if (g.ND > kMaxDesign || g.K > kMaxItr || box_blocks > kMaxBlocks || design_blocks > kMaxBlocks)
    return LKS_ERR_BUDGET;
  unsigned char* base = nullptr;
  r = scratch_address(&base);
  if (r != LKS_OK) return r;
  Ctrl* ctrl = (Ctrl*)(base + kOffCtrl);
  Moments* mom = (Moments*)(base + kOffMom);
  Dof* it = (Dof*)(base + kOffIt);
  double* kref = (double*)(base + kOffKref);
  double* partials = (double*)(base + kOffPartials);
  cudaStream_t st = (cudaStream_t)stream;

  // last-block counters and status must start at zero
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return LKS_ERR_CUDA;
  Dof s0;
  for (int a = 0; a < kNdofFree; ++a) s0.s[a] = (a < kNdofAxis) ? s_host[a] : 0.0;
  s0.cs = std::cos(s0.s[6]);
  s0.sn = std::sin(s0.s[6]);
  dof_views(&s0, false);
  // The device sees step 1 of a two-slot ring whose base selects the parity: slot (t-1) mod 2 is
  // read and slot t mod 2 written.
  const int parity = (t - 1) & 1;
  Slots<double> S{state_dev, 3 * g.N, 2};
  launch_prep<double>(g, gamma_dev, problem->kappa_max, problem->q, kref, mom, partials, ctrl, st);
  k_noalloc_seed<<<1, 1, 0, st>>>(ctrl, it, s0, parity);
  launch_stencil_fwd<double>(g, S, ctrl, 0, st);
  const long long pstride = 4LL * kMaxBlocks;  // halves of the double-buffered coupling partials
  for (int k = 1; k <= g.K; ++k) launch_couple<double>(g, S, ctrl, it, kref, mom, partials, pstride, k, nullptr, 1, 0, st);
  launch_couple_last<double>(g, ctrl, it, mom, partials, pstride, 1, st);
  Dof out;
  Ctrl c;
  if (cudaMemcpyAsync(&out, it + (g.K + 1), sizeof(Dof), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LKS_ERR_CUDA;
  if (cudaMemcpyAsync(&c, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess) return LKS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LKS_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return LKS_ERR_CUDA;
  for (int a = 0; a < 8; ++a) s_host[a] = out.s[a];
  if (c.status & (ST_BODY_OUTSIDE | ST_BOX_OVERFLOW)) return LKS_ERR_BODY_OUTSIDE;
  if (c.status & ST_NONFINITE) return LKS_ERR_NONFINITE;
  return LKS_OK;
}
