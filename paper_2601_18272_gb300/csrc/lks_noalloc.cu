// One time step of the coupled LKS / rigid-body march that allocates no device memory.
//
// Who needs this: lks_create allocates a workspace with cudaMalloc, and some callers cannot let a
// library do that -- real-time loops whose device memory must be fixed before they start, and
// host frameworks that own every device allocation and forbid libraries from making their own.
// For them, lks_step_noalloc keeps all of its scratch (kappa^ref, the design moments, the DOF
// iterates, the control block and the per-CTA partial sums of the force/torque reduction) in one
// fixed array of device memory declared below. The caller still passes the design field and the
// state.
//
// Costs and rules:
//   - every GPU that loads this library holds the array (kScratchBytes, about 0.7 MB) until the
//     process exits;
//   - the first call on a device looks up the array's device address (cudaGetSymbolAddress) with
//     that device current and caches it;
//   - all calls share the one array, which keeps the last call's contents: each call clears the
//     part that must start at zero, and calls that overlap on the GPU (two streams, two host
//     threads) race on it -- serialise them;
//   - each call waits for its stream and copies the new DOFs to the host before it returns;
//   - the problem is checked, and its geometry derived, by the same code as lks_create; sizes
//     beyond the array's limits are rejected with LKS_ERR_BUDGET, and what the step does not do
//     (3D, FP32 fields, the design chain) with LKS_ERR_UNSUPPORTED.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lks.h"
#include "lks_geo.h"
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

// Problem constants for one step (2D, FP64 fields) from the shared validation and geometry of
// lks_create, with the body box lks_forward would use for a march starting from s(t-1).
int make_geo(const lks_problem* P, const double* s_prev, Geo* g) {
  if (!P) return LKS_ERR_ARG;
  const int v = validate_problem(P);
  if (v != LKS_OK) return v;
  if (P->dim != 2 || P->field_precision != LKS_FP64) return LKS_ERR_UNSUPPORTED;
  // the design chain (cyclic expansion, filter, projection) needs workspace of its own
  if (P->filter_radius > 0.0 || P->proj_beta > 0.0 || P->cyclic_order > 1) return LKS_ERR_UNSUPPORTED;
  bool rot_ok = true;
  if (make_geometry(P, g, &rot_ok) != LKS_OK) return LKS_ERR_UNSUPPORTED;
  const bool rotated = (g->dof_mask & LKS_DOF_ROT) || s_prev[6] != 0.0;
  if (rotated && !rot_ok) return LKS_ERR_UNSUPPORTED;
  setup_box(g, P->design_radius, rotated);
  return LKS_OK;
}

}  // namespace

extern "C" int lks_step_noalloc(const lks_problem* problem, const double* gamma_dev, double* state_dev, int t,
                                double* s_host, void* stream) {
  if (!problem || !gamma_dev || !state_dev || !s_host || t < 1) return LKS_ERR_ARG;
  for (int a = 0; a < kNdofAxis; ++a)
    if (!std::isfinite(s_host[a])) return LKS_ERR_NONFINITE;
  for (int a = 0; a < 3; ++a)
    if (std::fabs(s_host[a]) > 1e9) return LKS_ERR_ARG;  // x^G far outside any grid
  Geo g;
  int r = make_geo(problem, s_host, &g);
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
  if ((c.status & ST_NONFINITE) || (c.prep_status & ST_NONFINITE)) return LKS_ERR_NONFINITE;
  return LKS_OK;
}
