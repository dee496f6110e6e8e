// C ABI of the library (include/lks.h): workspace, forward / adjoint scheduling, CUDA graphs.
//
// Forward (Algorithm 1, state loop): per step one stencil kernel over the grid and N_itr coupling
// kernels over the body box; the step index lives on the device (Ctrl::t), so one captured graph
// of L steps is replayed for every segment.
//   store-all : every state slot and the per-step u* of the body box are kept (plain form).
//   uniform   : ping-pong state, a checkpoint every k steps; the adjoint restores a checkpoint,
//               recomputes the segment (stencil + Brinkman update with the stored DOF iterates)
//               into a segment ring, then reverses it.
//   binomial  : s state snapshots placed along a binomial schedule (Griewank's optimal
//               checkpointing recursion for a fixed number of snapshots), built once as a list of
//               actions; the reverse sweep re-advances from the nearest snapshot and reverses one
//               step at a time.
// Adjoint (Algorithm 1, adjoint loop): per step, for k = N_itr..1 a cell-side and a design-side
// reverse kernel, then the transposed stencil.
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/lks.h"
#include "lks_geo.h"
#include "lks_kernels.h"

using namespace lks;

// ---- problem validation and constants (shared with the allocation-free step: lks_geo.h) ----
namespace lks {

namespace {
// Symmetric (to rounding) positive definite 3x3 matrix, by its leading minors.
bool spd3(const double* A) {
  double mx = 0.0;
  for (int i = 0; i < 9; ++i) {
    if (!std::isfinite(A[i])) return false;
    mx = std::max(mx, std::fabs(A[i]));
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(A[3 * i + j] - A[3 * j + i]) > 1e-12 * mx) return false;
  const double m2 = A[0] * A[4] - A[1] * A[3];
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  return A[0] > 0.0 && m2 > 0.0 && det > 0.0;
}

// Inverse of a symmetric 3x3 matrix: row i is c_(i+1) x c_(i+2) / det for the columns c.
void inverse_sym3(const double* A, double* inv) {
  const double c[3][3] = {{A[0], A[3], A[6]}, {A[1], A[4], A[7]}, {A[2], A[5], A[8]}};
  double rows[3][3];
  for (int i = 0; i < 3; ++i) {
    const double* u = c[(i + 1) % 3];
    const double* v = c[(i + 2) % 3];
    rows[i][0] = u[1] * v[2] - u[2] * v[1];
    rows[i][1] = u[2] * v[0] - u[0] * v[2];
    rows[i][2] = u[0] * v[1] - u[1] * v[0];
  }
  const double det = c[0][0] * rows[0][0] + c[0][1] * rows[0][1] + c[0][2] * rows[0][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) inv[3 * i + j] = rows[i][j] / det;
}

}  // namespace

int validate_problem(const lks_problem* P) {
  if (!P) return LKS_ERR_ARG;
  if (P->dim != 2 && P->dim != 3) return LKS_ERR_ARG;
  if (P->dim == 2 && (P->velocity_set != LKS_D2Q9 || P->nz != 1 || P->ndz != 1 || P->rot_axis != 2)) return LKS_ERR_ARG;
  if (P->dim == 3 && P->velocity_set != LKS_D3Q15) return LKS_ERR_ARG;
  if (P->nx < 4 || P->ny < 4 || (P->dim == 3 && P->nz < 4)) return LKS_ERR_ARG;
  if (P->ndx < 1 || P->ndy < 1 || P->ndz < 1) return LKS_ERR_ARG;
  if (P->rot_axis == LKS_ROT_FREE) {
    if (P->dim != 3 || !spd3(P->inertia_tensor)) return LKS_ERR_ARG;
  } else if (P->rot_axis < 0 || P->rot_axis > 2) {
    return LKS_ERR_ARG;
  }
  if (!(P->design_radius >= 0.0) || !std::isfinite(P->design_radius)) return LKS_ERR_ARG;
  if (!(P->filter_radius >= 0.0) || !std::isfinite(P->filter_radius)) return LKS_ERR_ARG;
  if (!(P->proj_beta >= 0.0) || !std::isfinite(P->proj_beta)) return LKS_ERR_ARG;
  if (P->proj_beta > 0.0 && !(P->proj_eta > 0.0 && P->proj_eta < 1.0)) return LKS_ERR_ARG;
  if (P->cyclic_order != 1 && P->cyclic_order != 2 && P->cyclic_order != 4) return LKS_ERR_ARG;
  if (P->cyclic_order > 1) {
    if (P->rot_axis == LKS_ROT_FREE) return LKS_ERR_ARG;
    const int nd[3] = {P->ndx, P->ndy, P->dim == 3 ? P->ndz : 1};
    const int b = (P->rot_axis + 1) % 3, c = (P->rot_axis + 2) % 3;
    if (P->cyclic_order == 4 && nd[b] != nd[c]) return LKS_ERR_ARG;
  }
  if (P->bc[0] != LKS_BC_PERIODIC && P->bc[0] != LKS_BC_INFLOW_OUTFLOW && P->bc[0] != LKS_BC_PRESSURE) return LKS_ERR_ARG;
  for (int a = 1; a < 3; ++a)
    if (P->bc[a] != LKS_BC_PERIODIC && P->bc[a] != LKS_BC_WALL) return LKS_ERR_ARG;
  if (!(P->nu > 0.0)) return LKS_ERR_UNSTABLE;
  if (P->n_steps < 1 || P->n_itr < 1) return LKS_ERR_ARG;
  if (P->weight_kind != LKS_W_COS4 && P->weight_kind != LKS_W_BILINEAR) return LKS_ERR_ARG;
  if (!(P->mass > 0.0) || !(P->inertia > 0.0)) return LKS_ERR_ARG;
  if (P->field_precision != LKS_FP32 && P->field_precision != LKS_FP64) return LKS_ERR_ARG;
  if (P->ckpt_policy != LKS_CKPT_STORE_ALL && P->ckpt_policy != LKS_CKPT_UNIFORM &&
      P->ckpt_policy != LKS_CKPT_BINOMIAL)
    return LKS_ERR_ARG;
  // binomial snapshots: a count, or 0 for as many as hbm_budget_bytes holds
  const bool bin_auto = P->ckpt_policy == LKS_CKPT_BINOMIAL && P->ckpt_every == 0 && P->hbm_budget_bytes > 0;
  if (P->ckpt_policy != LKS_CKPT_STORE_ALL && P->ckpt_every < 1 && !bin_auto) return LKS_ERR_ARG;
  if (P->ckpt_format != LKS_CKPT_NATIVE && P->ckpt_format != LKS_CKPT_BF16 && P->ckpt_format != LKS_CKPT_FP16)
    return LKS_ERR_ARG;
  // reduced-precision checkpoints: FP32 fields with uniform checkpoints or binomial snapshots
  if (P->ckpt_format != LKS_CKPT_NATIVE && (P->ckpt_policy == LKS_CKPT_STORE_ALL || P->field_precision != LKS_FP32))
    return LKS_ERR_UNSUPPORTED;
  // 3D: boundary pairs (x = 0,1 and nx-2,nx-1; y walls likewise) must share a stencil column
  // (2D strips choose their width so that they always do)
  if (P->dim == 3 && P->bc[0] != LKS_BC_PERIODIC && P->nx % kTileX == 1) return LKS_ERR_UNSUPPORTED;
  if (P->dim == 3 && P->bc[1] == LKS_BC_WALL && P->ny % kTileY3 == 1) return LKS_ERR_UNSUPPORTED;
  return LKS_OK;
}


void setup_box(Geo* gp, double design_radius, bool rotated) {
  Geo& g = *gp;
  double half[3] = {0, 0, 0};
  for (int a = 0; a < g.dim; ++a) half[a] = (g.nd[a] - 1) / 2.0;
  if (rotated && g.ax == AX_FREE) {
    const double r = std::sqrt(half[0] * half[0] + half[1] * half[1] + half[2] * half[2]);
    half[0] = half[1] = half[2] = r;
  } else if (rotated) {
    const double r = std::sqrt(half[g.axb] * half[g.axb] + half[g.axc] * half[g.axc]);
    half[g.axb] = half[g.axc] = r;
  }
  if (design_radius > 0.0)
    for (int a = 0; a < g.dim; ++a) half[a] = std::min(half[a], design_radius);
  g.margin = 1;
  g.box_cells = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < g.dim) {
      g.hb[a] = (int)std::ceil(half[a] - 1e-12);
      g.B[a] = 2 * g.hb[a] + 2 * g.s + 2 * g.margin + 2;
    } else {
      g.hb[a] = 0;
      g.B[a] = 1;
    }
    g.box_cells *= g.B[a];
  }
}

long long box_tiles(const Geo& g) {
  const long long cy = g.dim == 2 ? kBoxCtaCellsY2D : kBoxCtaCellsY;
  return ((g.B[0] + kBoxCtaCellsX - 1) / kBoxCtaCellsX) * ((g.B[1] + cy - 1) / cy) * (long long)g.B[2];
}

bool box_fits(const Geo& g) {
  for (int a = 0; a < g.dim; ++a)
    if (g.bc[a] == LKS_BC_PERIODIC && g.B[a] > g.n[a]) return false;
  return true;
}

int make_geometry(const lks_problem* P, Geo* gp, bool* rot_ok) {
  Geo& g = *gp;
  std::memset(&g, 0, sizeof(g));
  g.dim = P->dim;
  g.n[0] = P->nx;
  g.n[1] = P->ny;
  g.n[2] = P->dim == 3 ? P->nz : 1;
  g.N = (long long)g.n[0] * g.n[1] * g.n[2];
  for (int a = 0; a < 3; ++a) g.bc[a] = (a < g.dim) ? P->bc[a] : LKS_BC_PERIODIC;
  g.nd[0] = P->ndx;
  g.nd[1] = P->ndy;
  g.nd[2] = P->dim == 3 ? P->ndz : 1;
  g.ND = g.nd[0] * g.nd[1] * g.nd[2];
  for (int a = 0; a < 3; ++a) {
    g.xic[a] = (a < g.dim) ? (g.nd[a] - 1) / 2.0 : 0.0;
    g.xicf[a] = (float)g.xic[a];
  }
  if (P->rot_axis == LKS_ROT_FREE) {
    g.ax = AX_FREE;
    g.axb = 0;  // (unused with free rotation)
    g.axc = 1;
    g.ns = kNdofFree;
    inverse_sym3(P->inertia_tensor, g.Jinv);
  } else {
    g.ax = P->rot_axis;
    g.axb = (g.ax + 1) % 3;
    g.axc = (g.ax + 2) % 3;
    g.ns = kNdofAxis;
  }
  g.frad = P->filter_radius;
  g.pbeta = P->proj_beta;
  g.peta = P->proj_eta;
  g.cyc = P->cyclic_order;
  // design domain 4 |r_m|^2 <= rad4, compared in integers (4 |r_m|^2 is an integer)
  g.rad4 = INT_MAX;
  if (P->design_radius > 0.0) {
    const double q = std::floor(4.0 * P->design_radius * P->design_radius);
    g.rad4 = q < (double)INT_MAX ? (int)q : INT_MAX;
  }
  g.dof_mask = (int)P->dof_mask;
  g.wk = P->weight_kind;
  g.s = (P->weight_kind == LKS_W_BILINEAR) ? 1 : 2;
  g.K = P->n_itr;
  g.A = 4.5 * (1.0 / 6.0 - P->nu);
  g.A2 = (float)(2.0 * g.A);
  g.u_in = P->u_in;
  g.dp = P->dp;
  g.mass = P->mass;
  g.inertia = P->inertia;
  g.inv_mass = 1.0 / P->mass;
  g.inv_inertia = 1.0 / P->inertia;
  // the rotated (largest) box; a body without the rotational DOF whose rotated box would not fit a
  // periodic extent gets the axis-aligned box and may not start rotated
  setup_box(&g, P->design_radius, true);
  *rot_ok = box_fits(g);
  if (!*rot_ok) {
    setup_box(&g, P->design_radius, false);
    if ((g.dof_mask & LKS_DOF_ROT) || !box_fits(g)) return LKS_ERR_UNSUPPORTED;
  }
  return LKS_OK;
}

}  // namespace lks

namespace {

struct EventPair {
  cudaEvent_t a, b;
};

struct TimerFamily {
  std::vector<EventPair> pairs;
  size_t used = 0;
  double ms = 0.0;
  long long launches = 0;
};

// One action of the binomial checkpoint schedule (kinds LKS_BIN_* of the C ABI), built on the host
// once per handle and replayed by the forward (LKS_BIN_FWD_SNAPSHOT) and by the reverse sweep.
struct BinOp {
  int kind, a, b, c;
};

}  // namespace

struct lks_handle {
  lks_problem P;
  Geo g;
  int prec = 32;
  size_t esz = 4;
  // state rings
  void* ring = nullptr;  // store-all: N_t + 1 slots; uniform: segment of every + 1 slots
  int nring = 0;
  void* pp = nullptr;    // uniform: ping-pong forward state (2 slots)
  void* ckpt = nullptr;  // uniform: checkpoints at t = 0, k, 2k, ... (native format)
  unsigned short* ckq = nullptr;  // uniform, BF16/FP16: checkpoints at t = k, 2k, ... (t = 0 from init)
  unsigned* ckkeys = nullptr;     // their per-plane ranges
  int nckpt = 0;
  std::vector<BinOp> bin_plan;  // binomial: the schedule (the forward's snapshots, the reverse's actions)
  int bin_snapshots = 0;        // binomial: snapshot slots of the schedule
  long long slot_elems = 0;
  void* boxstore = nullptr;  // u* in the body box, one slab per step of the resident segment
  int nbox = 0;
  void* L = nullptr;  // adjoint fields, 2 slots
  void* acc = nullptr;
  void* scratch = nullptr;
  void* kref = nullptr;
  double* dkref = nullptr;
  double* gamma = nullptr;
  double* tmp_nd = nullptr;
  // design chain of the last forward (gbar feeds kappa^ref; gtil and the filter normaliser W serve
  // the transpose), of lks_constraint, and scratch for the transposes
  double *cg1 = nullptr, *cgtil = nullptr, *cgbar = nullptr, *cW = nullptr;
  double *kg1 = nullptr, *kgtil = nullptr, *kgbar = nullptr, *kW = nullptr;
  double *dv = nullptr, *dtmp = nullptr, *vol = nullptr;
  // terminal adjoint of the next reverse sweep (periodic warm start): fields in the field type
  void* term_L = nullptr;
  double* term_s = nullptr;
  bool has_term = false;
  // the paper-form adjoint (allocated by its first call): moment slots, box spread, equilibrium
  // vector Z, per-design-point sensitivity coefficients, design-CTA partials
  void* al_A = nullptr;
  void* al_box = nullptr;
  void* al_z = nullptr;
  void* al_sens = nullptr;
  void* al_part = nullptr;
  long long al_astride = 0;
  bool alks_mode = false, alks_done = false;
  Dof* it = nullptr;
  Ctrl* ctrl = nullptr;
  Moments* mom = nullptr;
  double* partials = nullptr;
  long long pstride = 0;  // elements per half of the double-buffered coupling partials
  double* init_p = nullptr;
  double* init_u = nullptr;
  double* init_s = nullptr;
  double* objw = nullptr;
  double host_s0[kNdofFree];
  size_t bytes = 0;
  std::vector<void*> allocs;
  cudaStream_t cap = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, int> graph_kernels;
  bool box_rot_ok = true;  // buffers hold the rotated box
  int coop_mode = 2;  // persistent coupling kernels: 0 off, 1 on (when the device holds their grid), 2 automatic
  // what the last calls left valid: a forward, an adjoint of it (either form: dkref), the exact
  // adjoint's lambda(0) and dJ/ds(0), the paper-form adjoint's moments
  bool fwd_done = false, adj_done = false, exact_done = false;
  long long launches = 0;
  bool timing = false;
  std::map<std::string, TimerFamily> timers;
  int chunk = 50;    // steps per captured graph in store-all mode
  int launch_error = 0;
};

namespace {

int g_last_cuda_error = 0;

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      g_last_cuda_error = (int)e_;            \
      return LKS_ERR_CUDA;                    \
    }                                         \
  } while (0)

int dalloc(lks_handle* h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (h->P.hbm_budget_bytes && h->bytes + bytes > h->P.hbm_budget_bytes) return LKS_ERR_BUDGET;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LKS_ERR_OOM;
  }
  h->bytes += bytes;
  h->allocs.push_back(*p);
  return LKS_OK;
}

#define TRY(call)           \
  do {                      \
    int r_ = (call);        \
    if (r_ != LKS_OK) {     \
      return r_;            \
    }                       \
  } while (0)

template <typename T>
Slots<T> ring_slots(lks_handle* h) {
  return Slots<T>{(T*)h->ring, h->slot_elems, h->nring};
}
template <typename T>
Slots<T> pp_slots(lks_handle* h) {
  return Slots<T>{(T*)h->pp, h->slot_elems, 2};
}

// Launch bookkeeping: counts kernels and, in timing mode, brackets them with events.
struct Launcher {
  lks_handle* h;
  cudaStream_t st;
  bool capturing;
  int kernels = 0;
  template <typename F>
  void operator()(const char* family, F&& f) {
    n(family, 1, f);
  }
  // one call that launches `count` kernels (timed together)
  template <typename F>
  void n(const char* family, int count, F&& f) {
    EventPair* ev = nullptr;
    if (h->timing && !capturing) {
      TimerFamily& tf = h->timers[family];
      if (tf.used == tf.pairs.size()) {
        EventPair p;
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        tf.pairs.push_back(p);
      }
      ev = &tf.pairs[tf.used++];
      tf.launches++;
      cudaEventRecord(ev->a, st);
    }
    f(st);
    if (ev) cudaEventRecord(ev->b, st);
    kernels += count;
    if (!capturing) h->launches += count;
  }
};

void collect_timers(lks_handle* h) {
  for (auto& kv : h->timers) {
    TimerFamily& tf = kv.second;
    for (size_t i = 0; i < tf.used; ++i) {
      float ms = 0.f;
      cudaEventSynchronize(tf.pairs[i].b);
      cudaEventElapsedTime(&ms, tf.pairs[i].a, tf.pairs[i].b);
      tf.ms += ms;
    }
    tf.used = 0;
  }
}

// Run `body` either directly (timing mode) or as a cached CUDA graph captured on a private stream.
template <typename Body>
int run_graph(lks_handle* h, const std::string& key, cudaStream_t st, Body&& body) {
  if (h->timing) {
    Launcher L{h, st, false};
    body(L);
    CK(cudaGetLastError());
    return LKS_OK;
  }
  auto itg = h->graphs.find(key);
  if (itg == h->graphs.end()) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    Launcher L{h, h->cap, true};
    body(L);
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) {
      g_last_cuda_error = (int)e;
      return LKS_ERR_CUDA;
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g_last_cuda_error = (int)e;
      return LKS_ERR_CUDA;
    }
    itg = h->graphs.emplace(key, exec).first;
    h->graph_kernels[key] = L.kernels;
  }
  CK(cudaGraphLaunch(itg->second, st));
  h->launches += h->graph_kernels[key];
  return LKS_OK;
}

void clear_graphs(lks_handle* h) {
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->graph_kernels.clear();
}

// Binomial checkpointing (Griewank's revolve schedule). The initial state and s snapshot slots are
// the c = s + 1 states a reversal can restart from. beta(c, r) = C(c + r, c) is the longest march
// that c such states reverse with each step advanced at most r times besides its own reverse
// step. A march of n steps is split after m steps: the last n - m are reversed from a snapshot of
// state(t0 + m) with one slot fewer, then the first m with all slots again. Every m in
// [max(beta(c, r-2), n - beta(c-1, r-1) - beta(c-2, r)), min(beta(c, r-1), n - beta(c-1, r-1))]
// (r the least with beta(c, r) >= n) gives the least total number of re-advanced steps,
// r n - beta(c+1, r-1); the upper end also leaves the most work to the snapshots the forward
// takes on its way (they cost no extra steps), so it is the split taken everywhere.
long long binomial_beta(int c, int r) {
  if (c < 0 || r < 0) return 0;
  long long b = 1;
  for (int i = 1; i <= c; ++i) {
    b = b * (r + i) / i;  // C(r + i, i), exact at every step
    if (b > (1LL << 50)) return 1LL << 50;
  }
  return b;
}
int binomial_split(int n, int s) {  // n >= 2, s >= 1
  const int c = s + 1;
  int r = 1;
  while (binomial_beta(c, r) < n) ++r;
  long long m = std::min(binomial_beta(c, r - 1), (long long)n - binomial_beta(c - 1, r - 1));
  if (m < 1) m = 1;
  if (m > n - 1) m = n - 1;
  return (int)m;
}

// Reverse of steps t0+1 .. t0+n with s free snapshot slots; state(t0) is the initial state (src < 0)
// or snapshot src. first: the snapshots of this branch's first descent are the forward's. Snapshot
// slot d belongs to recursion depth d.
void binomial_plan_rec(std::vector<BinOp>& ops, int t0, int n, int s, bool first, int src, int depth) {
  if (n <= 0) return;
  if (n == 1) {
    ops.push_back({LKS_BIN_RESTORE, src, t0, 0});
    ops.push_back({LKS_BIN_REVERSE, t0 + 1, t0, 0});
    return;
  }
  if (s == 0) {  // no snapshot left: re-advance for every step
    for (int j = n; j >= 1; --j) {
      ops.push_back({LKS_BIN_RESTORE, src, t0, 0});
      if (j > 1) ops.push_back({LKS_BIN_ADVANCE, t0, j - 1, 0});
      ops.push_back({LKS_BIN_REVERSE, t0 + j, t0, 0});
    }
    return;
  }
  const int m = binomial_split(n, s);
  if (first) {
    ops.push_back({LKS_BIN_FWD_SNAPSHOT, depth, t0 + m, 0});
  } else {
    ops.push_back({LKS_BIN_RESTORE, src, t0, 0});
    ops.push_back({LKS_BIN_ADVANCE, t0, m, 0});
    ops.push_back({LKS_BIN_STORE, depth, t0 + m, m});
  }
  binomial_plan_rec(ops, t0 + m, n - m, s - 1, first, depth, depth + 1);
  binomial_plan_rec(ops, t0, m, s, false, src, depth);
}
std::vector<BinOp> binomial_plan(int n, int s) {
  std::vector<BinOp> ops;
  binomial_plan_rec(ops, 0, n, s, true, -1, 0);
  return ops;
}

// Binomial snapshot slot a <- the state at src: a copy in the field precision, or BF16 / FP16 with
// the per-plane range of the reduced formats (FP32 fields).
int bin_snapshot(lks_handle* h, const void* src, int a, cudaStream_t st) {
  const size_t sb = h->slot_elems * h->esz;
  if (h->P.ckpt_format == LKS_CKPT_NATIVE) {
    CK(cudaMemcpyAsync((char*)h->ckpt + (size_t)a * sb, src, sb, cudaMemcpyDeviceToDevice, st));
  } else {
    launch_ckpt_pack_q_at(h->g, (const float*)src, h->ckq, h->ckkeys, h->P.ckpt_format, a, st);
    h->launches += 3;
  }
  return LKS_OK;
}

template <typename T>
void enqueue_fwd_steps(lks_handle* h, Launcher& L, const Slots<T>& S, int nsteps, bool store_box) {
  const Geo& g = h->g;
  T* bs = store_box ? (T*)h->boxstore : nullptr;
  for (int i = 0; i < nsteps; ++i) {
    L("stencil_fwd", [&](cudaStream_t s) { launch_stencil_fwd<T>(g, S, h->ctrl, i, s); });
    if (g.coop_fwd > 0) {  // all N_itr iterations and the last EOM in one persistent launch
      L("couple", [&](cudaStream_t s) {
        launch_couple_coop<T>(g, S, h->ctrl, h->it, (const T*)h->kref, h->mom, h->partials, h->pstride, bs, h->nbox,
                              i, s);
      });
      continue;
    }
    for (int k = 1; k <= g.K; ++k)
      L.n("couple", couple_kernels(g), [&](cudaStream_t s) {
        launch_couple<T>(g, S, h->ctrl, h->it, (const T*)h->kref, h->mom, h->partials, h->pstride, k, bs, h->nbox, i,
                         s);
      });
  }
}

template <typename T>
void enqueue_recompute(lks_handle* h, Launcher& L, const Slots<T>& S, int nsteps) {
  const Geo& g = h->g;
  for (int i = 0; i < nsteps; ++i) {
    L("stencil_fwd", [&](cudaStream_t s) { launch_stencil_fwd<T>(g, S, h->ctrl, i, s); });
    L("recompute", [&](cudaStream_t s) {
      launch_apply<T>(g, S, h->ctrl, h->it, (const T*)h->kref, (T*)h->boxstore, h->nbox, i, s);
    });
  }
}

template <typename T>
void enqueue_adj_steps(lks_handle* h, Launcher& L, const Slots<T>& S, int nsteps) {
  const Geo& g = h->g;
  if (h->alks_mode) {  // the paper-form adjoint: body at t, then the equilibrium's star moments at t-1
    for (int i = 0; i < nsteps; ++i) {
      L.n("alks_body", 5, [&](cudaStream_t s) {
        launch_alks_body<T>(g, S, h->ctrl, h->it, (const T*)h->kref, (T*)h->al_box, (T*)h->al_A, h->al_astride,
                            (T*)h->al_sens, h->al_part, h->dkref, i, s);
      });
      L.n("alks_stencil", alks_stencil_kernels(g.dim), [&](cudaStream_t s) {
        launch_alks_stencil<T>(g, S, h->ctrl, (T*)h->al_A, h->al_astride, (T*)h->al_z, i, s);
      });
    }
    return;
  }
  for (int i = 0; i < nsteps; ++i) {
    if (g.coop_adj > 0) {  // the N_itr reverse iterations in one persistent launch
      L("adj_body", [&](cudaStream_t s) {
        launch_adj_coop<T>(g, h->ctrl, h->it, (const T*)h->kref, (const T*)h->boxstore, h->nbox, (T*)h->L,
                           h->slot_elems, (T*)h->acc, (T*)h->scratch, h->dkref, h->partials, h->pstride, i, s);
      });
      L("stencil_adj", [&](cudaStream_t s) { launch_stencil_adj<T>(g, S, (T*)h->L, h->slot_elems, h->ctrl, i, s); });
      continue;
    }
    for (int k = g.K; k >= 1; --k) {
      L("adj_cell", [&](cudaStream_t s) {
        launch_adj_cell<T>(g, h->ctrl, h->it, (const T*)h->kref, (const T*)h->boxstore, h->nbox, (T*)h->L,
                           h->slot_elems, (T*)h->acc, (T*)h->scratch, k, i, s);
      });
      L.n("adj_design", 2, [&](cudaStream_t s) {
        launch_adj_design<T>(g, h->ctrl, h->it, (const T*)h->kref, (const T*)h->scratch, h->dkref, h->partials, k, i,
                             s);
      });
    }
    L("stencil_adj", [&](cudaStream_t s) { launch_stencil_adj<T>(g, S, (T*)h->L, h->slot_elems, h->ctrl, i, s); });
  }
}

template <typename T>
int forward_impl(lks_handle* h, cudaStream_t st) {
  const Geo& g = h->g;
  const int NT = h->P.n_steps;
  Launcher L0{h, st, false};
  CK(cudaMemsetAsync(&h->ctrl->sync_bar, 0, sizeof(unsigned), st));  // a barrier that timed out leaves it set
  if (h->P.ckpt_policy == LKS_CKPT_BINOMIAL) {
    // march in pieces between the snapshot steps of the first descent, snapshotting each
    Slots<T> S = pp_slots<T>(h);
    L0("init", [&](cudaStream_t s) { launch_init_forward<T>(g, S, h->init_p, h->init_u, h->init_s, h->it, h->ctrl, s); });
    std::vector<BinOp> stops;  // the forward's snapshots (ascending steps), then the end of the march
    for (const BinOp& op : h->bin_plan)
      if (op.kind == LKS_BIN_FWD_SNAPSHOT) stops.push_back(op);
    stops.push_back({-1, -1, NT, 0});
    int t = 0;
    for (const BinOp& stop : stops) {
      const int t1 = stop.b;
      const int n = t1 - t;
      if (n > 0) {
        L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t + 1, 0, s); });
        TRY(run_graph(h, "fwd_b_" + std::to_string(n), st, [&](Launcher& L) { enqueue_fwd_steps<T>(h, L, S, n, false); }));
      }
      if (stop.a >= 0) TRY(bin_snapshot(h, (char*)h->pp + (t1 & 1) * h->slot_elems * h->esz, stop.a, st));
      t = t1;
    }
  } else if (h->P.ckpt_policy == LKS_CKPT_STORE_ALL) {
    Slots<T> S = ring_slots<T>(h);
    L0("init", [&](cudaStream_t s) { launch_init_forward<T>(g, S, h->init_p, h->init_u, h->init_s, h->it, h->ctrl, s); });
    for (int t0 = 1; t0 <= NT; t0 += h->chunk) {
      const int n = std::min(h->chunk, NT - t0 + 1);
      L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t0, 0, s); });
      TRY(run_graph(h, "fwd_sa_" + std::to_string(n), st,
                    [&](Launcher& L) { enqueue_fwd_steps<T>(h, L, S, n, true); }));
    }
  } else {
    Slots<T> S = pp_slots<T>(h);
    const int every = h->P.ckpt_every;
    L0("init", [&](cudaStream_t s) { launch_init_forward<T>(g, S, h->init_p, h->init_u, h->init_s, h->it, h->ctrl, s); });
    const int fmt = h->P.ckpt_format;
    auto pack = [&](Launcher& L, int di) {
      if (fmt == LKS_CKPT_NATIVE)
        L("ckpt", [&](cudaStream_t s) { launch_ckpt_pack<T>(g, S, (T*)h->ckpt, h->slot_elems, every, h->ctrl, di, s); });
      else
        L("ckpt", [&](cudaStream_t s) {
          launch_ckpt_pack_q(g, reinterpret_cast<const Slots<float>&>(S), h->ckq, h->ckkeys, fmt, every, h->ctrl, di, s);
        });
    };
    if (fmt == LKS_CKPT_NATIVE) pack(L0, -1);  // reduced formats restart segment 0 from the initial state
    for (int t0 = 0; t0 < NT; t0 += every) {
      const int n = std::min(every, NT - t0);
      const bool do_pack = (t0 + n < NT);
      L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t0 + 1, 0, s); });
      TRY(run_graph(h, "fwd_u_" + std::to_string(n) + (do_pack ? "p" : ""), st, [&](Launcher& L) {
        enqueue_fwd_steps<T>(h, L, S, n, false);
        if (do_pack) pack(L, n - 1);
      }));
    }
  }
  if (g.coop_fwd == 0)  // the persistent kernel runs the last EOM itself
    L0("couple", [&](cudaStream_t s) { launch_couple_last<T>(g, h->ctrl, h->it, h->mom, h->partials, h->pstride, NT, s); });
  CK(cudaGetLastError());
  if (h->launch_error) return LKS_ERR_CUDA;
  return LKS_OK;
}

// The reverse sweep of the binomial schedule: its actions in order. The working pair (ring) holds
// state(t0) in slot 0 after a restore, so its slot base is t0; an advance by m leaves state(t0 + m)
// in slot m mod 2.
template <typename T>
int binomial_reverse(lks_handle* h, cudaStream_t st) {
  const Geo& g = h->g;
  Slots<T> W = ring_slots<T>(h);
  Launcher L0{h, st, false};
  const size_t sb = h->slot_elems * h->esz;
  for (const BinOp& op : h->bin_plan) {
    switch (op.kind) {
      case LKS_BIN_RESTORE:  // a: snapshot slot (-1: the initial state)
        if (op.a < 0)
          L0("ckpt", [&](cudaStream_t x) { launch_state_from_double<T>(g, (T*)h->ring, h->init_p, h->init_u, x); });
        else if (h->P.ckpt_format == LKS_CKPT_NATIVE)
          CK(cudaMemcpyAsync(h->ring, (char*)h->ckpt + (size_t)op.a * sb, sb, cudaMemcpyDeviceToDevice, st));
        else
          L0("ckpt", [&](cudaStream_t x) {
            launch_ckpt_restore_q(g, (float*)h->ring, h->ckq, h->ckkeys, h->P.ckpt_format, op.a, x);
          });
        break;
      case LKS_BIN_ADVANCE: {  // state(a) -> state(a + b)
        const int t0 = op.a, n = op.b;
        L0("init", [&](cudaStream_t x) { launch_set_step(h->ctrl, t0 + 1, t0, x); });
        TRY(run_graph(h, "bin_adv_" + std::to_string(n), st, [&](Launcher& L) { enqueue_recompute<T>(h, L, W, n); }));
        break;
      }
      case LKS_BIN_STORE:  // snapshot slot a <- state(b), c steps past the working pair's base
        TRY(bin_snapshot(h, (char*)h->ring + (size_t)(op.c & 1) * sb, op.a, st));
        break;
      case LKS_BIN_REVERSE: {  // step a from state(a - 1) in the working pair (base b)
        const int t = op.a, t0 = op.b;
        L0("init", [&](cudaStream_t x) { launch_set_step(h->ctrl, t, t0, x); });
        TRY(run_graph(h, h->alks_mode ? "alks_bin_rev1" : "bin_rev1", st, [&](Launcher& L) {
          enqueue_recompute<T>(h, L, W, 1);
          enqueue_adj_steps<T>(h, L, W, 1);
        }));
        break;
      }
      default:  // LKS_BIN_FWD_SNAPSHOT: taken by the forward
        break;
    }
  }
  return LKS_OK;
}

template <typename T>
int adjoint_impl(lks_handle* h, double seed, cudaStream_t st) {
  const Geo& g = h->g;
  const int NT = h->P.n_steps;
  Launcher L0{h, st, false};
  CK(cudaMemsetAsync(&h->ctrl->sync_bar, 0, sizeof(unsigned), st));
  if (h->alks_mode) {  // fluid multipliers zero at N_t + 1, terminal body multipliers
    CK(cudaMemsetAsync(h->al_A, 0, 2 * (size_t)h->al_astride * h->esz, st));
    L0("init", [&](cudaStream_t s) { launch_alks_init(g, h->ctrl, h->objw, seed, h->dkref, s); });
  } else {
    CK(cudaMemsetAsync(h->L, 0, 2 * h->slot_elems * h->esz, st));
    if (h->has_term)  // lambda(N_t) sits in slot N_t mod 2 of the adjoint pair
      CK(cudaMemcpyAsync((char*)h->L + (size_t)(NT & 1) * h->slot_elems * h->esz, h->term_L, h->slot_elems * h->esz,
                         cudaMemcpyDeviceToDevice, st));
    const double* term_s = h->has_term ? h->term_s : nullptr;
    L0("init", [&](cudaStream_t s) {
      launch_adj_init(g, h->ctrl, h->it, h->P.n_steps, h->objw, seed, term_s, h->dkref, g.ND, s);
    });
  }
  if (h->P.ckpt_policy == LKS_CKPT_BINOMIAL) {
    TRY(binomial_reverse<T>(h, st));
  } else if (h->P.ckpt_policy == LKS_CKPT_STORE_ALL) {
    Slots<T> S = ring_slots<T>(h);
    for (int t1 = NT; t1 >= 1; t1 -= h->chunk) {
      const int n = std::min(h->chunk, t1);
      L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t1, 0, s); });
      TRY(run_graph(h, (h->alks_mode ? "alks_sa_" : "adj_sa_") + std::to_string(n), st,
                    [&](Launcher& L) { enqueue_adj_steps<T>(h, L, S, n); }));
    }
  } else {
    Slots<T> S = ring_slots<T>(h);
    const int every = h->P.ckpt_every;
    const int nseg = (NT + every - 1) / every;
    for (int c = nseg - 1; c >= 0; --c) {
      const int t0 = c * every;
      const int n = std::min(every, NT - t0);
      if (h->P.ckpt_format == LKS_CKPT_NATIVE) {
        CK(cudaMemcpyAsync(h->ring, (char*)h->ckpt + (size_t)c * h->slot_elems * h->esz, h->slot_elems * h->esz,
                           cudaMemcpyDeviceToDevice, st));
      } else if (c == 0) {
        L0("ckpt", [&](cudaStream_t s) { launch_state_from_double<T>(g, (T*)h->ring, h->init_p, h->init_u, s); });
      } else {
        L0("ckpt", [&](cudaStream_t s) {
          launch_ckpt_restore_q(g, (float*)h->ring, h->ckq, h->ckkeys, h->P.ckpt_format, c, s);
        });
      }
      L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t0 + 1, t0, s); });
      TRY(run_graph(h, "rec_" + std::to_string(n), st, [&](Launcher& L) { enqueue_recompute<T>(h, L, S, n); }));
      L0("init", [&](cudaStream_t s) { launch_set_step(h->ctrl, t0 + n, t0, s); });
      TRY(run_graph(h, (h->alks_mode ? "alks_u_" : "adj_u_") + std::to_string(n), st,
                    [&](Launcher& L) { enqueue_adj_steps<T>(h, L, S, n); }));
    }
  }
  CK(cudaGetLastError());
  if (h->launch_error) return LKS_ERR_CUDA;
  return LKS_OK;
}

// Binomial schedule and its snapshot slots (native slots, or BF16 / FP16 values with per-plane
// ranges). ckpt_every snapshots, or with ckpt_every = 0 as many as hbm_budget_bytes holds after the
// rest of the workspace (at most n_steps - 1, the count beyond which the schedule cannot use more).
int allocate_snapshots(lks_handle* h, size_t slot_bytes) {
  const lks_problem& P = h->P;
  const int NT = P.n_steps, D = h->g.dim;
  const bool native = P.ckpt_format == LKS_CKPT_NATIVE;
  const size_t per_q = h->slot_elems * sizeof(unsigned short), per_keys = (size_t)(D + 1) * 2 * sizeof(unsigned);
  int s = P.ckpt_every;
  if (s == 0) {
    const size_t round = 256;  // each allocation is rounded up to 256 bytes
    const size_t have = P.hbm_budget_bytes > h->bytes + 2 * round ? P.hbm_budget_bytes - h->bytes - 2 * round : 0;
    const size_t per = native ? slot_bytes : per_q + per_keys;
    const size_t fit = have / per;
    s = (int)std::min<size_t>(fit, (size_t)std::max(NT - 1, 0));
  }
  h->bin_snapshots = s;
  h->bin_plan = binomial_plan(NT, s);
  h->nckpt = 0;  // the slots the schedule uses
  for (const BinOp& op : h->bin_plan)
    if (op.kind == LKS_BIN_FWD_SNAPSHOT || op.kind == LKS_BIN_STORE) h->nckpt = std::max(h->nckpt, op.a + 1);
  if (h->nckpt > 0 && native) {
    TRY(dalloc(h, &h->ckpt, (size_t)h->nckpt * slot_bytes));
  } else if (h->nckpt > 0) {  // snapshots in BF16 / FP16 with per-plane ranges
    TRY(dalloc(h, (void**)&h->ckq, (size_t)h->nckpt * per_q));
    TRY(dalloc(h, (void**)&h->ckkeys, (size_t)h->nckpt * per_keys));
  }
  return LKS_OK;
}

template <typename T>
int allocate(lks_handle* h) {
  Geo& g = h->g;
  const lks_problem& P = h->P;
  const int NT = P.n_steps, K = P.n_itr, D = g.dim;
  h->slot_elems = (long long)(D + 1) * g.N;
  const size_t slot_bytes = (size_t)h->slot_elems * sizeof(T);
  if (P.ckpt_policy == LKS_CKPT_STORE_ALL) {
    h->nring = NT + 1;
    h->nbox = NT;
  } else if (P.ckpt_policy == LKS_CKPT_BINOMIAL) {
    h->nring = 2;  // working pair of the reverse sweep
    h->nbox = 1;
    TRY(dalloc(h, &h->pp, 2 * slot_bytes));
    // the snapshots come last (allocate_snapshots): with ckpt_every = 0 their count is what the
    // budget holds after the rest of the workspace
  } else {
    h->nring = P.ckpt_every + 1;
    h->nbox = P.ckpt_every;
    h->nckpt = (NT + P.ckpt_every - 1) / P.ckpt_every;
    TRY(dalloc(h, &h->pp, 2 * slot_bytes));
    if (P.ckpt_format == LKS_CKPT_NATIVE) {
      TRY(dalloc(h, &h->ckpt, (size_t)h->nckpt * slot_bytes));
    } else {
      TRY(dalloc(h, (void**)&h->ckq, (size_t)h->nckpt * h->slot_elems * sizeof(unsigned short)));
      TRY(dalloc(h, (void**)&h->ckkeys, (size_t)h->nckpt * (D + 1) * 2 * sizeof(unsigned)));
    }
  }
  TRY(dalloc(h, &h->ring, (size_t)h->nring * slot_bytes));
  TRY(dalloc(h, &h->boxstore, (size_t)h->nbox * g.box_cells * D * sizeof(T)));
  TRY(dalloc(h, &h->L, 2 * slot_bytes));
  TRY(dalloc(h, &h->acc, (size_t)g.box_cells * D * sizeof(T)));
  TRY(dalloc(h, &h->scratch, (size_t)g.box_cells * (2 * D + 1) * sizeof(T)));
  TRY(dalloc(h, &h->kref, (size_t)g.ND * sizeof(T)));
  TRY(dalloc(h, (void**)&h->dkref, (size_t)g.ND * sizeof(double)));
  TRY(dalloc(h, (void**)&h->gamma, (size_t)g.ND * sizeof(double)));
  TRY(dalloc(h, (void**)&h->tmp_nd, (size_t)g.ND * sizeof(double)));
  double** chain_bufs[] = {&h->cg1, &h->cgtil, &h->cgbar, &h->cW, &h->kg1, &h->kgtil, &h->kgbar, &h->kW, &h->dv, &h->dtmp};
  for (double** b : chain_bufs) TRY(dalloc(h, (void**)b, (size_t)g.ND * sizeof(double)));
  TRY(dalloc(h, (void**)&h->vol, 2 * sizeof(double)));
  TRY(dalloc(h, &h->term_L, slot_bytes));
  TRY(dalloc(h, (void**)&h->term_s, kNdofFree * sizeof(double)));
  TRY(dalloc(h, (void**)&h->it, (size_t)(NT + 1) * (K + 1) * sizeof(Dof)));
  TRY(dalloc(h, (void**)&h->ctrl, sizeof(Ctrl)));
  TRY(dalloc(h, (void**)&h->mom, sizeof(Moments)));
  const long long bx = ((g.B[0] + kBoxCtaCellsX - 1) / kBoxCtaCellsX) * (long long)((g.B[1] + kBoxCtaCellsY - 1) / kBoxCtaCellsY) * g.B[2];
  const long long bd = ((long long)g.ND + kDesignPointsPerCta - 1) / kDesignPointsPerCta;
  const long long nblk = std::max(bx, bd) + 1;
  // per-CTA partials: up to 18 values (design-point reverse with free rotation), double-buffered
  TRY(dalloc(h, (void**)&h->partials, (size_t)nblk * 36 * sizeof(double)));
  h->pstride = 18 * nblk;  // two halves of up to 18 values per CTA (nblk >= the box tiles >= persistent CTAs)
  TRY(dalloc(h, (void**)&h->init_p, (size_t)g.N * sizeof(double)));
  TRY(dalloc(h, (void**)&h->init_u, (size_t)D * g.N * sizeof(double)));
  TRY(dalloc(h, (void**)&h->init_s, kNdofFree * sizeof(double)));
  TRY(dalloc(h, (void**)&h->objw, kNdofFree * sizeof(double)));
  if (P.ckpt_policy == LKS_CKPT_BINOMIAL) TRY(allocate_snapshots(h, slot_bytes));
  CK(cudaMemset(h->ctrl, 0, sizeof(Ctrl)));
  CK(cudaMemset(h->L, 0, 2 * slot_bytes));
  CK(cudaMemcpy(h->objw, P.obj_weights, g.ns * sizeof(double), cudaMemcpyHostToDevice));
  return LKS_OK;
}

int set_default_initial_state(lks_handle* h) {
  const Geo& g = h->g;
  std::vector<double> p((size_t)g.N, 0.0), u((size_t)g.dim * g.N, 0.0);
  for (long long n = 0; n < g.N; ++n) u[n] = h->P.u_in;
  CK(cudaMemcpy(h->init_p, p.data(), p.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->init_u, u.data(), u.size() * sizeof(double), cudaMemcpyHostToDevice));
  for (int a = 0; a < kNdofFree; ++a) h->host_s0[a] = 0.0;
  for (int a = 0; a < 3; ++a) h->host_s0[a] = h->P.body_centre[a];
  if (g.ax == AX_FREE) h->host_s0[S_R] = h->host_s0[S_R + 4] = h->host_s0[S_R + 8] = 1.0;  // R = I
  CK(cudaMemcpy(h->init_s, h->host_s0, g.ns * sizeof(double), cudaMemcpyHostToDevice));
  return LKS_OK;
}

// Box for the current initial state: the rotated (circumscribed) box if the body can rotate or
// starts rotated. The buffers were sized at creation for the largest box that fits.
int refresh_box(lks_handle* h) {
  bool start_rotated = h->host_s0[6] != 0.0;
  if (h->g.ax == AX_FREE) {
    start_rotated = false;
    for (int i = 0; i < 9; ++i) start_rotated = start_rotated || h->host_s0[S_R + i] != ((i % 4 == 0) ? 1.0 : 0.0);
  }
  const bool rotated = (h->g.dof_mask & LKS_DOF_ROT) || start_rotated;
  if (rotated && !h->box_rot_ok) return LKS_ERR_UNSUPPORTED;
  const int old[3] = {h->g.B[0], h->g.B[1], h->g.B[2]};
  setup_box(&h->g, h->P.design_radius, rotated);
  h->g.coop_fwd = h->g.coop_adj = 0;
  if (h->coop_mode != 0) setup_coop(&h->g, h->prec == LKS_FP64);
  if (h->coop_mode == 2 && (h->g.dim != 2 || box_tiles(h->g) <= h->g.coop_fwd))
    h->g.coop_fwd = h->g.coop_adj = 0;  // measured slower there: a grid barrier costs about twice a
                                         // kernel boundary in a graph; only multi-wave 2D boxes gain
  if (old[0] != h->g.B[0] || old[1] != h->g.B[1] || old[2] != h->g.B[2]) clear_graphs(h);
  return LKS_OK;
}

}  // namespace

extern "C" {

const char* lks_status_string(int s) {
  switch (s) {
    case LKS_OK: return "ok";
    case LKS_ERR_ARG: return "invalid argument";
    case LKS_ERR_OOM: return "device allocation failed";
    case LKS_ERR_BUDGET: return "workspace exceeds hbm_budget_bytes";
    case LKS_ERR_UNSTABLE: return "nu <= 0 (A >= 3/4)";
    case LKS_ERR_BODY_OUTSIDE: return "body reaches a non-periodic boundary layer";
    case LKS_ERR_NONFINITE: return "non-finite force, torque or state";
    case LKS_ERR_ORDER: return "call order (forward before adjoint before sensitivity)";
    case LKS_ERR_CUDA: return "CUDA runtime error";
    case LKS_ERR_UNSUPPORTED: return "unsupported configuration";
    case LKS_ERR_TIMEOUT: return "a bounded wait on the device timed out";
    default: return "unknown status";
  }
}

int lks_last_cuda_error(void) { return g_last_cuda_error; }

size_t lks_problem_size(void) { return sizeof(lks_problem); }

long long lks_binomial_plan(int n_steps, int snapshots, int* ops, long long capacity) {
  if (n_steps < 1 || snapshots < 0 || capacity < 0 || (capacity > 0 && !ops)) return -(long long)LKS_ERR_ARG;
  const std::vector<BinOp> plan = binomial_plan(n_steps, snapshots);
  const long long n = (long long)plan.size();
  for (long long i = 0; i < std::min(n, capacity); ++i) {
    ops[4 * i] = plan[i].kind;
    ops[4 * i + 1] = plan[i].a;
    ops[4 * i + 2] = plan[i].b;
    ops[4 * i + 3] = plan[i].c;
  }
  return n;
}

int lks_dof_count(const lks_problem* P) {
  if (!P) return 0;
  return P->rot_axis == LKS_ROT_FREE ? LKS_NDOF_FREE : LKS_NDOF_AXIS;
}

int lks_create(const lks_problem* P, lks_handle** out) {
  if (!out) return LKS_ERR_ARG;
  *out = nullptr;
  int v = validate_problem(P);
  if (v != LKS_OK) return v;
  lks_handle* h = new (std::nothrow) lks_handle();
  if (!h) return LKS_ERR_OOM;
  h->P = *P;
  h->prec = P->field_precision;
  h->esz = (h->prec == LKS_FP64) ? 8 : 4;
  bool rot_ok = true;
  if (make_geometry(P, &h->g, &rot_ok) != LKS_OK) {
    delete h;
    return LKS_ERR_UNSUPPORTED;
  }
  h->box_rot_ok = rot_ok;
  const Geo& g = h->g;
  int r = (h->prec == LKS_FP64) ? allocate<double>(h) : allocate<float>(h);
  if (r == LKS_OK) r = set_default_initial_state(h);
  if (r == LKS_OK && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) r = LKS_ERR_CUDA;
  if (r == LKS_OK && g.dim == 3) {
    if (h->prec == LKS_FP64) prepare_stencil3d<double>();
    else prepare_stencil3d<float>();
    if (cudaGetLastError() != cudaSuccess) r = LKS_ERR_CUDA;
  }
  if (r != LKS_OK) {
    lks_destroy(h);
    return r;
  }
  refresh_box(h);  // the default state starts unrotated: always fits
  *out = h;
  return LKS_OK;
}

int lks_set_initial_state(lks_handle* h, const double* p, const double* u, const double* s) {
  if (!h) return LKS_ERR_ARG;
  const Geo& g = h->g;
  // checked on the host before any device work: a NaN or an infinity is refused, not marched
  auto finite = [](const double* a, long long n) {
    for (long long i = 0; i < n; ++i)
      if (!std::isfinite(a[i])) return false;
    return true;
  };
  if ((p && !finite(p, g.N)) || (u && !finite(u, (long long)g.dim * g.N)) || (s && !finite(s, g.ns)))
    return LKS_ERR_NONFINITE;
  int r = set_default_initial_state(h);
  if (r != LKS_OK) return r;
  if (p) CK(cudaMemcpy(h->init_p, p, (size_t)g.N * sizeof(double), cudaMemcpyHostToDevice));
  if (u) CK(cudaMemcpy(h->init_u, u, (size_t)g.dim * g.N * sizeof(double), cudaMemcpyHostToDevice));
  if (s) {
    for (int a = 0; a < g.ns; ++a) h->host_s0[a] = s[a];
    CK(cudaMemcpy(h->init_s, h->host_s0, g.ns * sizeof(double), cudaMemcpyHostToDevice));
  }
  // the reverse sweep restores its first segment from the initial state: a new one voids the forward
  h->fwd_done = h->adj_done = h->exact_done = h->alks_done = false;
  return refresh_box(h);
}

int lks_forward(lks_handle* h, const double* gamma_dev, double* J_host, void* stream) {
  if (!h || !gamma_dev) return LKS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const Geo& g = h->g;
  h->fwd_done = h->adj_done = h->exact_done = h->alks_done = false;
  if ((const void*)gamma_dev != (const void*)h->gamma)
    CK(cudaMemcpyAsync(h->gamma, gamma_dev, (size_t)g.ND * sizeof(double), cudaMemcpyDeviceToDevice, st));
  Launcher L0{h, st, false};
  CK(cudaMemsetAsync((char*)h->ctrl + offsetof(Ctrl, prep_status), 0, sizeof(int), st));
  // design chain gamma -> gamma-bar (Sec. 3.2, 4.2), then kappa^ref of gamma-bar
  L0.n("prep", 2, [&](cudaStream_t s) { launch_design_chain(g, h->gamma, h->cg1, h->cgtil, h->cgbar, h->cW, s); });
  if (h->prec == LKS_FP64)
    L0("prep", [&](cudaStream_t s) { launch_prep<double>(g, h->cgbar, h->P.kappa_max, h->P.q, (double*)h->kref, h->mom, h->partials, h->ctrl, s); });
  else
    L0("prep", [&](cudaStream_t s) { launch_prep<float>(g, h->cgbar, h->P.kappa_max, h->P.q, (float*)h->kref, h->mom, h->partials, h->ctrl, s); });
  int r = (h->prec == LKS_FP64) ? forward_impl<double>(h, st) : forward_impl<float>(h, st);
  if (r != LKS_OK) return r;
  Dof last;
  Ctrl c;
  CK(cudaMemcpyAsync(&last, h->it + (size_t)h->P.n_steps * (g.K + 1), sizeof(Dof), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h->timing) collect_timers(h);
  double J = 0.0;
  for (int a = 0; a < g.ns; ++a) J += h->P.obj_weights[a] * last.s[a];
  if (J_host) *J_host = J;
  if (c.status & ST_SYNC_TIMEOUT) return LKS_ERR_TIMEOUT;
  if (c.status & ST_BODY_OUTSIDE) return LKS_ERR_BODY_OUTSIDE;
  if (c.status & ST_BOX_OVERFLOW) return LKS_ERR_BODY_OUTSIDE;
  if ((c.status & ST_NONFINITE) || (c.prep_status & ST_NONFINITE) || !std::isfinite(J)) return LKS_ERR_NONFINITE;
  h->fwd_done = true;
  return LKS_OK;
}

int lks_adjoint(lks_handle* h, double seed, void* stream) {
  if (!h) return LKS_ERR_ARG;
  if (!h->fwd_done) return LKS_ERR_ORDER;
  cudaStream_t st = (cudaStream_t)stream;
  h->adj_done = h->exact_done = false;
  int r = (h->prec == LKS_FP64) ? adjoint_impl<double>(h, seed, st) : adjoint_impl<float>(h, seed, st);
  if (r != LKS_OK) return r;
  // a grid barrier or tile copy whose wait timed out is reported through the status word
  if (h->g.coop_adj > 0 || lks_stencil_form(h) == 1) {
    int status = 0;
    CK(cudaMemcpyAsync(&status, (const char*)h->ctrl + offsetof(Ctrl, status), sizeof(int), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    if (status & ST_SYNC_TIMEOUT) return LKS_ERR_TIMEOUT;
  }
  if (h->timing) {
    CK(cudaStreamSynchronize(st));
    collect_timers(h);
  }
  h->adj_done = h->exact_done = true;
  return LKS_OK;
}

int lks_set_continuation(lks_handle* h, double q, double proj_beta) {
  if (!h) return LKS_ERR_ARG;
  if (!(q > 0.0) || !std::isfinite(q) || !(proj_beta >= 0.0) || !std::isfinite(proj_beta)) return LKS_ERR_ARG;
  if (proj_beta > 0.0 && !(h->P.proj_eta > 0.0 && h->P.proj_eta < 1.0)) return LKS_ERR_ARG;
  CK(cudaDeviceSynchronize());
  h->P.q = q;
  h->P.proj_beta = proj_beta;
  h->g.pbeta = proj_beta;
  clear_graphs(h);  // no captured launch may keep the old values
  h->fwd_done = h->adj_done = h->exact_done = h->alks_done = false;
  return LKS_OK;
}

int lks_adjoint_alks(lks_handle* h, double seed, void* stream) {
  if (!h) return LKS_ERR_ARG;
  if (!h->fwd_done) return LKS_ERR_ORDER;
  if (h->g.ax == AX_FREE || h->has_term) return LKS_ERR_UNSUPPORTED;
  const Geo& g = h->g;
  if (!h->al_A) {
    h->al_astride = (long long)alks_planes(g.dim) * g.N;
    TRY(dalloc(h, &h->al_A, 2 * (size_t)h->al_astride * h->esz));
    TRY(dalloc(h, &h->al_box, (size_t)(1 + 2 * g.dim) * g.box_cells * h->esz));
    TRY(dalloc(h, &h->al_z, (size_t)g.dim * g.N * h->esz));
    TRY(dalloc(h, &h->al_sens, (size_t)alks_sens_values(g.dim) * g.ND * h->esz));
    const long long nb = (g.ND + kDesignPointsPerCta - 1) / kDesignPointsPerCta;
    TRY(dalloc(h, &h->al_part, (size_t)nb * alks_partial_values(g.dim) * 2 * sizeof(double)));
  }
  cudaStream_t st = (cudaStream_t)stream;
  h->adj_done = h->alks_done = false;  // the exact adjoint's lambda(0) is untouched
  h->alks_mode = true;
  int r = (h->prec == LKS_FP64) ? adjoint_impl<double>(h, seed, st) : adjoint_impl<float>(h, seed, st);
  h->alks_mode = false;
  if (r != LKS_OK) return r;
  if (h->timing) {
    CK(cudaStreamSynchronize(st));
    collect_timers(h);
  }
  h->adj_done = h->alks_done = true;
  return LKS_OK;
}

int lks_get_alks_adjoint(lks_handle* h, double* p, double* u, double* s, double* body) {
  if (!h) return LKS_ERR_ARG;
  if (!h->alks_done) return LKS_ERR_ORDER;
  const int d = h->g.dim;
  const long long N = h->g.N, M = h->al_astride;
  std::vector<char> raw((size_t)M * h->esz);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(raw.data(), h->al_A, raw.size(), cudaMemcpyDeviceToHost));  // the moments at t = 0: slot 0
  auto val = [&](long long i) {
    return (h->esz == 8) ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
  };
  for (long long n = 0; n < N; ++n) {
    if (p) p[n] = val(n);
    for (int a = 0; a < d; ++a) {
      if (u) u[a * N + n] = val((1 + a) * N + n);
      for (int b = 0; b < d; ++b) {
        const int k = (a == b) ? a : (d == 2 ? 2 : (a + b == 1 ? 3 : (a + b == 2 ? 4 : 5)));
        if (s) s[((long long)a * d + b) * N + n] = val((1 + d + k) * N + n);
      }
    }
  }
  if (body) {
    Ctrl c;
    CK(cudaMemcpy(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    for (int a = 0; a < 8; ++a) body[a] = c.al_b[a];
  }
  return LKS_OK;
}

int lks_sensitivity(lks_handle* h, double* out, void* stream) {
  if (!h || !out) return LKS_ERR_ARG;
  if (!h->adj_done) return LKS_ERR_ORDER;
  cudaStream_t st = (cudaStream_t)stream;
  // dJ/dgamma-bar at gamma-bar, then the transpose of the design chain
  launch_sensitivity(h->g, h->cgbar, h->dkref, h->P.kappa_max, h->P.q, h->dv, st);
  launch_design_chain_T(h->g, h->cgtil, h->cW, h->dv, h->dtmp, out, st);
  h->launches += 4;
  CK(cudaGetLastError());
  return LKS_OK;
}

int lks_warm_start(lks_handle* h, int with_adjoint, void* stream) {
  if (!h) return LKS_ERR_ARG;
  if (!h->fwd_done || (with_adjoint && !h->exact_done)) return LKS_ERR_ORDER;
  cudaStream_t st = (cudaStream_t)stream;
  const Geo& g = h->g;
  const int NT = h->P.n_steps;
  const void* src = (h->P.ckpt_policy == LKS_CKPT_STORE_ALL)
                        ? (const char*)h->ring + (size_t)NT * h->slot_elems * h->esz
                        : (const char*)h->pp + (size_t)(NT & 1) * h->slot_elems * h->esz;
  if (h->prec == LKS_FP64)
    launch_state_to_double<double>(g, (const double*)src, h->init_p, h->init_u, st);
  else
    launch_state_to_double<float>(g, (const float*)src, h->init_p, h->init_u, st);
  Dof last;
  CK(cudaMemcpyAsync(&last, h->it + (size_t)NT * (g.K + 1), sizeof(Dof), cudaMemcpyDeviceToHost, st));
  if (with_adjoint) {
    CK(cudaMemcpyAsync(h->term_L, h->L, h->slot_elems * h->esz, cudaMemcpyDeviceToDevice, st));  // lambda(0)
    CK(cudaMemcpyAsync(h->term_s, (const char*)h->ctrl + offsetof(Ctrl, lam_s0), g.ns * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  h->launches += 1;
  for (int a = 0; a < kNdofFree; ++a) h->host_s0[a] = (a < g.ns) ? last.s[a] : 0.0;
  CK(cudaMemcpy(h->init_s, h->host_s0, g.ns * sizeof(double), cudaMemcpyHostToDevice));
  h->has_term = with_adjoint != 0;
  h->fwd_done = h->adj_done = h->exact_done = h->alks_done = false;
  return refresh_box(h);
}

int lks_constraint(lks_handle* h, const double* gamma_dev, double* G_host, double* dGdgamma_dev, void* stream) {
  if (!h || !gamma_dev || !G_host) return LKS_ERR_ARG;
  if (!(h->P.v_min > 0.0)) return LKS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const Geo& g = h->g;
  launch_design_chain(g, gamma_dev, h->kg1, h->kgtil, h->kgbar, h->kW, st);
  launch_volume(g, h->kgbar, h->vol, st);
  double vol[2];
  CK(cudaMemcpyAsync(vol, h->vol, sizeof(vol), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double scale = 1.0 / (h->P.v_min * vol[1]);
  *G_host = vol[0] * scale - 1.0;
  h->launches += 3;
  if (dGdgamma_dev) {
    launch_fill_domain(g, scale, h->dv, st);
    launch_design_chain_T(g, h->kgtil, h->kW, h->dv, h->dtmp, dGdgamma_dev, st);
    h->launches += 4;
  }
  CK(cudaGetLastError());
  return LKS_OK;
}

int lks_gradient_host(lks_handle* h, const double* gamma_host, double* J_host, double* dJdgamma_host, void* stream) {
  if (!h || !gamma_host) return LKS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nb = (size_t)h->g.ND * sizeof(double);
  CK(cudaMemcpyAsync(h->gamma, gamma_host, nb, cudaMemcpyHostToDevice, st));
  int r = lks_forward(h, h->gamma, J_host, stream);
  if (r != LKS_OK) return r;
  r = lks_adjoint(h, 1.0, stream);
  if (r != LKS_OK) return r;
  r = lks_sensitivity(h, h->tmp_nd, stream);
  if (r != LKS_OK) return r;
  if (dJdgamma_host) CK(cudaMemcpyAsync(dJdgamma_host, h->tmp_nd, nb, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return LKS_OK;
}

int lks_get_dof_history(lks_handle* h, double* buf, size_t n) {
  if (!h || !buf) return LKS_ERR_ARG;
  if (!h->fwd_done) return LKS_ERR_ORDER;
  const int NT = h->P.n_steps, K = h->g.K, ns = h->g.ns;
  if (n < (size_t)(NT + 1) * ns) return LKS_ERR_ARG;
  std::vector<Dof> rows((size_t)(NT + 1) * (K + 1));
  CK(cudaMemcpy(rows.data(), h->it, rows.size() * sizeof(Dof), cudaMemcpyDeviceToHost));
  for (int t = 0; t <= NT; ++t)
    for (int a = 0; a < ns; ++a) buf[(size_t)t * ns + a] = rows[(size_t)t * (K + 1)].s[a];
  return LKS_OK;
}

int lks_get_state(lks_handle* h, double* p, double* u) {
  if (!h) return LKS_ERR_ARG;
  if (!h->fwd_done) return LKS_ERR_ORDER;
  const int NT = h->P.n_steps;
  const void* src;
  if (h->P.ckpt_policy == LKS_CKPT_STORE_ALL)
    src = (const char*)h->ring + (size_t)NT * h->slot_elems * h->esz;
  else
    src = (const char*)h->pp + (size_t)(NT & 1) * h->slot_elems * h->esz;
  const long long M = h->slot_elems, N = h->g.N;
  std::vector<char> raw((size_t)M * h->esz);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost));
  for (long long i = 0; i < M; ++i) {
    const double v = (h->esz == 8) ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
    if (i < N) {
      if (p) p[i] = v;
    } else if (u) {
      u[i - N] = v;
    }
  }
  return LKS_OK;
}

int lks_get_initial_adjoint(lks_handle* h, double* lp, double* lu, double* ls) {
  if (!h) return LKS_ERR_ARG;
  if (!h->exact_done) return LKS_ERR_ORDER;
  const long long M = h->slot_elems, N = h->g.N;
  std::vector<char> raw((size_t)M * h->esz);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(raw.data(), h->L, raw.size(), cudaMemcpyDeviceToHost));  // lambda(0) sits in slot 0
  for (long long i = 0; i < M; ++i) {
    const double v = (h->esz == 8) ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
    if (i < N) {
      if (lp) lp[i] = v;
    } else if (lu) {
      lu[i - N] = v;
    }
  }
  if (ls) {
    Ctrl c;
    CK(cudaMemcpy(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    for (int a = 0; a < h->g.ns; ++a) ls[a] = c.lam_s0[a];
  }
  return LKS_OK;
}

int lks_support_sets(lks_handle* h, const double* s_host, int* box_host, long long* stats_host, size_t capacity) {
  if (!h || !s_host || !box_host) return LKS_ERR_ARG;
  Geo g = h->g;
  for (int a = 0; a < g.ns; ++a)
    if (!std::isfinite(s_host[a])) return LKS_ERR_NONFINITE;
  for (int a = 0; a < 3; ++a)
    if (std::fabs(s_host[a]) > 1e9) return LKS_ERR_ARG;
  Dof d;
  const bool free_rot = g.ax == AX_FREE;
  for (int a = 0; a < kNdofFree; ++a) d.s[a] = (a < g.ns) ? s_host[a] : 0.0;
  d.cs = free_rot ? 1.0 : std::cos(d.s[6]);
  d.sn = free_rot ? 0.0 : std::sin(d.s[6]);
  dof_views(&d, free_rot);
  // the box a march starting from s would use (as lks_set_initial_state chooses it)
  bool start_rotated = !free_rot && d.s[6] != 0.0;
  if (free_rot)
    for (int i = 0; i < 9; ++i) start_rotated = start_rotated || d.s[S_R + i] != ((i % 4 == 0) ? 1.0 : 0.0);
  const bool rotated = (g.dof_mask & LKS_DOF_ROT) || start_rotated;
  if (rotated && !h->box_rot_ok) return LKS_ERR_UNSUPPORTED;
  setup_box(&g, h->P.design_radius, rotated);
  for (int a = 0; a < 3; ++a) {
    box_host[a] = (a < g.dim) ? d.xi[a] - g.hb[a] - g.s - g.margin : 0;
    box_host[3 + a] = g.B[a];
  }
  if (!stats_host) return LKS_OK;
  if (capacity < (size_t)(5 * g.box_cells)) return LKS_ERR_ARG;
  long long* out = nullptr;
  CK(cudaMalloc((void**)&out, sizeof(long long) * 5 * (size_t)g.box_cells));
  if (h->prec == LKS_FP64)
    launch_support_sets<double>(g, d, (const double*)h->kref, out, 0);
  else
    launch_support_sets<float>(g, d, (const float*)h->kref, out, 0);
  cudaError_t e = cudaMemcpy(stats_host, out, sizeof(long long) * 5 * (size_t)g.box_cells, cudaMemcpyDeviceToHost);
  cudaFree(out);
  if (e != cudaSuccess) {
    g_last_cuda_error = (int)e;
    return LKS_ERR_CUDA;
  }
  h->launches += 1;
  return LKS_OK;
}

namespace {
// Sets or clears one bit of the control block's test-hook word.
int set_skip_bit(lks_handle* h, int bit, int on) {
  int v = 0;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&v, (char*)h->ctrl + offsetof(Ctrl, sync_skip), sizeof(int), cudaMemcpyDeviceToHost));
  v = on ? (v | bit) : (v & ~bit);
  CK(cudaMemcpy((char*)h->ctrl + offsetof(Ctrl, sync_skip), &v, sizeof(int), cudaMemcpyHostToDevice));
  return LKS_OK;
}
}  // namespace

int lks_debug_sync_skip(lks_handle* h, int skip) {
  if (!h) return LKS_ERR_ARG;
  return set_skip_bit(h, 1, skip);
}

int lks_debug_copy_skip(lks_handle* h, int skip) {
  if (!h) return LKS_ERR_ARG;
  return set_skip_bit(h, 2, skip);
}

int lks_persistent_coupling(lks_handle* h, int mode) {
  if (!h || mode < -1 || mode > 2) return -LKS_ERR_ARG;
  if (mode >= 0 && mode != h->coop_mode) {
    if (cudaDeviceSynchronize() != cudaSuccess) return -LKS_ERR_CUDA;
    h->coop_mode = mode;
    const int r = refresh_box(h);
    if (r != LKS_OK) return -r;
    clear_graphs(h);
  }
  return (h->g.coop_fwd > 0 && h->g.coop_adj > 0) ? 1 : 0;
}

long long lks_launch_count(const lks_handle* h) { return h ? h->launches : 0; }

int lks_set_kernel_timing(lks_handle* h, int enable) {
  if (!h) return LKS_ERR_ARG;
  h->timing = enable != 0;
  for (auto& kv : h->timers) {
    kv.second.ms = 0.0;
    kv.second.launches = 0;
    kv.second.used = 0;
  }
  return LKS_OK;
}

int lks_kernel_time(lks_handle* h, const char* family, double* ms, long long* launches) {
  if (!h || !family) return LKS_ERR_ARG;
  auto itf = h->timers.find(family);
  if (itf == h->timers.end()) {
    if (ms) *ms = 0.0;
    if (launches) *launches = 0;
    return LKS_OK;
  }
  if (ms) *ms = itf->second.ms;
  if (launches) *launches = itf->second.launches;
  return LKS_OK;
}

size_t lks_workspace_bytes(const lks_handle* h) { return h ? h->bytes : 0; }

int lks_checkpoint_slots(const lks_handle* h) {
  if (!h) return -LKS_ERR_ARG;
  if (h->P.ckpt_policy == LKS_CKPT_BINOMIAL) return h->bin_snapshots;
  if (h->P.ckpt_policy == LKS_CKPT_UNIFORM) return h->nckpt;
  return h->P.n_steps + 1;
}

int lks_stencil_form(const lks_handle* h) {
  if (!h) return -LKS_ERR_ARG;
  return (h->prec == LKS_FP32 && stencil3d_q_fits(h->g)) ? 1 : 0;
}

void lks_destroy(lks_handle* h) {
  if (!h) return;
  clear_graphs(h);
  for (auto& kv : h->timers)
    for (auto& p : kv.second.pairs) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
  for (void* p : h->allocs) cudaFree(p);
  if (h->cap) cudaStreamDestroy(h->cap);
  delete h;
}

}  // extern "C"
