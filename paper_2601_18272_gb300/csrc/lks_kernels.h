// Host-side launchers of the LKS kernels (internal to the library; the public boundary is
// include/lks.h).
#pragma once

#include "lks_device.cuh"

namespace lks {

// One launch path for every kernel of the library (grid, block, dynamic shared memory, stream).
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Cooperative launch (every CTA of the grid co-resident, or the launch fails): the persistent
// coupling kernels, whose CTAs meet at grid barriers.
template <typename... KArgs, typename... Args>
inline void launch_coop(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                        Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int kTileX = 32;  // 3D stencil column width (cells); boundary pairs must not straddle columns
constexpr int kTileY3 = 16;  // 3D stencil column height (the column marches over a chunk of z planes)
constexpr int kStripWarps = 4;  // 2D stencil: warps per CTA, each streaming its own strip of rows

// 2D stencil strips: W output columns per warp (<= 28), ntx column tiles, nstrip row strips.
struct StripPlan {
  int W, ntx, nstrip;
};
constexpr int kLanesPerCell = 4;                      // threads per box cell / design point in the body kernels
constexpr int kBoxCtaCellsX = 16, kBoxCtaCellsY = 8;  // box cells per body-kernel CTA in 3D (and for sizing)
constexpr int kBoxCtaCellsY2D = 16;                   // in 2D: 1024-thread CTAs, one per SM
constexpr int kDesignPointsPerCta = 64;               // design points per reverse design-side CTA

// Kernels that work on one time step take di: the step is ctrl->t0 + di (forward kernels) or
// ctrl->t0 - di (adjoint kernels), so one captured graph of L steps serves every chunk.

// Forward LKS predictor + boundary values for step t: slot(t-1) -> slot(t).
template <typename T>
void launch_stencil_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, int di, cudaStream_t st);

// Transpose of the predictor at the state slot(t-1): adjoint fields Lb[t&1] -> Lb[(t-1)&1]
// (each Lb slot holds dim+1 planes).
template <typename T>
void launch_stencil_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, const Ctrl* ctrl, int di,
                        cudaStream_t st);

// 3D forms (D3Q15), called by the launchers above; prepare_stencil3d sets their shared-memory
// attributes and must run once before the first launch (outside stream capture).
template <typename T>
void prepare_stencil3d();
template <typename T>
void launch_stencil3d_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, int di, cudaStream_t st);
template <typename T>
void launch_stencil3d_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, const Ctrl* ctrl, int di,
                          cudaStream_t st);
// Row-streamed FP32 forms (TMA-fed, packed FP32x2) for grids periodic in y and z with nx a multiple
// of 4 and at least 64 and ny at least 16: true if this geometry takes them. The launchers return false (launching
// nothing) where it does not, or where a tensor map cannot be encoded. A copy whose wait runs out
// (about a second) sets ST_SYNC_TIMEOUT in ctrl->status.
bool stencil3d_q_fits(const Geo& g);
void prepare_stencil3d_q();
bool launch_stencil3d_q_fwd(const Geo& g, const Slots<float>& S, const Ctrl* ctrl, int di, cudaStream_t st);
bool launch_stencil3d_q_adj(const Geo& g, const Slots<float>& S, float* Lb, long long lstride, const Ctrl* ctrl,
                            int di, cudaStream_t st);

// Design preparation: kappa^ref from gamma (Eq. brinkman_coefficient), moments.
template <typename T>
void launch_prep(const Geo& g, const double* gamma, double kappa_max, double q, T* kref, Moments* mom,
                 double* partials, Ctrl* ctrl, cudaStream_t st);

// Coupling iteration k (1..K) of step t: the EOM of the previous iteration (from the other half
// of the double-buffered partials, pstride elements apart), then spread, Brinkman, force/torque
// partials (float2 double-float pairs for FP32 fields, doubles for FP64). On k == K writes u(t) into
// slot(t) and optionally u* into the box store.
// Kernels one launch_couple issues: 2 when the previous iteration's finish runs as its own CTA.
int couple_kernels(const Geo& g);
template <typename T>
void launch_couple(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                   void* partials, long long pstride, int k, T* boxstore, int nbox, int di, cudaStream_t st);
// EOM of the last iteration of a forward run ending at step t_last.
template <typename T>
void launch_couple_last(const Geo& g, Ctrl* ctrl, Dof* it, const Moments* mom, const void* partials,
                        long long pstride, int t_last, cudaStream_t st);

// Persistent form of the N_itr coupling iterations of step t (one cooperative launch of
// g.coop_fwd CTAs that stride over the box tiles, with a bounded grid barrier after each
// iteration's partial sums): the same cell work and fixed-order sums as launch_couple, and the EOM
// of iteration N_itr too, so no finish kernel follows. Sets ctrl->coop fields through sync_bar.
template <typename T>
void launch_couple_coop(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                        void* partials, long long pstride, T* boxstore, int nbox, int di, cudaStream_t st);
// Persistent form of the reverse of the N_itr coupling iterations of step t (cell phase, barrier,
// design-point phase, barrier, finish with the EOM reverse in every CTA), one cooperative launch of
// g.coop_adj CTAs in place of launch_adj_cell + launch_adj_design for k = N_itr..1.
template <typename T>
void launch_adj_coop(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, double* dkref, void* partials, long long pstride, int di,
                     cudaStream_t st);
// CTAs of the cooperative kernels for this geometry and field type: the box tiles, at most as many
// as the device holds at once (0 if the kernel cannot be resident); sets g->coop_fwd, g->coop_adj.
void setup_coop(Geo* g, bool fp64);

// Recompute: Brinkman update with the stored iterate s^(K-1); writes u(t) and the box store of u*.
template <typename T>
void launch_apply(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, const Dof* it, const T* kref, T* boxstore,
                  int nbox, int di, cudaStream_t st);

// Reverse of coupling iteration k: cell side (Brinkman and interpolation reverse)...
template <typename T>
void launch_adj_cell(const Geo& g, const Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, int k, int di, cudaStream_t st);

// ... and design-point side (spread/transform reverse, dJ/dkappa^ref, per-CTA partials of
// dJ/ds^(k-1)), then a one-CTA finish kernel with the EOM reverse of the previous iteration.
template <typename T>
void launch_adj_design(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* scratch, double* dkref,
                       void* partials, int k, int di, cudaStream_t st);

// Test export: the design points the coupling's gather accepts for each cell of the box of the
// iterate s, as out[box cell][5] = (count, least index or -1, largest index, sum, sum of squares).
template <typename T>
void launch_support_sets(const Geo& g, const Dof& s, const T* kref, long long* out, cudaStream_t st);

// Design chain (cyclic expansion, density filter, Heaviside projection) gamma -> gbar, keeping the
// filtered field gtil and the filter normaliser W for the transpose; active unless every step is off.
bool design_chain_active(const Geo& g);
void launch_design_chain(const Geo& g, const double* gamma, double* g1, double* gtil, double* gbar, double* W,
                         cudaStream_t st);
// Transpose: out = (dgbar/dgamma)^T v; v and tmp are overwritten.
void launch_design_chain_T(const Geo& g, const double* gtil, const double* W, double* v, double* tmp, double* out,
                           cudaStream_t st);
// out2[0] = sum of gbar over the design domain, out2[1] = the domain's point count.
void launch_volume(const Geo& g, const double* gbar, double* out2, cudaStream_t st);
// out = value on the design domain, 0 elsewhere.
void launch_fill_domain(const Geo& g, double value, double* out, cudaStream_t st);

// Initial state (double) -> slot(0); s0 -> it row 0; ctrl reset for a forward (t0 = 1, base 0).
template <typename T>
void launch_init_forward(const Geo& g, const Slots<T>& S, const double* p0, const double* u0, const double* s0dev,
                         Dof* it, Ctrl* ctrl, cudaStream_t st);

// Set ctrl->t0 and ctrl->base.
void launch_set_step(Ctrl* ctrl, int t0, int base, cudaStream_t st);

// Adjoint initialisation: dJ/ds(N_t) = seed * w, EOM reverse of iteration K, zero dJ/dkappa^ref.
// term_s (device, nullable): a terminal DOF adjoint added to seed * w (the periodic warm start).
void launch_adj_init(const Geo& g, Ctrl* ctrl, const Dof* it, int nt, const double* objw, double seed,
                     const double* term_s, double* dkref, int nd, cudaStream_t st);
// A state slot (T) -> p0 [N], u0 [dim][N] as doubles.
template <typename T>
void launch_state_to_double(const Geo& g, const T* src, double* p0, double* u0, cudaStream_t st);

// dJ/dgamma-bar = dJ/dkappa^ref * dkappa^ref/dgamma-bar at gamma-bar (Eq. brinkman_coefficient).
void launch_sensitivity(const Geo& g, const double* gbar, const double* dkref, double kappa_max, double q,
                        double* out, cudaStream_t st);

// Reduced-precision checkpoint (FP32 fields) of the state at step ctrl->t0 + di into checkpoint
// c = step / every: per-plane range keys[c][plane][2] and q[c][plane][N] in BF16 or FP16.
void launch_ckpt_pack_q(const Geo& g, const Slots<float>& S, unsigned short* q, unsigned* keys, int fmt, int every,
                        const Ctrl* ctrl, int di, cudaStream_t st);
// The same for the state at src ((dim+1) planes of N floats) into checkpoint c.
void launch_ckpt_pack_q_at(const Geo& g, const float* src, unsigned short* q, unsigned* keys, int fmt, int c,
                           cudaStream_t st);
// Restore of checkpoint c into dst ((dim+1) planes of N floats).
void launch_ckpt_restore_q(const Geo& g, float* dst, const unsigned short* q, const unsigned* keys, int fmt, int c,
                           cudaStream_t st);
// State (p0 [N], u0 [dim][N] in FP64) into dst in the field type.
template <typename T>
void launch_state_from_double(const Geo& g, T* dst, const double* p0, const double* u0, cudaStream_t st);

// Checkpoint of the state at step ctrl->t0 + di into ckpt[step / every] (native precision).
template <typename T>
void launch_ckpt_pack(const Geo& g, const Slots<T>& S, T* ckpt, long long cstride, int every, const Ctrl* ctrl, int di,
                      cudaStream_t st);


// The paper-form adjoint (ALKS; lks_alks.cu). Moment slots Ab[t & 1] hold p~, u~[dim] and the
// distinct entries of s~ (alks_planes planes of N values); abox: kappa, u^S[dim], the omega~ source
// [dim] per box cell; sstore: alks_sens_values per design point; partials: alks_partial_values per
// design-point CTA.
int alks_partial_values(int dim);
int alks_sens_values(int dim);
int alks_planes(int dim);
int alks_stencil_kernels(int dim);  // kernels one launch_alks_stencil issues
void launch_alks_init(const Geo& g, Ctrl* ctrl, const double* objw, double seed, double* dkref, cudaStream_t st);
// Step t = ctrl->t0 - di: spread, coupling sums, fixed-point iterations, u~(t) in the box, the
// step's design sensitivity (5 kernels).
template <typename T>
void launch_alks_body(const Geo& g, const Slots<T>& S, Ctrl* ctrl, const Dof* it, const T* kref, T* abox, T* Ab,
                      long long astride, T* sstore, void* partials, double* dkref, int di, cudaStream_t st);
// Step t: the adjoint equilibrium at t and the star moments at t - 1 with boundary values (2 kernels).
template <typename T>
void launch_alks_stencil(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, T* Ab, long long astride, T* zb, int di,
                         cudaStream_t st);

}  // namespace lks
