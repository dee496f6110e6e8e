// Host-side launchers of the LKS kernels (internal to the library; the public boundary is
// include/lks.h).
#pragma once

#include "lks_device.cuh"

namespace lks {

constexpr int kTileX = 32;  // stencil tile width (cells); boundary pairs must not straddle tiles
constexpr int kTileY2 = 8;  // 2D stencil tile height
constexpr int kTileY3 = 4;  // 3D stencil tile height
constexpr int kTileZ3 = 4;  // 3D stencil tile depth

// Forward LKS predictor + boundary values for step ctrl->t: slot(t-1) -> slot(t).
template <typename T>
void launch_stencil_fwd(const Geo& g, const Slots<T>& S, const Ctrl* ctrl, cudaStream_t st);

// Transpose of the predictor at the state slot(t-1): adjoint fields Lb[t&1] -> Lb[(t-1)&1]
// (each Lb slot holds dim+1 planes); decrements ctrl->t.
template <typename T>
void launch_stencil_adj(const Geo& g, const Slots<T>& S, T* Lb, long long lstride, Ctrl* ctrl, cudaStream_t st);

// Design preparation: kappa^ref from gamma (Eq. brinkman_coefficient), moments.
template <typename T>
void launch_prep(const Geo& g, const double* gamma, double kappa_max, double q, T* kref, Moments* mom,
                 double* partials, Ctrl* ctrl, cudaStream_t st);

// Coupling iteration k (1..K) of step ctrl->t: spread, Brinkman, force/torque, EOM.
// On k == K writes u(t) into slot(t), optionally u* into the box store, and advances ctrl->t.
template <typename T>
void launch_couple(const Geo& g, const Slots<T>& S, Ctrl* ctrl, Dof* it, const T* kref, const Moments* mom,
                   double* partials, int k, T* boxstore, int nbox, cudaStream_t st);

// Recompute: Brinkman update with the stored iterate s^(K-1); writes u(t) and the box store of
// u*; advances ctrl->t.
template <typename T>
void launch_apply(const Geo& g, const Slots<T>& S, Ctrl* ctrl, const Dof* it, const T* kref, T* boxstore, int nbox,
                  cudaStream_t st);

// Adjoint of coupling iteration k, analysis-cell side (Brinkman and interpolation reverse).
template <typename T>
void launch_adj_cell(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* boxstore, int nbox, T* Lb,
                     long long lstride, T* acc, T* scratch, int k, cudaStream_t st);

// Adjoint of coupling iteration k, design-point side (spread/transform reverse, dJ/dkappa^ref,
// reduction to dJ/ds^(k-1) and the EOM reverse of the previous iteration).
template <typename T>
void launch_adj_design(const Geo& g, Ctrl* ctrl, const Dof* it, const T* kref, const T* scratch, double* dkref,
                       double* partials, int k, cudaStream_t st);

// Initial state (double) -> slot(0); s0 -> it row 0; ctrl reset for a forward.
template <typename T>
void launch_init_forward(const Geo& g, const Slots<T>& S, const double* p0, const double* u0, const double* s0dev,
                         Dof* it, Ctrl* ctrl, cudaStream_t st);

// Set ctrl->t and ctrl->base.
void launch_set_step(Ctrl* ctrl, int t, int base, cudaStream_t st);

// Adjoint initialisation: dJ/ds(N_t) = seed * w, EOM reverse of iteration K, zero dJ/dkappa^ref.
void launch_adj_init(const Geo& g, Ctrl* ctrl, const double* objw, double seed, double* dkref, int nd,
                     cudaStream_t st);

// dJ/dgamma = dJ/dkappa^ref * dkappa^ref/dgamma.
void launch_sensitivity(const Geo& g, const double* gamma, const double* dkref, double kappa_max, double q,
                        double* out, cudaStream_t st);

// Copy / convert one state slot.
template <typename T>
void launch_copy_slot(const Geo& g, const Slots<T>& S, int t_src, int src_base, T* dst, Ctrl* ctrl, cudaStream_t st);

// Checkpoint pack of the state at ctrl->t - 1 into ckpt[(t-1)/every] (native precision).
template <typename T>
void launch_ckpt_pack(const Geo& g, const Slots<T>& S, T* ckpt, long long cstride, int every, const Ctrl* ctrl,
                      cudaStream_t st);

}  // namespace lks
