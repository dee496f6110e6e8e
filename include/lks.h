/*
 * lks.h - C ABI of the GB300 library for the coupled lattice-kinetic-scheme (LKS) / rigid-body
 * forward march and its discrete adjoint.
 *
 * Method: "Topology optimization of passively moving rigid bodies in unsteady flows"
 * (arXiv 2601.18272). Per time step (Algorithm 1, inner loops):
 *   - LKS predictor p*, u* from the previous state (Sec. 2.2, Eqs. p_tmp, u_tmp with the
 *     equilibrium f^eq of Inamuro's LKS), boundary values prescribed directly (Sec. 2.2);
 *   - N_itr fixed-point iterations (Sec. 3.1) of: rigid transform of the design grid
 *     (Sec. 2.3, Eqs. rigid_body_position / rigid_body_velocity), spread of the Brinkman
 *     coefficient and solid velocity onto the analysis grid (Eqs. kappa_mapping, us_mapping),
 *     Brinkman update (Eq. u), fluid force and torque on the body and the explicit Euler
 *     equations of motion (Sec. 2.4);
 * and the reverse-time sweep giving dJ/dgamma for J = sum_d w_d s_d(N_t) (Sec. 2.5, 2.6).
 *
 * Conventions
 *   - Lattice units: dx = dt = 1, one design point per analysis cell spacing, pivot at the
 *     design-grid centre.
 *   - Fields are planes of nx*ny*nz values, x fastest. Design arrays have ndx*ndy*ndz values,
 *     x fastest.
 *   - DOF vector s: 8 doubles (xG_x, xG_y, xG_z, uG_x, uG_y, uG_z, theta, omega) for a body
 *     rotating about one axis; 21 doubles (xG[3], uG[3], h[3], omega[3], R[9] row-major) for a
 *     freely rotating 3D body (rot_axis = LKS_ROT_FREE), h the angular momentum and omega the
 *     angular velocity, both in the world frame. lks_dof_count gives the length.
 *   - Free rotation (six DOFs; the paper rotates about one axis and names Euler angles or
 *     quaternions as the extension, Sec. 2.1): explicit Euler, velocity first, with the inertia
 *     frozen over the step: h^(k) = h(t-1) + T^(k), omega^(k) = R(t-1) I_b^-1 R(t-1)^T h^(k),
 *     R^(k) = exp([omega^(k)]x) R(t-1) (Rodrigues' formula); iteration k's transform uses
 *     R^(k-1) and omega^(k-1).
 *   - Every call returns an lks_status code; nothing traps or exits. A handle is not
 *     thread-safe. All GPU work goes on the stream passed in (a cudaStream_t, or NULL for the
 *     legacy default stream).
 *   - Pointers named *_dev are device pointers owned by the caller; *_host are host pointers
 *     owned by the caller. The library owns its workspace (allocated in lks_create within
 *     hbm_budget_bytes, released in lks_destroy).
 */
#ifndef LKS_H_
#define LKS_H_

#include <stddef.h>

#if defined(__GNUC__)
#define LKS_API __attribute__((visibility("default")))
#else
#define LKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lks_status {
  LKS_OK = 0,
  LKS_ERR_ARG = 1,          /* invalid argument or problem description */
  LKS_ERR_OOM = 2,          /* device allocation failed */
  LKS_ERR_BUDGET = 3,       /* workspace would exceed hbm_budget_bytes */
  LKS_ERR_UNSTABLE = 4,     /* nu <= 0, i.e. A >= 3/4 in nu = (1/6 - 2A/9) dx (Sec. 2.2) */
  LKS_ERR_BODY_OUTSIDE = 5, /* the mapped body reaches a non-periodic boundary layer */
  LKS_ERR_NONFINITE = 6,    /* a non-finite force, torque or state was produced */
  LKS_ERR_ORDER = 7,        /* adjoint or sensitivity requested before a forward / adjoint */
  LKS_ERR_CUDA = 8,         /* a CUDA runtime call failed */
  LKS_ERR_UNSUPPORTED = 9,  /* valid but not supported by the library (e.g. grid/tile shape) */
  LKS_ERR_TIMEOUT = 10      /* a bounded wait on the device (a grid barrier of the persistent coupling
                             * kernels, or a tile copy of the row-streamed 3D stencils) waited longer
                             * than one second; the kernels returned early and the results of the call
                             * are void */
} lks_status;

enum { LKS_D2Q9 = 9, LKS_D3Q15 = 15 };                   /* velocity sets (Sec. 2.2) */
enum { LKS_BC_PERIODIC = 0, LKS_BC_INFLOW_OUTFLOW = 1, LKS_BC_WALL = 2, LKS_BC_PRESSURE = 3 };
enum { LKS_W_COS4 = 0, LKS_W_BILINEAR = 1 };              /* grid-separation weight (Sec. 2.3) */
enum { LKS_DOF_TX = 1, LKS_DOF_TY = 2, LKS_DOF_TZ = 4, LKS_DOF_ROT = 8 };
enum { LKS_ROT_FREE = -1 };                               /* rot_axis of a freely rotating 3D body */
enum { LKS_NDOF_AXIS = 8, LKS_NDOF_FREE = 21, LKS_MAX_DOF = 21 };  /* DOF vector lengths */
enum { LKS_FP32 = 32, LKS_FP64 = 64 };                    /* field storage / arithmetic type */
enum { LKS_CKPT_STORE_ALL = 0, LKS_CKPT_UNIFORM = 1, LKS_CKPT_BINOMIAL = 2 };
enum { LKS_CKPT_NATIVE = 0, LKS_CKPT_BF16 = 1, LKS_CKPT_FP16 = 2 };

/* Problem statement: grid, velocity set, design grid, body, fluid, run controls. */
typedef struct lks_problem {
  int dim;                /* 2 or 3 */
  int velocity_set;       /* LKS_D2Q9 (dim 2) or LKS_D3Q15 (dim 3) */
  int nx, ny, nz;         /* analysis grid in cells (nz = 1 for dim 2) */
  int ndx, ndy, ndz;      /* design grid in points (ndz = 1 for dim 2) */
  double body_centre[3];  /* x^G(0) in analysis coordinates */
  int rot_axis;           /* single rotation axis 0/1/2 (2 in 2D), or LKS_ROT_FREE (3D only) */
  unsigned dof_mask;      /* LKS_DOF_* bits of the free degrees of freedom (LKS_DOF_ROT: all rotation) */
  double mass;            /* M, constant (Sec. 2.1) */
  double inertia;         /* I about rot_axis, constant (Sec. 2.1); positive, unused with LKS_ROT_FREE */
  double inertia_tensor[9]; /* LKS_ROT_FREE: body-frame inertia tensor I_b about the pivot, row-major,
                           * symmetric positive definite, constant */
  double design_radius;   /* > 0: the design domain is the ball |r_m| <= design_radius (r_m = xi_m - xi^G);
                           * design points outside it take no part in any sum and get dJ/dgamma = 0.
                           * 0: the whole design grid */
  double filter_radius;   /* density filter radius R in design cells (Sec. 3.2, Eq. filter); 0: no filter */
  double proj_beta, proj_eta; /* Heaviside projection (Eq. projection); proj_beta 0: no projection,
                           * else 0 < proj_eta < 1 */
  double v_min;           /* minimum volume ratio of the constraint (Eq. constraint), used by lks_constraint */
  int cyclic_order;       /* cyclic periodic design (Sec. 4.2): 1 (none), 2 or 4; the design is expanded
                           * from each orbit's representative (smallest index) under rotations by
                           * 360/order degrees about the design-grid centre in the plane normal to
                           * rot_axis (order 4 needs equal extents in that plane; not with
                           * LKS_ROT_FREE) */
  double nu;              /* kinematic viscosity; A = 9/2 (1/6 - nu) */
  double u_in;            /* inflow speed for LKS_BC_INFLOW_OUTFLOW */
  double dp;              /* inlet pressure for LKS_BC_PRESSURE (outlet p = 0) */
  int bc[3];              /* per axis; x: periodic/inflow-outflow/pressure, y,z: periodic/wall */
  double kappa_max, q;    /* Brinkman interpolation (Eq. brinkman_coefficient) */
  int weight_kind;        /* LKS_W_COS4 (Eq. weight_function) or LKS_W_BILINEAR */
  int n_steps, n_itr;     /* N_t, N_itr (Sec. 3.1) */
  double obj_weights[LKS_MAX_DOF]; /* J = sum_d obj_weights[d] * s_d(N_t) over the DOF vector
                           * (Eqs. objective1, objective2); entries beyond lks_dof_count are ignored */
  int field_precision;    /* LKS_FP32 or LKS_FP64 */
  int ckpt_policy;        /* LKS_CKPT_STORE_ALL, LKS_CKPT_UNIFORM or LKS_CKPT_BINOMIAL */
  int ckpt_every;         /* UNIFORM: checkpoint interval k; BINOMIAL: number of state snapshots
                           * (the reverse sweep recomputes along a binomial schedule), or 0 with
                           * hbm_budget_bytes > 0: as many snapshots as the budget holds after the rest
                           * of the workspace (at most n_steps - 1) */
  int ckpt_format;        /* LKS_CKPT_NATIVE, LKS_CKPT_BF16 or LKS_CKPT_FP16 (FP32 fields; uniform
                           * checkpoints or binomial snapshots, 2 bytes per value and a per-plane range) */
  size_t hbm_budget_bytes;/* workspace limit, 0 = no limit */
} lks_problem;

typedef struct lks_handle lks_handle;

/* Validate the problem and allocate the workspace. On success *out owns the device memory.
 * The body box (the cells one step can touch) must fit every periodic extent; it is sized for a
 * rotating body unless that does not fit and dof_mask excludes rotation.
 * Errors: LKS_ERR_ARG, LKS_ERR_UNSTABLE, LKS_ERR_UNSUPPORTED, LKS_ERR_BUDGET, LKS_ERR_OOM. */
LKS_API int lks_create(const lks_problem* problem, lks_handle** out);

/* Length of the DOF vector of a problem: LKS_NDOF_AXIS, or LKS_NDOF_FREE with rot_axis =
 * LKS_ROT_FREE; 0 if problem is NULL. */
LKS_API int lks_dof_count(const lks_problem* problem);

/* sizeof(lks_problem) as compiled into the library, for bindings that mirror the struct. */
LKS_API size_t lks_problem_size(void);

/* Actions of the binomial checkpoint schedule (LKS_CKPT_BINOMIAL), in the order the library runs them. */
enum {
  LKS_BIN_FWD_SNAPSHOT = 0, /* the forward keeps state(b) in snapshot slot a on its way */
  LKS_BIN_RESTORE = 1,      /* the working state <- snapshot slot a (-1: the initial state), which holds state(b) */
  LKS_BIN_ADVANCE = 2,      /* re-advance the working state from state(a) by b steps */
  LKS_BIN_STORE = 3,        /* snapshot slot a <- the working state, state(b) (c steps past the last restore) */
  LKS_BIN_REVERSE = 4       /* reverse step a (its recompute from state(a - 1), then its adjoint) */
};

/* The binomial schedule (Griewank's revolve: the least total re-advanced steps for the given number
 * of snapshot slots, the initial state being restorable too) of an n_steps march with `snapshots`
 * slots, as the library builds it for lks_create with LKS_CKPT_BINOMIAL and ckpt_every =
 * snapshots. Host only (no device work). Writes min(count, capacity) actions as rows of four ints
 * (kind, a, b, c) into ops (host, [capacity][4]; may be NULL if capacity is 0) and returns the
 * action count, or -LKS_ERR_ARG for n_steps < 1, snapshots < 0 or capacity < 0. */
LKS_API long long lks_binomial_plan(int n_steps, int snapshots, int* ops, long long capacity);

/* Initial state for the next forward (Algorithm 1, "Initialize"). p [N], u [dim][N] and
 * s [lks_dof_count] are host arrays (copied). Any pointer may be NULL to keep the default: p = 0,
 * u = (u_in, 0, 0), body at rest at body_centre (R = identity with free rotation). The last
 * forward and its adjoints become invalid (the reverse sweep restarts from the initial state), so
 * lks_adjoint needs a new lks_forward.
 * Errors: LKS_ERR_ARG; LKS_ERR_NONFINITE if a given array holds a NaN or an infinity (checked on
 * the host before anything is copied: the previous state and results stay); LKS_ERR_UNSUPPORTED
 * if s starts the body rotated but the workspace was sized for an axis-aligned box (see
 * lks_create); LKS_ERR_CUDA. */
LKS_API int lks_set_initial_state(lks_handle* h, const double* p_host, const double* u_host, const double* s_host);

/* Forward march over n_steps (Algorithm 1, state loop) for the design field gamma_dev
 * [ndx*ndy*ndz] (device, values in [0,1]). Stores the DOF history and the checkpoints the
 * adjoint needs. Synchronises the stream once to return J (host scalar).
 * Errors: LKS_ERR_ARG, LKS_ERR_BODY_OUTSIDE, LKS_ERR_CUDA; LKS_ERR_NONFINITE if a force, torque or
 * DOF became non-finite, or if gamma_dev holds a NaN or an infinity (found on the device; those
 * points take part as void, kappa^ref = 0, so nothing non-finite enters the march). */
LKS_API int lks_forward(lks_handle* h, const double* gamma_dev, double* J_host, void* stream);

/* Reverse sweep (Algorithm 1, adjoint loop) seeded with dJ = seed. Enqueued on the stream; with the
 * persistent coupling kernels (lks_persistent_coupling) or the row-streamed 3D stencils
 * (lks_stencil_form = 1) it then synchronises the stream once to read the device status word.
 * Requires a prior lks_forward (else LKS_ERR_ORDER).
 * Errors: LKS_ERR_TIMEOUT, LKS_ERR_CUDA. */
LKS_API int lks_adjoint(lks_handle* h, double seed, void* stream);

/* Continuation step (Sec. 3.3): the convexity parameter q of Eq. brinkman_coefficient and the
 * projection steepness beta of Eq. projection for the following forward and adjoint calls (beta 0
 * turns the projection off; a positive beta needs 0 < proj_eta < 1 from lks_create). Synchronises
 * the device; the next lks_adjoint needs a new lks_forward. Errors: LKS_ERR_ARG. */
LKS_API int lks_set_continuation(lks_handle* h, double q, double proj_beta);

/* The paper's adjoint, ALKS (Sec. 2.5, Appendix A; Algorithm 1, adjoint loop), in place of the exact
 * discrete adjoint: the moments p~, u~, s~ of the adjoint distribution (the star moments gathered
 * from the adjoint equilibrium at x + c_i, Eqs. ap_tmp to as, with the boundary values prescribed)
 * and the body multipliers (Eqs. axg, aug, atheta, aomega, N_itr fixed-point iterations per step),
 * accumulating Eq. design_sensitivity; lks_sensitivity then returns its dJ/dgamma. A discretised
 * continuous adjoint: it approaches the exact gradient of lks_adjoint but is not equal to it.
 * Seeded with dJ = seed; enqueued on the stream. The exact adjoint's lambda(0) of an earlier
 * lks_adjoint of the same forward stays available. The first call allocates its buffers (about
 * (2 (1 + dim + dim(dim+1)/2) + dim) N field values). Single rotation axis only.
 * Errors: LKS_ERR_ORDER (no forward), LKS_ERR_UNSUPPORTED (free rotation, or a warm-start terminal
 * adjoint is set), LKS_ERR_OOM / LKS_ERR_BUDGET, LKS_ERR_CUDA. */
LKS_API int lks_adjoint_alks(lks_handle* h, double seed, void* stream);

/* After lks_adjoint_alks: the moments at t = 0, p~ [N], u~ [dim][N], s~ [dim][dim][N], and the body
 * multipliers at t = 1 (x~G[3], u~G[3], theta~, omega~; the paper's sign) as host doubles (any may
 * be NULL). Synchronous. Errors: LKS_ERR_ORDER. */
LKS_API int lks_get_alks_adjoint(lks_handle* h, double* p_host, double* u_host, double* s_host, double* body_host);

/* dJ/dgamma [ndx*ndy*ndz] (device, FP64) from the last adjoint: the accumulated dJ/dkappa^ref
 * chained through dkappa^ref/dgamma-bar (Eq. brinkman_coefficient) and the transpose of the design
 * chain (projection, filter, cyclic expansion: only orbit representatives receive sensitivity).
 * M and I are held constant. Requires a prior lks_adjoint (else LKS_ERR_ORDER). Enqueued, no
 * synchronisation. */
LKS_API int lks_sensitivity(lks_handle* h, double* dJdgamma_dev, void* stream);

/* Periodic warm start (Sec. 3.4): the last forward's final state and DOFs become the initial state
 * of the next forward, and (with_adjoint != 0) the last adjoint's initial adjoint lambda(0) and
 * dJ/ds(0) become the terminal adjoint of the next reverse sweep, which then differentiates
 * J + lambda(0).state(N_t). The copies stay on the device (the DOFs pass through the host). The
 * next lks_forward and lks_adjoint use them; lks_set_initial_state replaces the initial state
 * (the terminal adjoint stays until the next lks_warm_start). Synchronises the stream.
 * Errors: LKS_ERR_ORDER (no forward, or with_adjoint without an lks_adjoint of that forward: the
 * paper-form adjoint has no lambda(0) of the state), LKS_ERR_UNSUPPORTED (the
 * final DOFs start rotated but the workspace was sized for an axis-aligned box), LKS_ERR_CUDA. */
LKS_API int lks_warm_start(lks_handle* h, int with_adjoint, void* stream);

/* Volume constraint (Eq. constraint) of the design gamma_dev [N_D] (device): G = sum of gamma-bar over
 * the design domain / (v_min * its point count) - 1 into G_host, and dG/dgamma [N_D] (device, FP64,
 * through the design chain) into dGdgamma_dev if not NULL. Synchronises the stream to return G.
 * Errors: LKS_ERR_ARG (v_min <= 0, NULL pointers), LKS_ERR_CUDA. */
LKS_API int lks_constraint(lks_handle* h, const double* gamma_dev, double* G_host, double* dGdgamma_dev, void* stream);

/* End-to-end gradient with host buffers: copies gamma_host [N_D] to the device, runs forward,
 * adjoint (seed 1) and sensitivity, copies dJdgamma_host [N_D] back and returns J.
 * Synchronises the stream before returning. */
LKS_API int lks_gradient_host(lks_handle* h, const double* gamma_host, double* J_host, double* dJdgamma_host, void* stream);

/* DOF history of the last forward into host_buf [(n_steps+1)*lks_dof_count]; n = capacity in
 * doubles. */
LKS_API int lks_get_dof_history(lks_handle* h, double* host_buf, size_t n);

/* Final state of the last forward: p [N], u [dim][N] as doubles (host), any checkpoint policy.
 * Synchronous. Errors: LKS_ERR_ORDER (no forward since the last lks_create, lks_set_initial_state,
 * lks_set_continuation or lks_warm_start). */
LKS_API int lks_get_state(lks_handle* h, double* p_host, double* u_host);

/* Adjoint of the initial state after the last lks_adjoint: dJ/dp0 [N], dJ/du0 [dim][N],
 * dJ/ds0 [lks_dof_count] (host, any may be NULL). Synchronous. Errors: LKS_ERR_ORDER (no
 * lks_adjoint of the last forward; lks_adjoint_alks does not count). */
LKS_API int lks_get_initial_adjoint(lks_handle* h, double* lam_p_host, double* lam_u_host, double* lam_s_host);

/* For tests of the bit-exact integer indexing of the spread (Eqs. kappa_mapping, us_mapping,
 * weight_function): for the DOF vector s_host [lks_dof_count] (host), the body box a march starting
 * from s would use, box_host [6] = (unwrapped origin x, y, z; extent x, y, z) in cells, and, if
 * stats_host is not NULL, for each box cell (x fastest) the design points the coupling's gather
 * accepts (|x_n - x^ref_m| below the kernel's half-width on every axis, m in the design domain):
 * stats_host [box cells][5] = (count, least linear design index or -1, largest index, sum of the
 * indices, sum of their squares), capacity in values (at least 5 * box cells, else LKS_ERR_ARG).
 * The acceptance is decided in the field precision of the handle. Synchronous (legacy default
 * stream; allocates and frees a small device buffer). Errors: LKS_ERR_NONFINITE (s not finite),
 * LKS_ERR_UNSUPPORTED (s rotated but the workspace holds an axis-aligned box), LKS_ERR_CUDA. */
LKS_API int lks_support_sets(lks_handle* h, const double* s_host, int* box_host, long long* stats_host,
                             size_t capacity);

/* Test hook of the bounded grid barriers: skip != 0 makes the first CTA of every persistent coupling
 * kernel skip its barrier arrivals, so the other CTAs' waits run out (after one second) and the
 * forward or adjoint returns LKS_ERR_TIMEOUT; skip = 0 restores normal operation. Synchronises the
 * device. Errors: LKS_ERR_ARG, LKS_ERR_CUDA. */
LKS_API int lks_debug_sync_skip(lks_handle* h, int skip);

/* Test hook of the bounded copy waits of the row-streamed 3D stencils (lks_stencil_form = 1):
 * skip != 0 makes every CTA of those kernels withhold the copy of the third plane of its chunk, so
 * its wait runs out (after one second), the CTA waits (bounded) for the copies it did issue and
 * returns, and the forward or adjoint returns LKS_ERR_TIMEOUT; later launches of the same call
 * return at once. skip = 0 restores normal operation. Synchronises the device.
 * Errors: LKS_ERR_ARG, LKS_ERR_CUDA. */
LKS_API int lks_debug_copy_skip(lks_handle* h, int skip);

/* How the handle runs each step's N_itr coupling iterations (Sec. 3.1) and their reverse: mode 1 as
 * one persistent cooperative launch per step (grid barriers between the iterations) when the device
 * holds its grid, mode 0 as one launch per iteration (with the finish kernels), mode 2 (the default)
 * the persistent launch only where it measured faster (2D bodies whose box has more tiles than the
 * persistent grid has CTAs), mode -1 only asks. Returns 1 if the persistent kernels are in use after
 * the call, 0 if not, or -status on error (LKS_ERR_ARG, LKS_ERR_CUDA). Changing the mode
 * synchronises the device; results agree to rounding (the per-CTA partial sums are grouped
 * differently). */
LKS_API int lks_persistent_coupling(lks_handle* h, int mode);

/* Number of kernels this handle has launched (graph nodes counted per replay). */
LKS_API long long lks_launch_count(const lks_handle* h);

/* Kernel timing for the benchmark. enable = 1 runs later calls without CUDA graphs and brackets
 * every launch of the named kernel family with CUDA events on the launching stream.
 * lks_kernel_time returns the summed milliseconds and the launch count for the family
 * ("stencil_fwd", "stencil_adj", "couple", "adj_cell", "adj_design", "recompute", "adj_body" (the
 * persistent reverse coupling), and for lks_adjoint_alks "alks_body", "alks_stencil"); the coupling
 * and design-side families include their one-CTA finish kernels. */
LKS_API int lks_set_kernel_timing(lks_handle* h, int enable);
LKS_API int lks_kernel_time(lks_handle* h, const char* family, double* ms_total, long long* launches);

/* One time step of the march (LKS predictor, boundary values, N_itr coupling iterations) that
 * allocates no device memory. The paper has no counterpart: this is an interface for callers that
 * cannot let a library allocate -- real-time loops whose device memory is fixed up front, and
 * frameworks that own every device allocation and forbid libraries their own cudaMalloc. Its
 * scratch is one fixed device array (about 0.7 MB) that every GPU loading the library holds until
 * exit.
 *   problem   : checked by the same rules as lks_create (same errors), and the body box derived the
 *               same way; dim 2, LKS_FP64 and no design chain (filter_radius 0, proj_beta 0,
 *               cyclic_order 1) only, else LKS_ERR_UNSUPPORTED; at most 65536 design points,
 *               n_itr <= 16 and 4096 CTAs per reduction, else LKS_ERR_BUDGET
 *   gamma_dev : design field [ndx*ndy] (device, caller-owned), used as gamma-bar directly
 *   state_dev : two state slots [2][3][nx*ny] doubles (device, caller-owned): step t reads slot
 *               (t-1) mod 2 and writes p*, u(t) into slot t mod 2
 *   t         : step index >= 1 (only its parity matters)
 *   s_host    : DOF vector [8] (host): s(t-1) in, s(t) out; LKS_ERR_NONFINITE if it holds a NaN
 *               or an infinity
 * The first call on a device looks up the scratch array's address with that device current. All
 * calls share the array and each clears what must start at zero; calls that overlap on the GPU
 * race on it, so serialise them. The call waits for the stream (it copies s(t) to the host) before
 * it returns. */
LKS_API int lks_step_noalloc(const lks_problem* problem, const double* gamma_dev, double* state_dev, int t,
                             double* s_host, void* stream);

/* State copies the handle keeps for the reverse sweep: binomial snapshot slots (as chosen for
 * ckpt_every = 0), uniform checkpoints, or n_steps + 1 stored states; -LKS_ERR_ARG for NULL. */
LKS_API int lks_checkpoint_slots(const lks_handle* h);

/* Form of the 3D predictor and transpose kernels the handle launches: 1 for the row-streamed FP32
 * kernels (a 64-column window fed by one TMA box of 16 rows per plane, packed FP32x2 arithmetic;
 * taken for FP32 fields on grids periodic in y and z with nx a multiple of 4 and at least 64 and
 * ny at least 16, x not walled), 0 for the general kernels (2D problems, FP64 fields, walls, other
 * grids); -LKS_ERR_ARG for NULL. Both forms compute the predictor of Sec. 2.2 and its exact
 * transpose. */
LKS_API int lks_stencil_form(const lks_handle* h);

/* Bytes of device workspace held by the handle. */
LKS_API size_t lks_workspace_bytes(const lks_handle* h);

LKS_API void lks_destroy(lks_handle* h);

/* Static description of a status code. */
LKS_API const char* lks_status_string(int status);

/* The cudaError_t value of the most recent LKS_ERR_CUDA return (0 if none). */
LKS_API int lks_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LKS_H_ */
