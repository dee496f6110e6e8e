// Oracle for the coupled lattice-kinetic-scheme / rigid-body step and its discrete adjoint.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded FP64 CPU statement of
// what the method computes. Only the tests, the smoke check and the benchmark's CPU-baseline
// leg may load it. It shares no code, header or constant table with the CUDA library.
//
// Paper: "Topology optimization of passively moving rigid bodies in unsteady flows"
// (arXiv 2601.18272). Citations below name the paper's section / equation.
//
// Forward step t (Algorithm 1, inner loops), in the paper's order:
//   S1  LKS predictor p*, u* from the state at t-1          (Sec. 2.2, Eqs. p_tmp, u_tmp, f^eq)
//   S2  boundary values prescribed directly                  (Sec. 2.2, last paragraph)
//   S3  N_itr fixed-point iterations                         (Sec. 3.1)
//         rigid transform x^ref, u^S,ref                     (Sec. 2.3, Eqs. rigid_body_position/velocity)
//         spread kappa, u^S onto the analysis grid           (Sec. 2.3, Eqs. kappa_mapping, us_mapping)
//         Brinkman update u = (u* + kappa u^S)/(1 + kappa)   (Sec. 2.2, Eq. u)
//         interpolate u^ref to the design points             (Sec. 2.3, Eq. u_mapping)
//         force / torque sums and explicit Euler EOM         (Sec. 2.4)
// The adjoint is the exact reverse of that arithmetic (reverse-mode, written out by hand); the
// paper's continuous-adjoint ALKS (Sec. 2.5) has the same stencil structure (moments of the
// adjoint distribution gathered from x + c_i) but is a discretised continuous adjoint.
//
// Readings where the paper is silent or garbled (each repeated at its use):
//   lattice units dx = dt = 1, design-cell volume 1; D2Q9/D3Q15 velocity order (rest, axes,
//   diagonals); f^eq with -3/2|u|^2; velocity gradient by the isotropic central stencil
//   d_b u_a(y) = sum_j c_jb u_a(y + c_j) / sum_j c_jb^2; weight kernel w(r) = (1 + cos(pi r/2))/4
//   for |r| < 2 (or bilinear 1 - |r|); design spacing one cell with pivot at the design-grid
//   centre; DOF^(0) = DOF(t-1), u(t) from the last iteration, DOF(t) = DOF^(N_itr); lever arm
//   R(theta^(k-1)) r_m; M and I held constant.
//
// Free rotation in 3D (six DOFs; the paper treats one rotation axis and names Euler angles or
// quaternions as the extension). The DOF vector is s = (x^G[3], u^G[3], h[3], omega[3], R[9]),
// R row-major, h the angular momentum and omega the angular velocity (world frame). Explicit
// Euler with the body's inertia frozen over the step, velocity first as in the paper's scheme:
//   h^(k) = h(t-1) + T^(k),  omega^(k) = R(t-1) I_b^-1 R(t-1)^T h^(k),
//   R^(k) = exp([omega^(k)]x) R(t-1)   (Rodrigues' formula for the rotation by |omega| about omega),
// with I_b the body-frame inertia tensor about the pivot; the transform of iteration k uses
// R^(k-1) and omega^(k-1) (lever arm R r_m, solid velocity u^G + omega x R r_m). For a body whose
// rotation stays about one principal axis this is the single-axis scheme.
//
// Design domain: with design_radius > 0 only the design points with |r_m| <= design_radius
// belong to the body (a ball-shaped design domain); the others take no part in any sum and
// their sensitivity is zero.
//
// Design chain (Sec. 3.2, Sec. 4.2): the design variables gamma are first expanded cyclically
// (cyclic_order 2 or 4: the value at a point is that of its orbit's representative, the point of
// smallest index among its images under rotations by 360/order degrees about the design-grid
// centre in the plane normal to rot_axis), then filtered (Eq. filter: conic weights
// (R - |x_i - x_j|) / R within the filter radius R over the design domain, normalised), then
// projected (Eq. projection, parameters beta and eta); the result gamma-bar enters the Brinkman
// coefficient and the volume constraint G = sum gamma-bar / (V_min N_dom) - 1 (Eq. constraint, N_dom
// the number of design points in the domain). Radius 0, beta 0 or order 1 skip the step.
//
// Templated on the scalar type: double, and std::complex<double> for complex-step derivatives.
// Every branch (kernel support, floor, bilinear sign) is taken on the real part.

#include <cmath>
#include <complex>

// A timing build (compiled with -fopenmp) spreads the independent per-node loops marked below over
// the host's cores; every output is still computed by the same operations in the same order, so
// its results are those of the single-threaded build, bit for bit. The plain build ignores it.
#if defined(_OPENMP)
#include <omp.h>
#define LKS_ORACLE_PRAGMA(x) _Pragma(#x)
#define LKS_ORACLE_PARALLEL_FOR LKS_ORACLE_PRAGMA(omp parallel for schedule(static))
#else
#define LKS_ORACLE_PARALLEL_FOR
#endif
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <vector>

namespace {

typedef std::complex<double> cplx;

inline double re(double x) { return x; }
inline double re(const cplx& x) { return x.real(); }

const double kPi = 3.14159265358979323846;

enum { BC_PERIODIC = 0, BC_INFLOW_OUTFLOW = 1, BC_WALL = 2, BC_PRESSURE = 3 };
enum { W_COS4 = 0, W_BILINEAR = 1 };
enum { DOF_TX = 1, DOF_TY = 2, DOF_TZ = 4, DOF_ROT = 8 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_BODY_OUTSIDE = 2, ORC_ERR_NONFINITE = 3, ORC_ERR_UNSTABLE = 4 };

}  // namespace

// The oracle's own problem record (mirrored by oracle/oracle.py with ctypes).
extern "C" struct OracleProblem {
  int dim;             // 2 or 3
  int nx, ny, nz;      // analysis grid (nz = 1 in 2D)
  int ndx, ndy, ndz;   // design grid (ndz = 1 in 2D)
  int rot_axis;        // single rotation axis (2 = z in 2D), or -1: free rotation (3D)
  int dof_mask;        // DOF_TX | DOF_TY | DOF_TZ | DOF_ROT
  int bc[3];           // boundary kind per axis
  int weight_kind;     // W_COS4 or W_BILINEAR
  int n_steps;         // N_t
  int n_itr;           // N_itr
  double mass;         // M
  double inertia;      // I about rot_axis
  double nu;           // kinematic viscosity; A = 9/2 (1/6 - nu)
  double u_in;         // inflow speed
  double dp;           // pressure at the inlet for the pressure-driven boundary
  double kappa_max;    // kappa_max in the Brinkman interpolation
  double q;            // convexity parameter
  double obj_w[21];    // J = sum_d obj_w[d] * s_d(N_t) over the DOF vector
  double inertia_tensor[9];  // free rotation: body-frame inertia tensor about the pivot
  double design_radius;      // > 0: ball-shaped design domain |r_m| <= design_radius
  double filter_radius;      // density filter radius R (0: no filter)
  double proj_beta, proj_eta;  // Heaviside projection (beta 0: no projection)
  double v_min;              // minimum volume ratio of the constraint
  int cyclic_order;          // 1 (none), 2 or 4
};

namespace {

struct Lattice {
  int d = 2, Q = 9;
  int c[15][3];
  double w[15];
  double cn[3];  // sum_j c_jb^2, the normaliser of the gradient stencil
};

// Velocity sets and weights (Sec. 2.2). The paper gives the weights by index range; the vectors
// are drawn only in a figure, so the order used is rest, axis directions, diagonals.
Lattice make_lattice(int dim) {
  Lattice L;
  std::memset(L.c, 0, sizeof(L.c));
  if (dim == 2) {
    L.d = 2;
    L.Q = 9;
    const int c2[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int i = 0; i < 9; ++i) {
      L.c[i][0] = c2[i][0];
      L.c[i][1] = c2[i][1];
      L.c[i][2] = 0;
      L.w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else {
    L.d = 3;
    L.Q = 15;
    const int c3[15][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                           {0, 0, 1},   {0, 0, -1},  {1, 1, 1},  {-1, 1, 1}, {1, -1, 1},
                           {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};
    for (int i = 0; i < 15; ++i) {
      for (int a = 0; a < 3; ++a) L.c[i][a] = c3[i][a];
      L.w[i] = (i == 0) ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
  }
  for (int b = 0; b < 3; ++b) {
    L.cn[b] = 0;
    for (int j = 0; j < L.Q; ++j) L.cn[b] += L.c[j][b] * L.c[j][b];
  }
  return L;
}

struct Ctx {
  OracleProblem P;
  Lattice L;
  int d;
  int n[3];
  size_t N;
  int nd[3];
  size_t ND;
  double A;       // nu = (1/6 - 2A/9) dx (Sec. 2.2)
  int support;    // kernel half-width in cells
  int err = ORC_OK;
  std::vector<double> r;  // r_m = xi_m - xi^G, [ND][3]
  std::vector<char> dom;  // design point m belongs to the design domain
  std::vector<size_t> rep;  // representative of m's orbit under the cyclic rotations
  bool free_rot = false;  // six DOFs
  int ns = 8;             // DOF vector length: 8, or 21 with free rotation
  double Jinv[9];         // free rotation: I_b^-1
};

// Inverse of a symmetric positive definite 3x3 matrix (row-major) by cofactors; false unless
// the leading minors are positive.
bool invert3(const double* a, double* inv) {
  const double m1 = a[0], m2 = a[0] * a[4] - a[1] * a[3];
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  if (!(m1 > 0.0) || !(m2 > 0.0) || !(det > 0.0)) return false;
  const double c10 = a[2] * a[7] - a[1] * a[8], c11 = a[0] * a[8] - a[2] * a[6], c12 = a[1] * a[6] - a[0] * a[7];
  const double c20 = a[1] * a[5] - a[2] * a[4], c21 = a[2] * a[3] - a[0] * a[5], c22 = a[0] * a[4] - a[1] * a[3];
  // inverse = adjugate / det, the adjugate being the transposed cofactor matrix
  const double adj[9] = {c00, c10, c20, c01, c11, c21, c02, c12, c22};
  for (int i = 0; i < 9; ++i) inv[i] = adj[i] / det;
  return true;
}

// Orbit representatives of the cyclic expansion: the rotation by 90 degrees (order 4) or 180
// degrees (order 2) about the design-grid centre in the plane (b, c) normal to rot_axis maps
// (i_b, i_c) to (n - 1 - i_c, i_b) or (n_b - 1 - i_b, n_c - 1 - i_c).
bool make_cyclic(Ctx* C) {
  const int order = C->P.cyclic_order;
  C->rep.resize(C->ND);
  for (size_t m = 0; m < C->ND; ++m) C->rep[m] = m;
  if (order == 1) return true;
  if (order != 2 && order != 4) return false;
  if (C->P.rot_axis < 0) return false;
  const int ax = C->P.rot_axis, b = (ax + 1) % 3, c = (ax + 2) % 3;
  if (order == 4 && C->nd[b] != C->nd[c]) return false;
  for (size_t m = 0; m < C->ND; ++m) {
    int i[3] = {(int)(m % C->nd[0]), (int)((m / C->nd[0]) % C->nd[1]), (int)(m / ((size_t)C->nd[0] * C->nd[1]))};
    size_t best = m;
    for (int k = 1; k < order; ++k) {
      int j[3] = {i[0], i[1], i[2]};
      if (order == 4) {
        j[b] = C->nd[c] - 1 - i[c];
        j[c] = i[b];
      } else {
        j[b] = C->nd[b] - 1 - i[b];
        j[c] = C->nd[c] - 1 - i[c];
      }
      for (int a = 0; a < 3; ++a) i[a] = j[a];
      const size_t mj = (size_t)i[0] + C->nd[0] * ((size_t)i[1] + (size_t)C->nd[1] * i[2]);
      if (mj < best) best = mj;
    }
    C->rep[m] = best;
  }
  return true;
}

bool make_ctx(const OracleProblem* P, Ctx* C) {
  C->P = *P;
  C->d = P->dim;
  if (C->d != 2 && C->d != 3) return false;
  C->L = make_lattice(C->d);
  C->n[0] = P->nx;
  C->n[1] = P->ny;
  C->n[2] = (C->d == 3) ? P->nz : 1;
  C->nd[0] = P->ndx;
  C->nd[1] = P->ndy;
  C->nd[2] = (C->d == 3) ? P->ndz : 1;
  for (int a = 0; a < C->d; ++a)
    if (C->n[a] < 4 || C->nd[a] < 1) return false;
  C->N = (size_t)C->n[0] * C->n[1] * C->n[2];
  C->ND = (size_t)C->nd[0] * C->nd[1] * C->nd[2];
  if (P->bc[0] == BC_WALL) return false;  // x is periodic or open
  for (int a = 1; a < 3; ++a)
    if (P->bc[a] != BC_PERIODIC && P->bc[a] != BC_WALL) return false;
  if (C->d == 2 && P->rot_axis != 2) return false;
  C->free_rot = (C->d == 3 && P->rot_axis == -1);
  if (!C->free_rot && (P->rot_axis < 0 || P->rot_axis > 2)) return false;
  C->ns = C->free_rot ? 21 : 8;
  if (C->free_rot && !invert3(P->inertia_tensor, C->Jinv)) return false;
  if (P->n_itr < 1 || P->n_steps < 0) return false;
  C->A = 4.5 * (1.0 / 6.0 - P->nu);
  C->support = (P->weight_kind == W_BILINEAR) ? 1 : 2;
  C->r.assign(C->ND * 3, 0.0);
  for (int k = 0; k < C->nd[2]; ++k)
    for (int j = 0; j < C->nd[1]; ++j)
      for (int i = 0; i < C->nd[0]; ++i) {
        size_t m = (size_t)i + C->nd[0] * ((size_t)j + C->nd[1] * k);
        C->r[3 * m + 0] = i - (C->nd[0] - 1) / 2.0;
        C->r[3 * m + 1] = j - (C->nd[1] - 1) / 2.0;
        C->r[3 * m + 2] = (C->d == 3) ? k - (C->nd[2] - 1) / 2.0 : 0.0;
      }
  if (!make_cyclic(C)) return false;
  C->dom.assign(C->ND, 1);
  if (P->design_radius > 0.0)
    for (size_t m = 0; m < C->ND; ++m) {
      const double* r = &C->r[3 * m];
      C->dom[m] = (r[0] * r[0] + r[1] * r[1] + r[2] * r[2] <= P->design_radius * P->design_radius) ? 1 : 0;
    }
  return true;
}

inline size_t idx(const Ctx& C, int x, int y, int z) { return (size_t)x + C.n[0] * ((size_t)y + C.n[1] * z); }

inline int wrap(int v, int n) { return ((v % n) + n) % n; }

// Node on a boundary plane of a non-periodic axis?
inline bool on_boundary(const Ctx& C, int a, int v) {
  return C.P.bc[a] != BC_PERIODIC && (v == 0 || v == C.n[a] - 1);
}
inline bool is_interior(const Ctx& C, const int* x) {
  for (int a = 0; a < C.d; ++a)
    if (on_boundary(C, a, x[a])) return false;
  return true;
}

// Neighbour for the velocity-gradient stencil, with one ghost layer on non-periodic axes:
// open boundaries (inflow/outflow, pressure) copy the boundary node; no-slip walls take the odd
// reflection u(-1) = -u(1) (linear extrapolation through the wall value u = 0).
inline size_t grad_nbr(const Ctx& C, const int* x, const int* c, double* sgn) {
  int y[3] = {0, 0, 0};
  *sgn = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (a >= C.d) {
      y[a] = 0;
      continue;
    }
    int v = x[a] + c[a];
    int n = C.n[a];
    int bc = C.P.bc[a];
    if (bc == BC_PERIODIC) {
      v = wrap(v, n);
    } else if (v < 0 || v >= n) {
      if (bc == BC_WALL) {
        v = (v < 0) ? 1 : n - 2;
        *sgn = -*sgn;
      } else {
        v = (v < 0) ? 0 : n - 1;
      }
    }
    y[a] = v;
  }
  return idx(C, y[0], y[1], y[2]);
}

// Neighbour x - c_i for an interior node (always inside the grid on non-periodic axes).
inline size_t shift_nbr(const Ctx& C, const int* x, const int* c, int sign) {
  int y[3] = {0, 0, 0};
  for (int a = 0; a < C.d; ++a) y[a] = wrap(x[a] + sign * c[a], C.n[a]);
  return idx(C, y[0], y[1], y[2]);
}

inline void coords(const Ctx& C, size_t n, int* x) {
  x[0] = (int)(n % C.n[0]);
  x[1] = (int)((n / C.n[0]) % C.n[1]);
  x[2] = (int)(n / ((size_t)C.n[0] * C.n[1]));
}

template <class T>
struct Fields {
  std::vector<T> p;
  std::vector<T> u[3];
  void alloc(const Ctx& C) {
    p.assign(C.N, T(0));
    for (int a = 0; a < 3; ++a) u[a].assign(a < C.d ? C.N : 0, T(0));
  }
};

// ------------------------------------------------------------------------------------------
// S1 + S2: LKS predictor and boundary values (Sec. 2.2).
//   f_i^eq = w_i (3p + 3 c.u + 9/2 (c.u)^2 - 3/2 |u|^2) + w_i A (d_a u_b + d_b u_a) c_ia c_ib
//   p*(x) = 1/3 sum_i f_i^eq(x - c_i),  u*(x) = sum_i c_i f_i^eq(x - c_i)
// The paper prints "+3/2 u^2"; only "-3/2 |u|^2" makes sum_i f_i^eq = 3p, i.e. p* = p for a
// uniform state, which the paper's Eq. p = p* relies on; that sign is used.
// ------------------------------------------------------------------------------------------
template <class T>
void velocity_gradient(const Ctx& C, const Fields<T>& s, std::vector<T>* G) {
  const int d = C.d;
  G->assign((size_t)d * d * C.N, T(0));
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < C.N; ++n) {
    int x[3];
    coords(C, n, x);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        T acc = T(0);
        for (int j = 0; j < C.L.Q; ++j) {
          if (C.L.c[j][b] == 0) continue;
          double sg;
          size_t m = grad_nbr(C, x, C.L.c[j], &sg);
          acc += (double)C.L.c[j][b] * sg * s.u[a][m];
        }
        (*G)[((size_t)a * d + b) * C.N + n] = acc / C.L.cn[b];  // G_ab = d_b u_a
      }
  }
}

template <class T>
T feq(const Ctx& C, int i, const Fields<T>& s, const std::vector<T>& G, size_t n) {
  const int d = C.d;
  const int* c = C.L.c[i];
  T cu = T(0), uu = T(0), cgc = T(0);
  for (int a = 0; a < d; ++a) {
    cu += (double)c[a] * s.u[a][n];
    uu += s.u[a][n] * s.u[a][n];
  }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) cgc += (double)(c[a] * c[b]) * G[((size_t)a * d + b) * C.N + n];
  // A (d_a u_b + d_b u_a) c_a c_b summed over a, b equals 2 A sum_ab G_ab c_a c_b
  return C.L.w[i] * (3.0 * s.p[n] + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu) + C.L.w[i] * C.A * 2.0 * cgc;
}

template <class T>
void apply_boundaries(const Ctx& C, Fields<T>* o) {
  const int d = C.d;
  int x[3];
  // phase 1: y walls, for nodes whose x and z are interior
  // phase 2: z walls, for nodes whose x is interior
  for (int wa = 1; wa < d; ++wa) {
    if (C.P.bc[wa] != BC_WALL) continue;
    for (size_t n = 0; n < C.N; ++n) {
      coords(C, n, x);
      if (!(x[wa] == 0 || x[wa] == C.n[wa] - 1)) continue;
      if (on_boundary(C, 0, x[0])) continue;
      if (wa == 1 && d == 3 && on_boundary(C, 2, x[2])) continue;
      int y[3] = {x[0], x[1], x[2]};
      y[wa] = (x[wa] == 0) ? 1 : C.n[wa] - 2;
      o->p[n] = o->p[idx(C, y[0], y[1], y[2])];
      for (int a = 0; a < d; ++a) o->u[a][n] = T(0);
    }
  }
  // phase 3: open x boundaries, all rows
  const int bcx = C.P.bc[0];
  if (bcx == BC_PERIODIC) return;
  for (size_t n = 0; n < C.N; ++n) {
    coords(C, n, x);
    if (!(x[0] == 0 || x[0] == C.n[0] - 1)) continue;
    bool inlet = (x[0] == 0);
    size_t nin = idx(C, inlet ? 1 : C.n[0] - 2, x[1], x[2]);
    if (bcx == BC_INFLOW_OUTFLOW) {
      if (inlet) {
        o->p[n] = o->p[nin];  // zero-gradient pressure at the inlet
        o->u[0][n] = T(C.P.u_in);
        for (int a = 1; a < d; ++a) o->u[a][n] = T(0);
      } else {
        o->p[n] = T(0);  // pressure gauge fixed at the outlet
        for (int a = 0; a < d; ++a) o->u[a][n] = o->u[a][nin];
      }
    } else {  // BC_PRESSURE
      o->p[n] = inlet ? T(C.P.dp) : T(0);
      for (int a = 0; a < d; ++a) o->u[a][n] = o->u[a][nin];
    }
  }
}

template <class T>
void stencil_fwd(const Ctx& C, const Fields<T>& s, Fields<T>* o) {
  const int d = C.d, Q = C.L.Q;
  std::vector<T> G;
  velocity_gradient(C, s, &G);
  std::vector<T> f((size_t)Q * C.N);
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < C.N; ++n)
    for (int i = 0; i < Q; ++i) f[(size_t)i * C.N + n] = feq(C, i, s, G, n);
  o->alloc(C);
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < C.N; ++n) {
    int x[3];
    coords(C, n, x);
    if (!is_interior(C, x)) continue;
    T ps = T(0);
    T us[3] = {T(0), T(0), T(0)};
    for (int i = 0; i < Q; ++i) {
      T fi = f[(size_t)i * C.N + shift_nbr(C, x, C.L.c[i], -1)];  // f_i^eq(x - c_i)
      ps += fi;
      for (int a = 0; a < d; ++a) us[a] += (double)C.L.c[i][a] * fi;
    }
    o->p[n] = ps / 3.0;
    for (int a = 0; a < d; ++a) o->u[a][n] = us[a];
  }
  apply_boundaries(C, o);
}

// Exact transpose of stencil_fwd at the state s (the vector-Jacobian product).
// In: lps, lus = dJ/d(p*, u*). Out: lp, lu = dJ/d(p, u) at t-1.
template <class T>
void stencil_vjp(const Ctx& C, const Fields<T>& s, const Fields<T>& lam_star, Fields<T>* lam) {
  const int d = C.d, Q = C.L.Q;
  Fields<T> ls = lam_star;  // working copy, boundary phases reversed in place
  int x[3];
  // reverse phase 3 (open x boundaries)
  const int bcx = C.P.bc[0];
  if (bcx != BC_PERIODIC) {
    for (size_t n = 0; n < C.N; ++n) {
      coords(C, n, x);
      if (!(x[0] == 0 || x[0] == C.n[0] - 1)) continue;
      bool inlet = (x[0] == 0);
      size_t nin = idx(C, inlet ? 1 : C.n[0] - 2, x[1], x[2]);
      if (bcx == BC_INFLOW_OUTFLOW) {
        if (inlet) {
          ls.p[nin] += ls.p[n];
        } else {
          for (int a = 0; a < d; ++a) ls.u[a][nin] += ls.u[a][n];
        }
      } else {
        for (int a = 0; a < d; ++a) ls.u[a][nin] += ls.u[a][n];
      }
      ls.p[n] = T(0);
      for (int a = 0; a < d; ++a) ls.u[a][n] = T(0);
    }
  }
  // reverse phase 2 then phase 1 (walls)
  for (int wa = d - 1; wa >= 1; --wa) {
    if (C.P.bc[wa] != BC_WALL) continue;
    for (size_t n = 0; n < C.N; ++n) {
      coords(C, n, x);
      if (!(x[wa] == 0 || x[wa] == C.n[wa] - 1)) continue;
      if (on_boundary(C, 0, x[0])) continue;
      if (wa == 1 && d == 3 && on_boundary(C, 2, x[2])) continue;
      int y[3] = {x[0], x[1], x[2]};
      y[wa] = (x[wa] == 0) ? 1 : C.n[wa] - 2;
      ls.p[idx(C, y[0], y[1], y[2])] += ls.p[n];
      ls.p[n] = T(0);
      for (int a = 0; a < d; ++a) ls.u[a][n] = T(0);
    }
  }
  // interior gather transpose: fbar_i(x - c_i) += lps(x)/3 + c_i . lus(x)
  std::vector<T> fbar((size_t)Q * C.N, T(0));
  // (for a fixed i, x -> x - c_i is one-to-one on the interior: each fbar entry has one writer)
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < C.N; ++n) {
    int x[3];
    coords(C, n, x);
    if (!is_interior(C, x)) continue;
    for (int i = 0; i < Q; ++i) {
      T v = ls.p[n] / 3.0;
      for (int a = 0; a < d; ++a) v += (double)C.L.c[i][a] * ls.u[a][n];
      fbar[(size_t)i * C.N + shift_nbr(C, x, C.L.c[i], -1)] += v;
    }
  }
  // f^eq transpose (the gradient enters f^eq linearly, so only its adjoint is needed)
  lam->alloc(C);
  std::vector<T> lG((size_t)d * d * C.N, T(0));
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < C.N; ++n) {
    for (int i = 0; i < Q; ++i) {
      T fb = fbar[(size_t)i * C.N + n];
      const int* c = C.L.c[i];
      double wi = C.L.w[i];
      T cu = T(0);
      for (int a = 0; a < d; ++a) cu += (double)c[a] * s.u[a][n];
      lam->p[n] += 3.0 * wi * fb;
      for (int a = 0; a < d; ++a) lam->u[a][n] += wi * fb * (3.0 * c[a] + 9.0 * cu * (double)c[a] - 3.0 * s.u[a][n]);
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) lG[((size_t)a * d + b) * C.N + n] += wi * C.A * 2.0 * (double)(c[a] * c[b]) * fb;
    }
  }
  // velocity-gradient transpose: G_ab(n) = sum_j c_jb sgn u_a(nbr) / cn_b
  for (size_t n = 0; n < C.N; ++n) {
    coords(C, n, x);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        T g = lG[((size_t)a * d + b) * C.N + n];
        for (int j = 0; j < Q; ++j) {
          if (C.L.c[j][b] == 0) continue;
          double sg;
          size_t m = grad_nbr(C, x, C.L.c[j], &sg);
          lam->u[a][m] += (double)C.L.c[j][b] * sg * g / C.L.cn[b];
        }
      }
  }
}

// ------------------------------------------------------------------------------------------
// Grid separation (Sec. 2.3) and rigid motion.
// ------------------------------------------------------------------------------------------
template <class T>
T wk(int kind, T r) {
  double a = std::fabs(re(r));
  if (kind == W_BILINEAR) {
    if (a >= 1.0) return T(0);
    return re(r) >= 0.0 ? T(1.0) - r : T(1.0) + r;
  }
  if (a >= 2.0) return T(0);
  return 0.25 * (1.0 + std::cos(kPi * r / 2.0));  // the paper's "1 - cos" read as "1 + cos"
}

template <class T>
T dwk(int kind, T r) {  // dw/dr, the branch taken on the real part as in wk
  double a = std::fabs(re(r));
  if (kind == W_BILINEAR) {
    if (a >= 1.0) return T(0);
    return re(r) >= 0.0 ? T(-1.0) : T(1.0);
  }
  if (a >= 2.0) return T(0);
  return -0.125 * kPi * std::sin(kPi * r / 2.0);
}

// In-plane axes (b, c) of the rotation about axis a, right-handed.
inline void plane_axes(int a, int* b, int* c) {
  *b = (a + 1) % 3;
  *c = (a + 2) % 3;
}

// Design-point geometry for one DOF iterate (Eqs. rigid_body_position, rigid_body_velocity).
template <class T>
struct Geometry {
  std::vector<T> xref, usref, lev, dlev;  // [ND][3]; lev = R r, dlev = R' r = d(R r)/d theta
};

template <class T>
void transform(const Ctx& C, const T* s, Geometry<T>* g) {
  const size_t ND = C.ND;
  g->xref.assign(ND * 3, T(0));
  g->usref.assign(ND * 3, T(0));
  g->lev.assign(ND * 3, T(0));
  g->dlev.assign(ND * 3, T(0));
  if (C.free_rot) {
    // x^ref = x^G + R r, u^S,ref = u^G + omega x (R r); dlev unused
    const T* om = s + 9;
    const T* R = s + 12;
    for (size_t m = 0; m < ND; ++m) {
      const double* r = &C.r[3 * m];
      T l[3];
      for (int i = 0; i < 3; ++i) l[i] = R[3 * i + 0] * r[0] + R[3 * i + 1] * r[1] + R[3 * i + 2] * r[2];
      const T w[3] = {om[1] * l[2] - om[2] * l[1], om[2] * l[0] - om[0] * l[2], om[0] * l[1] - om[1] * l[0]};
      for (int a = 0; a < 3; ++a) {
        g->lev[3 * m + a] = l[a];
        g->xref[3 * m + a] = s[a] + l[a];
        g->usref[3 * m + a] = s[3 + a] + w[a];
      }
    }
    return;
  }
  int ax = C.P.rot_axis, b, c;
  plane_axes(ax, &b, &c);
  T ct = std::cos(s[6]), st = std::sin(s[6]);
  for (size_t m = 0; m < ND; ++m) {
    const double* r = &C.r[3 * m];
    T l[3], dl[3];
    l[ax] = T(r[ax]);
    dl[ax] = T(0);
    l[b] = ct * r[b] - st * r[c];
    l[c] = st * r[b] + ct * r[c];
    dl[b] = -st * r[b] - ct * r[c];
    dl[c] = ct * r[b] - st * r[c];
    for (int a = 0; a < 3; ++a) {
      g->lev[3 * m + a] = l[a];
      g->dlev[3 * m + a] = dl[a];
      g->xref[3 * m + a] = (a < C.d) ? s[a] + l[a] : T(0);
      g->usref[3 * m + a] = (a < C.d) ? s[3 + a] + s[7] * dl[a] : T(0);
    }
  }
}

// Support window of design point m: 2*support nodes per axis starting at floor(xref) - support + 1.
// Nodes on non-periodic axes must stay at least two cells inside the boundary planes.
struct WindowNode {
  size_t n;
  int off[3];
};

template <class T>
void window(Ctx& C, const T* xref, std::vector<WindowNode>* out, std::vector<T>* wv, std::vector<T>* dwv) {
  out->clear();
  wv->clear();
  dwv->clear();
  const int d = C.d, s = C.support, kind = C.P.weight_kind;
  int lo[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
  for (int a = 0; a < d; ++a) {
    lo[a] = (int)std::floor(re(xref[a])) - s + 1;
    cnt[a] = 2 * s;
  }
  for (int k = 0; k < cnt[2]; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i) {
        int pos[3] = {lo[0] + i, lo[1] + j, lo[2] + k};
        T w1[3], dw1[3];
        bool nz = true;
        for (int a = 0; a < 3; ++a) {
          if (a < d) {
            T rr = (double)pos[a] - xref[a];
            w1[a] = wk(kind, rr);
            dw1[a] = dwk(kind, rr);
            if (re(w1[a]) == 0.0 && re(dw1[a]) == 0.0) nz = false;
          } else {
            w1[a] = T(1);
            dw1[a] = T(0);
          }
        }
        if (!nz) continue;
        int node[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
          if (C.P.bc[a] == BC_PERIODIC) {
            node[a] = wrap(pos[a], C.n[a]);
          } else {
            if (pos[a] < 2 || pos[a] > C.n[a] - 3) {
              C.err = ORC_ERR_BODY_OUTSIDE;
              node[a] = pos[a] < 2 ? 2 : C.n[a] - 3;
            } else {
              node[a] = pos[a];
            }
          }
        }
        WindowNode wn;
        wn.n = idx(C, node[0], node[1], node[2]);
        wn.off[0] = i;
        wn.off[1] = j;
        wn.off[2] = k;
        out->push_back(wn);
        T W = w1[0] * w1[1] * w1[2];
        wv->push_back(W);
        // dW/dxref_e = -w'(x_e - xref_e) prod_{a != e} w(x_a - xref_a)
        for (int e = 0; e < 3; ++e) {
          T prod = T(1);
          for (int a = 0; a < 3; ++a) prod *= (a == e) ? dw1[a] : w1[a];
          dwv->push_back(e < d ? -prod : T(0));
        }
      }
}

// One coupling iteration's intermediate values (kept for the adjoint).
template <class T>
struct IterRecord {
  std::vector<T> kap, us[3], u[3];  // analysis-grid fields
  std::vector<T> uref;              // [ND][3]
  Geometry<T> geo;
  T F[3], Tq;  // force; torque about the rotation axis
  T Tv[3];     // free rotation: torque vector
};

// Rodrigues' formula: the rotation by |v| about v, Q = I + a [v]x + b [v]x^2 with
// a = sin|v| / |v| and b = (1 - cos|v|) / |v|^2, from their power series in x = v.v when |v| is
// small (terms to x^10, remainder below 1e-40 for |v| < 0.1).
template <class T>
void rodrigues(const T* v, T* Q) {
  const T x = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  T a, b;
  if (std::fabs(re(x)) < 1e-2) {
    T ta = T(1), tb = T(0.5);  // k = 0 terms: 1/1!, 1/2!
    a = ta;
    b = tb;
    for (int k = 1; k <= 10; ++k) {
      ta *= -x / double((2 * k) * (2 * k + 1));
      tb *= -x / double((2 * k + 1) * (2 * k + 2));
      a += ta;
      b += tb;
    }
  } else {
    const T th = std::sqrt(x);
    a = std::sin(th) / th;
    b = (1.0 - std::cos(th)) / x;
  }
  const T K[9] = {T(0), -v[2], v[1], v[2], T(0), -v[0], -v[1], v[0], T(0)};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T k2 = T(0);
      for (int l = 0; l < 3; ++l) k2 += K[3 * i + l] * K[3 * l + j];
      Q[3 * i + j] = (i == j ? T(1) : T(0)) + a * K[3 * i + j] + b * k2;
    }
}

// Explicit Euler EOM of one coupling iteration (Sec. 2.4), velocity first, masked by the DOFs:
// from s(t-1) = s0 and the iteration's force F and torque (Tq about the axis, or the vector Tv
// with free rotation) to s^(k).
template <class T>
void eom_apply(const Ctx& C, const T* s0, const T* F, T Tq, const T* Tv, T* out) {
  for (int a = 0; a < C.ns; ++a) out[a] = s0[a];
  const int mask = C.P.dof_mask;
  for (int a = 0; a < C.d; ++a) {
    if (!(mask & (1 << a))) continue;
    out[3 + a] = s0[3 + a] + F[a] / C.P.mass;
    out[a] = s0[a] + out[3 + a];
  }
  if (!(mask & DOF_ROT)) return;
  if (!C.free_rot) {
    out[7] = s0[7] + Tq / C.P.inertia;
    out[6] = s0[6] + out[7];
    return;
  }
  const T* R0 = s0 + 12;
  T h[3], v1[3], v2[3], w[3];
  for (int a = 0; a < 3; ++a) h[a] = s0[6 + a] + Tv[a];
  for (int j = 0; j < 3; ++j) v1[j] = R0[0 + j] * h[0] + R0[3 + j] * h[1] + R0[6 + j] * h[2];  // R0^T h
  for (int i = 0; i < 3; ++i) v2[i] = C.Jinv[3 * i + 0] * v1[0] + C.Jinv[3 * i + 1] * v1[1] + C.Jinv[3 * i + 2] * v1[2];
  for (int i = 0; i < 3; ++i) w[i] = R0[3 * i + 0] * v2[0] + R0[3 * i + 1] * v2[1] + R0[3 * i + 2] * v2[2];
  T Q[9];
  rodrigues(w, Q);
  for (int a = 0; a < 3; ++a) {
    out[6 + a] = h[a];
    out[9 + a] = w[a];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      out[12 + 3 * i + j] = Q[3 * i + 0] * R0[0 + j] + Q[3 * i + 1] * R0[3 + j] + Q[3 * i + 2] * R0[6 + j];
}

template <class T>
void coupling_iteration(Ctx& C, const std::vector<T>& kref, const T* s_prev_iter, const T* s_step_start,
                        const Fields<T>& star, IterRecord<T>* rec, T* s_new) {
  const int d = C.d;
  const size_t N = C.N, ND = C.ND;
  transform(C, s_prev_iter, &rec->geo);
  rec->kap.assign(N, T(0));
  for (int a = 0; a < 3; ++a) {
    rec->us[a].assign(a < d ? N : 0, T(0));
    rec->u[a].assign(a < d ? N : 0, T(0));
  }
  std::vector<WindowNode> wn;
  std::vector<T> wv, dwv;
  // spread (Eqs. kappa_mapping, us_mapping): scatter each design point over its window
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &rec->geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q) {
      rec->kap[wn[q].n] += wv[q] * kref[m];
      for (int a = 0; a < d; ++a) rec->us[a][wn[q].n] += wv[q] * rec->geo.usref[3 * m + a];
    }
  }
  // Brinkman update (Eq. u); p = p* is untouched
  LKS_ORACLE_PARALLEL_FOR
  for (size_t n = 0; n < N; ++n)
    for (int a = 0; a < d; ++a) rec->u[a][n] = (star.u[a][n] + rec->kap[n] * rec->us[a][n]) / (1.0 + rec->kap[n]);
  // interpolation to the design points (Eq. u_mapping)
  rec->uref.assign(ND * 3, T(0));
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &rec->geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q)
      for (int a = 0; a < d; ++a) rec->uref[3 * m + a] += wv[q] * rec->u[a][wn[q].n];
  }
  // force and torque from the design-grid sums (Sec. 2.4); lever arm x^ref - x^G = R r
  int ax = C.free_rot ? 2 : C.P.rot_axis, b, c;
  plane_axes(ax, &b, &c);
  T F[3] = {T(0), T(0), T(0)}, Tq = T(0), Tv[3] = {T(0), T(0), T(0)};
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    T D[3];
    for (int a = 0; a < 3; ++a) D[a] = (a < d) ? rec->uref[3 * m + a] - rec->geo.usref[3 * m + a] : T(0);
    for (int a = 0; a < d; ++a) F[a] += kref[m] * D[a];
    const T* l = &rec->geo.lev[3 * m];
    Tq += kref[m] * (l[b] * D[c] - l[c] * D[b]);
    Tv[0] += kref[m] * (l[1] * D[2] - l[2] * D[1]);
    Tv[1] += kref[m] * (l[2] * D[0] - l[0] * D[2]);
    Tv[2] += kref[m] * (l[0] * D[1] - l[1] * D[0]);
  }
  for (int a = 0; a < 3; ++a) {
    rec->F[a] = F[a];
    rec->Tv[a] = Tv[a];
  }
  rec->Tq = Tq;
  // explicit Euler EOM, velocity first (Eqs. equation_of_motion_*_discretized), masked by the DOFs
  eom_apply(C, s_step_start, F, Tq, Tv, s_new);
}

template <class T>
void forward_step(Ctx& C, const std::vector<T>& kref, const Fields<T>& prev, const T* s_prev, Fields<T>* next,
                  T* s_next, std::vector<T>* iters_out) {
  Fields<T> star;
  stencil_fwd(C, prev, &star);
  const int K = C.P.n_itr, ns = C.ns;
  std::vector<T> it((size_t)(K + 1) * ns);
  for (int a = 0; a < ns; ++a) it[a] = s_prev[a];
  IterRecord<T> rec;
  for (int k = 1; k <= K; ++k)
    coupling_iteration(C, kref, &it[(size_t)(k - 1) * ns], s_prev, star, &rec, &it[(size_t)k * ns]);
  next->p = star.p;
  for (int a = 0; a < 3; ++a) next->u[a] = rec.u[a];
  for (int a = 0; a < ns; ++a) s_next[a] = it[(size_t)K * ns + a];
  if (iters_out) *iters_out = it;
}

// The design chain (cyclic expansion, Eq. filter, Eq. projection) from gamma to gamma-bar.
template <class T>
struct Chain {
  std::vector<T> g1, g2, g3;  // expanded, filtered, projected
  std::vector<double> W;      // filter normaliser sum_j w_ij
};

// Filter neighbours of design point i: (j, w_ij) with |x_i - x_j| <= R, both in the domain.
void filter_nbrs(const Ctx& C, size_t i, std::vector<std::pair<size_t, double>>* out) {
  out->clear();
  const double R = C.P.filter_radius;
  const int rr = (int)std::floor(R);
  const int ii[3] = {(int)(i % C.nd[0]), (int)((i / C.nd[0]) % C.nd[1]), (int)(i / ((size_t)C.nd[0] * C.nd[1]))};
  const int ext[3] = {rr, rr, C.d == 3 ? rr : 0};
  for (int dz = -ext[2]; dz <= ext[2]; ++dz)
    for (int dy = -ext[1]; dy <= ext[1]; ++dy)
      for (int dx = -ext[0]; dx <= ext[0]; ++dx) {
        const int j[3] = {ii[0] + dx, ii[1] + dy, ii[2] + dz};
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && j[a] >= 0 && j[a] < C.nd[a];
        if (!ok) continue;
        const double dist = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (dist > R) continue;
        const size_t mj = (size_t)j[0] + C.nd[0] * ((size_t)j[1] + (size_t)C.nd[1] * j[2]);
        if (!C.dom[mj]) continue;
        out->push_back({mj, (R - dist) / R});
      }
}

template <class T>
T project(const Ctx& C, T x) {
  const double b = C.P.proj_beta, e = C.P.proj_eta;
  return (std::tanh(b * e) + std::tanh(b * (x - e))) / (std::tanh(b * e) + std::tanh(b * (1.0 - e)));
}

template <class T>
void design_chain(const Ctx& C, const T* gamma, Chain<T>* ch) {
  const size_t ND = C.ND;
  ch->g1.assign(ND, T(0));
  ch->g2.assign(ND, T(0));
  ch->g3.assign(ND, T(0));
  ch->W.assign(ND, 1.0);
  for (size_t m = 0; m < ND; ++m) ch->g1[m] = gamma[C.rep[m]];
  std::vector<std::pair<size_t, double>> nb;
  for (size_t i = 0; i < ND; ++i) {
    if (!C.dom[i]) continue;
    if (C.P.filter_radius > 0.0) {
      filter_nbrs(C, i, &nb);
      T acc = T(0);
      double W = 0.0;
      for (auto& q : nb) {
        acc += q.second * ch->g1[q.first];
        W += q.second;
      }
      ch->W[i] = W;
      ch->g2[i] = acc / W;
    } else {
      ch->g2[i] = ch->g1[i];
    }
    ch->g3[i] = (C.P.proj_beta > 0.0) ? project(C, ch->g2[i]) : ch->g2[i];
  }
}

// dJ/dgamma from dJ/dgamma-bar (gb3): the transposes of the projection, the filter (its weights are
// symmetric in i and j) and the cyclic expansion (a sum over each orbit onto its representative).
void design_chain_vjp(const Ctx& C, const Chain<double>& ch, const std::vector<double>& gb3, double* out) {
  const size_t ND = C.ND;
  std::vector<double> gb2(ND, 0.0), gb1(ND, 0.0);
  const double b = C.P.proj_beta, e = C.P.proj_eta;
  for (size_t i = 0; i < ND; ++i) {
    if (!C.dom[i]) continue;
    if (b > 0.0) {
      const double th = std::tanh(b * (ch.g2[i] - e));
      gb2[i] = gb3[i] * b * (1.0 - th * th) / (std::tanh(b * e) + std::tanh(b * (1.0 - e)));
    } else {
      gb2[i] = gb3[i];
    }
  }
  if (C.P.filter_radius > 0.0) {
    std::vector<std::pair<size_t, double>> nb;
    for (size_t i = 0; i < ND; ++i) {
      if (!C.dom[i]) continue;
      filter_nbrs(C, i, &nb);
      for (auto& q : nb) gb1[q.first] += q.second / ch.W[i] * gb2[i];
    }
  } else {
    gb1 = gb2;
  }
  for (size_t m = 0; m < ND; ++m) out[m] = 0.0;
  for (size_t m = 0; m < ND; ++m) out[C.rep[m]] += gb1[m];
}

// Brinkman interpolation (Eq. brinkman_coefficient) of gamma-bar, after the design chain.
template <class T>
std::vector<T> brinkman(const Ctx& C, const T* gamma, Chain<T>* keep = nullptr) {
  Chain<T> local;
  Chain<T>* ch = keep ? keep : &local;
  design_chain(C, gamma, ch);
  std::vector<T> k(C.ND);
  for (size_t m = 0; m < C.ND; ++m) {
    const T gb = ch->g3[m];
    k[m] = C.dom[m] ? C.P.kappa_max * C.P.q * gb / ((1.0 - gb) + C.P.q) : T(0);
  }
  return k;
}

template <class T>
void load_fields(const Ctx& C, const T* p, const T* u, Fields<T>* f) {
  f->alloc(C);
  for (size_t n = 0; n < C.N; ++n) f->p[n] = p[n];
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < C.N; ++n) f->u[a][n] = u[(size_t)a * C.N + n];
}

template <class T>
T objective(const Ctx& C, const T* s) {
  T J = T(0);
  for (int a = 0; a < C.ns; ++a) J += C.P.obj_w[a] * s[a];
  return J;
}

bool finite_fields(const Ctx& C, const Fields<double>& f) {
  for (size_t n = 0; n < C.N; ++n) {
    if (!std::isfinite(f.p[n])) return false;
    for (int a = 0; a < C.d; ++a)
      if (!std::isfinite(f.u[a][n])) return false;
  }
  return true;
}

// ------------------------------------------------------------------------------------------
// Adjoint of one coupling iteration k (exact reverse of coupling_iteration).
//   in : lam_sk = dJ/ds^(k) ; lam_uk_ext = dJ/du^(k) from outside the iteration (k = N_itr only)
//   out: lam_ustar += dJ/du* ; lam_prev += direct EOM part of dJ/ds(t-1) ;
//        lam_skm1 = dJ/ds^(k-1) through the transform ; dkref += dJ/dkappa^ref
// ------------------------------------------------------------------------------------------
// Reverse of the interpolation, Brinkman update and spread of one coupling iteration, given
// dJ/du^ref (l_uref): accumulates dJ/du* into lam_ustar, dJ/du^S,ref into l_usref, dJ/dx^ref into
// l_xref and the kernel-weight part of dJ/dkappa^ref into dkref.
void mapping_vjp(Ctx& C, const std::vector<double>& kref, const IterRecord<double>& rec,
                 const std::vector<double>& l_uref, const Fields<double>* lam_uk_ext, Fields<double>* lam_ustar,
                 std::vector<double>* l_usref_p, std::vector<double>* l_xref_p, std::vector<double>* dkref) {
  const int d = C.d;
  const size_t N = C.N, ND = C.ND;
  std::vector<double>& l_usref = *l_usref_p;
  std::vector<double>& l_xref = *l_xref_p;
  // interpolation reverse
  Fields<double> lam_uk;
  lam_uk.alloc(C);
  if (lam_uk_ext)
    for (int a = 0; a < d; ++a) lam_uk.u[a] = lam_uk_ext->u[a];
  std::vector<WindowNode> wn;
  std::vector<double> wv, dwv;
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &rec.geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q) {
      double ul = 0;
      for (int a = 0; a < d; ++a) {
        lam_uk.u[a][wn[q].n] += wv[q] * l_uref[3 * m + a];
        ul += rec.u[a][wn[q].n] * l_uref[3 * m + a];
      }
      for (int e = 0; e < d; ++e) l_xref[3 * m + e] += dwv[3 * q + e] * ul;
    }
  }
  // Brinkman reverse
  std::vector<double> l_kap(N, 0.0);
  std::vector<double> l_us[3];
  for (int a = 0; a < d; ++a) l_us[a].assign(N, 0.0);
  for (size_t n = 0; n < N; ++n) {
    double inv = 1.0 / (1.0 + rec.kap[n]);
    double lk = 0;
    for (int a = 0; a < d; ++a) {
      double lu = lam_uk.u[a][n];
      lam_ustar->u[a][n] += lu * inv;
      lk += lu * (rec.us[a][n] - rec.u[a][n]) * inv;
      l_us[a][n] = lu * rec.kap[n] * inv;
    }
    l_kap[n] = lk;
  }
  // spread reverse
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &rec.geo.xref[3 * m], &wn, &wv, &dwv);
    double dk = 0;
    for (size_t q = 0; q < wn.size(); ++q) {
      size_t n = wn[q].n;
      dk += wv[q] * l_kap[n];
      double su = kref[m] * l_kap[n];
      for (int a = 0; a < d; ++a) {
        l_usref[3 * m + a] += wv[q] * l_us[a][n];
        su += rec.geo.usref[3 * m + a] * l_us[a][n];
      }
      for (int e = 0; e < d; ++e) l_xref[3 * m + e] += dwv[3 * q + e] * su;
    }
    (*dkref)[m] += dk;
  }
}

// Reverse of eom_apply with free rotation, by complex-step derivatives: column j of the Jacobian
// of s^(k) with respect to the inputs (s0[21], F[3], Tv[3]) is Im eom_apply(input + i h e_j) / h,
// exact to rounding (no difference is taken). lam_in[j] = sum_i lam_out[i] d out_i / d in_j.
void eom_vjp_free(const Ctx& C, const double* s0, const double* F, const double* Tv, const double* lam_out,
                  double* lam_in) {
  const int ns = C.ns, nin = ns + 6;
  const double h = 1e-30;
  for (int j = 0; j < nin; ++j) {
    cplx in[27], out[21];
    for (int a = 0; a < ns; ++a) in[a] = cplx(s0[a], 0.0);
    for (int a = 0; a < 3; ++a) {
      in[ns + a] = cplx(F[a], 0.0);
      in[ns + 3 + a] = cplx(Tv[a], 0.0);
    }
    in[j] += cplx(0.0, h);
    eom_apply<cplx>(C, in, in + ns, cplx(0.0), in + ns + 3, out);
    double acc = 0.0;
    for (int i = 0; i < ns; ++i) acc += lam_out[i] * (out[i].imag() / h);
    lam_in[j] = acc;
  }
}

// Exact reverse of coupling_iteration with free rotation (see coupling_iteration_vjp).
void coupling_iteration_vjp_free(Ctx& C, const std::vector<double>& kref, const IterRecord<double>& rec,
                                 const double* s_km1, const double* s_step_start, const double* lam_sk,
                                 const Fields<double>* lam_uk_ext, Fields<double>* lam_ustar, double* lam_prev,
                                 double* lam_skm1, std::vector<double>* dkref) {
  const size_t ND = C.ND;
  const int ns = C.ns;
  // EOM reverse
  double lin[27];
  eom_vjp_free(C, s_step_start, rec.F, rec.Tv, lam_sk, lin);
  for (int a = 0; a < ns; ++a) lam_prev[a] += lin[a];
  const double* lF = lin + ns;
  const double* lT = lin + ns + 3;
  // force / torque reverse: F = sum_m kappa_m D_m, T = sum_m kappa_m l_m x D_m, D = u^ref - u^S,ref
  std::vector<double> l_uref(ND * 3, 0.0), l_usref(ND * 3, 0.0), l_lev(ND * 3, 0.0), l_xref(ND * 3, 0.0);
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    const double* l = &rec.geo.lev[3 * m];
    double D[3];
    for (int a = 0; a < 3; ++a) D[a] = rec.uref[3 * m + a] - rec.geo.usref[3 * m + a];
    const double txl[3] = {lT[1] * l[2] - lT[2] * l[1], lT[2] * l[0] - lT[0] * l[2], lT[0] * l[1] - lT[1] * l[0]};
    const double dxt[3] = {D[1] * lT[2] - D[2] * lT[1], D[2] * lT[0] - D[0] * lT[2], D[0] * lT[1] - D[1] * lT[0]};
    double dk = 0;
    for (int a = 0; a < 3; ++a) {
      const double lD = kref[m] * (lF[a] + txl[a]);  // d/dD of lF.D + lT.(l x D) = D.(lT x l)
      l_uref[3 * m + a] = lD;
      l_usref[3 * m + a] = -lD;
      l_lev[3 * m + a] += kref[m] * dxt[a];           // lT.(l x D) = l.(D x lT)
      dk += lF[a] * D[a] + txl[a] * D[a];
    }
    (*dkref)[m] += dk;
  }
  mapping_vjp(C, kref, rec, l_uref, lam_uk_ext, lam_ustar, &l_usref, &l_xref, dkref);
  // transform reverse: xref = xG + R r, usref = uG + omega x (R r), lev = R r
  for (int a = 0; a < ns; ++a) lam_skm1[a] = 0.0;
  const double* om = s_km1 + 9;
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    const double* l = &rec.geo.lev[3 * m];
    const double* r = &C.r[3 * m];
    const double* lu = &l_usref[3 * m];
    const double lxu[3] = {l[1] * lu[2] - l[2] * lu[1], l[2] * lu[0] - l[0] * lu[2], l[0] * lu[1] - l[1] * lu[0]};
    const double uxo[3] = {lu[1] * om[2] - lu[2] * om[1], lu[2] * om[0] - lu[0] * om[2], lu[0] * om[1] - lu[1] * om[0]};
    for (int a = 0; a < 3; ++a) {
      lam_skm1[a] += l_xref[3 * m + a];
      lam_skm1[3 + a] += lu[a];
      lam_skm1[9 + a] += lxu[a];  // lu.(omega x l) = omega.(l x lu)
    }
    for (int i = 0; i < 3; ++i) {
      const double gl = l_lev[3 * m + i] + l_xref[3 * m + i] + uxo[i];  // lu.(omega x l) = l.(lu x omega)
      for (int j = 0; j < 3; ++j) lam_skm1[12 + 3 * i + j] += gl * r[j];
    }
  }
}

void coupling_iteration_vjp(Ctx& C, const std::vector<double>& kref, const IterRecord<double>& rec,
                            const double* s_km1, const double* s_step_start, const double* lam_sk,
                            const Fields<double>* lam_uk_ext, Fields<double>* lam_ustar, double* lam_prev,
                            double* lam_skm1, std::vector<double>* dkref) {
  const int d = C.d;
  const size_t ND = C.ND;
  const int mask = C.P.dof_mask;
  if (C.free_rot) {
    coupling_iteration_vjp_free(C, kref, rec, s_km1, s_step_start, lam_sk, lam_uk_ext, lam_ustar, lam_prev, lam_skm1,
                                dkref);
    return;
  }
  // EOM reverse
  double lF[3] = {0, 0, 0}, lT = 0;
  for (int a = 0; a < 3; ++a) {
    bool free_a = (a < d) && (mask & (1 << a));
    if (free_a) {
      double lug = lam_sk[3 + a] + lam_sk[a];
      lF[a] = lug / C.P.mass;
      lam_prev[a] += lam_sk[a];
      lam_prev[3 + a] += lug;
    } else {
      lam_prev[a] += lam_sk[a];
      lam_prev[3 + a] += lam_sk[3 + a];
    }
  }
  if (mask & DOF_ROT) {
    double lom = lam_sk[7] + lam_sk[6];
    lT = lom / C.P.inertia;
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lom;
  } else {
    lam_prev[6] += lam_sk[6];
    lam_prev[7] += lam_sk[7];
  }
  // force / torque reverse
  int ax = C.P.rot_axis, b, c;
  plane_axes(ax, &b, &c);
  std::vector<double> l_uref(ND * 3, 0.0), l_usref(ND * 3, 0.0), l_lev(ND * 3, 0.0), l_xref(ND * 3, 0.0);
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    double D[3];
    for (int a = 0; a < 3; ++a) D[a] = (a < d) ? rec.uref[3 * m + a] - rec.geo.usref[3 * m + a] : 0.0;
    const double* l = &rec.geo.lev[3 * m];
    double lD[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) lD[a] += kref[m] * lF[a];
    lD[c] += kref[m] * lT * l[b];
    lD[b] -= kref[m] * lT * l[c];
    for (int a = 0; a < d; ++a) {
      l_uref[3 * m + a] = lD[a];
      l_usref[3 * m + a] = -lD[a];
    }
    l_lev[3 * m + b] += lT * kref[m] * D[c];
    l_lev[3 * m + c] -= lT * kref[m] * D[b];
    double dk = 0;
    for (int a = 0; a < d; ++a) dk += lF[a] * D[a];
    dk += lT * (l[b] * D[c] - l[c] * D[b]);
    (*dkref)[m] += dk;
  }
  mapping_vjp(C, kref, rec, l_uref, lam_uk_ext, lam_ustar, &l_usref, &l_xref, dkref);
  // transform reverse: xref = xG + R r, usref = uG + omega R' r, lev = R r
  for (int a = 0; a < 8; ++a) lam_skm1[a] = 0.0;
  const double om = s_km1[7];
  for (size_t m = 0; m < ND; ++m) {
    if (!C.dom[m]) continue;
    const double* l = &rec.geo.lev[3 * m];
    const double* dl = &rec.geo.dlev[3 * m];
    double ddl[3];  // R'' r = -(R r) in the rotation plane, 0 along the axis
    for (int a = 0; a < 3; ++a) ddl[a] = (a == ax) ? 0.0 : -l[a];
    for (int a = 0; a < d; ++a) {
      lam_skm1[a] += l_xref[3 * m + a];
      lam_skm1[3 + a] += l_usref[3 * m + a];
    }
    for (int a = 0; a < 3; ++a) {
      double lx = (a < d) ? l_xref[3 * m + a] : 0.0;
      double lus = (a < d) ? l_usref[3 * m + a] : 0.0;
      lam_skm1[6] += (lx + l_lev[3 * m + a]) * dl[a] + om * lus * ddl[a];
      lam_skm1[7] += lus * dl[a];
    }
  }
}

// Full forward with every state and DOF iterate stored, then the exact reverse sweep.
struct Trajectory {
  std::vector<Fields<double>> states;  // t = 0..N_t
  std::vector<std::vector<double>> iters;  // per step t = 1..N_t: (K+1)*ns
  std::vector<double> s;               // (N_t+1)*ns
};

int run_forward(Ctx& C, const std::vector<double>& kref, const double* p0, const double* u0, const double* dof0,
                Trajectory* tr, bool keep) {
  const int NT = C.P.n_steps;
  Fields<double> cur;
  load_fields(C, p0, u0, &cur);
  const int ns = C.ns;
  tr->s.assign((size_t)(NT + 1) * ns, 0.0);
  for (int a = 0; a < ns; ++a) tr->s[a] = dof0[a];
  if (keep) {
    tr->states.clear();
    tr->states.push_back(cur);
    tr->iters.clear();
  }
  for (int t = 1; t <= NT; ++t) {
    Fields<double> nxt;
    std::vector<double> it;
    forward_step(C, kref, cur, &tr->s[(size_t)(t - 1) * ns], &nxt, &tr->s[(size_t)t * ns], keep ? &it : nullptr);
    cur.p.swap(nxt.p);
    for (int a = 0; a < 3; ++a) cur.u[a].swap(nxt.u[a]);
    if (keep) {
      tr->states.push_back(cur);
      tr->iters.push_back(it);
    }
  }
  if (!keep) {
    tr->states.clear();
    tr->states.push_back(cur);
  }
  return C.err;
}

// ------------------------------------------------------------------------------------------
// The paper's adjoint, ALKS (Sec. 2.5, Appendix A): a discretised continuous adjoint, kept beside
// the exact discrete adjoint above for comparison. Its variables are the moments of the adjoint
// distribution, p~ = sum_i w_i f~_i, u~ = sum_i w_i c_i f~_i, s~ = sum_i w_i c_i c_i f~_i, and the
// body multipliers x~G, u~G, theta~, omega~, with the paper's sign (the multipliers of the
// residuals of the Lagrangian, minus the derivatives of J).
//
// Adjoint loop of Algorithm 1, per step t = N_t, ..., 1:
//   with the converged DOFs s(t) and the state u(t): N_itr fixed-point iterations of Eq. au (p~ and
//   s~ equal their star moments, Eqs. ap and as, since J has no field term) and of Eqs. axg, aug,
//   atheta, aomega; then the step's term of Eq. design_sensitivity;
//   the star moments at t - 1 from the adjoint equilibrium at t (Eqs. ap_tmp, au_tmp, as_tmp),
//   with the boundary values prescribed.
// Readings where the paper is silent:
//   - the terminal values x~G = -dJ/dxG, M u~G = -dJ/duG, theta~ = -dJ/dtheta, I omega~ = -dJ/domega
//     belong to a step N_t + 1, so that the equations hold at every coupled step 1..N_t; the fluid
//     multipliers at N_t + 1 are zero (J has no field term);
//   - iteration k evaluates Eq. au with the body multipliers of iteration k - 1, and the body
//     equations with the fluid multiplier of iteration k and u~G, omega~ of iteration k - 1 (x~G and
//     theta~ of iteration k enter Eqs. aug and aomega); iteration 0 takes the values of step t + 1;
//   - the derivative in f~eq is the forward's velocity-gradient stencil, with a ghost node that
//     copies the boundary node;
//   - boundary values: a quantity the forward prescribes (inlet and wall velocity, outlet pressure,
//     the pressure of a pressure boundary) has a zero multiplier; one the forward copies from the
//     inward neighbour copies the neighbour's multiplier, except the velocity at the outlet plane,
//     which follows the outflow condition of the convective adjoint, (u . n) u~ + nu du~/dn = 0
//     (a plain copy there made the sweep grow without bound once the outflow was fast); s~ is
//     copied on every boundary;
//   - single rotation axis only (the paper's setting); the derivative of the lever arm and of the
//     solid velocity with respect to theta follow Eqs. rigid_body_position and rigid_body_velocity.
// ------------------------------------------------------------------------------------------

// Adjoint moments p~ [N], u~ [d][N] and s~ [3 a + b][N] (a, b < d; stored in full).
struct AdjMoments {
  std::vector<double> p;
  std::vector<double> u[3];
  std::vector<double> s[9];
  void alloc(const Ctx& C) {
    p.assign(C.N, 0.0);
    for (int a = 0; a < 3; ++a) u[a].assign(a < C.d ? C.N : 0, 0.0);
    for (int k = 0; k < 9; ++k) s[k].assign((k / 3 < C.d && k % 3 < C.d) ? C.N : 0, 0.0);
  }
};

// Neighbour x + c for the derivative in f~eq: wrapped on periodic axes, the boundary node itself
// beyond a non-periodic boundary.
inline size_t copy_nbr(const Ctx& C, const int* x, const int* c) {
  int y[3] = {0, 0, 0};
  for (int a = 0; a < C.d; ++a) {
    int v = x[a] + c[a];
    if (C.P.bc[a] == BC_PERIODIC)
      v = wrap(v, C.n[a]);
    else
      v = std::min(std::max(v, 0), C.n[a] - 1);
    y[a] = v;
  }
  return idx(C, y[0], y[1], y[2]);
}

// Adjoint equilibrium at every node (Sec. 2.5, Appendix A):
//   f~eq_i = p~ + 3 c_ia (u~_a + 3 s~_ab u_b - p~ u_a) - A c_ia d_b (s~_ab + s~_ba),
// with the forward's velocity u at the same node and time. F [Q][N].
void alks_feq_field(const Ctx& C, const AdjMoments& a, const Fields<double>& st, std::vector<double>* F) {
  const int d = C.d, Q = C.L.Q;
  std::vector<double> Dv((size_t)d * C.N, 0.0);  // Dv_a = sum_b d_b (s~_ab + s~_ba)
  int x[3];
  for (size_t n = 0; n < C.N; ++n) {
    coords(C, n, x);
    for (int ia = 0; ia < d; ++ia) {
      double acc = 0.0;
      for (int b = 0; b < d; ++b) {
        double g = 0.0;
        for (int j = 0; j < Q; ++j) {
          if (C.L.c[j][b] == 0) continue;
          const size_t m = copy_nbr(C, x, C.L.c[j]);
          g += (double)C.L.c[j][b] * (a.s[3 * ia + b][m] + a.s[3 * b + ia][m]);
        }
        acc += g / C.L.cn[b];
      }
      Dv[(size_t)ia * C.N + n] = acc;
    }
  }
  F->assign((size_t)Q * C.N, 0.0);
  for (size_t n = 0; n < C.N; ++n)
    for (int i = 0; i < Q; ++i) {
      const int* c = C.L.c[i];
      double v = a.p[n];
      for (int ia = 0; ia < d; ++ia) {
        double su = 0.0;
        for (int b = 0; b < d; ++b) su += a.s[3 * ia + b][n] * st.u[b][n];
        v += 3.0 * c[ia] * (a.u[ia][n] + 3.0 * su - a.p[n] * st.u[ia][n]);
        v -= C.A * c[ia] * Dv[(size_t)ia * C.N + n];
      }
      (*F)[(size_t)i * C.N + n] = v;
    }
}

// The outlet multiplier of u~ (reading above). A test may plant another rule in its place, to check
// that the tests of the paper-form adjoint tell the rules apart: 1 copies u~ (factor 1), 2 zeroes
// it, 3 takes the complement max(u_x, 0) / (nu + max(u_x, 0)), 4 doubles the outflow speed.
int g_alks_outlet_rule = 0;
double alks_outlet_factor(double nu, double ux) {
  const double up = std::max(ux, 0.0);
  switch (g_alks_outlet_rule) {
    case 1: return 1.0;
    case 2: return 0.0;
    case 3: return up / (nu + up);
    case 4: return nu / (nu + 2.0 * up);
    default: return nu / (nu + up);
  }
}

// Boundary values of the adjoint moments (reading above), in the forward's phase order: walls zero
// u~ and copy p~, s~; the inlet copies p~ (inflow/outflow) or zeroes it (pressure), zeroes u~
// (inflow/outflow) or copies it (pressure); the outlet zeroes p~ and scales the inward u~ by
// nu / (nu + u_x) (the state's outflow velocity there); s~ is copied.
void alks_boundaries(const Ctx& C, const Fields<double>& st, AdjMoments* o) {
  const int d = C.d;
  int x[3];
  auto copy_s = [&](size_t n, size_t m) {
    for (int k = 0; k < 9; ++k)
      if (!o->s[k].empty()) o->s[k][n] = o->s[k][m];
  };
  for (int wa = 1; wa < d; ++wa) {
    if (C.P.bc[wa] != BC_WALL) continue;
    for (size_t n = 0; n < C.N; ++n) {
      coords(C, n, x);
      if (!(x[wa] == 0 || x[wa] == C.n[wa] - 1)) continue;
      if (on_boundary(C, 0, x[0])) continue;
      if (wa == 1 && d == 3 && on_boundary(C, 2, x[2])) continue;
      int y[3] = {x[0], x[1], x[2]};
      y[wa] = (x[wa] == 0) ? 1 : C.n[wa] - 2;
      const size_t m = idx(C, y[0], y[1], y[2]);
      o->p[n] = o->p[m];                             // the wall pressure is copied
      for (int a = 0; a < d; ++a) o->u[a][n] = 0.0;  // the wall velocity is prescribed
      copy_s(n, m);
    }
  }
  const int bcx = C.P.bc[0];
  if (bcx == BC_PERIODIC) return;
  for (size_t n = 0; n < C.N; ++n) {
    coords(C, n, x);
    if (!(x[0] == 0 || x[0] == C.n[0] - 1)) continue;
    const bool inlet = (x[0] == 0);
    const size_t m = idx(C, inlet ? 1 : C.n[0] - 2, x[1], x[2]);
    const bool p_fixed = (bcx == BC_PRESSURE) || !inlet;      // outlet, or either pressure plane
    const bool u_fixed = (bcx == BC_INFLOW_OUTFLOW) && inlet;
    // outlet: the outflow condition of the convective adjoint, (u . n) u~ + nu du~/dn = 0, with a
    // one-sided difference: u~(outlet) = nu / (nu + max(u_x, 0)) u~(inward neighbour)
    const double fac = inlet ? 1.0 : alks_outlet_factor(C.P.nu, st.u[0][n]);
    o->p[n] = p_fixed ? 0.0 : o->p[m];
    for (int a = 0; a < d; ++a) o->u[a][n] = u_fixed ? 0.0 : fac * o->u[a][m];
    copy_s(n, m);
  }
}

// Star moments at t - 1 from the adjoint equilibrium at t (Eqs. ap_tmp, au_tmp, as_tmp):
//   p~*(x) = sum_i w_i f~eq_i(x + c_i), u~*_a(x) = sum_i w_i c_ia f~eq_i(x + c_i),
//   s~*_ab(x) = sum_i w_i c_ia c_ib f~eq_i(x + c_i),
// at the interior nodes; the boundary nodes by alks_boundaries. st is the state at t.
void alks_gather(const Ctx& C, const AdjMoments& a, const Fields<double>& st, AdjMoments* o) {
  const int d = C.d, Q = C.L.Q;
  std::vector<double> F;
  alks_feq_field(C, a, st, &F);
  o->alloc(C);
  int x[3];
  for (size_t n = 0; n < C.N; ++n) {
    coords(C, n, x);
    if (!is_interior(C, x)) continue;
    for (int i = 0; i < Q; ++i) {
      const int* c = C.L.c[i];
      const double fw = C.L.w[i] * F[(size_t)i * C.N + shift_nbr(C, x, c, +1)];
      o->p[n] += fw;
      for (int ia = 0; ia < d; ++ia) {
        o->u[ia][n] += c[ia] * fw;
        for (int b = 0; b < d; ++b) o->s[3 * ia + b][n] += (double)(c[ia] * c[b]) * fw;
      }
    }
  }
  alks_boundaries(C, st, o);
}

// (a x b) along the rotation axis ax.
template <class T>
T cross_axis(int ax, const T* a, const T* b) {
  int bb, cc;
  plane_axes(ax, &bb, &cc);
  return a[bb] * b[cc] - a[cc] * b[bb];
}

// The coupling part of the paper's Lagrangian at one step (the forcing term of R_1, and R_3, R_5):
//   Lambda = sum_n 3 kappa_n (u_n - uS_n) . u~_n - u~G . F - omega~ T,
//   F = sum_m kappa_m (u^ref_m - uS,ref_m),  T = sum_m kappa_m (l_m x (u^ref_m - uS,ref_m))_axis,
// with the multipliers u~, u~G, omega~ held fixed and kappa_n, uS_n, u^ref_m, l_m = x^ref_m - x^G
// evaluated at the DOFs s. Eq. au and the coupling terms of Eqs. axg, aug, atheta, aomega and of
// Eq. design_sensitivity are its derivatives (the tests check them by complex step).
template <class T>
T alks_lambda(Ctx& C, const std::vector<T>& kref, const T* s, const std::vector<T>* u, const std::vector<double>* ut,
              const double* ug, double om) {
  const int d = C.d, ax = C.P.rot_axis;
  Geometry<T> geo;
  transform(C, s, &geo);
  std::vector<T> kap(C.N, T(0)), us[3], uref(3 * C.ND, T(0));
  for (int a = 0; a < 3; ++a) us[a].assign(C.N, T(0));
  std::vector<WindowNode> wn;
  std::vector<T> wv, dwv;
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q) {
      const size_t n = wn[q].n;
      kap[n] += wv[q] * kref[m];
      for (int a = 0; a < d; ++a) {
        us[a][n] += wv[q] * geo.usref[3 * m + a];
        uref[3 * m + a] += wv[q] * u[a][n];
      }
    }
  }
  T L = T(0);
  for (size_t n = 0; n < C.N; ++n)
    for (int a = 0; a < d; ++a) L += 3.0 * kap[n] * (u[a][n] - us[a][n]) * ut[a][n];
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    T D[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < d; ++a) D[a] = uref[3 * m + a] - geo.usref[3 * m + a];
    for (int a = 0; a < d; ++a) L -= ug[a] * kref[m] * D[a];
    L -= om * kref[m] * cross_axis(ax, &geo.lev[3 * m], D);
  }
  return L;
}

// The spread quantities of one step at the converged DOFs s(t) and the state u(t).
struct AlksGeom {
  Geometry<double> geo;
  std::vector<std::vector<WindowNode>> win;  // per design point: its support window
  std::vector<std::vector<double>> W, dW;    // W(x_n, x^ref_m) and dW/dx^ref (3 per node)
  std::vector<double> kap;                   // kappa(x_n) = sum_m kappa_m W
  std::vector<double> us[3];                 // uS(x_n) = sum_m W uS,ref_m
  std::vector<double> tq[3];                 // sum_m kappa_m W (e_axis x l_m), the omega~ source of Eq. au
  std::vector<double> uref;                  // u^ref_m = sum_n W u(x_n)  [3 per m]
};

void alks_geometry(Ctx& C, const std::vector<double>& kref, const double* s, const Fields<double>& st, AlksGeom* G) {
  const int d = C.d;
  transform(C, s, &G->geo);
  G->win.assign(C.ND, {});
  G->W.assign(C.ND, {});
  G->dW.assign(C.ND, {});
  G->kap.assign(C.N, 0.0);
  for (int a = 0; a < 3; ++a) {
    G->us[a].assign(C.N, 0.0);
    G->tq[a].assign(C.N, 0.0);
  }
  G->uref.assign(3 * C.ND, 0.0);
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &G->geo.xref[3 * m], &G->win[m], &G->W[m], &G->dW[m]);
    for (size_t q = 0; q < G->win[m].size(); ++q) {
      const size_t n = G->win[m][q].n;
      const double w = G->W[m][q];
      G->kap[n] += w * kref[m];
      for (int a = 0; a < d; ++a) {
        G->us[a][n] += w * G->geo.usref[3 * m + a];
        G->tq[a][n] += kref[m] * w * G->geo.dlev[3 * m + a];
        G->uref[3 * m + a] += w * st.u[a][n];
      }
    }
  }
}

// Eq. au: u~ = (u~* + (u~G kappa + omega~ sum_m kappa_m W (e_axis x l_m)) / 3) / (1 + kappa).
void alks_fluid(const Ctx& C, const AlksGeom& G, const std::vector<double>* ustar, const double* ug, double om,
                std::vector<double>* ut) {
  for (int a = 0; a < C.d; ++a) {
    ut[a].assign(C.N, 0.0);
    for (size_t n = 0; n < C.N; ++n)
      ut[a][n] = (ustar[a][n] + (G.kap[n] * ug[a] + om * G.tq[a][n]) / 3.0) / (1.0 + G.kap[n]);
  }
}

// The coupling terms of the body equations at step t for the fluid multiplier ut and the body
// multipliers ug (u~G) and om (omega~), written as printed (sums over the design points m and the
// nodes n of their supports); omega_t is the state's omega(t):
//   X  : Eq. axg without x~G(t+1) and dJ/dxG,   U  : the bracket of Eq. aug without x~G(t) and dJ/duG,
//   Th : Eq. atheta without theta~(t+1) and dJ/dtheta,   Om : the bracket of Eq. aomega without
//   theta~(t) and dJ/domega.
void alks_terms(const Ctx& C, const std::vector<double>& kref, const AlksGeom& G, const Fields<double>& st,
                const std::vector<double>* ut, const double* ug, double om, double omega_t, double* X, double* U,
                double* Th, double* Om) {
  const int d = C.d, ax = C.P.rot_axis;
  int b, c;
  plane_axes(ax, &b, &c);
  for (int a = 0; a < 3; ++a) X[a] = U[a] = 0.0;
  *Th = *Om = 0.0;
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    const double km = kref[m];
    const double* l = &G.geo.lev[3 * m];     // x^ref - x^G
    const double* pm = &G.geo.dlev[3 * m];   // dx^ref/dtheta = duS,ref/domega
    const double* usr = &G.geo.usref[3 * m];
    double dus[3] = {0.0, 0.0, 0.0};         // duS,ref/dtheta = -omega (l_b, l_c) in the plane
    dus[b] = -omega_t * l[b];
    dus[c] = -omega_t * l[c];
    double D[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a) D[a] = G.uref[3 * m + a] - usr[a];
    double ugdus = 0.0, ugp = 0.0;
    for (int a = 0; a < d; ++a) {
      double ea[3] = {0.0, 0.0, 0.0};
      ea[a] = 1.0;
      U[a] -= ug[a] * km;
      U[a] -= om * cross_axis(ax, l, ea) * km;
      ugdus += ug[a] * dus[a];
      ugp += ug[a] * pm[a];
    }
    *Th -= ugdus * km;
    *Th += om * cross_axis(ax, pm, D) * km;
    *Th -= om * cross_axis(ax, l, dus) * km;
    *Om -= ugp * km;
    *Om -= om * cross_axis(ax, l, pm) * km;
    for (size_t q = 0; q < G.win[m].size(); ++q) {
      const size_t n = G.win[m][q].n;
      const double w = G.W[m][q];
      const double* dw = &G.dW[m][3 * q];
      double un[3] = {0.0, 0.0, 0.0}, v_ut = 0.0, ut_usr = 0.0, ut_dus = 0.0, ut_p = 0.0, ugu = 0.0, dwp = 0.0;
      for (int a = 0; a < d; ++a) {
        un[a] = st.u[a][n];
        v_ut += (un[a] - G.us[a][n]) * ut[a][n];
        ut_usr += ut[a][n] * usr[a];
        ut_dus += ut[a][n] * dus[a];
        ut_p += ut[a][n] * pm[a];
        ugu += ug[a] * un[a];
        dwp += dw[a] * pm[a];
      }
      const double lu = cross_axis(ax, l, un);
      const double kn = G.kap[n];
      for (int al = 0; al < d; ++al) {
        X[al] += -3.0 * km * dw[al] * v_ut + 3.0 * kn * ut_usr * dw[al] + ugu * km * dw[al] + om * lu * km * dw[al];
        U[al] += 3.0 * kn * ut[al][n] * w;
      }
      *Th += -3.0 * km * dwp * v_ut + 3.0 * kn * ut_dus * w + 3.0 * kn * ut_usr * dwp + ugu * km * dwp +
             om * lu * km * dwp;
      *Om += 3.0 * kn * ut_p * w;
    }
  }
}

// The step's term of Eq. design_sensitivity per design point:
//   sum_n 3 W (u - uS) . u~ - u~G . (u^ref - uS,ref) - omega~ (l x (u^ref - uS,ref))_axis.
void alks_sens_step(const Ctx& C, const AlksGeom& G, const Fields<double>& st, const std::vector<double>* ut,
                    const double* ug, double om, double* sens) {
  const int d = C.d, ax = C.P.rot_axis;
  for (size_t m = 0; m < C.ND; ++m) {
    sens[m] = 0.0;
    if (!C.dom[m]) continue;
    double acc = 0.0;
    for (size_t q = 0; q < G.win[m].size(); ++q) {
      const size_t n = G.win[m][q].n;
      for (int a = 0; a < d; ++a) acc += 3.0 * G.W[m][q] * (st.u[a][n] - G.us[a][n]) * ut[a][n];
    }
    double D[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a) D[a] = G.uref[3 * m + a] - G.geo.usref[3 * m + a];
    for (int a = 0; a < d; ++a) acc -= ug[a] * D[a];
    acc -= om * cross_axis(ax, &G.geo.lev[3 * m], D);
    sens[m] = acc;
  }
}

// One step of the paper's adjoint at the converged DOFs s = s(t) and the state st = (p, u)(t):
// N_itr fixed-point iterations of Eq. au and Eqs. axg, aug, atheta, aomega, then the step's term of
// Eq. design_sensitivity added to dk. nxt: the body multipliers at t + 1 (DOF-vector order x~G[3],
// u~G[3], theta~, omega~); out_b: those at t; star: the star moments at t; out: the moments at t.
void alks_body_step(Ctx& C, const std::vector<double>& kref, const double* s, const Fields<double>& st,
                    const AdjMoments& star, const double* nxt, int K, AdjMoments* out, double* out_b,
                    std::vector<double>* dk) {
  AlksGeom G;
  alks_geometry(C, kref, s, st, &G);
  const int d = C.d, mask = C.P.dof_mask;
  double cur[8];
  for (int a = 0; a < 8; ++a) cur[a] = nxt[a];
  *out = star;
  for (int k = 1; k <= K; ++k) {
    alks_fluid(C, G, star.u, &cur[3], cur[7], out->u);
    double X[3], U[3], Th, Om;
    alks_terms(C, kref, G, st, out->u, &cur[3], cur[7], s[7], X, U, &Th, &Om);
    double nw[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int a = 0; a < d; ++a) {
      if (!(mask & (1 << a))) continue;
      nw[a] = nxt[a] + X[a];                               // Eq. axg
      nw[3 + a] = nxt[3 + a] + (nw[a] + U[a]) / C.P.mass;  // Eq. aug
    }
    if (mask & DOF_ROT) {
      nw[6] = nxt[6] + Th;                                 // Eq. atheta
      nw[7] = nxt[7] + (nw[6] + Om) / C.P.inertia;         // Eq. aomega
    }
    for (int a = 0; a < 8; ++a) cur[a] = nw[a];
  }
  for (int a = 0; a < 8; ++a) out_b[a] = cur[a];
  std::vector<double> sens(C.ND, 0.0);
  alks_sens_step(C, G, st, out->u, &cur[3], cur[7], sens.data());
  for (size_t m = 0; m < C.ND; ++m) (*dk)[m] += sens[m];
}

// Terminal body multipliers for J = sum_d w_d s_d(N_t), at the step N_t + 1 (reading above).
void alks_terminal(const Ctx& C, double* b) {
  for (int a = 0; a < 8; ++a) b[a] = 0.0;
  for (int a = 0; a < C.d; ++a) {
    if (!(C.P.dof_mask & (1 << a))) continue;
    b[a] = -C.P.obj_w[a];
    b[3 + a] = -C.P.obj_w[3 + a] / C.P.mass;
  }
  if (C.P.dof_mask & DOF_ROT) {
    b[6] = -C.P.obj_w[6];
    b[7] = -C.P.obj_w[7] / C.P.inertia;
  }
}

void alks_load_moments(const Ctx& C, const double* p, const double* u, const double* s, AdjMoments* a) {
  a->alloc(C);
  for (size_t n = 0; n < C.N; ++n) a->p[n] = p ? p[n] : 0.0;
  for (int i = 0; i < C.d; ++i)
    for (size_t n = 0; n < C.N; ++n) a->u[i][n] = u ? u[(size_t)i * C.N + n] : 0.0;
  for (int i = 0; i < C.d; ++i)
    for (int j = 0; j < C.d; ++j)
      for (size_t n = 0; n < C.N; ++n) a->s[3 * i + j][n] = s ? s[((size_t)i * C.d + j) * C.N + n] : 0.0;
}

void alks_store_moments(const Ctx& C, const AdjMoments& a, double* p, double* u, double* s) {
  if (p)
    for (size_t n = 0; n < C.N; ++n) p[n] = a.p[n];
  if (u)
    for (int i = 0; i < C.d; ++i)
      for (size_t n = 0; n < C.N; ++n) u[(size_t)i * C.N + n] = a.u[i][n];
  if (s)
    for (int i = 0; i < C.d; ++i)
      for (int j = 0; j < C.d; ++j)
        for (size_t n = 0; n < C.N; ++n) s[((size_t)i * C.d + j) * C.N + n] = a.s[3 * i + j][n];
}

void alks_load_velocity(const Ctx& C, const double* u, Fields<double>* st) {
  st->alloc(C);
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < C.N; ++n) st->u[a][n] = u[(size_t)a * C.N + n];
}

}  // namespace

// ============================================================================================
// C API (ctypes). Field arrays: p [N], u [dim][N] planes, x fastest. DOF vectors: ns doubles,
// ns = 8 (xG_x, xG_y, xG_z, uG_x, uG_y, uG_z, theta, omega) for a single rotation axis, or 21
// (xG[3], uG[3], h[3], omega[3], R[9] row-major) for free rotation. Return: 0 ok, else an
// ORC_ERR_* code.
// ============================================================================================
extern "C" {

int oracle_abi_version(void) { return 1; }

// Test hook: the outlet rule of the paper-form adjoint (0: the reading; 1..4: planted mistakes, see
// alks_outlet_factor). Returns the previous rule.
int oracle_set_alks_outlet_rule(int rule) {
  const int prev = g_alks_outlet_rule;
  g_alks_outlet_rule = rule;
  return prev;
}

// Threads the per-node loops use: 1 in the plain build, the OpenMP team size in the timing build.
int oracle_threads(void) {
#if defined(_OPENMP)
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_sizeof_problem(void) { return (int)sizeof(OracleProblem); }

// Length of the DOF vector of the problem (0 if the problem is invalid).
int oracle_dof_count(const OracleProblem* P) {
  Ctx C;
  if (!make_ctx(P, &C)) return 0;
  return C.ns;
}

// Forward march: final fields, DOF history [(n_steps+1)*ns] (optional), J (optional).
int oracle_forward(const OracleProblem* P, const double* gamma, const double* p0, const double* u0,
                   const double* dof0, double* p_out, double* u_out, double* dof_hist, double* J) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  if (P->nu <= 0.0) return ORC_ERR_UNSTABLE;
  std::vector<double> kref = brinkman(C, gamma);
  Trajectory tr;
  run_forward(C, kref, p0, u0, dof0, &tr, false);
  const Fields<double>& f = tr.states.back();
  if (p_out)
    for (size_t n = 0; n < C.N; ++n) p_out[n] = f.p[n];
  if (u_out)
    for (int a = 0; a < C.d; ++a)
      for (size_t n = 0; n < C.N; ++n) u_out[(size_t)a * C.N + n] = f.u[a][n];
  if (dof_hist) std::memcpy(dof_hist, tr.s.data(), tr.s.size() * sizeof(double));
  if (J) *J = objective(C, &tr.s[(size_t)P->n_steps * C.ns]);
  if (C.err) return C.err;
  if (!finite_fields(C, f)) return ORC_ERR_NONFINITE;
  return ORC_OK;
}

// Forward + exact discrete adjoint with seed dJ = 1. Outputs J, dJ/dgamma [ND] and, when the
// pointers are non-null, the adjoint of the initial state: dJ/dp0 [N], dJ/du0 [dim][N],
// dJ/ds0 [ns], and dJ/dkappa^ref [ND].
// The same with a terminal adjoint (the warm start of periodic problems, Sec. 3.4): the reverse sweep
// starts from dJ/dp(N_t) = lam_pT [N], dJ/du(N_t) = lam_uT [dim][N] and dJ/ds(N_t) = w + lam_sT [ns],
// i.e. it differentiates J + lam_pT.p(N_t) + lam_uT.u(N_t) + lam_sT.s(N_t). Any of the three may be NULL.
int oracle_gradient_terminal(const OracleProblem* P, const double* gamma, const double* p0, const double* u0,
                             const double* dof0, const double* lam_pT, const double* lam_uT, const double* lam_sT,
                             double* J, double* dJdgamma, double* lam_p0, double* lam_u0, double* lam_dof0,
                             double* dJdkref);

int oracle_gradient(const OracleProblem* P, const double* gamma, const double* p0, const double* u0,
                    const double* dof0, double* J, double* dJdgamma, double* lam_p0, double* lam_u0,
                    double* lam_dof0, double* dJdkref) {
  return oracle_gradient_terminal(P, gamma, p0, u0, dof0, nullptr, nullptr, nullptr, J, dJdgamma, lam_p0, lam_u0,
                                  lam_dof0, dJdkref);
}

int oracle_gradient_terminal(const OracleProblem* P, const double* gamma, const double* p0, const double* u0,
                             const double* dof0, const double* lam_pT, const double* lam_uT, const double* lam_sT,
                             double* J, double* dJdgamma, double* lam_p0, double* lam_u0, double* lam_dof0,
                             double* dJdkref) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  if (P->nu <= 0.0) return ORC_ERR_UNSTABLE;
  Chain<double> chain;
  std::vector<double> kref = brinkman(C, gamma, &chain);
  Trajectory tr;
  run_forward(C, kref, p0, u0, dof0, &tr, true);
  if (C.err) return C.err;
  const int NT = P->n_steps, K = P->n_itr, d = C.d, ns = C.ns;
  if (J) *J = objective(C, &tr.s[(size_t)NT * ns]);
  // terminal adjoint: the objective depends on the DOFs only
  Fields<double> lam;
  lam.alloc(C);
  double lam_s[21];
  for (int a = 0; a < ns; ++a) lam_s[a] = P->obj_w[a] + (lam_sT ? lam_sT[a] : 0.0);
  if (lam_pT)
    for (size_t n = 0; n < C.N; ++n) lam.p[n] = lam_pT[n];
  if (lam_uT)
    for (int a = 0; a < d; ++a)
      for (size_t n = 0; n < C.N; ++n) lam.u[a][n] = lam_uT[(size_t)a * C.N + n];
  std::vector<double> dk(C.ND, 0.0);
  for (int t = NT; t >= 1; --t) {
    const Fields<double>& prev = tr.states[t - 1];
    const std::vector<double>& it = tr.iters[t - 1];
    Fields<double> star;
    stencil_fwd(C, prev, &star);
    std::vector<IterRecord<double>> recs(K + 1);
    for (int k = 1; k <= K; ++k) {
      double tmp[21];
      coupling_iteration(C, kref, &it[(size_t)(k - 1) * ns], &it[0], star, &recs[k], tmp);
    }
    Fields<double> lam_star;
    lam_star.alloc(C);
    lam_star.p = lam.p;  // p(t) = p*(t)
    double lam_prev[21] = {0};
    double lam_sk[21];
    for (int a = 0; a < ns; ++a) lam_sk[a] = lam_s[a];
    for (int k = K; k >= 1; --k) {
      double lam_skm1[21];
      coupling_iteration_vjp(C, kref, recs[k], &it[(size_t)(k - 1) * ns], &it[0], lam_sk,
                             (k == K) ? &lam : nullptr, &lam_star, lam_prev, lam_skm1, &dk);
      if (k > 1) {
        for (int a = 0; a < ns; ++a) lam_sk[a] = lam_skm1[a];
      } else {
        for (int a = 0; a < ns; ++a) lam_prev[a] += lam_skm1[a];
      }
    }
    Fields<double> lam_prev_fields;
    stencil_vjp(C, prev, lam_star, &lam_prev_fields);
    lam.p.swap(lam_prev_fields.p);
    for (int a = 0; a < 3; ++a) lam.u[a].swap(lam_prev_fields.u[a]);
    for (int a = 0; a < ns; ++a) lam_s[a] = lam_prev[a];
  }
  if (C.err) return C.err;
  std::vector<double> gb3(C.ND, 0.0);
  for (size_t m = 0; m < C.ND; ++m) {
    // dkappa/dgamma-bar at gamma-bar (Eq. brinkman_coefficient), then the chain's transpose
    const double den = (1.0 - chain.g3[m]) + P->q;
    gb3[m] = C.dom[m] ? dk[m] * P->kappa_max * P->q * (1.0 + P->q) / (den * den) : 0.0;
    if (dJdkref) dJdkref[m] = dk[m];
  }
  if (dJdgamma) design_chain_vjp(C, chain, gb3, dJdgamma);
  if (lam_p0)
    for (size_t n = 0; n < C.N; ++n) lam_p0[n] = lam.p[n];
  if (lam_u0)
    for (int a = 0; a < d; ++a)
      for (size_t n = 0; n < C.N; ++n) lam_u0[(size_t)a * C.N + n] = lam.u[a][n];
  if (lam_dof0)
    for (int a = 0; a < ns; ++a) lam_dof0[a] = lam_s[a];
  return ORC_OK;
}

// Complex-step directional derivative of J along (dgamma, dp0, du0, ddof0): dJ = Im J(x + i h v) / h.
int oracle_forward_cs(const OracleProblem* P, const double* gamma, const double* dgamma, const double* p0,
                      const double* dp0, const double* u0, const double* du0, const double* dof0,
                      const double* ddof0, double h, double* J, double* dJ) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  const size_t N = C.N, ND = C.ND;
  const int d = C.d;
  std::vector<cplx> g(ND);
  for (size_t m = 0; m < ND; ++m) g[m] = cplx(gamma[m], dgamma ? h * dgamma[m] : 0.0);
  std::vector<cplx> kref = brinkman(C, g.data());
  std::vector<cplx> pc(N), uc((size_t)d * N);
  for (size_t n = 0; n < N; ++n) pc[n] = cplx(p0[n], dp0 ? h * dp0[n] : 0.0);
  for (size_t n = 0; n < (size_t)d * N; ++n) uc[n] = cplx(u0[n], du0 ? h * du0[n] : 0.0);
  Fields<cplx> cur;
  load_fields(C, pc.data(), uc.data(), &cur);
  cplx s[21];
  for (int a = 0; a < C.ns; ++a) s[a] = cplx(dof0[a], ddof0 ? h * ddof0[a] : 0.0);
  for (int t = 1; t <= P->n_steps; ++t) {
    Fields<cplx> nxt;
    cplx sn[21];
    forward_step<cplx>(C, kref, cur, s, &nxt, sn, nullptr);
    cur.p.swap(nxt.p);
    for (int a = 0; a < 3; ++a) cur.u[a].swap(nxt.u[a]);
    for (int a = 0; a < C.ns; ++a) s[a] = sn[a];
  }
  cplx Jc = objective(C, s);
  if (J) *J = Jc.real();
  if (dJ) *dJ = Jc.imag() / h;
  return C.err;
}

// Complex-step derivative along dgamma of J + lam_pT.p(N_t) + lam_uT.u(N_t) + lam_sT.s(N_t).
int oracle_forward_cs_terminal(const OracleProblem* P, const double* gamma, const double* dgamma, const double* p0,
                               const double* u0, const double* dof0, const double* lam_pT, const double* lam_uT,
                               const double* lam_sT, double h, double* dJ) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  const size_t N = C.N, ND = C.ND;
  const int d = C.d;
  std::vector<cplx> g(ND);
  for (size_t m = 0; m < ND; ++m) g[m] = cplx(gamma[m], h * dgamma[m]);
  std::vector<cplx> kref = brinkman(C, g.data());
  std::vector<cplx> pc(N), uc((size_t)d * N);
  for (size_t n = 0; n < N; ++n) pc[n] = cplx(p0[n], 0.0);
  for (size_t n = 0; n < (size_t)d * N; ++n) uc[n] = cplx(u0[n], 0.0);
  Fields<cplx> cur;
  load_fields(C, pc.data(), uc.data(), &cur);
  cplx s[21];
  for (int a = 0; a < C.ns; ++a) s[a] = cplx(dof0[a], 0.0);
  for (int t = 1; t <= P->n_steps; ++t) {
    Fields<cplx> nxt;
    cplx sn[21];
    forward_step<cplx>(C, kref, cur, s, &nxt, sn, nullptr);
    cur.p.swap(nxt.p);
    for (int a = 0; a < 3; ++a) cur.u[a].swap(nxt.u[a]);
    for (int a = 0; a < C.ns; ++a) s[a] = sn[a];
  }
  cplx Jc = objective(C, s);
  for (int a = 0; a < C.ns; ++a) Jc += lam_sT[a] * s[a];
  for (size_t n = 0; n < N; ++n) Jc += lam_pT[n] * cur.p[n];
  for (int a = 0; a < d; ++a)
    for (size_t n = 0; n < N; ++n) Jc += lam_uT[(size_t)a * N + n] * cur.u[a][n];
  if (dJ) *dJ = Jc.imag() / h;
  return C.err;
}

// ---- sub-steps, for unit tests -------------------------------------------------------------

// S1 + S2 only: p*, u* from (p, u).
int oracle_stencil(const OracleProblem* P, const double* p, const double* u, double* ps, double* us) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Fields<double> s, o;
  load_fields(C, p, u, &s);
  stencil_fwd(C, s, &o);
  for (size_t n = 0; n < C.N; ++n) ps[n] = o.p[n];
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < C.N; ++n) us[(size_t)a * C.N + n] = o.u[a][n];
  return ORC_OK;
}

// Complex-step Jacobian-vector product of S1 + S2 along (dp, du).
int oracle_stencil_jvp(const OracleProblem* P, const double* p, const double* dp, const double* u,
                       const double* du, double h, double* dps, double* dus) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  const size_t N = C.N;
  std::vector<cplx> pc(N), uc((size_t)C.d * N);
  for (size_t n = 0; n < N; ++n) pc[n] = cplx(p[n], h * dp[n]);
  for (size_t n = 0; n < (size_t)C.d * N; ++n) uc[n] = cplx(u[n], h * du[n]);
  Fields<cplx> s, o;
  load_fields(C, pc.data(), uc.data(), &s);
  stencil_fwd(C, s, &o);
  for (size_t n = 0; n < N; ++n) dps[n] = o.p[n].imag() / h;
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < N; ++n) dus[(size_t)a * N + n] = o.u[a][n].imag() / h;
  return ORC_OK;
}

// Vector-Jacobian product of S1 + S2 at (p, u).
int oracle_stencil_vjp(const OracleProblem* P, const double* p, const double* u, const double* lps,
                       const double* lus, double* lp, double* lu) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Fields<double> s, ls, l;
  load_fields(C, p, u, &s);
  load_fields(C, lps, lus, &ls);
  stencil_vjp(C, s, ls, &l);
  for (size_t n = 0; n < C.N; ++n) lp[n] = l.p[n];
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < C.N; ++n) lu[(size_t)a * C.N + n] = l.u[a][n];
  return ORC_OK;
}

// One full forward step from (p, u, s); outputs the next state, the DOF iterates [(n_itr+1)*ns].
int oracle_step(const OracleProblem* P, const double* gamma, const double* p, const double* u, const double* s,
                double* p_out, double* u_out, double* s_out, double* iters) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  std::vector<double> kref = brinkman(C, gamma);
  Fields<double> cur, nxt;
  load_fields(C, p, u, &cur);
  std::vector<double> it;
  forward_step(C, kref, cur, s, &nxt, s_out, &it);
  for (size_t n = 0; n < C.N; ++n) p_out[n] = nxt.p[n];
  for (int a = 0; a < C.d; ++a)
    for (size_t n = 0; n < C.N; ++n) u_out[(size_t)a * C.N + n] = nxt.u[a][n];
  if (iters) std::memcpy(iters, it.data(), it.size() * sizeof(double));
  return C.err;
}

// Spread of kappa^ref and u^S,ref at the DOF vector s (Eqs. kappa_mapping, us_mapping), and the
// number of design points with a non-zero weight at each analysis node.
int oracle_spread(const OracleProblem* P, const double* gamma, const double* s, double* kappa, double* us,
                  int* count) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  std::vector<double> kref = brinkman(C, gamma);
  Geometry<double> geo;
  transform(C, s, &geo);
  std::vector<WindowNode> wn;
  std::vector<double> wv, dwv;
  for (size_t n = 0; n < C.N; ++n) {
    if (kappa) kappa[n] = 0;
    if (count) count[n] = 0;
    if (us)
      for (int a = 0; a < C.d; ++a) us[(size_t)a * C.N + n] = 0;
  }
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q) {
      if (wv[q] == 0.0) continue;
      if (kappa) kappa[wn[q].n] += wv[q] * kref[m];
      if (count) count[wn[q].n] += 1;
      if (us)
        for (int a = 0; a < C.d; ++a) us[(size_t)a * C.N + wn[q].n] += wv[q] * geo.usref[3 * m + a];
    }
  }
  return C.err;
}

// Index sets of the spread at the DOF vector s (Eqs. kappa_mapping, weight_function): for every
// analysis node n, the design points m of the design domain whose support window holds n, i.e.
// |x_n - x^ref_m| < support on every axis, summarised as stats [N][5] = (count, least index or -1,
// largest index, sum of the indices, sum of their squares). The windows are those of the scatter
// per design point above.
int oracle_support_sets(const OracleProblem* P, const double* s, long long* stats) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Geometry<double> geo;
  transform(C, s, &geo);
  for (size_t n = 0; n < C.N; ++n) {
    stats[5 * n + 0] = 0;
    stats[5 * n + 1] = -1;
    stats[5 * n + 2] = -1;
    stats[5 * n + 3] = 0;
    stats[5 * n + 4] = 0;
  }
  std::vector<WindowNode> wn;
  std::vector<double> wv, dwv;
  for (size_t m = 0; m < C.ND; ++m) {
    if (!C.dom[m]) continue;
    window(C, &geo.xref[3 * m], &wn, &wv, &dwv);
    const long long mm = (long long)m;
    for (size_t q = 0; q < wn.size(); ++q) {
      long long* st = &stats[5 * wn[q].n];
      if (st[0] == 0 || mm < st[1]) st[1] = mm;
      if (mm > st[2]) st[2] = mm;
      st[0] += 1;
      st[3] += mm;
      st[4] += mm * mm;
    }
  }
  return C.err;
}

// Interpolation of an analysis-grid velocity to the design points (Eq. u_mapping): uref [ND][3].
int oracle_interp(const OracleProblem* P, const double* s, const double* u, double* uref) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Geometry<double> geo;
  transform(C, s, &geo);
  std::vector<WindowNode> wn;
  std::vector<double> wv, dwv;
  for (size_t m = 0; m < C.ND; ++m) {
    for (int a = 0; a < 3; ++a) uref[3 * m + a] = 0;
    if (!C.dom[m]) continue;
    window(C, &geo.xref[3 * m], &wn, &wv, &dwv);
    for (size_t q = 0; q < wn.size(); ++q)
      for (int a = 0; a < C.d; ++a) uref[3 * m + a] += wv[q] * u[(size_t)a * C.N + wn[q].n];
  }
  return C.err;
}

// gamma-bar [ND] of the design chain (cyclic expansion, filter, projection) for gamma [ND].
int oracle_design_chain(const OracleProblem* P, const double* gamma, double* gbar) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Chain<double> ch;
  design_chain(C, gamma, &ch);
  for (size_t m = 0; m < C.ND; ++m) gbar[m] = ch.g3[m];
  return ORC_OK;
}

// Transpose of the design chain at gamma: out = (d gamma-bar / d gamma)^T v, v [ND].
int oracle_design_chain_vjp(const OracleProblem* P, const double* gamma, const double* v, double* out) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  Chain<double> ch;
  design_chain(C, gamma, &ch);
  std::vector<double> gb3(v, v + C.ND);
  design_chain_vjp(C, ch, gb3, out);
  return ORC_OK;
}

// Complex-step directional derivative of gamma-bar along dgamma: out = Im gbar(gamma + i h v) / h.
int oracle_design_chain_jvp(const OracleProblem* P, const double* gamma, const double* v, double h, double* out) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  std::vector<cplx> g(C.ND);
  for (size_t m = 0; m < C.ND; ++m) g[m] = cplx(gamma[m], h * v[m]);
  Chain<cplx> ch;
  design_chain(C, g.data(), &ch);
  for (size_t m = 0; m < C.ND; ++m) out[m] = ch.g3[m].imag() / h;
  return ORC_OK;
}

// Volume constraint (Eq. constraint) G = sum_dom gamma-bar / (V_min N_dom) - 1 and dG/dgamma.
int oracle_constraint(const OracleProblem* P, const double* gamma, double* G, double* dGdgamma) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  if (!(P->v_min > 0.0)) return ORC_ERR_ARG;
  Chain<double> ch;
  design_chain(C, gamma, &ch);
  size_t ndom = 0;
  double sum = 0.0;
  for (size_t m = 0; m < C.ND; ++m)
    if (C.dom[m]) {
      ++ndom;
      sum += ch.g3[m];
    }
  const double scale = 1.0 / (P->v_min * (double)ndom);
  if (G) *G = sum * scale - 1.0;
  if (dGdgamma) {
    std::vector<double> gb3(C.ND, 0.0);
    for (size_t m = 0; m < C.ND; ++m) gb3[m] = C.dom[m] ? scale : 0.0;
    design_chain_vjp(C, ch, gb3, dGdgamma);
  }
  return ORC_OK;
}

// One weight-kernel value w(r) and derivative, for the kernel tests.
double oracle_weight(int kind, double r, double* dw) {
  if (dw) *dw = dwk<double>(kind, r);
  return wk<double>(kind, r);
}


// ------------------------------------------------------------------------------------------
// The paper's adjoint (ALKS, Sec. 2.5): entry points. Adjoint moments: p~ [N], u~ [dim][N],
// s~ [dim][dim][N]. Body multipliers: 8 doubles in the DOF-vector order (x~G[3], u~G[3], theta~,
// omega~). Single rotation axis only (ORC_ERR_ARG with free rotation).
// ------------------------------------------------------------------------------------------

// Forward + the paper's adjoint with dJ = 1: J, dJ/dgamma [ND] (Eq. design_sensitivity through the
// design chain), dJ/dkappa^ref [ND], the moments at t = 0 and the body multipliers at t = 1.
int oracle_gradient_alks(const OracleProblem* P, const double* gamma, const double* p0, const double* u0,
                         const double* dof0, double* J, double* dJdgamma, double* dJdkref, double* adj_p0,
                         double* adj_u0, double* adj_s0, double* body1) {
  Ctx C;
  if (!make_ctx(P, &C) || C.free_rot) return ORC_ERR_ARG;
  if (P->nu <= 0.0) return ORC_ERR_UNSTABLE;
  Chain<double> chain;
  std::vector<double> kref = brinkman(C, gamma, &chain);
  Trajectory tr;
  run_forward(C, kref, p0, u0, dof0, &tr, true);
  if (C.err) return C.err;
  const int NT = P->n_steps, ns = C.ns;
  if (J) *J = objective(C, &tr.s[(size_t)NT * ns]);
  double nxt[8];
  alks_terminal(C, nxt);
  AdjMoments star;
  star.alloc(C);
  std::vector<double> dk(C.ND, 0.0);
  for (int t = NT; t >= 1; --t) {
    AdjMoments at, prev;
    double b[8];
    alks_body_step(C, kref, &tr.s[(size_t)t * ns], tr.states[t], star, nxt, P->n_itr, &at, b, &dk);
    alks_gather(C, at, tr.states[t], &prev);
    star = prev;
    for (int a = 0; a < 8; ++a) nxt[a] = b[a];
  }
  if (C.err) return C.err;
  alks_store_moments(C, star, adj_p0, adj_u0, adj_s0);
  if (body1)
    for (int a = 0; a < 8; ++a) body1[a] = nxt[a];
  std::vector<double> gb3(C.ND, 0.0);
  for (size_t m = 0; m < C.ND; ++m) {
    const double den = (1.0 - chain.g3[m]) + P->q;
    gb3[m] = C.dom[m] ? dk[m] * P->kappa_max * P->q * (1.0 + P->q) / (den * den) : 0.0;
    if (dJdkref) dJdkref[m] = dk[m];
  }
  if (dJdgamma) design_chain_vjp(C, chain, gb3, dJdgamma);
  return ORC_OK;
}

// The adjoint equilibrium f~eq [Q][N] of the moments (ap, au, as_) at the velocity u [dim][N].
int oracle_alks_feq(const OracleProblem* P, const double* ap, const double* au, const double* as_, const double* u,
                    double* F) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  AdjMoments a;
  alks_load_moments(C, ap, au, as_, &a);
  Fields<double> st;
  alks_load_velocity(C, u, &st);
  std::vector<double> f;
  alks_feq_field(C, a, st, &f);
  std::memcpy(F, f.data(), f.size() * sizeof(double));
  return ORC_OK;
}

// Complex-step derivative along df of sum_{n,j} phi_j(n) f^eq_j(n), where f^eq is the forward's
// equilibrium of the moments p = sum_i f_i / 3, u = sum_i c_i f_i of the distributions f [Q][N].
int oracle_feq_adjoint_cs(const OracleProblem* P, const double* f, const double* df, const double* phi, double h,
                          double* out) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  const int Q = C.L.Q, d = C.d;
  Fields<cplx> s;
  s.alloc(C);
  for (size_t n = 0; n < C.N; ++n)
    for (int i = 0; i < Q; ++i) {
      const cplx fi(f[(size_t)i * C.N + n], h * df[(size_t)i * C.N + n]);
      s.p[n] += fi / 3.0;
      for (int a = 0; a < d; ++a) s.u[a][n] += (double)C.L.c[i][a] * fi;
    }
  std::vector<cplx> G;
  velocity_gradient(C, s, &G);
  cplx acc(0.0, 0.0);
  for (size_t n = 0; n < C.N; ++n)
    for (int i = 0; i < Q; ++i) acc += phi[(size_t)i * C.N + n] * feq(C, i, s, G, n);
  *out = acc.imag() / h;
  return ORC_OK;
}

// Star moments at t - 1 (with the boundary values) from the moments at t and the velocity u(t).
int oracle_alks_gather(const OracleProblem* P, const double* ap, const double* au, const double* as_,
                       const double* u, double* op, double* ou, double* os) {
  Ctx C;
  if (!make_ctx(P, &C)) return ORC_ERR_ARG;
  AdjMoments a, o;
  alks_load_moments(C, ap, au, as_, &a);
  Fields<double> st;
  alks_load_velocity(C, u, &st);
  alks_gather(C, a, st, &o);
  alks_store_moments(C, o, op, ou, os);
  return ORC_OK;
}

// One evaluation of the step's equations at the DOFs s [8] and the velocity u [dim][N], for given
// star moment ustar [dim][N] and body multipliers ug [3], om: the fluid multiplier of Eq. au into
// ut [dim][N], the coupling terms (X[3], U[3], Th, Om; see alks_terms) with that ut into terms [8],
// and the step's term of Eq. design_sensitivity into sens [ND].
int oracle_alks_parts(const OracleProblem* P, const double* gamma, const double* s, const double* u,
                      const double* ustar, const double* ug, double om, double* ut, double* terms, double* sens) {
  Ctx C;
  if (!make_ctx(P, &C) || C.free_rot) return ORC_ERR_ARG;
  std::vector<double> kref = brinkman(C, gamma);
  Fields<double> st;
  alks_load_velocity(C, u, &st);
  AlksGeom G;
  alks_geometry(C, kref, s, st, &G);
  std::vector<double> us[3], uo[3];
  for (int a = 0; a < C.d; ++a) us[a].assign(ustar + (size_t)a * C.N, ustar + (size_t)(a + 1) * C.N);
  alks_fluid(C, G, us, ug, om, uo);
  for (int a = 0; a < C.d; ++a) std::memcpy(ut + (size_t)a * C.N, uo[a].data(), C.N * sizeof(double));
  alks_terms(C, kref, G, st, uo, ug, om, s[7], &terms[0], &terms[3], &terms[6], &terms[7]);
  alks_sens_step(C, G, st, uo, ug, om, sens);
  return C.err;
}

// Complex-step derivative of the step Lagrangian (alks_lambda) along dkref [ND], ds [8] and du
// [dim][N] (each may be NULL), at kappa^ref(gamma), the DOFs s and the velocity u, with the
// multipliers ut [dim][N], ug [3], om held fixed.
int oracle_alks_lambda_cs(const OracleProblem* P, const double* gamma, const double* dkref, const double* s,
                          const double* ds, const double* u, const double* du, const double* ut, const double* ug,
                          double om, double h, double* out) {
  Ctx C;
  if (!make_ctx(P, &C) || C.free_rot) return ORC_ERR_ARG;
  std::vector<double> kr = brinkman(C, gamma);
  std::vector<cplx> kref(C.ND);
  for (size_t m = 0; m < C.ND; ++m) kref[m] = cplx(kr[m], dkref ? h * dkref[m] : 0.0);
  cplx sc[8];
  for (int a = 0; a < 8; ++a) sc[a] = cplx(s[a], ds ? h * ds[a] : 0.0);
  std::vector<cplx> uc[3];
  std::vector<double> utv[3];
  for (int a = 0; a < C.d; ++a) {
    uc[a].resize(C.N);
    utv[a].assign(ut + (size_t)a * C.N, ut + (size_t)(a + 1) * C.N);
    for (size_t n = 0; n < C.N; ++n) uc[a][n] = cplx(u[(size_t)a * C.N + n], du ? h * du[(size_t)a * C.N + n] : 0.0);
  }
  const cplx L = alks_lambda(C, kref, sc, uc, utv, ug, om);
  *out = L.imag() / h;
  return C.err;
}

// One step of the paper's adjoint with K fixed-point iterations (alks_body_step): from the star
// moment ustar [dim][N] and the body multipliers nxt [8] at t + 1 to u~ [dim][N] and out_b [8] at t,
// and the step's design sensitivity sens [ND].
int oracle_alks_body_step(const OracleProblem* P, const double* gamma, const double* s, const double* u,
                          const double* ustar, const double* nxt, int K, double* ut, double* out_b, double* sens) {
  Ctx C;
  if (!make_ctx(P, &C) || C.free_rot || K < 1) return ORC_ERR_ARG;
  std::vector<double> kref = brinkman(C, gamma);
  Fields<double> st;
  alks_load_velocity(C, u, &st);
  AdjMoments star, out;
  alks_load_moments(C, nullptr, ustar, nullptr, &star);
  std::vector<double> dk(C.ND, 0.0);
  alks_body_step(C, kref, s, st, star, nxt, K, &out, out_b, &dk);
  for (int a = 0; a < C.d; ++a) std::memcpy(ut + (size_t)a * C.N, out.u[a].data(), C.N * sizeof(double));
  if (sens) std::memcpy(sens, dk.data(), C.ND * sizeof(double));
  return C.err;
}

}  // extern "C"

extern "C" {
// The velocity set and weights used for dimension dim: c [Q][3], w [Q]; returns Q.
int oracle_lattice(int dim, int* c, double* w) {
  Lattice L = make_lattice(dim);
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
  }
  return L.Q;
}
}  // extern "C"
