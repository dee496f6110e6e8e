// Helpers shared by the body kernels (lks_body.cu) and the paper-form adjoint (lks_alks.cu):
// the box-cell thread layout, the cell gather of the design-point sums, the box grid and the
// dispatch on the dimension and rotation axis.
#pragma once

#include "lks_kernels.h"

namespace lks {

namespace {

// Box-cell kernels: LN consecutive threads share one cell's gather (candidate rows split among
// them), CX x CY cells per CTA. Design-point kernel: LN threads per point (rows, or planes in 3D,
// of its support window), kDesignPointsPerCta points per CTA. The split multiplies the resident
// warps of these latency-bound kernels by LN.
constexpr int LN = kLanesPerCell;
// Box-cell CTA shape: 16 x 16 cells in 2D (fewer CTAs: each runs the fused finish, its FP64 chain
// and block reductions once; measured 763 against 772 ms on the 512x256 gradient), 16 x 8 in 3D
// (where the larger CTAs measured 7 % slower).
template <int D>
struct BoxCta {
  static constexpr int X = kBoxCtaCellsX, Y = (D == 2) ? kBoxCtaCellsY2D : kBoxCtaCellsY;
  static constexpr int threads = X * Y * LN;
  static constexpr int min_blocks = threads >= 1024 ? 1 : 2;  // resident CTAs the register budget allows
};
constexpr int kDesignBlock = kDesignPointsPerCta * LN;
constexpr int kFinishThreads = 256;
// Coupling: up to this many CTAs every CTA finishes the previous iteration itself (fused; saves a
// launch); above it a one-CTA kernel does it once (the fused form loads every CTA's partials in
// every CTA).
constexpr int kFusedFinishMaxParts = 640;

struct CellSlot {
  int j0, j1, j2, lane;
  bool active;  // inside the box
};

template <int D>
__device__ __forceinline__ CellSlot cell_slot(const Geo& g) {
  constexpr int CX = BoxCta<D>::X, CY = BoxCta<D>::Y;
  CellSlot c;
  const int q = threadIdx.x / LN;
  c.lane = threadIdx.x % LN;
  c.j0 = blockIdx.x * CX + q % CX;
  c.j1 = blockIdx.y * CY + q / CX;
  c.j2 = blockIdx.z;
  c.active = c.j0 < g.B[0] && c.j1 < g.B[1];
  return c;
}

// The same for box tile `tile` of the box grid (x fastest) in the persistent kernels, whose CTAs
// stride over the tiles.
template <int D>
__device__ __forceinline__ CellSlot cell_slot_tile(const Geo& g, int tile, int gx, int gy) {
  constexpr int CX = BoxCta<D>::X, CY = BoxCta<D>::Y;
  CellSlot c;
  const int q = threadIdx.x / LN;
  c.lane = threadIdx.x % LN;
  const int bx = tile % gx, by = (tile / gx) % gy, bz = tile / (gx * gy);
  c.j0 = bx * CX + q % CX;
  c.j1 = by * CY + q / CX;
  c.j2 = bz;
  c.active = c.j0 < g.B[0] && c.j1 < g.B[1];
  return c;
}

__device__ __forceinline__ int block_linear() { return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z); }

// R and omega of a free-rotation iterate in the field type.
template <typename T>
struct FreeView;
template <>
struct FreeView<float> {
  float R[9], om[3];
  __device__ __forceinline__ explicit FreeView(const Dof& d) {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = d.Rf[i];
#pragma unroll
    for (int a = 0; a < 3; ++a) om[a] = d.omf[a];
  }
};
template <>
struct FreeView<double> {
  double R[9], om[3];
  __device__ __forceinline__ explicit FreeView(const Dof& d) {
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = d.s[S_R + i];
#pragma unroll
    for (int a = 0; a < 3; ++a) om[a] = d.s[S_OM + a];
  }
};

// Gather of the cell's design-point sums under the iterate's rotation, and from them the
// rotational part of the solid velocity (omega R' sum W r, or omega x R sum W r) and the lever
// sum L_n = R sum W kappa r.
template <typename T, int D, int AX>
__device__ __forceinline__ void gather_cell(const Geo& g, const T* __restrict__ kref, const Dof& sk,
                                            const DofView<T>& V, const T (&d)[3], int lane, bool active, Acc<T>& A,
                                            T (&rotv)[3], T (&L)[3]) {
  if constexpr (AX == AX_FREE) {
    const FreeView<T> FV(sk);
    gather_free_lanes<T, LN>(g, kref, d, FV.R, lane, active, A);
    T Rwr[3];
    matvec3(FV.R, A.wr, Rwr);
    cross3(FV.om, Rwr, rotv);
    matvec3(FV.R, A.kr, L);
  } else {
    gather_lanes<T, D, AX, LN>(g, kref, d, V.cs, V.sn, lane, active, A);
    T dwr[3];
    drot<AX>(V.cs, V.sn, A.wr, dwr);
#pragma unroll
    for (int a = 0; a < 3; ++a) rotv[a] = V.om * dwr[a];
    rot<AX>(V.cs, V.sn, A.kr, L);
  }
}

// Design-point kernels: one CTA per kDesignPointsPerCta points up to kMaxDesignCtas CTAs (two waves
// at their occupancy), grid-strided beyond, so the one-CTA finish sums at most that many partials.
constexpr int kMaxDesignCtas = 912;
inline int design_ctas(const Geo& g) {
  const int n = (g.ND + kDesignPointsPerCta - 1) / kDesignPointsPerCta;
  return n < kMaxDesignCtas ? n : kMaxDesignCtas;
}

__host__ __device__ inline int box_threads(const Geo& g) { return kBoxCtaCellsX * (g.dim == 2 ? kBoxCtaCellsY2D : kBoxCtaCellsY) * LN; }
__host__ __device__ inline dim3 box_grid(const Geo& g) {
  const int cx = kBoxCtaCellsX, cy = g.dim == 2 ? kBoxCtaCellsY2D : kBoxCtaCellsY;
  return dim3((g.B[0] + cx - 1) / cx, (g.B[1] + cy - 1) / cy, g.dim == 3 ? g.B[2] : 1);
}

}  // namespace

// Dispatch on the dimension and the (runtime) rotation axis to the compile-time instantiation.
#define LKS_BOX_DISPATCH(KERNEL, GRID, BLOCK, ...)          \
  do {                                                      \
    if (g.dim == 2)                                         \
      launch(KERNEL<T, 2, 2>, GRID, BLOCK, 0, st, __VA_ARGS__); \
    else if (g.ax == 0)                                     \
      launch(KERNEL<T, 3, 0>, GRID, BLOCK, 0, st, __VA_ARGS__); \
    else if (g.ax == 1)                                     \
      launch(KERNEL<T, 3, 1>, GRID, BLOCK, 0, st, __VA_ARGS__); \
    else if (g.ax == 2)                                     \
      launch(KERNEL<T, 3, 2>, GRID, BLOCK, 0, st, __VA_ARGS__); \
    else                                                    \
      launch(KERNEL<T, 3, AX_FREE>, GRID, BLOCK, 0, st, __VA_ARGS__); \
  } while (0)

}  // namespace lks
