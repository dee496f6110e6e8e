// Helpers shared by the 2D and 3D LKS predictor kernels (boundary classification and the ghost
// rule of the velocity-gradient stencil).
#pragma once

#include "lks_device.cuh"

namespace lks {

// 2A in the field type (the FP32 copy for FP32 fields, exact for FP64 fields).
template <typename T>
__device__ __forceinline__ T two_a(const Geo& g);
template <>
__device__ __forceinline__ float two_a<float>(const Geo& g) { return g.A2; }
template <>
__device__ __forceinline__ double two_a<double>(const Geo& g) { return 2.0 * g.A; }

// Interior along one axis: every node of a periodic axis, else 1 .. n-2.
__device__ __forceinline__ bool interior_axis(int bc, int n, int v) {
  return bc == BC_PERIODIC || (v >= 1 && v <= n - 2);
}

// Gradient ghost rule along one axis: periodic axes wrap; one ghost layer beyond a non-periodic
// boundary copies the boundary node (open planes) or reflects it with a sign flip of u (walls,
// u(-1) = -u(1)). Returns false beyond the ghost layer.
__device__ __forceinline__ bool ghost_axis(int bc, int n, int* v, int* sgn) {
  if (bc == BC_PERIODIC) {
    *v = wrapi(*v, n);
    return true;
  }
  if (*v >= 0 && *v < n) return true;
  if (bc == BC_WALL) {
    if (*v == -1) {
      *v = 1;
      *sgn = -*sgn;
      return true;
    }
    if (*v == n) {
      *v = n - 2;
      *sgn = -*sgn;
      return true;
    }
    return false;
  }
  if (*v == -1) {
    *v = 0;
    return true;
  }
  if (*v == n) {
    *v = n - 1;
    return true;
  }
  return false;
}

}  // namespace lks
