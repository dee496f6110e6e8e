// Reduced-precision checkpoints of the FP32 state (the memory strategy of the checkpointed
// gradient; the paper does not prescribe one).
//
// Per checkpoint and per plane (p, u_x, u_y[, u_z]) the plane's range [lo, hi] is found first; each
// value is then stored as q = (v - m) / s in BF16 or FP16, rounded to nearest even, with
// m = (hi + lo) / 2 and s = (hi - lo) / 2 (so q lies in [-1, 1]); the restore computes
// v = s q + m. A constant plane (s = 0) is restored exactly. The forward keeps marching from its
// exact FP32 state; only the recompute segments of the adjoint start from a restored state, so
// the objective is unaffected and the gradient carries the quantisation error.
//
// The range is reduced with order-preserving integer keys and atomicMin / atomicMax, one update
// per CTA and plane: the result (a min and a max) does not depend on the order of the updates.
//
// Traffic per cell and checkpoint: read the plane values (4 B each) twice, write 2 B each; the
// restore reads 2 B and writes 4 B per value.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lks_kernels.h"

namespace lks {

namespace {

constexpr int kQB = 256;  // threads per CTA

// Order-preserving map of floats to unsigned keys (and back).
__device__ __forceinline__ unsigned fkey(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float funkey(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ unsigned short to_q(float q, int fmt) {
  return fmt == CKQ_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(q)) : __half_as_ushort(__float2half_rn(q));
}
__device__ __forceinline__ float from_q(unsigned short b, int fmt) {
  return fmt == CKQ_BF16 ? __bfloat162float(__ushort_as_bfloat16(b)) : __half2float(__ushort_as_half(b));
}

// checkpoint index of the step the graph node works on
__device__ __forceinline__ int ckpt_index(const Ctrl* ctrl, int di, int every) { return (ctrl->t0 + di) / every; }

__device__ __forceinline__ void ckq_init_body(unsigned* keys, int nplanes, int c) {
  const int a = threadIdx.x;
  if (a < nplanes) {
    keys[(c * nplanes + a) * 2 + 0] = 0xffffffffu;  // min
    keys[(c * nplanes + a) * 2 + 1] = 0u;           // max
  }
}

__global__ void k_ckq_init(unsigned* keys, int nplanes, int every, const Ctrl* ctrl, int di) {
  ckq_init_body(keys, nplanes, ckpt_index(ctrl, di, every));
}

// Range of plane a of the state v (N values per plane) into its key pair kp.
__device__ __forceinline__ void ckq_range_body(const Geo& g, const float* __restrict__ v, unsigned* kp) {
  __shared__ float smin[kQB / 32], smax[kQB / 32];
  float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
  for (long long i = blockIdx.x * (long long)kQB + threadIdx.x; i < g.N; i += (long long)gridDim.x * kQB) {
    const float x = v[i];
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    smin[w] = lo;
    smax[w] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kQB / 32; ++q) {
      lo = fminf(lo, smin[q]);
      hi = fmaxf(hi, smax[q]);
    }
    atomicMin(&kp[0], fkey(lo));
    atomicMax(&kp[1], fkey(hi));
  }
}

__global__ void __launch_bounds__(kQB) k_ckq_range(Geo g, Slots<float> S, unsigned* keys, int every,
                                                   const Ctrl* ctrl, int di) {
  const int tn = ctrl->t0 + di, c = tn / every, a = blockIdx.y, nplanes = g.dim + 1;
  ckq_range_body(g, slot_ptr(S, tn, ctrl->base) + (long long)a * g.N, keys + (c * nplanes + a) * 2);
}

// m and s of a plane from its key pair; inv = 1/s (0 for a constant plane)
__device__ __forceinline__ void plane_scale(const unsigned* kp, float* m, float* s, float* inv) {
  const float lo = funkey(kp[0]), hi = funkey(kp[1]);
  *m = 0.5f * (hi + lo);
  *s = 0.5f * (hi - lo);
  *inv = *s > 0.0f ? 1.0f / *s : 0.0f;
}

// Plane values v -> q[] in the reduced format with the plane's scale from its key pair kp.
__device__ __forceinline__ void ckq_store_body(const Geo& g, const float* __restrict__ v, const unsigned* kp,
                                               unsigned short* __restrict__ out, int fmt) {
  float m, s, inv;
  plane_scale(kp, &m, &s, &inv);
  for (long long i = blockIdx.x * (long long)kQB + threadIdx.x; i < g.N; i += (long long)gridDim.x * kQB)
    out[i] = to_q((v[i] - m) * inv, fmt);
}

__global__ void __launch_bounds__(kQB) k_ckq_store(Geo g, Slots<float> S, const unsigned* keys, unsigned short* q,
                                                   int fmt, int every, const Ctrl* ctrl, int di) {
  const int tn = ctrl->t0 + di, c = tn / every, a = blockIdx.y, nplanes = g.dim + 1;
  ckq_store_body(g, slot_ptr(S, tn, ctrl->base) + (long long)a * g.N, keys + (c * nplanes + a) * 2,
                 q + ((long long)c * nplanes + a) * g.N, fmt);
}

// The same three steps for the state at src into checkpoint c (the binomial snapshots, whose slots
// and steps the host schedule names).
__global__ void k_ckq_init_at(unsigned* keys, int nplanes, int c) { ckq_init_body(keys, nplanes, c); }
__global__ void __launch_bounds__(kQB) k_ckq_range_at(Geo g, const float* src, unsigned* keys, int c) {
  const int a = blockIdx.y, nplanes = g.dim + 1;
  ckq_range_body(g, src + (long long)a * g.N, keys + (c * nplanes + a) * 2);
}
__global__ void __launch_bounds__(kQB) k_ckq_store_at(Geo g, const float* src, const unsigned* keys,
                                                      unsigned short* q, int fmt, int c) {
  const int a = blockIdx.y, nplanes = g.dim + 1;
  ckq_store_body(g, src + (long long)a * g.N, keys + (c * nplanes + a) * 2, q + ((long long)c * nplanes + a) * g.N,
                 fmt);
}

__global__ void __launch_bounds__(kQB) k_ckq_restore(Geo g, float* dst, const unsigned* keys,
                                                     const unsigned short* q, int fmt, int c) {
  const int a = blockIdx.y, nplanes = g.dim + 1;
  float m, s, inv;
  plane_scale(keys + (c * nplanes + a) * 2, &m, &s, &inv);
  const unsigned short* __restrict__ in = q + ((long long)c * nplanes + a) * g.N;
  float* __restrict__ out = dst + (long long)a * g.N;
  for (long long i = blockIdx.x * (long long)kQB + threadIdx.x; i < g.N; i += (long long)gridDim.x * kQB)
    out[i] = fmaf(s, from_q(in[i], fmt), m);
}

template <typename T>
__global__ void k_state_from_double(Geo g, T* dst, const double* __restrict__ p0, const double* __restrict__ u0) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    dst[n] = (T)p0[n];
    for (int a = 0; a < g.dim; ++a) dst[(a + 1) * N + n] = (T)u0[a * N + n];
  }
}

template <typename T>
__global__ void k_state_to_double(Geo g, const T* __restrict__ src, double* p0, double* u0) {
  const long long N = g.N;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
    p0[n] = (double)src[n];
    for (int a = 0; a < g.dim; ++a) u0[a * N + n] = (double)src[(a + 1) * N + n];
  }
}

inline unsigned q_blocks(const Geo& g) {
  const long long nb = (g.N + kQB - 1) / kQB;
  return (unsigned)(nb < 1024 ? nb : 1024);
}

}  // namespace

void launch_ckpt_pack_q(const Geo& g, const Slots<float>& S, unsigned short* q, unsigned* keys, int fmt, int every,
                        const Ctrl* ctrl, int di, cudaStream_t st) {
  const int nplanes = g.dim + 1;
  launch(k_ckq_init, 1, 32, 0, st, keys, nplanes, every, ctrl, di);
  const dim3 grid(q_blocks(g), nplanes);
  launch(k_ckq_range, grid, kQB, 0, st, g, S, keys, every, ctrl, di);
  launch(k_ckq_store, grid, kQB, 0, st, g, S, (const unsigned*)keys, q, fmt, every, ctrl, di);
}

void launch_ckpt_pack_q_at(const Geo& g, const float* src, unsigned short* q, unsigned* keys, int fmt, int c,
                           cudaStream_t st) {
  const int nplanes = g.dim + 1;
  launch(k_ckq_init_at, 1, 32, 0, st, keys, nplanes, c);
  const dim3 grid(q_blocks(g), nplanes);
  launch(k_ckq_range_at, grid, kQB, 0, st, g, src, keys, c);
  launch(k_ckq_store_at, grid, kQB, 0, st, g, src, (const unsigned*)keys, q, fmt, c);
}

void launch_ckpt_restore_q(const Geo& g, float* dst, const unsigned short* q, const unsigned* keys, int fmt, int c,
                           cudaStream_t st) {
  const dim3 grid(q_blocks(g), g.dim + 1);
  launch(k_ckq_restore, grid, kQB, 0, st, g, dst, keys, q, fmt, c);
}

template <typename T>
void launch_state_from_double(const Geo& g, T* dst, const double* p0, const double* u0, cudaStream_t st) {
  const long long nb = (g.N + 255) / 256;
  launch(k_state_from_double<T>, (unsigned)(nb < 4096 ? nb : 4096), 256, 0, st, g, dst, p0, u0);
}

template <typename T>
void launch_state_to_double(const Geo& g, const T* src, double* p0, double* u0, cudaStream_t st) {
  const long long nb = (g.N + 255) / 256;
  launch(k_state_to_double<T>, (unsigned)(nb < 4096 ? nb : 4096), 256, 0, st, g, src, p0, u0);
}

template void launch_state_to_double<float>(const Geo&, const float*, double*, double*, cudaStream_t);
template void launch_state_to_double<double>(const Geo&, const double*, double*, double*, cudaStream_t);
template void launch_state_from_double<float>(const Geo&, float*, const double*, const double*, cudaStream_t);
template void launch_state_from_double<double>(const Geo&, double*, const double*, const double*, cudaStream_t);

}  // namespace lks
