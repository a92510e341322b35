// FP64 mass reduction and precision conversions between the FP64 host-facing
// staging buffer and the working precision.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kReduceThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_w[kReduceThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  v = (threadIdx.x < kReduceThreads / 32) ? s_w[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

// Stage 1: each block sums a grid-stride slice of x into partials[blockIdx.x].
template <typename real>
__global__ void __launch_bounds__(kReduceThreads)
sum_partials_kernel(const real* __restrict__ x, long long n, double* __restrict__ partials) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kReduceThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kReduceThreads)
    acc += static_cast<double>(x[i]);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Stage 2: one block sums the partials.
__global__ void __launch_bounds__(kReduceThreads)
sum_final_kernel(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += kReduceThreads) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// The latest step's mass: the collide-stream kernel's warp partials added in a fixed
// order; with limit > 0, a mass outside [-limit, limit] (or not finite) sets bit 1 of flag.
// FP32 forms store each warp's partial as a float pair (hi, lo) in the 8-byte slot (pair = 1):
// its value is hi + lo, formed here in FP64 (exact for such a pair).
__global__ void __launch_bounds__(kReduceThreads)
step_mass_kernel(const double* __restrict__ partials, int nparts, int pair, double* __restrict__ out, double limit,
                 int* __restrict__ flag) {
  double acc = 0.0;
  if (pair) {
    const float2* p2 = reinterpret_cast<const float2*>(partials);
    for (int i = threadIdx.x; i < nparts; i += kReduceThreads) {
      const float2 v = p2[i];
      acc += static_cast<double>(v.x) + static_cast<double>(v.y);
    }
  } else {
    for (int i = threadIdx.x; i < nparts; i += kReduceThreads) acc += partials[i];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) {
    *out = acc;
    if (limit > 0.0 && !(fabs(acc) <= limit)) atomicOr(flag, 1);
  }
}

template <typename real>
__global__ void convert_in_kernel(const double* __restrict__ src, real* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = static_cast<real>(src[i]);
}

template <typename real>
__global__ void convert_out_kernel(const real* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = static_cast<double>(src[i]);
}

// dst[i] = sum_{s < k} src[s * stride + i] (FP32, added in order of s), as FP64
__global__ void sum_partials_out_kernel(const float* __restrict__ src, int k, long long stride,
                                        double* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float acc = src[i];
    for (int s = 1; s < k; ++s) acc += src[s * stride + i];
    dst[i] = static_cast<double>(acc);
  }
}

__global__ void sum_partials_kernel(const float* __restrict__ src, int k, long long stride, float* __restrict__ dst,
                                    long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float acc = src[i];
    for (int s = 1; s < k; ++s) acc += src[s * stride + i];
    dst[i] = acc;
  }
}

int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  const long long cap = 16LL * device_sms();
  if (b > cap) b = cap;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

int reduce_blocks_for(long long n) {
  long long b = (n + 4LL * kReduceThreads - 1) / (4LL * kReduceThreads);
  if (b > 1024) b = 1024;
  return static_cast<int>(b < 1 ? 1 : b);
}

cudaError_t launch_mass(const lbm_s* h, const void* C, cudaStream_t s) {
  const long long n = h->sp.nodes;
  const int nb = h->reduce_blocks;
  if (h->elem == 8)
    sum_partials_kernel<double><<<nb, kReduceThreads, 0, s>>>((const double*)C, n, h->dev.partials);
  else
    sum_partials_kernel<float><<<nb, kReduceThreads, 0, s>>>((const float*)C, n, h->dev.partials);
  sum_final_kernel<<<1, kReduceThreads, 0, s>>>(h->dev.partials, nb, h->dev.scalar);
  return cudaGetLastError();
}

cudaError_t launch_step_mass(const lbm_s* h, double limit, cudaStream_t s) {
  step_mass_kernel<<<1, kReduceThreads, 0, s>>>(h->cs_part, h->cs_nparts * kMassSlots, h->elem == 4 ? 1 : 0,
                                                 h->dev.scalar, limit, h->dev.flag);
  return cudaGetLastError();
}

cudaError_t launch_convert_in(const void* src, void* dst, int elem, long long n, cudaStream_t s) {
  if (elem == 8) convert_in_kernel<double><<<blocks_for(n), 256, 0, s>>>((const double*)src, (double*)dst, n);
  else convert_in_kernel<float><<<blocks_for(n), 256, 0, s>>>((const double*)src, (float*)dst, n);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials_out(const float* src, int k, long long stride, double* dst, long long n,
                                    cudaStream_t s) {
  sum_partials_out_kernel<<<blocks_for(n), 256, 0, s>>>(src, k, stride, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const float* src, int k, long long stride, float* dst, long long n, cudaStream_t s) {
  sum_partials_kernel<<<blocks_for(n), 256, 0, s>>>(src, k, stride, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_out(const void* src, int elem, double* dst, long long n, cudaStream_t s) {
  if (elem == 8) convert_out_kernel<double><<<blocks_for(n), 256, 0, s>>>((const double*)src, dst, n);
  else convert_out_kernel<float><<<blocks_for(n), 256, 0, s>>>((const float*)src, dst, n);
  return cudaGetLastError();
}

}  // namespace lbm
