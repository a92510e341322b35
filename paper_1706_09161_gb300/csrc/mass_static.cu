// FP64 sum of a device array with its scratch in static device memory.
//
// Same reduction as lbm_mass (block partial sums in FP64, then one final pass),
// for callers that cannot allocate device memory themselves: code that runs as a
// plug-in of a host framework which owns all GPU memory and hands out only
// pointers, and code that must not call cudaMalloc because an allocation can
// synchronise the device.  The partial sums live in g_partials, a file-scope
// __device__ array that every GPU which loads this library keeps until exit.
#include <mutex>

#include "lbm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr long long kPerBlock = (long long)kThreads * kPerThread;  // elements summed per partial
constexpr long long kMaxPartials = 65536;                          // 512 KiB of FP64
constexpr long long kMaxElements = kMaxPartials * kPerBlock;       // 67,108,864
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[kMaxPartials];

std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {nullptr};

// Device address of g_partials on the current device, looked up once per device.
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return LBM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) return LBM_ECUDA;
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return LBM_OK;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s_w[kThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  v = (threadIdx.x < kThreads / 32) ? s_w[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

// Block b sums elements [b*kPerBlock, (b+1)*kPerBlock) into partials[b]; every
// partial that the final pass reads is written here, so nothing needs clearing.
template <typename T>
__global__ void __launch_bounds__(kThreads)
static_partials_kernel(const T* __restrict__ x, long long n, double* __restrict__ partials) {
  const long long base = blockIdx.x * kPerBlock;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const long long i = base + (long long)k * kThreads + threadIdx.x;
    if (i < n) acc += static_cast<double>(x[i]);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads)
static_final_kernel(const double* __restrict__ partials, long long nparts, double* __restrict__ out) {
  double acc = 0.0;
  for (long long i = threadIdx.x; i < nparts; i += kThreads) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

}  // namespace

extern "C" int lbm_mass_static(const void* x_dev, int elem_bytes, long long n, double* sum_dev, void* stream) {
  if (!x_dev || !sum_dev || (elem_bytes != 4 && elem_bytes != 8) || n < 0) return LBM_EINVAL;
  if (n > kMaxElements) return LBM_ETOOBIG;
  double* partials = nullptr;
  int rc = scratch_address(&partials);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long nparts = (n + kPerBlock - 1) / kPerBlock;
  if (nparts > 0) {
    if (elem_bytes == 8)
      static_partials_kernel<double><<<(unsigned)nparts, kThreads, 0, s>>>(static_cast<const double*>(x_dev), n, partials);
    else
      static_partials_kernel<float><<<(unsigned)nparts, kThreads, 0, s>>>(static_cast<const float*>(x_dev), n, partials);
  }
  static_final_kernel<<<1, kThreads, 0, s>>>(partials, nparts, sum_dev);
  return (cudaGetLastError() == cudaSuccess) ? LBM_OK : LBM_ECUDA;
}
