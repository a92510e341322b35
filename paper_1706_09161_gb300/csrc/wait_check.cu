// Check of the bounded device-side wait.
//
// Every pipelined kernel of this library waits on mbarrier phases (TMA completions,
// MMA commits, the fused step's grid barrier) through mbar_wait, which gives up after a
// %globaltimer limit, sets bit 2 of the handle's status word and lets the kernel run to
// its end, so that a lost completion surfaces as LBM_ERR_TIMEOUT on the host instead of
// a hung GPU.  lbm_wait_check runs that wait on a barrier whose phase is (or, on
// request, is not) completed and reports what the host reads back.
#include "lbm_internal.h"
#include "tc_dev.cuh"

namespace lbm {
namespace {

__global__ void wait_check_kernel(int complete, long long limit_ns, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (complete) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  mbar_wait(&bar, 0, status, limit_ns);  // bit 2 of *status when it gives up
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

}  // namespace
}  // namespace lbm

int lbm_wait_check(int complete, int limit_us, void* stream) {
  if (limit_us < 1 || limit_us > 1000000) return LBM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return LBM_ENOMEM;
  int host = 0;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    lbm::wait_check_kernel<<<1, 32, 0, s>>>(complete ? 1 : 0, 1000LL * limit_us, status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(status);
  if (e != cudaSuccess) return LBM_ECUDA;
  return (host & 2) ? LBM_ERR_TIMEOUT : LBM_OK;
}
