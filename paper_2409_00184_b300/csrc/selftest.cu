// Failure-detection self-test: the bounded mbarrier wait of the TMA and tensor-core kernels, run on
// a barrier that nothing arrives on, must give up and report MFA_DEV_TIMEOUT in the status word.
#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace mfa {
namespace {

__global__ void wait_timeout_kernel(uint32_t* status, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);  // expects one arrival, which never comes
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0, polls)) flag(status, MFA_DEV_TIMEOUT);
}

}  // namespace
}  // namespace mfa

extern "C" int mfa_selftest_wait_timeout(mfa_ctx* ctx, int32_t polls, void* stream) {
  if (!ctx || polls < 1 || (uint32_t)polls > mfa::kWaitPolls) return MFA_ERR_INVALID_ARG;
  mfa::wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ctx->d_status, (uint32_t)polls);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}
