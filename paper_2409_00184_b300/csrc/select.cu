// In-level adaptive encoding (Sec. 4.2.2, Eq. 4): per block, the smallest NCP among the candidates
// whose error is below the bound. One thread per block reads its column of the candidate-major error
// table (coalesced across threads for every candidate).
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

constexpr int kMaxCand = 64;

struct SelectParams {
  const double* errors;
  int ncand;
  int64_t nblocks;
  double bound;
  int32_t* out;
  int32_t ncp[kMaxCand];
};

__global__ void __launch_bounds__(256) select_ncp_kernel(SelectParams prm) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= prm.nblocks) return;
  int best = -1;
  for (int c = 0; c < prm.ncand; ++c) {
    const double e = prm.errors[(int64_t)c * prm.nblocks + b];
    if (e < prm.bound && (best < 0 || prm.ncp[c] < best)) best = prm.ncp[c];  // NaN compares false
  }
  prm.out[b] = best;
}

}  // namespace
}  // namespace mfa

extern "C" int mfa_select_ncp(mfa_ctx* ctx, const double* d_errors, int32_t ncand, const int32_t* h_ncp,
                              int64_t nblocks, double bound, int32_t* d_ncp_out, void* stream) {
  using namespace mfa;
  if (!ctx || !h_ncp) return MFA_ERR_INVALID_ARG;
  if (ncand < 1 || ncand > kMaxCand || nblocks < 0 || std::isnan(bound)) return MFA_ERR_INVALID_ARG;
  SelectParams prm;
  for (int c = 0; c < ncand; ++c) {
    if (h_ncp[c] < 1) return MFA_ERR_INVALID_ARG;
    prm.ncp[c] = h_ncp[c];
  }
  if (nblocks == 0) return MFA_OK;  // the device pointers may be null then
  if (!d_errors || !d_ncp_out) return MFA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_errors) % 8 != 0 || reinterpret_cast<uintptr_t>(d_ncp_out) % 4 != 0)
    return MFA_ERR_INVALID_ARG;
  prm.errors = d_errors;
  prm.ncand = ncand;
  prm.nblocks = nblocks;
  prm.bound = bound;
  prm.out = d_ncp_out;
  const int64_t grid = (nblocks + 255) / 256;
  if (grid > 0x7fffffff) return MFA_ERR_INVALID_ARG;
  select_ncp_kernel<<<(unsigned)grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}
