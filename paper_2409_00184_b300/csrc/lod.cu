// Multi-resolution partition of a sampled field (Sec. 4.2, Algorithm 1): the micro-blocks of one level
// of detail, each n^3 samples taken every `stride` samples from a block of n*stride per axis.
// One CTA per block, threads over its n^3 samples (x fastest, so reads of stride 1 coalesce).
#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

struct LodParams {
  const float* field;
  int64_t dims[3];
  int B[3];
  int n, stride;
  const int32_t* ids;
  int nblocks;
  float* out;
  int64_t slot_stride;
  uint32_t* status;
};

__global__ void __launch_bounds__(256) lod_gather_kernel(LodParams prm) {
  const int e = blockIdx.x;
  const int64_t nb = (int64_t)prm.B[0] * prm.B[1] * prm.B[2];
  const int id = prm.ids ? prm.ids[e] : e;
  if (id < 0 || id >= nb) {
    if (threadIdx.x == 0) flag(prm.status, MFA_DEV_BAD_LIST);
    return;
  }
  const int bx = id % prm.B[0], by = (id / prm.B[0]) % prm.B[1], bz = id / (prm.B[0] * prm.B[1]);
  const int n = prm.n, s = prm.stride;
  const int64_t n3 = (int64_t)n * n * n;
  float* out = prm.out + (int64_t)e * prm.slot_stride;
  for (int64_t v = threadIdx.x; v < n3; v += blockDim.x) {
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((int64_t)n * n));
    const int64_t x = (int64_t)(bx * n + i) * s, y = (int64_t)(by * n + j) * s, z = (int64_t)(bz * n + k) * s;
    out[v] = __ldg(prm.field + (z * prm.dims[1] + y) * prm.dims[0] + x);
  }
}

}  // namespace
}  // namespace mfa

extern "C" int mfa_lod_gather(mfa_ctx* ctx, const float* d_field, const int32_t dims[3], int32_t n, int32_t stride,
                              const int32_t* d_ids, int32_t nblocks, float* d_out, int64_t slot_stride,
                              void* stream) {
  using namespace mfa;
  if (!ctx || !dims || n < 2 || n > MFA_MAX_NSAMP || stride < 1 || nblocks < 0) return MFA_ERR_INVALID_ARG;
  LodParams prm;
  int64_t nb = 1;
  for (int a = 0; a < 3; ++a) {
    const int64_t span = (int64_t)n * stride;
    if (dims[a] < 1 || dims[a] % span != 0) return MFA_ERR_INVALID_ARG;
    prm.dims[a] = dims[a];
    prm.B[a] = (int)(dims[a] / span);
    nb *= prm.B[a];
  }
  if (nb > 0x7fffffff || (!d_ids && nblocks > nb)) return MFA_ERR_INVALID_ARG;
  if (slot_stride < (int64_t)n * n * n) return MFA_ERR_INVALID_ARG;
  if (nblocks == 0) return MFA_OK;
  if (!d_field || !d_out) return MFA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_field) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4 ||
      (d_ids && reinterpret_cast<uintptr_t>(d_ids) % 4))
    return MFA_ERR_INVALID_ARG;
  prm.field = d_field;
  prm.n = n;
  prm.stride = stride;
  prm.ids = d_ids;
  prm.nblocks = nblocks;
  prm.out = d_out;
  prm.slot_stride = slot_stride;
  prm.status = ctx->d_status;
  lod_gather_kernel<<<nblocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}
