// Per-axis basis tables of one block (span index and the p+1 nonzero N, N'), exposed so the
// span search and Cox-de Boor recurrence used by every kernel can be checked on their own.
#include "common.cuh"
#include "kernels.h"

namespace mfa {

__global__ void basis_tables_kernel(const mfa_block_desc* d, const float* knots, int64_t knots_len,
                                    int32_t* span, float* basis, uint32_t* status) {
  const int a = blockIdx.x;  // axis
  const int i = threadIdx.x; // sample
  const int p = d->degree[a], C = d->ncp[a], n = d->nsamp[a];
  const int64_t off = d->knot_off[a];
  if (p < 1 || p > MFA_MAX_DEGREE || C < p + 1 || C > MFA_MAX_NCP || n < 2 || n > MFA_MAX_NSAMP ||
      off < 0 || off + C + p + 1 > knots_len) {
    if (i == 0) flag(status, MFA_DEV_BAD_DESC);
    return;
  }
  if (i >= n) return;
  const float* t = knots + off;
  const float u = sample_param(i, n);
  const int s = find_span(t, p, C, u);
  float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
  basis_funs<MFA_MAX_DEGREE>(t, p, s, u, N, dN);
  span[a * MFA_MAX_NSAMP + i] = s;
  for (int r = 0; r <= MFA_MAX_DEGREE; ++r) {
    basis[((a * MFA_MAX_NSAMP + i) * 2 + 0) * 4 + r] = N[r];
    basis[((a * MFA_MAX_NSAMP + i) * 2 + 1) * 4 + r] = dN[r];
  }
}

int basis_tables(mfa_ctx* ctx, const mfa_block_desc* d_desc, const float* d_knots, int64_t knots_len,
                 int32_t* d_span, float* d_basis, cudaStream_t stream) {
  basis_tables_kernel<<<3, MFA_MAX_NSAMP, 0, stream>>>(d_desc, d_knots, knots_len, d_span, d_basis, ctx->d_status);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
