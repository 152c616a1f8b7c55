// Multi-resolution partition of a sampled field (Sec. 4.2, Algorithm 1): the micro-blocks of one level
// of detail, each n^3 samples taken every `stride` samples from a block of n*stride per axis, or, with
// shared boundaries (Sec. 4.2: neighbouring blocks share one sample on the boundary), from a block of
// (n-1)*stride intervals whose last samples are the next block's first.
// One CTA per block, threads over its n^3 samples (x fastest, so reads of stride 1 coalesce).
// Also the per-frame selection of a level of detail for every block by its distance from the point of
// view (Sec. 5.1.3).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

struct LodParams {
  const float* field;
  int64_t dims[3];
  int B[3];
  int n, stride;
  int pitch;  // first sample of block b along an axis: b * pitch * stride (n, or n - 1 when shared)
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
    const int P = prm.pitch;
    const int64_t x = (int64_t)(bx * P + i) * s, y = (int64_t)(by * P + j) * s, z = (int64_t)(bz * P + k) * s;
    out[v] = __ldg(prm.field + (z * prm.dims[1] + y) * prm.dims[0] + x);
  }
}

struct SelectParams {
  float eye[3];
  float r2[MFA_MAX_LEVELS];  // squared range of level l >= 1 (FP32 product of the range with itself)
  int B0, n, levels;
  int off[MFA_MAX_LEVELS];   // first global id of every level
  int32_t* table;
};

// Whether the block of first node g0 and extent E (finest nodes) lies at distance >= r from the eye, in
// FP32 one rounded operation at a time: c = (2 g0 + E) / (N - 1) - 1, d^2 = ((dx^2 + dy^2) + dz^2).
__device__ __forceinline__ bool far_enough(const SelectParams& p, const int g0[3], int E, float r2) {
  const float nm1 = (float)(p.B0 * (p.n - 1));
  float d2 = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float c = __fsub_rn(__fdiv_rn((float)(2 * g0[a] + E), nm1), 1.0f);
    const float d = __fsub_rn(c, p.eye[a]);
    d2 = a == 0 ? __fmul_rn(d, d) : __fadd_rn(d2, __fmul_rn(d, d));
  }
  return d2 >= r2;
}

// One thread per finest block: the coarsest ancestor level l >= 1 that is far enough for its range (the
// first block a top-down walk of the levels would stop at), else level 0; writes that block's global id.
__global__ void lod_select_kernel(SelectParams p) {
  const int64_t nb = (int64_t)p.B0 * p.B0 * p.B0;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nb; f += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(f % p.B0), y = (int)((f / p.B0) % p.B0), z = (int)(f / ((int64_t)p.B0 * p.B0));
    int chosen = 0;
    for (int l = p.levels - 1; l >= 1; --l) {
      const int E = (p.n - 1) << l;
      const int g0[3] = {(x >> l) * E, (y >> l) * E, (z >> l) * E};
      if (far_enough(p, g0, E, p.r2[l])) {
        chosen = l;
        break;
      }
    }
    const int Bl = p.B0 >> chosen;
    p.table[f] = p.off[chosen] + ((z >> chosen) * Bl + (y >> chosen)) * Bl + (x >> chosen);
  }
}

}  // namespace
}  // namespace mfa

extern "C" int mfa_lod_gather(mfa_ctx* ctx, const float* d_field, const int32_t dims[3], int32_t n, int32_t stride,
                              const int32_t* d_ids, int32_t nblocks, float* d_out, int64_t slot_stride,
                              void* stream) {
  return mfa_lod_gather_ex(ctx, d_field, dims, n, stride, d_ids, nblocks, d_out, slot_stride, 0u, stream);
}

extern "C" int mfa_lod_gather_ex(mfa_ctx* ctx, const float* d_field, const int32_t dims[3], int32_t n,
                                 int32_t stride, const int32_t* d_ids, int32_t nblocks, float* d_out,
                                 int64_t slot_stride, uint32_t flags, void* stream) {
  using namespace mfa;
  if (!ctx || !dims || n < 2 || n > MFA_MAX_NSAMP || stride < 1 || nblocks < 0) return MFA_ERR_INVALID_ARG;
  if (flags & ~MFA_LOD_SHARED_BOUNDARY) return MFA_ERR_INVALID_ARG;
  const bool shared = (flags & MFA_LOD_SHARED_BOUNDARY) != 0;
  LodParams prm;
  prm.pitch = shared ? n - 1 : n;
  int64_t nb = 1;
  for (int a = 0; a < 3; ++a) {
    const int64_t span = (int64_t)prm.pitch * stride;
    const int64_t extent = shared ? (int64_t)dims[a] - 1 : (int64_t)dims[a];
    if (dims[a] < 1 || extent < span || extent % span != 0) return MFA_ERR_INVALID_ARG;
    prm.dims[a] = dims[a];
    prm.B[a] = (int)(extent / span);
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

extern "C" int mfa_lod_select(mfa_ctx* ctx, const float eye[3], int32_t fine_blocks, int32_t n, int32_t levels,
                              const float* ranges, int32_t* d_table, void* stream) {
  using namespace mfa;
  if (!ctx || !eye || !d_table || n < 2 || n > MFA_MAX_NSAMP || levels < 1 || levels > MFA_MAX_LEVELS ||
      fine_blocks < 1 || (levels > 1 && !ranges))
    return MFA_ERR_INVALID_ARG;
  if (fine_blocks % (1 << (levels - 1)) != 0 || (int64_t)fine_blocks * (n - 1) >= (1 << 23) ||
      reinterpret_cast<uintptr_t>(d_table) % 4)
    return MFA_ERR_INVALID_ARG;
  SelectParams p;
  int64_t acc = 0;
  for (int l = 0; l < levels; ++l) {
    p.off[l] = (int)acc;
    const int64_t Bl = fine_blocks >> l;
    acc += Bl * Bl * Bl;
    p.r2[l] = 0.f;
    if (l >= 1) {
      const float r = ranges[l - 1];
      if (!(r >= 0.f) || !std::isfinite(r)) return MFA_ERR_INVALID_ARG;
      p.r2[l] = r * r;  // FP32 product, as the selection rule states
    }
  }
  if (acc > 0x7fffffff) return MFA_ERR_CAPACITY;
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(eye[a])) return MFA_ERR_INVALID_ARG;
    p.eye[a] = eye[a];
  }
  p.B0 = fine_blocks;
  p.n = n;
  p.levels = levels;
  p.table = d_table;
  const int64_t nb = (int64_t)fine_blocks * fine_blocks * fine_blocks;
  const int grid = (int)std::min<int64_t>((nb + 255) / 256, (int64_t)ctx->num_sms * 8);
  lod_select_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(p);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}
