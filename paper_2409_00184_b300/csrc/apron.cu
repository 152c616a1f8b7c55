// Apron of the decoded cache (MFA_DECODE_APRON): every brick of n^3 voxels is stored in rows of
// apron_pitch(n) = n + 1 rounded up to even voxels, planes of n + 1 rows and n + 1 planes, and the planes
// x = n, y = n, z = n hold the neighbouring bricks' voxels at local 0 on those axes. The ray caster's cells
// then never reach outside their brick: the eight corners of the cell at local (lx, ly, lz),
// lx, ly, lz < n, sit at local lx .. lx+1 (and so on) of the same slot. A column x = n + 1 (even n) is
// padding and becomes zero. With an even n and an even slot stride every row of float4 starts on a
// 32-byte sector, so the decode's rows and the apron column written here never share a sector.
//
// One CTA per brick of the brick table. The eight slots of the brick and its +x, +y, +z neighbours
// (-1 when absent or outside the volume) are looked up once into shared memory. The apron voxels are
// numbered in three faces:
//   face x = n: (n+1)^2 voxels (y, z in 0..n) from brick (+1, [y = n], [z = n]) at local
//               (0, y mod n, z mod n), each with its padding voxel x = n + 1 when the pitch has one;
//   face y = n: (n+1) n voxels (x < n, z in 0..n) from brick (0, +1, [z = n]) at local (x, 0, z mod n);
//   face z = n: n^2 voxels (x < n, y < n) from brick (0, 0, +1) at local (x, y, 0).
// Each thread takes kBatch voxels of that numbering at a time and issues all their loads before any of
// their stores (loads and stores address the same cache, so the compiler would not move a load above an
// earlier store): the batch's loads are in flight together instead of one latency per voxel. An absent
// source gives zeros, as the ray caster reads an absent brick's voxels.
#include "common.cuh"
#include "kernels.h"

namespace mfa {

namespace {

constexpr int kApronThreads = 256;
constexpr int kBatch = 13;  // 256 x 13 >= 3169: a 32^3 brick's apron in one round of loads

__global__ void __launch_bounds__(kApronThreads, 3) apron_fill_kernel(ApronParams prm) {
  __shared__ int s_nb[8];  // slot of the brick at offset (e & 1, (e >> 1) & 1, e >> 2)
  const int brick = blockIdx.x;
  const int B0 = prm.B[0], B1 = prm.B[1], B2 = prm.B[2];
  const int bx = brick % B0, by = (brick / B0) % B1, bz = brick / (B0 * B1);
  if (threadIdx.x < 8) {
    const int e = threadIdx.x;
    const int sx = bx + (e & 1), sy = by + ((e >> 1) & 1), sz = bz + (e >> 2);
    int s = -1;
    if (sx < B0 && sy < B1 && sz < B2) s = prm.table[(sz * B1 + sy) * B0 + sx];
    s_nb[e] = (s >= 0 && s < prm.nslots) ? s : -1;
  }
  __syncthreads();
  const int dst_slot = s_nb[0];
  if (dst_slot < 0) return;
  const int n = prm.n, p = n + 1, px = apron_pitch(n);  // rows per plane, row pitch
  const int fx = p * p, fy = p * n, total = fx + fy + n * n;
  const bool pad = px > p;
  float4* dst = prm.cache + (int64_t)dst_slot * prm.slot_stride;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * kApronThreads) {
    float4 v[kBatch];
    int d[kBatch];
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      const int e = e0 + q * kApronThreads;
      int nb = -1, so = 0, di = -1;
      if (e < fx) {  // face x = n
        const int y = e % p, z = e / p;
        nb = 1 + 2 * (y == n) + 4 * (z == n);
        so = ((z == n ? 0 : z) * p + (y == n ? 0 : y)) * px;
        di = (z * p + y) * px + n;
      } else if (e < fx + fy) {  // face y = n
        const int f = e - fx, x = f % n, z = f / n;
        nb = 2 + 4 * (z == n);
        so = (z == n ? 0 : z) * p * px + x;
        di = (z * p + n) * px + x;
      } else if (e < total) {  // face z = n
        const int f = e - fx - fy, x = f % n, y = f / n;
        nb = 4;
        so = y * px + x;
        di = (n * p + y) * px + x;
      }
      const int s = nb >= 0 ? s_nb[nb] : -1;
      v[q] = s >= 0 ? __ldg(prm.cache + (int64_t)s * prm.slot_stride + so) : zero;
      d[q] = di;
    }
#pragma unroll
    for (int q = 0; q < kBatch; ++q) {
      if (d[q] < 0) continue;
      dst[d[q]] = v[q];
      if (pad && e0 + q * kApronThreads < fx) dst[d[q] + 1] = zero;
    }
  }
}

}  // namespace

int apron_fill(mfa_ctx* ctx, const ApronParams& prm, cudaStream_t stream) {
  const int64_t bricks = (int64_t)prm.B[0] * prm.B[1] * prm.B[2];
  if (bricks < 1 || bricks > (int64_t)1 << 31) return MFA_ERR_INVALID_ARG;
  apron_fill_kernel<<<(unsigned)bricks, kApronThreads, 0, stream>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
