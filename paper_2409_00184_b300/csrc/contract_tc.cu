// Transposed three-axis contraction on the tensor cores (tcgen05), for the least-squares fit (the model()
// of Algorithm 1: P = D x_1 Px x_2 Py x_3 Pz with the per-axis pseudo-inverses Pa = (Na^T Na)^-1 Na^T) and
// the adjoint of the decode (dP = R x_1 Nx^T x_2 Ny^T x_3 Nz^T), in BF16 or split-BF16 (A*B ~ Ahi*Bhi +
// Ahi*Blo + Alo*Bhi) with FP32 accumulation in tensor memory.
//
// Shapes: 32 samples and at most 16 control points per axis. Per block, with X the 32^3 sample grid
// ([k][j][i], FP32 in global memory) and A_a the n x C matrix of axis a (basis or pseudo-inverse, transposed):
//   stage x  T1[(k,j)][a] = sum_i X[(k,j)][i] Ax[i][a]   M = 1024 rows (8 tiles), K = i, N = 16 columns
//   stage y  T2[(k,a)][b] = sum_j T1[(k,j)][a] Ay[j][b]   M = 512 rows (4 tiles),  K = j
//   stage z  Y[(b,a)][c]  = sum_k T2[(k,a)][b] Az[k][c]   M = 256 rows (2 tiles),  K = k
// K = 32 is two MMA steps of 16. The sample grid arrives in two batches of 16 planes: each thread loads its
// share of a batch into registers (coalesced 16-byte loads), splits it into BF16 hi (and lo) parts and
// writes the stage-x A operand; the next batch (and, after the last one, the next block's first batch) is
// loaded while the MMAs of the current one run. Stage outputs are read from tensor memory, split again and
// written transposed as the next stage's A operand; the B operands (the three A_a^T, zero beyond C) are
// built per block. One thread issues the MMAs; completion is an mbarrier armed by tcgen05.commit and waited
// on with a bounded poll that reports MFA_DEV_TIMEOUT.
#include <algorithm>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mfa {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcN = 32;                  // samples per axis (the contraction's K)
constexpr int kTcC = 16;                  // padded control points per axis (the MMA N)
constexpr uint32_t kLBO32 = 128, kSBO32 = 512;  // K-major core-matrix strides for K = 32
constexpr int kRowB = 64;                 // bytes of one operand row (32 x 16-bit)
constexpr int kBatchRows = 512;           // 16 planes x 32 rows
constexpr int kF4PerThread = kBatchRows * 8 / kTcThreads;  // float4 loads per thread and batch (16)

// Shared-memory layout (bytes): every operand is stored hi, then lo at +half its region.
constexpr int kA1 = 0, kA1Lo = kBatchRows * kRowB;                  // stage-x A: 512 rows
constexpr int kA2 = kA1 + 2 * kBatchRows * kRowB, kA2Lo = 512 * kRowB;  // stage-y A: 512 rows (k,a)
constexpr int kA3 = kA2 + 2 * 512 * kRowB, kA3Lo = 256 * kRowB;       // stage-z A: 256 rows (b,a)
constexpr int kB = kA3 + 2 * 256 * kRowB, kBLo = kTcC * kRowB;        // B_x, B_y, B_z: 16 rows each
constexpr int kBasisOff = kB + 3 * 2 * kTcC * kRowB;                 // adjoint: per axis and sample
constexpr int kTcSmem = kBasisOff + 3 * kTcN * 32 + 1024;            // + slack for 1024-byte alignment
static_assert(kTcSmem <= 227 * 1024, "shared memory budget");
// tensor-memory columns: T1 8 x 16, T2 4 x 16, Y 2 x 16
constexpr uint32_t kT1 = 0, kT2 = 128, kT3 = 192, kTcCols = 256;

struct TcBand {  // one sample of one axis: first nonzero basis index and the p+1 values there
  int off;
  float N[4];
  int pad[3];
};

struct TcGeom {  // validated block, as the kernel needs it
  int ok;
  int C[3], p[3];
  int slot;
  int64_t cp_off;
  int64_t koff[3];  // adjoint: knots of each axis
  int cls[3];       // fit: axis classes of the plan
};

template <bool SPLIT>
__device__ __forceinline__ void put_pair(unsigned char* sm, uint32_t off, uint32_t lo, float x0, float x1) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  *reinterpret_cast<__nv_bfloat162*>(sm + off) = h;
  if (SPLIT) {
    const float2 hf = __bfloat1622float2(h);
    *reinterpret_cast<__nv_bfloat162*>(sm + lo + off) = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  }
}
template <bool SPLIT>
__device__ __forceinline__ void put_one(unsigned char* sm, uint32_t off, uint32_t lo, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  *reinterpret_cast<__nv_bfloat16*>(sm + off) = h;
  if (SPLIT) *reinterpret_cast<__nv_bfloat16*>(sm + lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
}

__device__ __forceinline__ uint32_t off32(int r, int k) { return kmajor_off(r, k, kLBO32, kSBO32); }

// Reads and checks work item `item` (fit: plan item and classes; adjoint: descriptor and knots' range).
__device__ __forceinline__ uint32_t load_tc_item(const ContractParams& prm, int item, TcGeom& g) {
  g.ok = 0;
  if (prm.mode == kFit) {
    const EncItem it = prm.items[item];
    for (int a = 0; a < 3; ++a) {
      const EncClass& c = prm.classes[it.cls[a]];
      g.cls[a] = it.cls[a];
      g.C[a] = c.C;
      g.p[a] = c.p;
      if (c.n != kTcN || c.C > kTcC) return MFA_DEV_BAD_DESC;
    }
    g.slot = it.slot;
    g.cp_off = it.cp_off;
    if (g.slot < 0 || g.slot >= prm.nslots) return MFA_DEV_BAD_RANGE;
  } else {
    BlockGeom bg;
    const uint32_t bad = load_desc(prm.desc + item, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                                   prm.slot_stride, bg);
    if (bad) return bad;
    for (int a = 0; a < 3; ++a) {
      if (bg.n[a] != kTcN || bg.C[a] > kTcC) return MFA_DEV_BAD_DESC;
      g.C[a] = bg.C[a];
      g.p[a] = bg.p[a];
      g.koff[a] = bg.knot_off[a];
    }
    g.slot = bg.slot;
    g.cp_off = bg.cp_off;
  }
  if ((int64_t)g.slot * prm.slot_stride + kTcN * kTcN * kTcN > prm.nslots * prm.slot_stride) return MFA_DEV_BAD_RANGE;
  g.ok = 1;
  return 0;
}

template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) contract_tc_kernel(ContractParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TcGeom s_g[2];
  __shared__ float s_kn[3][kKnotMax];
  __shared__ int s_bad;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, group = warp >> 2;
  TcBand* band = reinterpret_cast<TcBand*>(sm + kBasisOff);  // [axis][sample]

  if (warp == 0) {
    tmem_alloc(&s_tmem, kTcCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_addr(sm);
  const uint32_t idesc = idesc_f16(128, kTcC, true);
  uint32_t phase = 0;
  bool timed_out = false;

  // D (+)= A * B^T over K = 32 (two steps of 16), A and B at byte offsets with their lo parts further on
  auto mma32 = [&](uint32_t d, uint32_t a, uint32_t a_lo, uint32_t b) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t ko = s * 2 * kLBO32;
      mma_f16(d, desc_kmajor(sbase + a + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + ko, kLBO32, kSBO32), idesc,
              s > 0);
      if (SPLIT) {
        mma_f16(d, desc_kmajor(sbase + a + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + kBLo + ko, kLBO32, kSBO32),
                idesc, 1);
        mma_f16(d, desc_kmajor(sbase + a + a_lo + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + ko, kLBO32, kSBO32),
                idesc, 1);
      }
    }
  };
  auto wait_mma = [&]() {  // all threads
    const bool ok = mbar_wait_bounded(&s_bar, phase);
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      if (tid == 0) flag(prm.status, MFA_DEV_TIMEOUT);
      mbar_wait_bounded(&s_bar, phase);  // a second bounded wait for the MMAs still in flight
    }
    phase ^= 1;
    tc_fence_after();
  };
  auto operands_ready = [&]() {  // generic-proxy smem writes -> visible to the MMA (async proxy)
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };
  // thread 0: the next valid work item into s_g[buf] (ok = 0 when the queue is empty)
  auto fetch = [&](int buf) {
    for (;;) {
      const int item = (int)atomicAdd(prm.counter, 1u);
      if (item >= prm.nblocks) {
        s_g[buf].ok = 0;
        return;
      }
      const uint32_t bad = load_tc_item(prm, item, s_g[buf]);
      if (!bad) return;
      flag(prm.status, bad);
    }
  };
  float4 xr[kF4PerThread];
  // this thread's share of batch h (16 planes) of the block in s_g[buf]
  auto load_batch = [&](int buf, int h) {
    const float4* src = reinterpret_cast<const float4*>(prm.x + (int64_t)s_g[buf].slot * prm.slot_stride +
                                                        (int64_t)h * kBatchRows * kTcN);
#pragma unroll
    for (int s = 0; s < kF4PerThread; ++s) xr[s] = __ldg(src + s * kTcThreads + tid);
  };
  auto store_batch = [&]() {
#pragma unroll
    for (int s = 0; s < kF4PerThread; ++s) {
      const int e = s * kTcThreads + tid, row = e >> 3, k4 = (e & 7) * 4;
      const uint32_t o = kA1 + off32(row, k4);
      put_pair<SPLIT>(sm, o, kA1Lo, xr[s].x, xr[s].y);
      put_pair<SPLIT>(sm, o + 4, kA1Lo, xr[s].z, xr[s].w);
    }
  };

  if (tid == 0) fetch(0);
  __syncthreads();
  int cur = 0;
  if (s_g[0].ok) load_batch(0, 0);

  while (s_g[cur].ok && !timed_out) {
    const TcGeom& g = s_g[cur];
    // ---- B operands: B_a[c][i] = A_a[i][c] for c < C_a, else 0 ----
    if (prm.mode == kAdjoint) {
      if (tid < 3 * kKnotMax) {
        const int a = tid / kKnotMax, i = tid - a * kKnotMax;
        if (i < g.C[a] + g.p[a] + 1) s_kn[a][i] = prm.knots[g.koff[a] + i];
      }
      if (tid == 0) s_bad = 0;
      __syncthreads();
      if (tid < 3 && !knots_ok(s_kn[tid], g.p[tid], g.C[tid])) {
        atomicOr(&s_bad, 1);
        flag(prm.status, MFA_DEV_BAD_KNOTS);
      }
      if (tid < 3 * kTcN) {
        const int a = tid / kTcN, i = tid - a * kTcN;
        const float u = sample_param(i, kTcN);
        const int s = find_span(s_kn[a], g.p[a], g.C[a], u);
        float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
        basis_funs<MFA_MAX_DEGREE>(s_kn[a], g.p[a], s, u, N, dN);
        TcBand b;
        b.off = s - g.p[a];
        for (int r = 0; r < 4; ++r) b.N[r] = N[r];
        band[a * kTcN + i] = b;
      }
      __syncthreads();
    }
    for (int e = tid; e < 3 * kTcC * kTcN; e += kTcThreads) {
      const int a = e / (kTcC * kTcN), rem = e - a * (kTcC * kTcN), c = rem / kTcN, i = rem - c * kTcN;
      float v = 0.f;
      if (c < g.C[a]) {
        if (prm.mode == kFit) {
          const EncClass& cl = prm.classes[g.cls[a]];
          v = prm.pinv[cl.pinv_off + i * cl.C + c];
        } else {
          const TcBand& b = band[a * kTcN + i];
          const int d = c - b.off;
          if (d >= 0 && d <= g.p[a]) v = b.N[d];
        }
      }
      put_one<SPLIT>(sm, kB + a * 2 * kTcC * kRowB + off32(c, i), kBLo, v);
    }
    const bool skip = prm.mode == kAdjoint && s_bad;  // s_bad is only read after the barriers above
    // ---- stage x, two batches of 16 planes; the next loads are in flight while the MMAs run ----
    for (int h = 0; h < 2 && !timed_out; ++h) {
      store_batch();
      operands_ready();
      if (tid == 0 && !skip) {
#pragma unroll
        for (int t = 0; t < 4; ++t)
          mma32(tmem + kT1 + 16 * (4 * h + t), kA1 + t * 16 * kSBO32, kA1Lo, kB);
      }
      if (tid == 0) {
        if (h == 1) fetch(cur ^ 1);  // the next block, whose first batch loads during this block's stages
        if (!skip) mma_commit(&s_bar);
      }
      __syncthreads();
      if (h == 0) load_batch(cur, 1);
      else if (s_g[cur ^ 1].ok) load_batch(cur ^ 1, 0);
      if (!skip) wait_mma();
    }
    if (timed_out) break;
    if (!skip) {
      // ---- T1 -> A2: row (k,a) = 16k + a, K = j ----
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int t = group + 2 * tt, k = 4 * t + quarter, j = lane;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + kT1 + 16 * t, r);
        tmem_ld_wait();
#pragma unroll
        for (int a = 0; a < kTcC; ++a) put_one<SPLIT>(sm, kA2 + off32(16 * k + a, j), kA2Lo, __uint_as_float(r[a]));
      }
      operands_ready();
      if (tid == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) mma32(tmem + kT2 + 16 * u, kA2 + u * 16 * kSBO32, kA2Lo, kB + 2 * kTcC * kRowB);
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
      // ---- T2 -> A3: T2 row (k,a) = 128u + 32q + lane; A3 row (b,a) = 16b + a, K = k ----
#pragma unroll
      for (int uu = 0; uu < 2; ++uu) {
        const int u = group + 2 * uu, R = 128 * u + 32 * quarter + lane, k = R >> 4, a = R & 15;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + kT2 + 16 * u, r);
        tmem_ld_wait();
#pragma unroll
        for (int b = 0; b < kTcC; ++b) put_one<SPLIT>(sm, kA3 + off32(16 * b + a, k), kA3Lo, __uint_as_float(r[b]));
      }
      operands_ready();
      if (tid == 0) {
#pragma unroll
        for (int v = 0; v < 2; ++v) mma32(tmem + kT3 + 16 * v, kA3 + v * 16 * kSBO32, kA3Lo, kB + 4 * kTcC * kRowB);
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
      // ---- Y row (b,a) = 128v + 32q + lane, columns c -> out[cp_off + (c Cy + b) Cx + a] ----
      {
        const int R = 128 * group + 32 * quarter + lane, b = R >> 4, a = R & 15;
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + kT3 + 16 * group, r);
        tmem_ld_wait();
        const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2];
        if (a < Cx && b < Cy) {
          float* out = prm.out + g.cp_off + (int64_t)b * Cx + a;
#pragma unroll
          for (int c = 0; c < kTcC; ++c)
            if (c < Cz) out[(int64_t)c * Cy * Cx] = __uint_as_float(r[c]);
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the operands, s_g[cur] and the tensor memory are reused by the next block
    tc_fence_after();
    cur ^= 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTcCols);
}

template <bool SPLIT>
int launch_contract_tc(mfa_ctx* ctx, const ContractParams& prm, cudaStream_t stream) {
  if (cudaFuncSetAttribute(contract_tc_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) !=
      cudaSuccess)
    return MFA_ERR_CUDA;
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  const int grid = std::min(ctx->num_sms, prm.nblocks);
  contract_tc_kernel<SPLIT><<<grid, kTcThreads, kTcSmem, stream>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace

int contract_tc(mfa_ctx* ctx, const ContractParams& prm, int precision, cudaStream_t stream) {
  const bool shape_ok = prm.maxN == kTcN && prm.maxC <= kTcC;
  const bool mode_ok = (prm.mode == kFit && prm.rmse == nullptr) || (prm.mode == kAdjoint && prm.cps == nullptr);
  const bool aligned = reinterpret_cast<uintptr_t>(prm.x) % 16 == 0 && prm.slot_stride % 4 == 0;
  if (!shape_ok || !mode_ok || !aligned) return MFA_ERR_UNSUPPORTED;
  if (prm.nblocks < 1) return MFA_OK;
  if (precision == MFA_PREC_SPLIT_BF16) return launch_contract_tc<true>(ctx, prm, stream);
  if (precision == MFA_PREC_BF16) return launch_contract_tc<false>(ctx, prm, stream);
  return MFA_ERR_UNSUPPORTED;
}

}  // namespace mfa
