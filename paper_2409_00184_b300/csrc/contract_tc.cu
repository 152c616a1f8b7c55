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
// K = 32 is two MMA steps of 16. The sample grid arrives in four batches of 8 planes: each thread loads its
// share of a batch (coalesced 16-byte loads), splits it into BF16 hi (and lo) parts and writes the stage-x A
// operand. Stage outputs are read from tensor memory, split again and written transposed as the next stage's
// A operand (stage y in two halves of 16 planes); the B operands (the three A_a^T, zero beyond C) are built
// per block, or kept when the previous block of the CTA had the same axis classes (fit) or knots, degrees and
// control-point counts (adjoint). The fit contracts the samples minus the mid-range of the block's first load
// round and adds it back to the control points (the fit reproduces constants). One 32 KB operand region serves every A operand in turn, and a CTA (one warpgroup) holds 128
// tensor-memory columns, so four CTAs share an SM and one's loads and conversions overlap the others' MMAs.
// One thread issues the MMAs; completion is an mbarrier armed by tcgen05.commit and waited on with a
// bounded poll that reports MFA_DEV_TIMEOUT.
#include <algorithm>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mfa {
namespace {

constexpr int kTcThreads = 128;           // one warpgroup: warp w reads tensor-memory lanes 32w .. 32w+31
constexpr int kTcN = 32;                  // samples per axis (the contraction's K)
constexpr int kTcC = 16;                  // padded control points per axis (the MMA N)
// K-major core-matrix strides for K = 32: the four K-adjacent core matrices (8 rows x 16 bytes) of a row group
// lie 144 bytes apart instead of back to back, so the same row of consecutive K chunks falls in different
// shared-memory banks (a warp writing one row's 32 K entries, or one K entry of 8 rows, hits no bank twice).
constexpr uint32_t kLBO32 = 144, kSBO32 = 4 * kLBO32;
constexpr int kOpRows = 256;              // rows of the operand region (two 128-row tiles)
constexpr int kBatches = 4;               // 8 planes (256 rows of 32 samples) per batch
constexpr int kF4Round = 8;               // float4 loads per thread in flight
constexpr int kF4PerThread = kOpRows * 8 / kTcThreads;  // float4 loads per thread and batch (16)

// Shared-memory layout (bytes). One operand region serves the stage-x A (a batch), the stage-y A (half of
// its rows) and the stage-z A in turn: each is written only after the MMAs that read the previous one have
// completed. Every operand is stored hi, then lo at +half its region.
constexpr int kOp = 0, kOpLo = kOpRows / 8 * kSBO32;                  // 256 rows: 18 KB (+18 KB lo)
constexpr int kB = kOp + 2 * kOpLo, kBLo = kTcC / 8 * kSBO32;        // B_x, B_y, B_z: 16 rows each (+lo)
constexpr int kBasisOff = kB + 3 * 2 * kBLo;                         // adjoint: per axis and sample
constexpr int kTcUsed = kBasisOff + 3 * kTcN * 32 + 1024;            // + slack for 1024-byte alignment
// requested per CTA: at most four CTAs share an SM (4 x 128 tensor-memory columns)
constexpr int kTcSmem = 48 * 1024;
static_assert(kTcUsed <= kTcSmem, "shared memory budget");
// tensor-memory columns: T1 8 tiles x 16 (then T2 over the first 64, Y over the next 32)
constexpr uint32_t kT1 = 0, kT2 = 0, kT3 = 64, kTcCols = 128;

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
__global__ void __launch_bounds__(kTcThreads, 4) contract_tc_kernel(ContractParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ TcGeom s_g;
  __shared__ float s_kn[3][kKnotMax];
  __shared__ int s_bad;
  // the key of the B operands in shared memory (fit: the three axis classes; adjoint: knots, degrees and
  // control-point counts); a block with the same key keeps them
  __shared__ int64_t s_bkey[9];
  __shared__ int s_bkey_ok, s_bsame;
  __shared__ float s_lo[kTcThreads / 32], s_hi[kTcThreads / 32];  // fit: per warp, least and greatest sample
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  TcBand* band = reinterpret_cast<TcBand*>(sm + kBasisOff);  // [axis][sample]

  if (warp == 0) {
    tmem_alloc(&s_tmem, kTcCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_bkey_ok = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes
  const uint32_t sbase = smem_addr(sm);
  const uint32_t idesc = idesc_f16(128, kTcC, true);
  uint32_t phase = 0;
  bool timed_out = false;

  // D (+)= A * B^T over K = 32 (two steps of 16); A at byte offset a in the operand region, B at offset b
  auto mma32 = [&](uint32_t d, uint32_t a, uint32_t b) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint32_t ko = s * 2 * kLBO32;
      mma_f16(d, desc_kmajor(sbase + a + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + ko, kLBO32, kSBO32), idesc,
              s > 0);
      if (SPLIT) {
        mma_f16(d, desc_kmajor(sbase + a + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + kBLo + ko, kLBO32, kSBO32),
                idesc, 1);
        mma_f16(d, desc_kmajor(sbase + a + kOpLo + ko, kLBO32, kSBO32), desc_kmajor(sbase + b + ko, kLBO32, kSBO32),
                idesc, 1);
      }
    }
  };
  // the two 128-row tiles of the operand region against B, into tensor-memory columns d0 and d1
  auto mma_tiles = [&](uint32_t d0, uint32_t d1, uint32_t b) {
    if (tid == 0) {
      mma32(tmem + d0, kOp, b);
      mma32(tmem + d1, kOp + 16 * kSBO32, b);
      mma_commit(&s_bar);
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

  for (;;) {
    if (tid == 0) {  // the next valid work item (ok = 0 when the queue is empty)
      for (;;) {
        const int item = (int)atomicAdd(prm.counter, 1u);
        if (item >= prm.nblocks) {
          s_g.ok = 0;
          break;
        }
        const uint32_t bad = load_tc_item(prm, item, s_g);
        if (!bad) break;
        flag(prm.status, bad);
      }
      s_bad = 0;
      if (s_g.ok) {
        int64_t key[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 3; ++a) {
          if (prm.mode == kFit) {
            key[a] = s_g.cls[a];
          } else {
            key[a] = s_g.koff[a];
            key[3 + a] = s_g.p[a];
            key[6 + a] = s_g.C[a];
          }
        }
        bool same = s_bkey_ok;
        for (int q = 0; q < 9; ++q) same = same && s_bkey[q] == key[q];
        s_bsame = same;
        if (!same) {
          for (int q = 0; q < 9; ++q) s_bkey[q] = key[q];
          s_bkey_ok = 0;  // valid once this block's operands are built and its knots checked
        }
      }
    }
    __syncthreads();
    if (!s_g.ok || timed_out) break;
    const TcGeom& g = s_g;
    // ---- B operands: B_a[c][i] = A_a[i][c] for c < C_a, else 0 (kept from the previous block when its key
    //      is the same) ----
    const bool bsame = s_bsame;
    if (!bsame) {
    if (prm.mode == kAdjoint) {
      if (tid < 3 * kKnotMax) {
        const int a = tid / kKnotMax, i = tid - a * kKnotMax;
        if (i < g.C[a] + g.p[a] + 1) s_kn[a][i] = prm.knots[g.koff[a] + i];
      }
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
      put_one<SPLIT>(sm, kB + a * 2 * kBLo + off32(c, i), kBLo, v);
    }
    }  // !bsame
    if (prm.mode == kAdjoint && s_bad) {  // (s_bad is read after the barriers above)
      __syncthreads();
      continue;
    }
    if (tid == 0 && !bsame) s_bkey_ok = 1;  // read by the next block's fetch, after this block's barriers
    // ---- stage x: four batches of 8 planes (256 rows of 32 samples) through the operand region ----
    // Each batch is loaded in two rounds of kF4Round float4 per thread; the first round of the next batch is
    // in flight while the current batch's MMAs run. The fit contracts X - m, m the mid-range of the first
    // round's samples (4 of the 32 planes), and adds m to every control point: the least-squares fit
    // reproduces constants (the basis functions sum to 1), so P(X) = m + P(X - m), and the 16-bit roundings
    // scale with the samples' spread rather than their offset.
    const float4* src = reinterpret_cast<const float4*>(prm.x + (int64_t)g.slot * prm.slot_stride);
    float4 xr[kF4Round];
    float shift = 0.f;
    auto load_round = [&](int h, int s0) {
#pragma unroll
      for (int s = 0; s < kF4Round; ++s) xr[s] = __ldg(src + (h * kF4PerThread + s0 + s) * kTcThreads + tid);
    };
    auto store_round = [&](int s0) {
      if (prm.mode == kFit) {  // X - m, as packed FP32x2 subtractions
        const float2 m2 = make_float2(-shift, -shift);
#pragma unroll
        for (int s = 0; s < kF4Round; ++s) {
          const float2 a = __fadd2_rn(make_float2(xr[s].x, xr[s].y), m2);
          const float2 b = __fadd2_rn(make_float2(xr[s].z, xr[s].w), m2);
          xr[s] = make_float4(a.x, a.y, b.x, b.y);
        }
      }
#pragma unroll
      for (int s = 0; s < kF4Round; ++s) {
        const int e = (s0 + s) * kTcThreads + tid, row = e >> 3, k4 = (e & 7) * 4;
        const uint32_t o = kOp + off32(row, k4);
        put_pair<SPLIT>(sm, o, kOpLo, xr[s].x, xr[s].y);
        put_pair<SPLIT>(sm, o + 4, kOpLo, xr[s].z, xr[s].w);
      }
    };
    static_assert(kF4PerThread == 2 * kF4Round, "two rounds per batch");
    load_round(0, 0);
    if (prm.mode == kFit) {
      float lo = __int_as_float(0x7f800000), hi = -lo;
#pragma unroll
      for (int s = 0; s < kF4Round; ++s) {
        lo = fminf(fminf(lo, fminf(xr[s].x, xr[s].y)), fminf(xr[s].z, xr[s].w));
        hi = fmaxf(fmaxf(hi, fmaxf(xr[s].x, xr[s].y)), fmaxf(xr[s].z, xr[s].w));
      }
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
      __syncthreads();
      for (int w = 0; w < kTcThreads / 32; ++w) { lo = fminf(lo, s_lo[w]); hi = fmaxf(hi, s_hi[w]); }
      shift = 0.5f * (lo + hi);
    }
    for (int h = 0; h < kBatches && !timed_out; ++h) {
      if (h > 0) wait_mma();  // the previous batch's MMAs have read the region
      if (timed_out) break;
      store_round(0);
      load_round(h, kF4Round);
      store_round(kF4Round);
      operands_ready();
      mma_tiles(kT1 + 32 * h, kT1 + 32 * h + 16, kB);
      if (h + 1 < kBatches) load_round(h + 1, 0);
    }
    if (timed_out) break;
    wait_mma();
    if (timed_out) break;
    // ---- stage y in two halves of 16 planes: T1 (row (k,j) = 32k + j) -> operand rows 16(k - 16 half) + a ----
    for (int half = 0; half < 2 && !timed_out; ++half) {
      uint32_t r4[4][16];  // the half's four tiles are loaded together, then one wait
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) tmem_ld16(tlane + kT1 + 16 * (4 * half + tt), r4[tt]);
      tmem_ld_wait();
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int kl = 4 * tt + warp;  // T1 tile 4 half + tt, row 32 warp + lane: k = 4t + warp
        const uint32_t* r = r4[tt];
        // Lanes j and j^1 trade values so that each writes one 32-bit word (K = j & ~1 and its successor):
        // the even lane the word of row (kl, a), the odd lane that of row (kl, a + 8). Those two rows lie
        // in different bank halves, so the warp's 32 words hit 32 banks.
        const bool even = (lane & 1) == 0;
#pragma unroll
        for (int a = 0; a < kTcC / 2; ++a) {
          const float va = __uint_as_float(r[a]), vb = __uint_as_float(r[a + 8]);
          const float got = __shfl_xor_sync(0xffffffffu, even ? vb : va, 1);
          const int row = 16 * kl + (even ? a : a + 8);
          put_pair<SPLIT>(sm, kOp + off32(row, lane & ~1), kOpLo, even ? va : got, even ? got : vb);
        }
      }
      operands_ready();
      mma_tiles(kT2 + 32 * half, kT2 + 32 * half + 16, kB + 2 * kBLo);
      wait_mma();
    }
    if (timed_out) break;
    // ---- stage z: T2 (row (k,a) = 16k + a) -> operand rows (b,a) = 16b + a, K = k ----
    {
      uint32_t r4[4][16];  // the four tiles are loaded together, then one wait
#pragma unroll
      for (int u = 0; u < 4; ++u) tmem_ld16(tlane + kT2 + 16 * u, r4[u]);
      tmem_ld_wait();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int R = 128 * u + 32 * warp + lane, k = R >> 4, a = R & 15;
#pragma unroll
        for (int b = 0; b < kTcC; ++b) put_one<SPLIT>(sm, kOp + off32(16 * b + a, k), kOpLo, __uint_as_float(r4[u][b]));
      }
    }
    operands_ready();
    mma_tiles(kT3, kT3 + 16, kB + 4 * kBLo);
    wait_mma();
    if (timed_out) break;
    // ---- Y row (b,a) = 128v + 32 warp + lane, columns c -> out[cp_off + (c Cy + b) Cx + a] ----
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int R = 128 * v + 32 * warp + lane, b = R >> 4, a = R & 15;
      uint32_t r[16];
      tmem_ld16(tlane + kT3 + 16 * v, r);
      tmem_ld_wait();
      const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2];
      if (a < Cx && b < Cy) {
        float* out = prm.out + g.cp_off + (int64_t)b * Cx + a;
#pragma unroll
        for (int c = 0; c < kTcC; ++c)
          if (c < Cz) out[(int64_t)c * Cy * Cx] = __uint_as_float(r[c]) + shift;
      }
    }
    tc_fence_before();
    __syncthreads();  // the operands, s_g and the tensor memory are reused by the next block
    tc_fence_after();
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
  if (cudaFuncSetAttribute(contract_tc_kernel<SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return MFA_ERR_CUDA;
  // resident CTAs per SM from the kernel's registers and shared memory (and the SM's register file and
  // shared memory), at most four: every resident CTA holds 128 of the SM's 512 tensor-memory columns
  cudaFuncAttributes fa;
  int smem_sm = 0, regs_sm = 0;
  if (cudaFuncGetAttributes(&fa, contract_tc_kernel<SPLIT>) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device) != cudaSuccess)
    return MFA_ERR_CUDA;
  const int by_regs = regs_sm / std::max(1, fa.numRegs * kTcThreads);
  const int by_smem = smem_sm / (int)(kTcSmem + fa.sharedSizeBytes + 1024);
  const int per_sm = std::max(1, std::min(512 / (int)kTcCols, std::min(by_regs, by_smem)));
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  const int grid = std::min(ctx->num_sms * per_sm, prm.nblocks);
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
