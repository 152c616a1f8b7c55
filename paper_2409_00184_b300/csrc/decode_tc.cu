// Batched micro-model decode on the tensor cores (tcgen05): the three mode products of the decode
// (Sec. 4.2 model, Algorithm 4 value and gradient queries) as dense 16-bit MMAs with FP32 accumulation
// in tensor memory, for BF16, FP16 and split-BF16 operands.
//
// Work unit = one sub-cube of a block, taken from an atomic queue and decoded in slabs of 8 z-planes (four
// for 32 planes). Per axis a sub-cube has 32 samples when the axis has at most 16 control points, else 16
// samples; it only touches the window of control points c0 .. c0+W-1 that its samples' bands cover, and
// W <= 16 holds for uniform knots up to about 24 control points (a wider window, possible only for strongly
// clustered knots, sets MFA_DEV_BAD_DESC for that sub-cube). So every MMA has K = 16 (the window, padded);
// every index is padded to 16 control points and 32 samples, and basis rows are written densely (zero
// outside each band and for the samples past the sub-cube's end). n is at most 64 per axis. The output is
// the row layout or the apron layout (MFA_DECODE_APRON), with or without the gradient. A block's control
// points arrive by one 1-D bulk copy (TMA) on an mbarrier when the copy, widened to 16-byte boundaries, fits
// the free operand area and stays inside the control-point array; else the threads load the window. The
// stage-z operands (P and its differences) do not depend on the slab and are built once per unit; the value
// chain carries P - m, m the mid-range of the window, and the readout adds m back (the basis functions on
// the sub-cube sum to 1). One kernel per
// precision; BF16 and FP16 keep no "lo" operands, which halves the shared memory and lets two CTAs share an
// SM (2 x 256 TMEM columns). Split-BF16 (one CTA per SM) holds all 512 columns and runs stage z once per
// unit for all 32 planes (N = 64) into columns 256..511; the slabs then start at stage y. Derivatives use
// the B-spline derivative identity: d/du sum_a N_{a,p}(u) c_a = sum_a N_{a,p-1}(u) q_a with
// q_a = p (c_{a+1} - c_a) / (t_{a+p+1} - t_{a+1}) on the knots t_1 .. t_{C+p-1}. The four outputs are four independent chains of mode products on the control points
// P and their FP32 differences DxP, DyP, DzP, taken before any rounding: every 16-bit operand is then a
// weighted average of exact differences, and no product cancels against another.
//   chain 0 (f):   P   x N_z x N_y x N_x          chain 1 (f_u): DxP x N_z x N_y       x N_x^(p-1)
//   chain 2 (f_v): DyP x N_z x N_y^(p-1) x N_x    chain 3 (f_w): DzP x N_z^(p-1) x N_y x N_x
//   stage z:  rows (b,a) of each chain (M = 256, two tiles) x [N_z | 0], [0 | N_z^(p-1)] or [0 | N_z]
//   stage y:  transposed, one M = 128 tile for all chains: rows 32c + j hold chain c, N = 128 columns
//             (k,a); the A operand of chain c is the basis placed at rows 32c .. 32c+31, zero elsewhere,
//             so the four MMAs accumulate into one 128 x 128 result
//   stage x:  rows (k,j) of each chain (M = 256, two tiles) x [N_x ; N_x^(p-1)], f | f_u | f_v | f_w in
//             columns 0..127 of the tile
// Each stage's FP32 results are read from tensor memory, rounded (or split into hi + lo) and written as
// the next stage's operand. Split-BF16 forms A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi (three MMAs into the
// same accumulator). The (f, f_u, f_v, f_w) rows leave through a swizzled per-warp staging area so
// each global store instruction writes whole 128-byte lines. One thread issues the MMAs; completion is
// an mbarrier armed by tcgen05.commit, waited on with a bounded poll that reports MFA_DEV_TIMEOUT.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace mfa {
namespace {

constexpr int kThreadsTC = 256;
constexpr int kN = 32;       // samples per axis of one work unit (sub-cube)
constexpr int kK = 16;       // padded control points per axis (one MMA K step)
constexpr int kKS = 8;       // z-planes per slab
constexpr int kSlabs = kN / kKS;
constexpr int kRowBytes = 32;                  // one K-major operand row: 16 x 16-bit
constexpr uint32_t kLBO = 128, kSBO = 256;     // core-matrix strides for K = 16

enum Prec { kBF16 = 0, kFP16 = 1, kSplit = 2 };
// Split-BF16 runs one CTA per SM (its shared memory) and takes all 512 tensor-memory columns: its stage z runs
// once per block, for all 32 planes, into columns 256..511. BF16 and FP16 run two CTAs of 256 columns each
// and a stage z per slab.
template <int PREC> constexpr bool kZOnce = PREC == kSplit;
template <int PREC> constexpr uint32_t kTmemColsOf = kZOnce<PREC> ? 512 : 256;
constexpr uint32_t kZCols = 256;  // first column of the whole-block stage-z result

constexpr int kOp256 = 256 * kRowBytes, kOp128 = 128 * kRowBytes, kOp64 = 64 * kRowBytes, kOp16 = 16 * kRowBytes;
constexpr int kZRows = 224;                   // stage-y basis buffer: 96 zero rows, 32 basis rows, 96 zero rows
constexpr int kOpZ = kZRows * kRowBytes;
constexpr int kStageBytes = 8 * 32 * 128;     // readout staging: 8 warps x 32 rows x 8 float4
constexpr int kPBytes = kK * kK * kK * 4;     // control points, FP32

// Shared-memory layout (bytes) for one precision; every operand is stored hi, then (split-BF16 only) lo.
template <int PREC>
struct TcLayout {
  static constexpr int NL = PREC == kSplit ? 2 : 1;
  static constexpr int Az = 0;                             // stage z A: chains 0..3, per block
  static constexpr int R1 = Az + 4 * kOp256 * NL;          // stage x A; aliases P (block set-up) and staging
  static constexpr int R1Bytes = std::max(4 * kOp256 * NL, std::max(kPBytes, kStageBytes));
  // stage z B, per slab (16 rows: 8 planes) or per block (64 rows: 32 planes):
  // B_z0 = [N_z | 0], B_z1 = [0 | N_z^(p-1)], B_z2 = [0 | N_z]
  static constexpr int BzOp = kZOnce<PREC> ? kOp64 : kOp16;
  static constexpr int Bz = R1 + R1Bytes;
  static constexpr int Ty = Bz + 3 * BzOp * NL;            // stage y B: chains 0..3, rows (k,a), K = b
  static constexpr int Zy = Ty + 4 * kOp128 * NL;          // stage y A: N_y and N_y^(p-1), zero-padded
  static constexpr int Bx = Zy + 2 * kOpZ * NL;            // stage x B: rows [N_x ; N_x^(p-1)]
  static constexpr int Basis = Bx + kOp64 * NL;            // per axis and sample: TcBasis (48 B)
  static constexpr int Knots = Basis + 3 * kN * 48;
  static constexpr int Dsc = Knots + 3 * kKnotMax * 4;     // per axis: p / (t_{c+p+1} - t_{c+1})
  static constexpr int Total = Dsc + 3 * kN * 4 + 1024;    // + slack for 1024-byte alignment
  // lo-part distances (0 when unused)
  static constexpr int dAz = 4 * kOp256, dAx = 4 * kOp256, dBz = 3 * BzOp, dTy = 4 * kOp128, dZy = 2 * kOpZ, dBx = kOp64;
  static_assert(Total <= 227 * 1024, "shared memory budget");
};

template <int PREC>
__device__ __forceinline__ uint16_t to16(float x) {
  if (PREC == kFP16) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <int PREC>
__device__ __forceinline__ float from16(uint16_t v) {
  if (PREC == kFP16) return __half2float(__ushort_as_half(v));
  return __bfloat162float(__ushort_as_bfloat16(v));
}
// Writes x (and, for split-BF16, its remainder x - hi at lo_delta further) at byte offset `off`.
template <int PREC>
__device__ __forceinline__ void put(unsigned char* base, uint32_t off, uint32_t lo_delta, float x) {
  const uint16_t h = to16<PREC>(x);
  *reinterpret_cast<uint16_t*>(base + off) = h;
  if (PREC == kSplit) *reinterpret_cast<uint16_t*>(base + lo_delta + off) = to16<PREC>(x - from16<PREC>(h));
}
// Writes two consecutive K entries (x0 first) as one 32-bit word and, for split-BF16, their remainders.
template <int PREC>
__device__ __forceinline__ void put2(unsigned char* base, uint32_t off, uint32_t lo_delta, float x0, float x1) {
  const uint16_t h0 = to16<PREC>(x0), h1 = to16<PREC>(x1);
  *reinterpret_cast<uint32_t*>(base + off) = (uint32_t)h0 | ((uint32_t)h1 << 16);
  if (PREC == kSplit)
    *reinterpret_cast<uint32_t*>(base + lo_delta + off) =
        (uint32_t)to16<PREC>(x0 - from16<PREC>(h0)) | ((uint32_t)to16<PREC>(x1 - from16<PREC>(h1)) << 16);
}
// Writes 8 consecutive K entries of one operand row (16 bytes) and, for split-BF16, their remainders.
template <int PREC>
__device__ __forceinline__ void put8(unsigned char* base, uint32_t off, uint32_t lo_delta, const uint32_t* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float x0 = __uint_as_float(x[2 * i]), x1 = __uint_as_float(x[2 * i + 1]);
    const uint16_t h0 = to16<PREC>(x0), h1 = to16<PREC>(x1);
    h[i] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    if (PREC == kSplit)
      l[i] = (uint32_t)to16<PREC>(x0 - from16<PREC>(h0)) | ((uint32_t)to16<PREC>(x1 - from16<PREC>(h1)) << 16);
  }
  *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  if (PREC == kSplit) *reinterpret_cast<uint4*>(base + lo_delta + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

struct TcBasis {  // one sample: first nonzero index (both degrees) and the band values of degree p, p-1
  int off;
  int pad[3];
  float N[4], Nm[4];
};

template <int PREC>
__global__ void __launch_bounds__(kThreadsTC, PREC == kSplit ? 1 : 2) decode_tc_kernel(DecodeParams prm) {
  using L = TcLayout<PREC>;
  constexpr bool split = PREC == kSplit;
  constexpr bool bf = PREC != kFP16;
  constexpr bool zonce = kZOnce<PREC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ int s_item, s_bad, s_same;
  __shared__ int s_w0[3], s_m[3];  // first sample and number of samples of the sub-cube per axis
  __shared__ int s_c0[3];          // first control point of the sub-cube's window per axis
  __shared__ float s_lo[kThreadsTC / 32], s_hi[kThreadsTC / 32];  // per warp: least and greatest P loaded
  __shared__ float s_mid;  // mid-range of the unit's window of P
  __shared__ BlockGeom s_g;
  __shared__ int64_t s_key[15];  // knots, degrees, sizes and sub-cube of the unit whose bases are in shared memory
  __shared__ int s_key_ok;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(8) uint64_t s_pbar;  // the bulk copy of a unit's control points
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, group = warp >> 2;
  float* P = reinterpret_cast<float*>(sm + L::R1);
  TcBasis* bas = reinterpret_cast<TcBasis*>(sm + L::Basis);  // [axis][sample]
  float* kn = reinterpret_cast<float*>(sm + L::Knots);
  float* dsc = reinterpret_cast<float*>(sm + L::Dsc);          // [axis][control index]

  if (warp == 0) {
    tmem_alloc(&s_tmem, kTmemColsOf<PREC>);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    mbar_init(&s_pbar, 1);
    fence_mbar_init();
    s_key_ok = 0;
  }
  // the zero rows of the stage-y basis buffers are written once; the basis rows per block
  for (int e = tid * 16; e < 2 * kOpZ * L::NL; e += kThreadsTC * 16)
    *reinterpret_cast<uint4*>(sm + L::Zy + e) = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t sbase = smem_addr(sm);
  uint32_t phase = 0, pphase = 0;
  bool timed_out = false;

  int count = prm.list ? (prm.count ? *prm.count : prm.list_len) : prm.nblocks;
  if (prm.list && (count < 0 || count > prm.list_len)) {
    if (blockIdx.x == 0 && tid == 0) flag(prm.status, MFA_DEV_BAD_LIST);
    count = max(0, min(count, prm.list_len));
  }
  // work units: every item has Sa^3 sub-cube positions G apart per axis (G = 16 when some axis may have more
  // than 16 control points, else 32; Sa = ceil(max_nsamp / G)); a block takes the positions on its own
  // sub-cube grid (32 or 16 samples per axis) inside its n, the others are empty
  const int G = prm.bounds.max_ncp > kK ? kN / 2 : kN;
  const int Sa = (prm.bounds.max_nsamp + G - 1) / G, S = Sa * Sa * Sa;
  const int units = count * S;

  // D (+)= A * B^T for operands at byte offsets a, b (lo parts at a_lo, b_lo); acc0 = accumulate into D
  auto mma = [&](uint32_t d, uint32_t a, uint32_t a_lo, uint32_t b, uint32_t b_lo, int N, uint32_t acc0) {
    const uint32_t id = idesc_f16(128, N, bf);
    mma_f16(d, desc_kmajor(sbase + a, kLBO, kSBO), desc_kmajor(sbase + b, kLBO, kSBO), id, acc0);
    if (split) {
      mma_f16(d, desc_kmajor(sbase + a, kLBO, kSBO), desc_kmajor(sbase + b_lo, kLBO, kSBO), id, 1);
      mma_f16(d, desc_kmajor(sbase + a_lo, kLBO, kSBO), desc_kmajor(sbase + b, kLBO, kSBO), id, 1);
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
    __syncthreads();
    if (tid == 0) {
      s_item = (int)atomicAdd(prm.counter, 1u);
      s_bad = 0;
      if (s_item < units) {
        const int item = s_item / S, sub = s_item - item * S;
        s_w0[0] = (sub % Sa) * G;
        s_w0[1] = ((sub / Sa) % Sa) * G;
        s_w0[2] = (sub / (Sa * Sa)) * G;
        const int b = prm.list ? prm.list[item] : item;
        const bool list_slots = (prm.flags & MFA_DECODE_LIST_SLOTS) != 0;
        uint32_t bad = 0;
        if (b < 0 || b >= prm.nblocks) bad = MFA_DEV_BAD_LIST;
        else bad = load_desc(prm.desc + b, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots, prm.slot_stride,
                             s_g, !list_slots);
        if (!bad && list_slots) {
          if (item >= prm.nslots) bad = MFA_DEV_BAD_RANGE;
          s_g.slot = item;
        }
        if (!bad && (prm.flags & MFA_DECODE_APRON) &&
            (int64_t)apron_pitch(s_g.n[0]) * (s_g.n[1] + 1) * (s_g.n[2] + 1) > prm.slot_stride)
          bad = MFA_DEV_BAD_RANGE;
        if (bad) { flag(prm.status, bad); s_bad = 1; }
        // positions off the block's sub-cube grid, or past its own sample count, have nothing to decode
        if (!bad)
          for (int a = 0; a < 3; ++a) {
            const int E = s_g.C[a] <= kK ? kN : kN / 2;
            if (s_w0[a] % E != 0 || s_w0[a] >= s_g.n[a]) s_bad = 1;
            s_m[a] = min(E, s_g.n[a] - s_w0[a]);
          }
        // the bases, difference scales and basis operands only depend on (knots, degree, C, n, sub-cube) per
        // axis: a unit that repeats the previous unit's keeps them
        const int64_t key[15] = {s_g.knot_off[0], s_g.knot_off[1], s_g.knot_off[2], s_g.p[0], s_g.p[1], s_g.p[2],
                                 s_g.C[0],        s_g.C[1],        s_g.C[2],        s_g.n[0], s_g.n[1], s_g.n[2],
                                 s_w0[0],         s_w0[1],         s_w0[2]};
        bool same = s_key_ok && !s_bad;
        for (int q = 0; q < 15; ++q) same = same && s_key[q] == key[q];
        s_same = same;
        if (!s_bad && !same) {
          for (int q = 0; q < 15; ++q) s_key[q] = key[q];
          s_key_ok = 0;  // valid once this unit's set-up has passed its checks
        }
      }
    }
    __syncthreads();
    if (s_item >= units || timed_out) break;
    if (s_bad) continue;
    const int Cx = s_g.C[0], Cy = s_g.C[1], Cz = s_g.C[2];
    const bool same = s_same;
    // z-slabs of this sub-cube; a block of 32^3 samples and at most 16 control points per axis is one whole
    // sub-cube
    const int nslab = (s_m[2] + kKS - 1) / kKS;
    const bool whole = s_g.n[0] == kN && s_g.n[1] == kN && s_g.n[2] == kN && s_m[0] == kN && s_m[1] == kN &&
                       s_m[2] == kN;
    const bool apron = (prm.flags & MFA_DECODE_APRON) != 0;

    // ---- per unit: knots, basis bands of degree p and p-1, control windows, difference scales (unless
    //      kept), the window of P ----
    if (!same) {
    if (tid < 3 * kKnotMax) {
      const int a = tid / kKnotMax, i = tid - a * kKnotMax;
      if (i < s_g.C[a] + s_g.p[a] + 1) kn[tid] = prm.knots[s_g.knot_off[a] + i];
    }
    __syncthreads();
    if (tid < 3 && !knots_ok(kn + tid * kKnotMax, s_g.p[tid], s_g.C[tid])) {
      atomicOr(&s_bad, 1);
      flag(prm.status, MFA_DEV_BAD_KNOTS);
    }
    if (tid < 3 * kN) {
      const int a = tid / kN, i = tid - a * kN;
      const int p = s_g.p[a];
      const float* t = kn + a * kKnotMax;
      TcBasis tb;
      tb.off = 0;
      tb.pad[0] = tb.pad[1] = tb.pad[2] = 0;
      for (int r = 0; r < 4; ++r) { tb.N[r] = 0.f; tb.Nm[r] = 0.f; }
      if (i < s_m[a]) {  // a sample of this sub-cube (the rows past its end stay zero)
        const float u = sample_param(s_w0[a] + i, s_g.n[a]);
        const int s = find_span(t, p, s_g.C[a], u);
        float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1], Nm[MFA_MAX_DEGREE + 1], dNm[MFA_MAX_DEGREE + 1];
        basis_funs<MFA_MAX_DEGREE>(t, p, s, u, N, dN);
        // degree p-1 on the knots t_1 .. t_{C+p-1}: span s-1, nonzero functions s-p .. s-1
        basis_funs<MFA_MAX_DEGREE>(t + 1, p - 1, s - 1, u, Nm, dNm);
        tb.off = s - p;
        for (int r = 0; r < 4; ++r) { tb.N[r] = N[r]; tb.Nm[r] = Nm[r]; }
      }
      bas[a * kN + i] = tb;
      // difference scale of control index i (i < C-1)
      float sc = 0.f;
      if (i < s_g.C[a] - 1) {
        const float den = t[i + p + 1] - t[i + 1];
        if (den > 0.f) sc = (float)p / den;
      }
      dsc[a * kN + i] = sc;
    }
    __syncthreads();
    // control window per axis: from the first sample's band to the last one's (spans do not decrease)
    if (tid < 3 && !s_bad) {
      const int c0 = bas[tid * kN].off, last = bas[tid * kN + s_m[tid] - 1].off;
      s_c0[tid] = c0;
      if (last + s_g.p[tid] + 1 - c0 > kK) {
        atomicOr(&s_bad, 1);
        flag(prm.status, MFA_DEV_BAD_DESC);
      }
    }
    __syncthreads();
    if (s_bad) continue;
    if (tid < 3 * kN && tid % kN < s_m[tid / kN]) bas[tid].off -= s_c0[tid / kN];  // band offsets in the window
    if (tid == 0) s_key_ok = 1;
    __syncthreads();
    // stage-y A: rows 96..127 of the two zero-padded buffers = N_y(u_j) and N_y^(p-1)(u_j), K = b;
    // stage-x B: rows n < 32 = N_x(u_n), rows 32..63 = N_x^(p-1)(u_{n-32}), K = a
    for (int e = tid; e < 2 * 64 * kK; e += kThreadsTC) {
      const int which = e / (64 * kK), rem = e - which * (64 * kK), n = rem / kK, c = rem - (rem / kK) * kK;
      const int axis = which == 0 ? 1 : 0;
      const TcBasis& tb = bas[axis * kN + (n & 31)];
      const int d = c - tb.off;
      float v = 0.f;
      const int cw = c + s_c0[axis];  // control index
      if (n < 32) { if (d >= 0 && d <= 3 && cw < s_g.C[axis]) v = tb.N[d]; }
      else if (d >= 0 && d <= 3 && cw < s_g.C[axis] - 1) v = tb.Nm[d];
      if (which == 0)
        put<PREC>(sm + L::Zy + (n < 32 ? 0 : kOpZ), kmajor_off(96 + (n & 31), c, kLBO, kSBO), L::dZy, v);
      else
        put<PREC>(sm + L::Bx, kmajor_off(n, c, kLBO, kSBO), L::dBx, v);
    }
    // per-block stage-z B: rows n < 32 of B_z0 = N_z(u_n); rows 32..63 of B_z1 = N_z^(p-1)(u_{n-32}) and of
    // B_z2 = N_z(u_{n-32}); K = c
    if (zonce)
      for (int e = tid; e < 3 * 64 * kK; e += kThreadsTC) {
        const int which = e / (64 * kK), n = (e >> 4) & 63, c = e & 15;
        float v = 0.f;
        if ((n < 32) == (which == 0)) {
          const TcBasis& tb = bas[2 * kN + (n & 31)];
          const int d = c - tb.off, cw = c + s_c0[2];
          if (d >= 0 && d <= 3) {
            if (which == 1) { if (cw < Cz - 1) v = tb.Nm[d]; }
            else if (cw < Cz) v = tb.N[d];
          }
        }
        put<PREC>(sm + L::Bz + which * kOp64, kmajor_off(n, c, kLBO, kSBO), L::dBz, v);
      }
    }  // !same
    {  // the window of P, control (c0_z + c, c0_y + b, c0_x + a) at Pw[c sz + b sy + a]
    const int x0 = s_c0[0], y0 = s_c0[1], z0 = s_c0[2];
    const int Wx = min(kK, Cx - x0), Wy = min(kK, Cy - y0), Wz = min(kK, Cz - z0);
    // The block's control points arrive by one bulk copy (TMA) when the copy, widened to 16-byte boundaries,
    // fits the R1 area (free until the stage-x operand is written) and stays inside the control-point array;
    // then Pw has the block's own strides. Else the threads load the window into a dense 16 x 16 x 16 box.
    const int64_t b0 = s_g.cp_off * 4, e0 = (s_g.cp_off + (int64_t)Cx * Cy * Cz) * 4;
    const int64_t a0 = b0 & ~int64_t(15), a1 = (e0 + 15) & ~int64_t(15);
    const bool bulk = (reinterpret_cast<uintptr_t>(prm.cps) & 15) == 0 && a1 - a0 <= L::R1Bytes && a1 <= prm.cps_len * 4;
    const int sy = bulk ? Cx : kK, sz = bulk ? Cx * Cy : kK * kK;
    const float* Pw = bulk ? P + (b0 - a0) / 4 + ((int64_t)z0 * Cy + y0) * Cx + x0 : P;
    float lo = __int_as_float(0x7f800000), hi = -lo;
    if (bulk) {
      if (tid == 0) {
        fence_async_smem();  // the threads' earlier accesses to the P area come before the copy's writes
        mbar_arrive_expect_tx(&s_pbar, (uint32_t)(a1 - a0));
        bulk_load(P, reinterpret_cast<const unsigned char*>(prm.cps) + a0, (uint32_t)(a1 - a0), &s_pbar);
      }
      const bool ok = mbar_wait_bounded(&s_pbar, pphase);
      if (__syncthreads_or(!ok)) {
        timed_out = true;
        if (tid == 0) flag(prm.status, MFA_DEV_TIMEOUT);
        mbar_wait_bounded(&s_pbar, pphase);  // a second bounded wait for the copy still in flight
        break;
      }
      pphase ^= 1;
      for (int e = tid; e < kK * kK * kK; e += kThreadsTC) {
        const int c = e >> 8, b = (e >> 4) & 15, a = e & 15;
        if (a < Wx && b < Wy && c < Wz) {
          const float v = Pw[c * sz + b * sy + a];
          lo = fminf(lo, v);
          hi = fmaxf(hi, v);
        }
      }
    } else {
      for (int e = tid; e < kK * kK * kK; e += kThreadsTC) {
        const int c = e >> 8, b = (e >> 4) & 15, a = e & 15;
        if (a < Wx && b < Wy && c < Wz) {
          const float v = __ldg(prm.cps + s_g.cp_off + ((z0 + c) * Cy + y0 + b) * Cx + x0 + a);
          P[e] = v;
          lo = fminf(lo, v);
          hi = fmaxf(hi, v);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
    __syncthreads();
    // The value chain carries P - m, m the mid-range of the window's P, and the readout adds m back: the
    // sub-cube's samples have all their nonzero basis functions in the window and they sum to 1, so
    // f = m + sum N (P - m), while the 16-bit roundings now scale with |P - m| instead of |P|.
    for (int w = 0; w < kThreadsTC / 32; ++w) { lo = fminf(lo, s_lo[w]); hi = fmaxf(hi, s_hi[w]); }
    const float mid = 0.5f * (lo + hi);
    if (tid == 0) s_mid = mid;  // read by the value readouts of this unit's slabs
    // stage-z A: chains P - m, DxP, DyP, DzP at rows (b,a) = 16b + a, K = c (z control index in the window),
    // two K at a time. A difference whose second point lies past the window is never used (its degree p-1
    // basis function is zero on the sub-cube's samples) and is written as 0.
    for (int e = tid; e < 256 * kK / 2; e += kThreadsTC) {
      const int R = e >> 3, c0 = 2 * (e & 7), b = R >> 4, a = R & 15;
      float v0[2] = {0.f, 0.f}, vu[2] = {0.f, 0.f}, vv[2] = {0.f, 0.f}, vw[2] = {0.f, 0.f};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = c0 + h;
        if (a < Wx && b < Wy && c < Wz) {
          const int idx = c * sz + b * sy + a;
          const float p0 = Pw[idx];
          v0[h] = p0 - mid;
          if (a + 1 < Wx) vu[h] = dsc[x0 + a] * (Pw[idx + 1] - p0);
          if (b + 1 < Wy) vv[h] = dsc[kN + y0 + b] * (Pw[idx + sy] - p0);
          if (c + 1 < Wz) vw[h] = dsc[2 * kN + z0 + c] * (Pw[idx + sz] - p0);
        }
      }
      const uint32_t off = kmajor_off(R, c0, kLBO, kSBO);
      put2<PREC>(sm + L::Az, off, L::dAz, v0[0], v0[1]);
      put2<PREC>(sm + L::Az + kOp256, off, L::dAz, vu[0], vu[1]);
      put2<PREC>(sm + L::Az + 2 * kOp256, off, L::dAz, vv[0], vv[1]);
      put2<PREC>(sm + L::Az + 3 * kOp256, off, L::dAz, vw[0], vw[1]);
    }
    }
    // (P in R1 is dead from here on: R1 becomes the stage-x operand and the readout staging)
    if (zonce) {
      operands_ready();
      // ---- stage z for all 32 planes, per 128-row tile t at column 256 + 128t:
      //      [chain 0 | chain 3 | chain 2 | chain 1], 32 planes each ----
      if (tid == 0) {
        for (int t = 0; t < 2; ++t) {
          const uint32_t ro = t * 16 * kSBO, d = tmem + kZCols + 128 * t;
          mma(d, L::Az + ro, L::Az + L::dAz + ro, L::Bz, L::Bz + L::dBz, 64, 0);
          mma(d, L::Az + 3 * kOp256 + ro, L::Az + 3 * kOp256 + L::dAz + ro, L::Bz + kOp64, L::Bz + kOp64 + L::dBz,
              64, 1);
          mma(d + 64, L::Az + 2 * kOp256 + ro, L::Az + 2 * kOp256 + L::dAz + ro, L::Bz, L::Bz + L::dBz, 64, 0);
          mma(d + 64, L::Az + kOp256 + ro, L::Az + kOp256 + L::dAz + ro, L::Bz + 2 * kOp64,
              L::Bz + 2 * kOp64 + L::dBz, 64, 1);
        }
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
    }

    for (int slab = 0; slab < nslab && !timed_out; ++slab) {
      const int k0 = slab * kKS;
      if (!zonce) {
      for (int e = tid; e < 3 * 16 * kK; e += kThreadsTC) {  // B_z0, B_z1, B_z2: 16 x 16 each
        const int which = e >> 8, n = (e >> 4) & 15, c = e & 15;
        const int kl = n & 7;
        float v = 0.f;
        if ((n < 8) == (which == 0)) {
          const TcBasis& tb = bas[2 * kN + k0 + kl];
          const int d = c - tb.off, cw = c + s_c0[2];
          if (d >= 0 && d <= 3) {
            if (which == 1) { if (cw < Cz - 1) v = tb.Nm[d]; }
            else if (cw < Cz) v = tb.N[d];
          }
        }
        put<PREC>(sm + L::Bz + which * kOp16, kmajor_off(n, c, kLBO, kSBO), L::dBz, v);
      }
      operands_ready();
      // ---- stage z, per 128-row tile t: columns 16t: [chain 0 | chain 3], 32 + 16t: [chain 2 | chain 1] ----
      if (tid == 0) {
        for (int t = 0; t < 2; ++t) {
          const uint32_t ro = t * 16 * kSBO;
          mma(tmem + 16 * t, L::Az + ro, L::Az + L::dAz + ro, L::Bz, L::Bz + L::dBz, 16, 0);
          mma(tmem + 16 * t, L::Az + 3 * kOp256 + ro, L::Az + 3 * kOp256 + L::dAz + ro, L::Bz + kOp16,
              L::Bz + kOp16 + L::dBz, 16, 1);
          mma(tmem + 32 + 16 * t, L::Az + 2 * kOp256 + ro, L::Az + 2 * kOp256 + L::dAz + ro, L::Bz, L::Bz + L::dBz,
              16, 0);
          mma(tmem + 32 + 16 * t, L::Az + kOp256 + ro, L::Az + kOp256 + L::dAz + ro, L::Bz + 2 * kOp16,
              L::Bz + 2 * kOp16 + L::dBz, 16, 1);
        }
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
      }  // !zonce
      // readout z -> stage-y B of chain c: element (row 16k + a, K = b); every entry of all 128 rows is written.
      // r0 = [chain 0 | chain 3], r1 = [chain 2 | chain 1] of planes k0 .. k0+7
      {
        const int R = 128 * group + 32 * quarter + lane, b = R >> 4, a = R & 15;
        uint32_t r0[16], r1[16];
        if (zonce) {
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + kZCols + 128 * group + k0;
          tmem_ld8(ta, *reinterpret_cast<uint32_t(*)[8]>(r0));
          tmem_ld8(ta + 32, *reinterpret_cast<uint32_t(*)[8]>(r0 + 8));
          tmem_ld8(ta + 64, *reinterpret_cast<uint32_t(*)[8]>(r1));
          tmem_ld8(ta + 96, *reinterpret_cast<uint32_t(*)[8]>(r1 + 8));
        } else {
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + 16 * group;
          tmem_ld16(ta, r0);
          tmem_ld16(ta + 32, r1);
        }
        tmem_ld_wait();
        // Lanes L and L + 16 hold the same (k, a) at b and b + 1 (adjacent K): they trade values so that
        // the lower lane writes the 32-bit words (b, b + 1) of chains 0 and 1, the upper one those of chains 2
        // and 3.
        const bool low = (lane & 16) == 0;
        unsigned char* dst0 = sm + L::Ty + (low ? 0 : 2 * kOp128);
        unsigned char* dst1 = sm + L::Ty + (low ? kOp128 : 3 * kOp128);
#pragma unroll
        for (int kl = 0; kl < kKS; ++kl) {
          const float v0 = __uint_as_float(r0[kl]), v1 = __uint_as_float(r1[8 + kl]);
          const float v2 = __uint_as_float(r1[kl]), v3 = __uint_as_float(r0[8 + kl]);
          const float g0 = __shfl_xor_sync(0xffffffffu, low ? v2 : v0, 16);
          const float g1 = __shfl_xor_sync(0xffffffffu, low ? v3 : v1, 16);
          const uint32_t off = kmajor_off(kl * 16 + a, b & ~1, kLBO, kSBO);
          put2<PREC>(dst0, off, L::dTy, low ? v0 : g0, low ? g0 : v2);
          put2<PREC>(dst1, off, L::dTy, low ? v1 : g1, low ? g1 : v3);
        }
      }
      operands_ready();
      // ---- stage y: D[32c + j][(k,a)] = sum_b basis_c(u_j)_b T_c[(k,a)][b], chains accumulated ----
      if (tid == 0) {
        for (int c = 0; c < 4; ++c) {
          const uint32_t za = L::Zy + (c == 2 ? kOpZ : 0) + (uint32_t)((96 - 32 * c) / 8) * kSBO;
          mma(tmem, za, za + L::dZy, L::Ty + c * kOp128, L::Ty + c * kOp128 + L::dTy, 128, c > 0);
        }
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
      // readout y: warp (quarter c, group g) holds chain c, sample j = lane, planes k = 4g .. 4g+3;
      // stage-x A of chain c: element (row 32k + j, K = a), 16 consecutive K entries = two 16-byte stores
      {  // the four loads are issued together, then one wait
        uint32_t r[4][16];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 16 * (4 * group + kk), r[kk]);
        tmem_ld_wait();
        unsigned char* base = sm + L::R1 + quarter * kOp256;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kmajor_off((4 * group + kk) * 32 + lane, 0, kLBO, kSBO);
          put8<PREC>(base, off, L::dAx, r[kk]);
          put8<PREC>(base, off + kLBO, L::dAx, r[kk] + 8);
        }
      }
      operands_ready();
      // ---- stage x per 128-row tile: f | f_u | f_v | f_w in columns 0..127 of the tile ----
      if (tid == 0) {
        for (int t = 0; t < 2; ++t) {
          const uint32_t d = tmem + 128 * t, ro = t * 16 * kSBO;
          for (int c = 0; c < 4; ++c) {
            const uint32_t bo = c == 1 ? 4 * kSBO : 0;
            mma(d + 32 * c, L::R1 + c * kOp256 + ro, L::R1 + c * kOp256 + L::dAx + ro, L::Bx + bo,
                L::Bx + L::dBx + bo, 32, 0);
          }
        }
        mma_commit(&s_bar);
      }
      wait_mma();
      if (timed_out) break;
      if (prm.flags & MFA_DECODE_VALUE_ONLY) {
        // value only (one float per voxel): each lane writes f of its row (k, j), voxel row
        // (w0_z + k0 + k, w0_y + j), for the 16 voxels of each column half inside the sub-cube
        float* outf = prm.cache + (int64_t)s_g.slot * prm.slot_stride;
        const int Rg = 128 * group + 32 * quarter + lane, kl = k0 + (Rg >> 5), j = Rg & 31;
        const int rows = apron ? s_g.n[1] + 1 : s_g.n[1], pitch = apron ? apron_pitch(s_g.n[0]) : s_g.n[0];
        float* row = outf + ((int64_t)(s_w0[2] + kl) * rows + s_w0[1] + j) * pitch + s_w0[0];
        for (int h = 0; h < 2; ++h) {
          uint32_t f[16];
          tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + 128 * group + 16 * h, f);
          tmem_ld_wait();
          if (kl < s_m[2] && j < s_m[1]) {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (16 * h + q < s_m[0]) __stcs(row + 16 * h + q, __uint_as_float(f[q]) + s_mid);
          }
        }
      } else
      // readout x: warp group g takes tile g; each warp stages its 32 rows, 8 voxels at a time, and writes
      // the voxels inside the sub-cube: row (k, j) of the tile is voxel row (w0_z + k0 + k, w0_y + j)
      {
        float4* stg = reinterpret_cast<float4*>(sm + L::R1 + warp * 32 * 128);
        float4* out = reinterpret_cast<float4*>(prm.cache) + (int64_t)s_g.slot * prm.slot_stride;

        for (int h = 0; h < 2; ++h) {
          uint32_t f[16], fu[16], fv[16], fw[16];
          const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + 128 * group + 16 * h;
          tmem_ld16(ta, f);
          tmem_ld16(ta + 32, fu);
          tmem_ld16(ta + 64, fv);
          tmem_ld16(ta + 96, fw);
          tmem_ld_wait();
#pragma unroll
          for (int half = 0; half < 2; ++half) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              const int q = 8 * half + v;
              stg[lane * 8 + (v ^ (lane & 7))] = make_float4(__uint_as_float(f[q]) + s_mid, __uint_as_float(fu[q]),
                                                             __uint_as_float(fv[q]), __uint_as_float(fw[q]));
            }
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 8; ++it) {
              const int rr = 4 * it + (lane >> 3), v = lane & 7;
              const int Rg = 128 * group + 32 * quarter + rr, i = 16 * h + 8 * half + v;
              if (whole) {  // row (k, j) of the tile at (k0 + k) 32^2 + 32 j, or with an apron at
                            // ((k0 + k) 33 + j) apron_pitch(32)
                constexpr int AP = apron_pitch(kN);
                const int row = apron ? ((k0 + (Rg >> 5)) * (kN + 1) + (Rg & 31)) * AP : k0 * kN * kN + Rg * kN;
                __stcs(out + (row + i), stg[rr * 8 + (v ^ (rr & 7))]);
              } else {  // voxel (w0_z + k0 + k, w0_y + j, w0_x + i) when inside the sub-cube; with an apron in
                        // rows of apron_pitch(n_x) and planes of n_y + 1 rows
                const int kl = k0 + (Rg >> 5), j = Rg & 31;
                if (kl < s_m[2] && j < s_m[1] && i < s_m[0]) {
                  const int rows = apron ? s_g.n[1] + 1 : s_g.n[1], pitch = apron ? apron_pitch(s_g.n[0]) : s_g.n[0];
                  __stcs(out + (((s_w0[2] + kl) * rows + s_w0[1] + j) * pitch + s_w0[0] + i),
                         stg[rr * 8 + (v ^ (rr & 7))]);
                }
              }
            }
            __syncwarp();
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // staging (R1) and the tensor memory are reused by the next slab
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemColsOf<PREC>);
}

template <int PREC>
int launch_tc(mfa_ctx* ctx, DecodeParams prm, cudaStream_t stream) {
  using L = TcLayout<PREC>;
  const size_t smem = L::Total;
  if (cudaFuncSetAttribute(decode_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return MFA_ERR_CUDA;
  // all of the SM's unified L1 / shared memory as shared memory, so that two BF16 / FP16 CTAs fit
  if (cudaFuncSetAttribute(decode_tc_kernel<PREC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return MFA_ERR_CUDA;
  // resident CTAs per SM from the kernel's registers and shared memory (and the SM's register file and shared
  // memory); the resident CTAs share the SM's 512 tensor-memory columns
  cudaFuncAttributes fa;
  int smem_sm = 0, regs_sm = 0;
  if (cudaFuncGetAttributes(&fa, decode_tc_kernel<PREC>) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device) != cudaSuccess)
    return MFA_ERR_CUDA;
  const int by_regs = regs_sm / std::max(1, fa.numRegs * kThreadsTC);
  const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
  const int per_sm = std::max(1, std::min((int)(512 / kTmemColsOf<PREC>), std::min(by_regs, by_smem)));
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  decode_tc_kernel<PREC><<<ctx->num_sms * per_sm, kThreadsTC, smem, stream>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace

int decode_tc(mfa_ctx* ctx, DecodeParams prm, int precision, cudaStream_t stream) {
  if (prm.bounds.max_nsamp > 2 * kN) return MFA_ERR_UNSUPPORTED;
  prm.ks = kKS;
  prm.slabs = kSlabs;
  if (precision == MFA_PREC_BF16) return launch_tc<kBF16>(ctx, prm, stream);
  if (precision == MFA_PREC_FP16) return launch_tc<kFP16>(ctx, prm, stream);
  return launch_tc<kSplit>(ctx, prm, stream);
}

}  // namespace mfa
