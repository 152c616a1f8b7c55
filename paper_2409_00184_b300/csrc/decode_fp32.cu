// Batched micro-model decode on the CUDA cores in FP32 (value + parametric gradient).
//
// Each micro-block's model f(u,v,w) = sum N_a(u) N_b(v) N_c(w) P_abc (Sec. 4.2) is evaluated on
// its regular sample grid as three banded mode products, so each output costs p+1 FMAs per
// stage instead of (p+1)^3:
//   stage z:  T[k][b][a] = (sum_c P[c][b][a] N_c(w_k), same with N'_c)              (float2)
//   stage y:  U[k][j][a] = (T0 N_b(v_j), T0 N'_b(v_j), T1 N_b(v_j)) summed over b      (float4)
//   stage x:  (f, f_u, f_v, f_w)[k][j][i] = sum_a (U0 N_a, U0 N'_a, U1 N_a, U2 N_a)(u_i)
// Work unit = (block, group of slabs of `ks` z-planes each); a persistent grid pulls units from an
// atomic counter. A unit loads the block's knots and control points and builds its basis tables
// once, then runs the three stages slab by slab. Control points, basis tables and the stage outputs
// live in shared memory; only the final float4 per voxel goes to HBM (coalesced 512-byte rows per
// warp).
// Stage outputs are interleaved so stage x reads one 16-byte word per (row, control index), and
// the loops advance their (k, j, a) indices incrementally instead of dividing.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mfa {

struct DecodeSmem {
  int knots, boff, bN, bdN, T, P, U, total;  // offsets in 4-byte words
};

static int r4(int v) { return (v + 3) & ~3; }

constexpr int kUnitPlanes = 32;

__device__ __forceinline__ void compare_sample(const DecodeParams& prm, int64_t idx, float r, float& ksum,
                                               float& kcomp);
constexpr int kPrefetch = 8;  // rows per thread whose samples are loaded together (decode with comparison)  // z-planes per work unit (the set-up is shared by its slabs)

// [knots | basis tables | T | P | U]. With one slab per unit (`alias`), U (stage y output) overwrites
// P, which stage z has consumed; units of several slabs keep P for all of them.
static DecodeSmem decode_smem_layout(bool value_only, int maxC, int maxN, int ks, bool alias) {
  DecodeSmem L;
  int o = 0;
  L.knots = o; o += r4(3 * kKnotMax);
  L.boff = o;  o += r4(3 * maxN);
  L.bN = o;    o += 3 * maxN * 4;   // float4 per sample: N_{s-p..s} (zero padded)
  L.bdN = o;   o += 3 * maxN * 4;   // float4 per sample: N'
  L.T = o;     o += r4(maxC * maxC * ks * (value_only ? 1 : 2));
  const int pw = r4(maxC * maxC * maxC), uw = r4(maxC * maxN * ks * (value_only ? 1 : 4));
  L.P = o;
  if (alias) {
    L.U = o;
    o += std::max(pw, uw);
  } else {
    L.U = o + pw;
    o += pw + uw;
  }
  L.total = o;
  return L;
}

// LAYOUT of the cache: kLayoutRows [z][y][x], kLayoutCubes, kLayoutApron ([z][y][x] in rows of apron_pitch(n), planes of n + 1 rows)
enum CacheLayout { kLayoutRows = 0, kLayoutCubes = 1, kLayoutApron = 2 };

template <int PMAX, bool VALUE_ONLY, bool COMPARE, int LAYOUT>
__global__ void __launch_bounds__(kDecodeThreads, LAYOUT == kLayoutApron ? 4 : 0)  // 0: no minimum
decode_fp32_kernel(DecodeParams prm, DecodeSmem L) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_unit, s_bad, s_item;
  __shared__ double s_red[kDecodeThreads / 32];
  __shared__ BlockGeom s_g;
  constexpr int Q = PMAX + 1;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int maxN = prm.bounds.max_nsamp;
  float* s_knots = sm + L.knots;
  int* s_boff = reinterpret_cast<int*>(sm + L.boff);
  float4* s_bN = reinterpret_cast<float4*>(sm + L.bN);
  float4* s_bdN = reinterpret_cast<float4*>(sm + L.bdN);
  float* s_P = sm + L.P;

  int count = prm.list ? (prm.count ? *prm.count : prm.list_len) : prm.nblocks;
  if (prm.list && (count < 0 || count > prm.list_len)) {
    if (blockIdx.x == 0 && tid == 0) flag(prm.status, MFA_DEV_BAD_LIST);
    count = max(0, min(count, prm.list_len));
  }
  const int64_t total_units = (int64_t)count * prm.slabs;

  for (;;) {
    __syncthreads();  // previous unit finished with shared memory
    if (tid == 0) {
      s_unit = atomicAdd(prm.counter, 1u);
      s_bad = 0;
      const int64_t unit = s_unit;
      if (unit < total_units) {
        const int item = (int)(unit / prm.slabs);
        s_item = item;
        const int b = prm.list ? prm.list[item] : item;
        const bool list_slots = (prm.flags & MFA_DECODE_LIST_SLOTS) != 0;
        uint32_t bad = 0;
        if (b < 0 || b >= prm.nblocks) bad = MFA_DEV_BAD_LIST;
        else bad = load_desc(prm.desc + b, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                             prm.slot_stride, s_g, !list_slots);
        if (!bad && list_slots) {
          if (item >= prm.nslots) bad = MFA_DEV_BAD_RANGE;
          s_g.slot = item;
        }
        if (!bad && COMPARE && (int64_t)s_g.n[0] * s_g.n[1] * s_g.n[2] > prm.data_stride) bad = MFA_DEV_BAD_RANGE;
        if (!bad && (prm.flags & MFA_DECODE_CUBES) && ((s_g.n[0] | s_g.n[1] | s_g.n[2]) & 1)) bad = MFA_DEV_BAD_DESC;
        if (!bad && (prm.flags & MFA_DECODE_APRON) &&
            (int64_t)apron_pitch(s_g.n[0]) * (s_g.n[1] + 1) * (s_g.n[2] + 1) > prm.slot_stride)
          bad = MFA_DEV_BAD_RANGE;
        if (bad) { flag(prm.status, bad); s_bad = 1; }
      }
    }
    __syncthreads();
    if ((int64_t)s_unit >= total_units) break;
    if (s_bad) continue;
    const int part = (int)((int64_t)s_unit % prm.slabs);
    const int kz0 = part * prm.ks * prm.group;  // first z-plane of this unit
    const int nz = s_g.n[2];
    if (kz0 >= nz) continue;
    const int kzn = min(prm.ks * prm.group, nz - kz0);  // z-planes of this unit
    const int Cx = s_g.C[0], Cy = s_g.C[1], Cz = s_g.C[2];
    const int nx = s_g.n[0], ny = s_g.n[1];
    const int px = s_g.p[0], py = s_g.p[1], pz = s_g.p[2];

    // knots -> shared; control points -> shared (coalesced)
    if (tid < 3 * kKnotMax) {
      const int a = tid / kKnotMax, i = tid - a * kKnotMax;
      if (i < s_g.C[a] + s_g.p[a] + 1) s_knots[tid] = prm.knots[s_g.knot_off[a] + i];
    }
    const int ncps = Cx * Cy * Cz;
    const float* gP = prm.cps + s_g.cp_off;
    for (int e = tid; e < ncps; e += nthr) s_P[e] = __ldg(gP + e);
    __syncthreads();
    if (tid < 3 && !knots_ok(s_knots + tid * kKnotMax, s_g.p[tid], s_g.C[tid])) {
      atomicOr(&s_bad, 1);
      flag(prm.status, MFA_DEV_BAD_KNOTS);
    }
    // basis tables: x (nx samples), y (ny samples), z (the unit's kzn samples)
    for (int e = tid; e < nx + ny + kzn; e += nthr) {
      int a, i, smp;
      if (e < nx) { a = 0; i = e; smp = e; }
      else if (e < nx + ny) { a = 1; i = e - nx; smp = i; }
      else { a = 2; i = e - nx - ny; smp = kz0 + i; }
      {
        const float* t = s_knots + a * kKnotMax;
        const float u = sample_param(smp, s_g.n[a]);
        const int s = find_span(t, s_g.p[a], s_g.C[a], u);
        float N[4] = {0.f, 0.f, 0.f, 0.f}, dN[4] = {0.f, 0.f, 0.f, 0.f};
        float Nq[Q], dNq[Q];
        basis_funs<PMAX>(t, s_g.p[a], s, u, Nq, dNq);
#pragma unroll
        for (int r = 0; r < Q; ++r) { N[r] = Nq[r]; dN[r] = dNq[r]; }
        s_boff[a * maxN + i] = s - s_g.p[a];
        s_bN[a * maxN + i] = make_float4(N[0], N[1], N[2], N[3]);
        s_bdN[a * maxN + i] = make_float4(dN[0], dN[1], dN[2], dN[3]);
      }
    }
    __syncthreads();
    if (s_bad) continue;

    float ksum = 0.f, kcomp = 0.f;  // squared differences to the samples (COMPARE), Kahan-summed per thread
    for (int k0 = kz0; k0 < kz0 + kzn; k0 += prm.ks) {  // slabs of the unit
      const int kc = min(prm.ks, kz0 + kzn - k0);
      const int zt = 2 * maxN + (k0 - kz0);  // z-table row of the slab's first plane

      // ---- stage z: T[kl][b][a] over the slab, flat index e = kl*plane + ab ----
      {
        const int plane = Cx * Cy;
        const int tot = plane * kc;
        int kl = tid / plane, ab = tid - (tid / plane) * plane;
        for (int e = tid; e < tot; e += nthr) {
          const int oz = s_boff[zt + kl];
          const float4 Nz = s_bN[zt + kl];
          const float4 dNz = s_bdN[zt + kl];
          const float Nzv[4] = {Nz.x, Nz.y, Nz.z, Nz.w}, dNzv[4] = {dNz.x, dNz.y, dNz.z, dNz.w};
          const float* Pc = s_P + oz * plane + ab;
          float t0 = 0.f, t1 = 0.f;
#pragma unroll
          for (int d = 0; d < Q; ++d) {
            if (d <= pz) {
              const float pv = Pc[d * plane];
              t0 = fmaf(pv, Nzv[d], t0);
              if (!VALUE_ONLY) t1 = fmaf(pv, dNzv[d], t1);
            }
          }
          if (VALUE_ONLY) sm[L.T + e] = t0;
          else reinterpret_cast<float2*>(sm + L.T)[e] = make_float2(t0, t1);
          ab += nthr;
          while (ab >= plane) { ab -= plane; ++kl; }
        }
      }
      __syncthreads();
      // ---- stage y: U[kl][j][a]; thread keeps its column a, rows r = (kl, j) advance by step ----
      {
        const int step = nthr / Cx;
        const int g = tid / Cx;
        if (g < step) {
          const int a = tid - g * Cx;
          const int rows = ny * kc;
          int kl = g / ny, j = g - (g / ny) * ny;
          for (int r = g; r < rows; r += step) {
            const int oy = s_boff[maxN + j];
            const float4 Ny = s_bN[maxN + j];
            const float Nyv[4] = {Ny.x, Ny.y, Ny.z, Ny.w};
            const int tb = (kl * Cy + oy) * Cx + a;
            if (VALUE_ONLY) {
              float u0 = 0.f;
#pragma unroll
              for (int d = 0; d < Q; ++d)
                if (d <= py) u0 = fmaf(sm[L.T + tb + d * Cx], Nyv[d], u0);
              sm[L.U + r * Cx + a] = u0;
            } else {
              const float4 dNy = s_bdN[maxN + j];
              const float dNyv[4] = {dNy.x, dNy.y, dNy.z, dNy.w};
              const float2* T = reinterpret_cast<const float2*>(sm + L.T);
              float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
              for (int d = 0; d < Q; ++d) {
                if (d <= py) {
                  const float2 tv = T[tb + d * Cx];
                  u0 = fmaf(tv.x, Nyv[d], u0);
                  u1 = fmaf(tv.x, dNyv[d], u1);
                  u2 = fmaf(tv.y, Nyv[d], u2);
                }
              }
              reinterpret_cast<float4*>(sm + L.U)[r * Cx + a] = make_float4(u0, u1, u2, 0.f);
            }
            j += step;
            while (j >= ny) { j -= ny; ++kl; }
          }
        }
      }
      __syncthreads();
      // ---- stage x + store: thread owns one x sample, loops over (k, j) rows ----
      {
        const int rows_per_pass = nthr / nx;
        const int i = tid % nx;
        const int r0 = tid / nx;
        if (r0 < rows_per_pass) {
          const int ox = s_boff[i];
          const float4 Nx4 = s_bN[i], dNx4 = s_bdN[i];
          const float Nx[4] = {Nx4.x, Nx4.y, Nx4.z, Nx4.w}, dNx[4] = {dNx4.x, dNx4.y, dNx4.z, dNx4.w};
          const int rows = ny * kc;
          const int64_t base = (int64_t)s_g.slot * prm.slot_stride + (int64_t)k0 * ny * nx + i;
          // cache index of row r's voxel: [z][y][x], the cube layout, or [z][y][x] with rows of
          // apron_pitch(nx) and planes of ny + 1 rows (apron)
          const int64_t sbase = (int64_t)s_g.slot * prm.slot_stride;
          const float inv_ny = 1.0f / (float)ny;
          // apron: row r = kl * ny + j of the chunk sits at ((k0 + kl) * (ny + 1) + j) * ax + i, which is
          // a0 + (r + kl) * ax
          // (offsets inside a slot stay below 65^3, so 32 bits hold them)
          const int ax = apron_pitch(nx), a0 = k0 * (ny + 1) * ax + i;
          auto cidx = [&](int r) -> int64_t {
            if (LAYOUT == kLayoutRows) return base + (int64_t)r * nx;
            const int kl = __float2int_rz(((float)r + 0.5f) * inv_ny);  // r / ny, exact for r < 2^12
            if (LAYOUT == kLayoutCubes) return sbase + cube_index(i, r - kl * ny, k0 + kl, nx, ny);
            return sbase + (a0 + (r + kl) * ax);
          };
          const int64_t dbase = COMPARE ? (int64_t)s_g.slot * prm.data_stride + (int64_t)k0 * ny * nx + i : 0;
          // rows in chunks of kPrefetch per thread: with COMPARE the chunk's samples D are loaded before its
          // arithmetic, so the loads overlap instead of each row waiting for its own
          if (COMPARE) {
            for (int rc = r0; rc < rows; rc += kPrefetch * rows_per_pass) {
              float dpre[kPrefetch];
#pragma unroll
              for (int q = 0; q < kPrefetch; ++q) {
                const int r = rc + q * rows_per_pass;
                dpre[q] = r < rows ? __ldg(prm.data + dbase + (int64_t)r * nx) : 0.f;
              }
#pragma unroll
              for (int q = 0; q < kPrefetch; ++q) {
                const int r = rc + q * rows_per_pass;
                if (r >= rows) break;
                float f = 0.f;
                if (VALUE_ONLY) {
                  const float* U = sm + L.U + ox;
#pragma unroll
                  for (int d = 0; d < Q; ++d)
                    if (d <= px) f = fmaf(U[r * Cx + d], Nx[d], f);
                  __stcs(prm.cache + cidx(r), f);
                } else {
                  const float4* U = reinterpret_cast<const float4*>(sm + L.U) + ox;
                  float fu = 0.f, fv = 0.f, fw = 0.f;
#pragma unroll
                  for (int d = 0; d < Q; ++d) {
                    if (d <= px) {
                      const float4 uv = U[r * Cx + d];
                      f = fmaf(uv.x, Nx[d], f);
                      fu = fmaf(uv.x, dNx[d], fu);
                      fv = fmaf(uv.y, Nx[d], fv);
                      fw = fmaf(uv.z, Nx[d], fw);
                    }
                  }
                  __stcs(reinterpret_cast<float4*>(prm.cache) + cidx(r),
                         make_float4(f, fu, fv, fw));
                }
                compare_sample(prm, dbase + (int64_t)r * nx, f - dpre[q], ksum, kcomp);
              }
            }
          } else if (VALUE_ONLY) {
            const float* U = sm + L.U + ox;
            for (int r = r0; r < rows; r += rows_per_pass) {
              float f = 0.f;
#pragma unroll
              for (int d = 0; d < Q; ++d)
                if (d <= px) f = fmaf(U[r * Cx + d], Nx[d], f);
              __stcs(prm.cache + cidx(r), f);
            }
          } else {
            const float4* U = reinterpret_cast<const float4*>(sm + L.U) + ox;
            float4* out = reinterpret_cast<float4*>(prm.cache);
            for (int r = r0; r < rows; r += rows_per_pass) {
              float f = 0.f, fu = 0.f, fv = 0.f, fw = 0.f;
#pragma unroll
              for (int d = 0; d < Q; ++d) {
                if (d <= px) {
                  const float4 uv = U[r * Cx + d];
                  f = fmaf(uv.x, Nx[d], f);
                  fu = fmaf(uv.x, dNx[d], fu);
                  fv = fmaf(uv.y, Nx[d], fv);
                  fw = fmaf(uv.z, Nx[d], fw);
                }
              }
              __stcs(out + cidx(r), make_float4(f, fu, fv, fw));
            }
          }
        }
      }
    }
    if (COMPARE && prm.sq) {  // the unit's sum of squared differences, added to its item in FP64
      double v = (double)ksum - (double)kcomp;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nthr / 32; ++w) tot += s_red[w];
        atomicAdd(prm.sq + s_item, tot);
      }
    }
  }
}

// The difference r = f - D of one decoded voxel: written when asked, r^2 into the thread's Kahan sum.
__device__ __forceinline__ void compare_sample(const DecodeParams& prm, int64_t idx, float r, float& ksum,
                                               float& kcomp) {
  if (prm.residual) __stcs(prm.residual + idx, r);
  const float y = r * r - kcomp;
  const float t = ksum + y;
  kcomp = (t - ksum) - y;
  ksum = t;
}

// RMSE of every selected item from its sum of squared differences: sqrt(sum / voxels), NaN for an
// item whose block failed its checks (it was not decoded).
__global__ void rmse_finish_kernel(DecodeParams prm, int max_items) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  int count = prm.list ? (prm.count ? *prm.count : prm.list_len) : prm.nblocks;
  count = max(0, min(count, max_items));
  if (item >= count) return;
  const int b = prm.list ? prm.list[item] : item;
  BlockGeom g;
  const bool list_slots = (prm.flags & MFA_DECODE_LIST_SLOTS) != 0;
  if (b < 0 || b >= prm.nblocks ||
      load_desc(prm.desc + b, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots, prm.slot_stride, g, !list_slots)) {
    prm.sq[item] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  const double vox = (double)g.n[0] * g.n[1] * g.n[2];
  prm.sq[item] = sqrt(prm.sq[item] / vox);
}

template <int PMAX, bool VO>
static cudaError_t launch_one(mfa_ctx* ctx, const DecodeParams& prm, const DecodeSmem& L, int ctas_per_sm,
                              cudaStream_t stream) {
  const int layout = (prm.flags & MFA_DECODE_CUBES) ? kLayoutCubes : (prm.flags & MFA_DECODE_APRON) ? kLayoutApron : kLayoutRows;
  auto pick = [&](auto rows, auto cubes, auto apron) { return layout == kLayoutCubes ? cubes : layout == kLayoutApron ? apron : rows; };
  auto kern = prm.data ? pick(decode_fp32_kernel<PMAX, VO, true, kLayoutRows>, decode_fp32_kernel<PMAX, VO, true, kLayoutCubes>,
                              decode_fp32_kernel<PMAX, VO, true, kLayoutApron>)
                       : pick(decode_fp32_kernel<PMAX, VO, false, kLayoutRows>, decode_fp32_kernel<PMAX, VO, false, kLayoutCubes>,
                              decode_fp32_kernel<PMAX, VO, false, kLayoutApron>);
  const size_t smem = (size_t)L.total * 4;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kDecodeThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
  const int grid = std::max(1, ctx->num_sms * occ);
  kern<<<grid, kDecodeThreads, smem, stream>>>(prm, L);
  ctx->launches++;
  return cudaGetLastError();
}

int decode_fp32(mfa_ctx* ctx, DecodeParams prm, const DecodeTuning& tune, cudaStream_t stream) {
  const int maxN = prm.bounds.max_nsamp, maxC = prm.bounds.max_ncp, pmax = prm.bounds.max_degree;
  const bool vo = (prm.flags & MFA_DECODE_VALUE_ONLY) != 0;
  // default slab depth from the tiling sweep on 32^3 blocks: 4 planes, 2 when C > 16 (larger T and U)
  int ks = tune.ks > 0 ? std::min(tune.ks, maxN) : std::min(maxC > 16 ? 2 : 4, maxN);
  // units of kUnitPlanes z-planes (several slabs) share one set-up of knots, control points and basis
  // tables; when P and U do not both fit, one slab per unit with U over P
  int group = std::max(1, std::min(kUnitPlanes, maxN) / ks);
  DecodeSmem L = decode_smem_layout(vo, maxC, maxN, ks, group == 1);
  if ((size_t)L.total * 4 > kMaxDynSmem && group > 1) {
    group = 1;
    L = decode_smem_layout(vo, maxC, maxN, ks, true);
  }
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = decode_smem_layout(vo, maxC, maxN, ks, true);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  prm.ks = ks;
  prm.group = group;
  prm.slabs = (maxN + ks * group - 1) / (ks * group);
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  const int max_items = prm.list ? prm.list_len : prm.nblocks;
  if (prm.data && prm.sq && cudaMemsetAsync(prm.sq, 0, sizeof(double) * (size_t)max_items, stream) != cudaSuccess)
    return MFA_ERR_CUDA;
  cudaError_t e;
  switch (pmax) {
    case 1: e = vo ? launch_one<1, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<1, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    case 2: e = vo ? launch_one<2, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<2, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    case 3: e = vo ? launch_one<3, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<3, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    default: return MFA_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return MFA_ERR_CUDA;
  if (prm.data && prm.sq && max_items > 0) {
    rmse_finish_kernel<<<(max_items + 255) / 256, 256, 0, stream>>>(prm, max_items);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) return MFA_ERR_CUDA;
  }
  return MFA_OK;
}

}  // namespace mfa
