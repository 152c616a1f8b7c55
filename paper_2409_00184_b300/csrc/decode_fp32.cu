// Batched micro-model decode on the CUDA cores in FP32 (value + parametric gradient).
//
// Each micro-block's model f(u,v,w) = sum N_a(u) N_b(v) N_c(w) P_abc (Sec. 4.2) is evaluated on
// its regular sample grid as three banded mode products, so each output costs p+1 FMAs per
// stage instead of (p+1)^3:
//   stage z:  T0[k][b][a] = sum_c P[c][b][a] N_c(w_k),     T1 = same with N'_c
//   stage y:  U0[k][j][a] = sum_b T0[k][b][a] N_b(v_j),    U1 = T0 with N'_b,  U2 = T1 with N_b
//   stage x:  (f, f_u, f_v, f_w)[k][j][i] = sum_a (U0 N_a, U0 N'_a, U1 N_a, U2 N_a)(u_i)
// Work unit = (block, slab of `ks` z-planes); a persistent grid pulls units from an atomic
// counter. Control points, basis tables and the stage outputs of one unit live in shared
// memory; only the final float4 per voxel goes to HBM (coalesced 512-byte rows per warp).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mfa {

struct DecodeSmem {
  int knots, boff, bN, bdN, P, T0, T1, U0, U1, U2, total;  // offsets in 4-byte words
};

static DecodeSmem decode_smem_layout(int pmax, int maxC, int maxN, int ks) {
  DecodeSmem L;
  int o = 0;
  const int q = pmax + 1;
  L.knots = o; o += 3 * (MFA_MAX_NCP + MFA_MAX_DEGREE + 1);
  L.boff = o;  o += 3 * maxN;
  L.bN = o;    o += 3 * maxN * q;
  L.bdN = o;   o += 3 * maxN * q;
  o = (o + 3) & ~3;
  L.P = o;     o += maxC * maxC * maxC;
  L.T0 = o;    o += maxC * maxC * ks;
  L.T1 = o;    o += maxC * maxC * ks;
  L.U0 = o;    o += maxC * maxN * ks;
  L.U1 = o;    o += maxC * maxN * ks;
  L.U2 = o;    o += maxC * maxN * ks;
  L.total = o;
  return L;
}

template <int PMAX, bool VALUE_ONLY>
__global__ void __launch_bounds__(kDecodeThreads)
decode_fp32_kernel(DecodeParams prm, DecodeSmem L) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_unit, s_block, s_bad;
  __shared__ BlockGeom s_g;
  constexpr int Q = PMAX + 1;
  const int tid = threadIdx.x;
  const int maxN = prm.bounds.max_nsamp;
  float* s_knots = sm + L.knots;
  int* s_boff = reinterpret_cast<int*>(sm + L.boff);
  float* s_bN = sm + L.bN;
  float* s_bdN = sm + L.bdN;
  float* s_P = sm + L.P;
  float* s_T0 = sm + L.T0;
  float* s_T1 = sm + L.T1;
  float* s_U0 = sm + L.U0;
  float* s_U1 = sm + L.U1;
  float* s_U2 = sm + L.U2;

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
      int b = -1;
      if (unit < total_units) {
        const int item = (int)(unit / prm.slabs);
        b = prm.list ? prm.list[item] : item;
        uint32_t bad = 0;
        const bool list_slots = (prm.flags & MFA_DECODE_LIST_SLOTS) != 0;
        if (b < 0 || b >= prm.nblocks) bad = MFA_DEV_BAD_LIST;
        else bad = load_desc(prm.desc + b, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                             prm.slot_stride, s_g, !list_slots);
        if (!bad && list_slots) {
          if (item >= prm.nslots) bad = MFA_DEV_BAD_RANGE;
          s_g.slot = item;
        }
        if (bad) { flag(prm.status, bad); s_bad = 1; }
      }
      s_block = b;
    }
    __syncthreads();
    if ((int64_t)s_unit >= total_units) break;
    if (s_bad) continue;
    const BlockGeom g = s_g;
    const int slab = (int)((int64_t)s_unit % prm.slabs);
    const int k0 = slab * prm.ks;
    if (k0 >= g.n[2]) continue;
    const int kc = min(prm.ks, g.n[2] - k0);
    const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2];
    const int nx = g.n[0], ny = g.n[1];

    // knots -> shared
    for (int a = 0; a < 3; ++a) {
      const int len = g.C[a] + g.p[a] + 1;
      for (int i = tid; i < len; i += blockDim.x)
        s_knots[a * (MFA_MAX_NCP + MFA_MAX_DEGREE + 1) + i] = prm.knots[g.knot_off[a] + i];
    }
    // control points -> shared (coalesced)
    const int ncps = Cx * Cy * Cz;
    const float* gP = prm.cps + g.cp_off;
    for (int e = tid; e < ncps; e += blockDim.x) s_P[e] = gP[e];
    __syncthreads();
    if (tid < 3) {
      const float* t = s_knots + tid * (MFA_MAX_NCP + MFA_MAX_DEGREE + 1);
      if (!knots_ok(t, g.p[tid], g.C[tid])) { atomicOr(&s_bad, 1); flag(prm.status, MFA_DEV_BAD_KNOTS); }
    }
    // basis tables: x (nx samples), y (ny samples), z (the slab's kc samples)
    {
      int a = -1, i = 0, smp = 0;
      if (tid < nx) { a = 0; i = tid; smp = tid; }
      else if (tid < nx + ny) { a = 1; i = tid - nx; smp = i; }
      else if (tid < nx + ny + kc) { a = 2; i = tid - nx - ny; smp = k0 + i; }
      if (a >= 0) {
        const float* t = s_knots + a * (MFA_MAX_NCP + MFA_MAX_DEGREE + 1);
        const float u = sample_param(smp, g.n[a]);
        const int s = find_span(t, g.p[a], g.C[a], u);
        float N[Q], dN[Q];
        basis_funs<PMAX>(t, g.p[a], s, u, N, dN);
        s_boff[a * maxN + i] = s - g.p[a];
#pragma unroll
        for (int r = 0; r < Q; ++r) {
          s_bN[(a * maxN + i) * Q + r] = N[r];
          s_bdN[(a * maxN + i) * Q + r] = dN[r];
        }
      }
    }
    __syncthreads();
    if (s_bad) continue;

    // stage z
    {
      const int pz = g.p[2];
      const int plane = Cx * Cy;
      const int tot = plane * kc;
      for (int e = tid; e < tot; e += blockDim.x) {
        const int kl = e / plane;
        const int ab = e - kl * plane;
        const int oz = s_boff[2 * maxN + kl];
        const float* Nz = s_bN + (2 * maxN + kl) * Q;
        const float* dNz = s_bdN + (2 * maxN + kl) * Q;
        float t0 = 0.f, t1 = 0.f;
#pragma unroll
        for (int d = 0; d < Q; ++d) {
          if (d <= pz) {
            const float pv = s_P[(oz + d) * plane + ab];
            t0 = fmaf(pv, Nz[d], t0);
            if (!VALUE_ONLY) t1 = fmaf(pv, dNz[d], t1);
          }
        }
        s_T0[e] = t0;
        if (!VALUE_ONLY) s_T1[e] = t1;
      }
    }
    __syncthreads();
    // stage y
    {
      const int py = g.p[1];
      const int tot = Cx * ny * kc;
      for (int e = tid; e < tot; e += blockDim.x) {
        const int a = e % Cx;
        const int r = e / Cx;  // kl * ny + j
        const int j = r % ny;
        const int kl = r / ny;
        const int oy = s_boff[maxN + j];
        const float* Ny = s_bN + (maxN + j) * Q;
        const float* dNy = s_bdN + (maxN + j) * Q;
        const float* T0 = s_T0 + (kl * Cy + oy) * Cx + a;
        const float* T1 = s_T1 + (kl * Cy + oy) * Cx + a;
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
        for (int d = 0; d < Q; ++d) {
          if (d <= py) {
            const float tv = T0[d * Cx];
            u0 = fmaf(tv, Ny[d], u0);
            if (!VALUE_ONLY) {
              u1 = fmaf(tv, dNy[d], u1);
              u2 = fmaf(T1[d * Cx], Ny[d], u2);
            }
          }
        }
        s_U0[e] = u0;
        if (!VALUE_ONLY) { s_U1[e] = u1; s_U2[e] = u2; }
      }
    }
    __syncthreads();
    // stage x + store: thread owns one x sample, loops over (k, j) rows
    {
      const int rows_per_pass = blockDim.x / nx;
      const int i = tid % nx;
      const int r0 = tid / nx;
      if (r0 < rows_per_pass) {
        const int px = g.p[0];
        const int ox = s_boff[i];
        float Nx[Q], dNx[Q];
#pragma unroll
        for (int d = 0; d < Q; ++d) {
          Nx[d] = s_bN[i * Q + d];
          dNx[d] = s_bdN[i * Q + d];
        }
        const int rows = ny * kc;
        const int64_t base = (int64_t)g.slot * prm.slot_stride + (int64_t)k0 * ny * nx + i;
        for (int r = r0; r < rows; r += rows_per_pass) {
          const float* u0 = s_U0 + r * Cx + ox;
          float f = 0.f, fu = 0.f, fv = 0.f, fw = 0.f;
          if (VALUE_ONLY) {
#pragma unroll
            for (int d = 0; d < Q; ++d)
              if (d <= px) f = fmaf(u0[d], Nx[d], f);
            __stcs(prm.cache + base + (int64_t)r * nx, f);
          } else {
            const float* u1 = s_U1 + r * Cx + ox;
            const float* u2 = s_U2 + r * Cx + ox;
#pragma unroll
            for (int d = 0; d < Q; ++d) {
              if (d <= px) {
                const float a0 = u0[d];
                f = fmaf(a0, Nx[d], f);
                fu = fmaf(a0, dNx[d], fu);
                fv = fmaf(u1[d], Nx[d], fv);
                fw = fmaf(u2[d], Nx[d], fw);
              }
            }
            __stcs(reinterpret_cast<float4*>(prm.cache) + base + (int64_t)r * nx, make_float4(f, fu, fv, fw));
          }
        }
      }
    }
  }
}

template <int PMAX, bool VO>
static cudaError_t launch_one(mfa_ctx* ctx, const DecodeParams& prm, const DecodeSmem& L, int ctas_per_sm,
                              cudaStream_t stream) {
  auto kern = decode_fp32_kernel<PMAX, VO>;
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
  int ks = tune.ks > 0 ? std::min(tune.ks, maxN) : 8;
  DecodeSmem L = decode_smem_layout(pmax, maxC, maxN, ks);
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = decode_smem_layout(pmax, maxC, maxN, ks);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  prm.ks = ks;
  prm.slabs = (maxN + ks - 1) / ks;
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  const bool vo = (prm.flags & MFA_DECODE_VALUE_ONLY) != 0;
  cudaError_t e;
  switch (pmax) {
    case 1: e = vo ? launch_one<1, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<1, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    case 2: e = vo ? launch_one<2, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<2, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    case 3: e = vo ? launch_one<3, true>(ctx, prm, L, tune.ctas_per_sm, stream) : launch_one<3, false>(ctx, prm, L, tune.ctas_per_sm, stream); break;
    default: return MFA_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
