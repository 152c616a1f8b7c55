// Adjoint of the micro-model decode: dP_abc = sum_{k,j,i} R[k][j][i] N_a(u_i) N_b(v_j) N_c(w_k).
// (Entry point; the common case runs on the dense contraction kernel of contract3.cu. The banded
// gather kernel below is the general path for shapes that kernel does not take: shared memory
// beyond its budget, or the fused gradient on sample rows the TMA path cannot load.)
//
// The gradient of 0.5*||decode(P) - D||^2 with respect to the control points, i.e. the transposed
// contraction that makes the least-squares encode of Algorithm 1's model() a gradient method.
// One CTA per block (persistent queue); the block's samples stream through shared memory in
// z-slabs and the banded transposed products run as gathers:
//   x^T:  V[k][j][a] = sum_{i : a in band(i)} N_a(u_i) R[k][j][i]
//   y^T:  W[k][b][a] = sum_{j : b in band(j)} N_b(v_j) V[k][j][a]
//   z^T:  G[c][b][a] += sum_{k in slab : c in band(k)} N_c(w_k) W[k][b][a]
// The bands are contiguous sample ranges because spans grow with the sample index. The basis is
// recomputed from the knots in every CTA rather than stored. With control points given, R is
// formed in the kernel as decode_value(P) - D, slab by slab, without an HBM round trip.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"

namespace mfa {

namespace {

constexpr int kThreads = 256;
constexpr int kKnotStride = MFA_MAX_NCP + MFA_MAX_DEGREE + 1;

struct AdjSmem {
  int knots, boff, bN, lo, hi, P, G, T, U, R, total;
};

AdjSmem adj_layout(int pmax, int maxC, int maxN, int ks) {
  AdjSmem L;
  int o = 0;
  const int q = pmax + 1;
  L.knots = o; o += 3 * kKnotStride;
  L.boff = o;  o += 3 * maxN;
  L.bN = o;    o += 3 * maxN * q;
  L.lo = o;    o += 3 * MFA_MAX_NCP;
  L.hi = o;    o += 3 * MFA_MAX_NCP;
  o = (o + 3) & ~3;
  L.P = o;     o += maxC * maxC * maxC;
  L.G = o;     o += maxC * maxC * maxC;
  L.T = o;     o += maxC * std::max(maxC, maxN) * ks;   // T0 (forward) then W
  L.U = o;     o += maxC * maxN * ks;                   // U0 (forward) then V
  L.R = o;     o += maxN * maxN * ks;
  L.total = o;
  return L;
}

template <int PMAX>
__global__ void __launch_bounds__(kThreads) adjoint_kernel(AdjointParams prm, AdjSmem L, int ks) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item, s_bad;
  __shared__ BlockGeom s_g;
  constexpr int Q = PMAX + 1;
  const int tid = threadIdx.x;
  const int maxN = prm.bounds.max_nsamp;
  float* s_knots = sm + L.knots;
  int* s_boff = reinterpret_cast<int*>(sm + L.boff);
  float* s_bN = sm + L.bN;
  int* s_lo = reinterpret_cast<int*>(sm + L.lo);
  int* s_hi = reinterpret_cast<int*>(sm + L.hi);
  float* s_P = sm + L.P;
  float* s_G = sm + L.G;
  float* s_T = sm + L.T;
  float* s_U = sm + L.U;
  float* s_R = sm + L.R;
  const bool fused = prm.cps != nullptr;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = atomicAdd(prm.counter, 1u);
      s_bad = 0;
      if (s_item < prm.nblocks) {
        uint32_t bad = load_desc(prm.desc + s_item, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                                 prm.slot_stride, s_g);
        if (bad) { flag(prm.status, bad); s_bad = 1; }
      }
    }
    __syncthreads();
    if (s_item >= prm.nblocks) break;
    if (s_bad) continue;
    const BlockGeom g = s_g;
    const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int ncps = Cx * Cy * Cz;

    for (int a = 0; a < 3; ++a) {
      const int len = g.C[a] + g.p[a] + 1;
      for (int i = tid; i < len; i += blockDim.x) s_knots[a * kKnotStride + i] = prm.knots[g.knot_off[a] + i];
    }
    for (int e = tid; e < ncps; e += blockDim.x) {
      s_G[e] = 0.f;
      if (fused) s_P[e] = prm.cps[g.cp_off + e];
    }
    __syncthreads();
    if (tid < 3) {
      if (!knots_ok(s_knots + tid * kKnotStride, g.p[tid], g.C[tid])) {
        atomicOr(&s_bad, 1);
        flag(prm.status, MFA_DEV_BAD_KNOTS);
      }
    }
    // basis tables for every sample of every axis (n <= 64 per axis, 3*64 <= 256 threads)
    {
      const int a = tid < nx ? 0 : (tid < nx + ny ? 1 : (tid < nx + ny + nz ? 2 : -1));
      if (a >= 0) {
        const int i = a == 0 ? tid : (a == 1 ? tid - nx : tid - nx - ny);
        const float* t = s_knots + a * kKnotStride;
        const float u = sample_param(i, g.n[a]);
        const int s = find_span(t, g.p[a], g.C[a], u);
        float N[Q], dN[Q];
        basis_funs<PMAX>(t, g.p[a], s, u, N, dN);
        s_boff[a * maxN + i] = s - g.p[a];
#pragma unroll
        for (int r = 0; r < Q; ++r) s_bN[(a * maxN + i) * Q + r] = N[r];
      }
    }
    __syncthreads();
    if (s_bad) continue;
    // sample range of each control index: the i with boff_i <= c <= boff_i + p
    if (tid < Cx + Cy + Cz) {
      const int a = tid < Cx ? 0 : (tid < Cx + Cy ? 1 : 2);
      const int c = a == 0 ? tid : (a == 1 ? tid - Cx : tid - Cx - Cy);
      int lo = g.n[a], hi = -1;
      for (int i = 0; i < g.n[a]; ++i) {
        const int o = s_boff[a * maxN + i];
        if (o <= c && c <= o + g.p[a]) { lo = min(lo, i); hi = max(hi, i); }
      }
      s_lo[a * MFA_MAX_NCP + c] = lo;
      s_hi[a * MFA_MAX_NCP + c] = hi;
    }
    __syncthreads();

    for (int k0 = 0; k0 < nz; k0 += ks) {
      const int kc = min(ks, nz - k0);
      // ---- residual slab R[kl][j][i] ----
      const float* src = prm.residual + (int64_t)g.slot * prm.slot_stride + (int64_t)k0 * ny * nx;
      if (fused) {
        const int plane = Cx * Cy;
        for (int e = tid; e < plane * kc; e += blockDim.x) {  // stage z (value)
          const int kl = e / plane, ab = e - kl * plane;
          const int oz = s_boff[2 * maxN + k0 + kl];
          const float* Nz = s_bN + (2 * maxN + k0 + kl) * Q;
          float acc = 0.f;
#pragma unroll
          for (int d = 0; d < Q; ++d)
            if (d <= g.p[2]) acc = fmaf(s_P[(oz + d) * plane + ab], Nz[d], acc);
          s_T[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < Cx * ny * kc; e += blockDim.x) {  // stage y (value)
          const int a = e % Cx, r = e / Cx, j = r % ny, kl = r / ny;
          const int oy = s_boff[maxN + j];
          const float* Ny = s_bN + (maxN + j) * Q;
          float acc = 0.f;
#pragma unroll
          for (int d = 0; d < Q; ++d)
            if (d <= g.p[1]) acc = fmaf(s_T[(kl * Cy + oy + d) * Cx + a], Ny[d], acc);
          s_U[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < nx * ny * kc; e += blockDim.x) {  // stage x (value) minus data
          const int i = e % nx, r = e / nx;
          const int ox = s_boff[i];
          const float* Nx = s_bN + i * Q;
          float acc = 0.f;
#pragma unroll
          for (int d = 0; d < Q; ++d)
            if (d <= g.p[0]) acc = fmaf(s_U[r * Cx + ox + d], Nx[d], acc);
          s_R[e] = acc - src[e];
        }
      } else {
        for (int e = tid; e < nx * ny * kc; e += blockDim.x) s_R[e] = src[e];
      }
      __syncthreads();
      // ---- x^T: V[kl][j][a] (stored in U) ----
      for (int e = tid; e < Cx * ny * kc; e += blockDim.x) {
        const int a = e % Cx, r = e / Cx;
        const int lo = s_lo[a], hi = s_hi[a];
        float acc = 0.f;
        for (int i = lo; i <= hi; ++i) acc = fmaf(s_bN[i * Q + (a - s_boff[i])], s_R[r * nx + i], acc);
        s_U[e] = acc;
      }
      __syncthreads();
      // ---- y^T: W[kl][b][a] (stored in T) ----
      for (int e = tid; e < Cx * Cy * kc; e += blockDim.x) {
        const int a = e % Cx, r = e / Cx, b = r % Cy, kl = r / Cy;
        const int lo = s_lo[MFA_MAX_NCP + b], hi = s_hi[MFA_MAX_NCP + b];
        float acc = 0.f;
        for (int j = lo; j <= hi; ++j)
          acc = fmaf(s_bN[(maxN + j) * Q + (b - s_boff[maxN + j])], s_U[(kl * ny + j) * Cx + a], acc);
        s_T[e] = acc;
      }
      __syncthreads();
      // ---- z^T: accumulate into G ----
      for (int e = tid; e < ncps; e += blockDim.x) {
        const int ab = e % (Cx * Cy), c = e / (Cx * Cy);
        const int lo = max(s_lo[2 * MFA_MAX_NCP + c], k0), hi = min(s_hi[2 * MFA_MAX_NCP + c], k0 + kc - 1);
        float acc = s_G[e];
        for (int k = lo; k <= hi; ++k)
          acc = fmaf(s_bN[(2 * maxN + k) * Q + (c - s_boff[2 * maxN + k])], s_T[(k - k0) * Cx * Cy + ab], acc);
        s_G[e] = acc;
      }
      __syncthreads();
    }
    for (int e = tid; e < ncps; e += blockDim.x) prm.grad[g.cp_off + e] = s_G[e];
  }
}

template <int PMAX>
cudaError_t launch_adj(mfa_ctx* ctx, const AdjointParams& prm, const AdjSmem& L, int ks, cudaStream_t stream) {
  auto kern = adjoint_kernel<PMAX>;
  const size_t smem = (size_t)L.total * 4;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(ctx->num_sms * occ, prm.nblocks));
  kern<<<grid, kThreads, smem, stream>>>(prm, L, ks);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

int adjoint(mfa_ctx* ctx, const AdjointParams& prm, cudaStream_t stream) {
  // the dense contraction kernel first (N^T R, or M P - N^T D for the fused gradient); this banded
  // gather kernel only serves block shapes whose buffers do not fit that kernel's shared memory. The
  // 16-bit precisions run on the tensor-core contraction only.
  {
    ContractParams c;
    std::memset(&c, 0, sizeof(c));
    c.mode = prm.cps ? kGradient : kAdjoint;
    c.nblocks = prm.nblocks;
    c.desc = prm.desc;
    c.knots = prm.knots;
    c.knots_len = prm.knots_len;
    c.bounds = prm.bounds;
    c.cps = prm.cps;
    c.x = prm.residual;
    c.slot_stride = prm.slot_stride;
    c.nslots = prm.nslots;
    c.out = prm.grad;
    c.cps_len = prm.cps_len;
    c.status = prm.status;
    c.counter = prm.counter;
    c.maxC = prm.bounds.max_ncp;
    c.maxN = prm.bounds.max_nsamp;
    c.pmax = prm.bounds.max_degree;
    c.rows32 = prm.bounds.max_nsamp == 32;
    if (prm.precision != MFA_PREC_FP32) return contract_tc(ctx, c, prm.precision, stream);
    const int rc = contract3(ctx, c, stream);
    if (rc != MFA_ERR_CAPACITY && rc != MFA_ERR_UNSUPPORTED) return rc;
  }
  const int maxN = prm.bounds.max_nsamp, maxC = prm.bounds.max_ncp, pmax = prm.bounds.max_degree;
  int ks = std::min(8, maxN);
  AdjSmem L = adj_layout(pmax, maxC, maxN, ks);
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = adj_layout(pmax, maxC, maxN, ks);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  cudaError_t e;
  switch (pmax) {
    case 1: e = launch_adj<1>(ctx, prm, L, ks, stream); break;
    case 2: e = launch_adj<2>(ctx, prm, L, ks, stream); break;
    case 3: e = launch_adj<3>(ctx, prm, L, ks, stream); break;
    default: return MFA_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
