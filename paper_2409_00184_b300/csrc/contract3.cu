// Transposed three-axis contraction of per-block sample grids, shared by the least-squares fit and
// the adjoint:
//     Y[c][b][a] = sum_{k,j,i} X[k][j][i] Ax[i][a] Ay[j][b] Az[k][c]
//   kFit:      A = (N^T N)^{-1} N^T per axis (from the encode plan) -> least-squares control points,
//              then optionally the FP64 RMSE of the fitted model over the samples (Table 1's metric);
//   kAdjoint:  A = N (collocation matrix, built from the knots in the CTA) -> N^T R;
//   kGradient: G = (M_x (x) M_y (x) M_z) P - N^T D with M = N^T N, the gradient of
//              0.5*||decode(P) - D||^2 (= N^T (N P - D)) without a forward decode of the samples.
// One CTA per block, persistent queue. The grid streams through in z-slabs of ks planes:
//   x:  Y1[(k,j)][a] = sum_i X[k][j][i] Ax[i][a]   thread per sample row, all columns in registers,
//                                                  the row read with 16-byte loads, Ax rows broadcast
//   y:  Y2[k][b][a]  = sum_j Y1[(k,j)][a] Ay[j][b]  4 columns b per thread
//   z:  Y[c][b][a]  += sum_k Y2[k][b][a] Az[k][c]   4 columns c per thread
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

constexpr int kThreads = 256;

struct C3Smem {
  int A[3], M[3], tab[3], knots, Y1, Y2, Y, P, Z, total;  // offsets in 4-byte words
};

int round4(int v) { return (v + 3) & ~3; }

C3Smem c3_layout(int mode, int CP, int maxC, int maxN, int ks, bool rmse) {
  const int CPs = (CP % 8 == 0) ? CP + 4 : CP;
  C3Smem L;
  int o = 0;
  for (int a = 0; a < 3; ++a) { L.A[a] = o; o += maxN * CP; }
  for (int a = 0; a < 3; ++a) { L.M[a] = o; if (mode == kGradient) o += maxC * maxC; }
  for (int a = 0; a < 3; ++a) { L.tab[a] = o; if (mode == kFit && rmse) o += maxN * (int)(sizeof(TabEntry) / 4); }
  L.knots = o; if (mode != kFit) o += 3 * kKnotMax;
  o = round4(o);
  L.Y1 = o; o += ks * maxN * CPs;
  L.Y2 = o; o += round4(ks * maxC * maxC);
  L.Y = o;  o += round4(maxC * maxC * maxC);
  L.P = o;  if (mode == kGradient) o += round4(maxC * maxC * maxC);
  L.Z = o;  if (mode == kGradient) o += round4(maxC * maxC * maxC);
  L.total = o;
  return L;
}

template <int CP>
__global__ void __launch_bounds__(kThreads) contract3_kernel(ContractParams prm, C3Smem L, int ks, int vec_ok) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item, s_bad, s_slot;
  __shared__ int s_p[3], s_C[3], s_n[3], s_cls[3];
  __shared__ int64_t s_cpoff, s_koff[3];
  __shared__ double s_red[kThreads / 32];
  constexpr int CPs = (CP % 8 == 0) ? CP + 4 : CP;
  constexpr int Q4 = CP / 4;
  const int tid = threadIdx.x;
  const int mode = prm.mode;

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = atomicAdd(prm.counter, 1u);
      s_bad = 0;
      if (s_item < prm.nblocks) {
        if (mode == kFit) {
          const EncItem it = prm.items[s_item];
          for (int a = 0; a < 3; ++a) {
            const EncClass& c = prm.classes[it.cls[a]];
            s_p[a] = c.p; s_C[a] = c.C; s_n[a] = c.n; s_cls[a] = it.cls[a];
          }
          s_slot = it.slot;
          s_cpoff = it.cp_off;
        } else {
          BlockGeom g;
          const uint32_t bad = load_desc(prm.desc + s_item, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                                         prm.slot_stride, g);
          if (bad) {
            flag(prm.status, bad);
            s_bad = 1;
          } else {
            for (int a = 0; a < 3; ++a) { s_p[a] = g.p[a]; s_C[a] = g.C[a]; s_n[a] = g.n[a]; s_koff[a] = g.knot_off[a]; }
            s_slot = g.slot;
            s_cpoff = g.cp_off;
          }
        }
      }
    }
    __syncthreads();
    if (s_item >= prm.nblocks) break;
    if (s_bad) continue;
    const int Cx = s_C[0], Cy = s_C[1], Cz = s_C[2];
    const int nx = s_n[0], ny = s_n[1], nz = s_n[2];
    const int plane = Cx * Cy, ncps = plane * Cz;
    const int64_t cp_off = s_cpoff;
    const float* X = prm.x + (int64_t)s_slot * prm.slot_stride;
    float* Ax = sm + L.A[0];
    float* Ay = sm + L.A[1];
    float* Az = sm + L.A[2];

    // ---- set-up: the three n x CP matrices (zero-padded columns) ----
    if (mode == kFit) {
      for (int a = 0; a < 3; ++a) {
        const EncClass& c = prm.classes[s_cls[a]];
        float* A = sm + L.A[a];
        for (int e = tid; e < c.n * CP; e += blockDim.x) {
          const int i = e / CP, col = e - i * CP;
          A[e] = col < c.C ? prm.pinv[c.pinv_off + i * c.C + col] : 0.f;
        }
        if (prm.rmse) {
          TabEntry* tb = reinterpret_cast<TabEntry*>(sm + L.tab[a]);
          for (int e = tid; e < c.n; e += blockDim.x) tb[e] = prm.tabs[c.tab_off + e];
        }
      }
    } else {
      float* kn = sm + L.knots;
      for (int a = 0; a < 3; ++a) {
        for (int i = tid; i < s_C[a] + s_p[a] + 1; i += blockDim.x) kn[a * kKnotMax + i] = prm.knots[s_koff[a] + i];
        for (int e = tid; e < s_n[a] * CP; e += blockDim.x) sm[L.A[a] + e] = 0.f;
      }
      __syncthreads();
      if (tid < 3 && !knots_ok(kn + tid * kKnotMax, s_p[tid], s_C[tid])) {
        atomicOr(&s_bad, 1);
        flag(prm.status, MFA_DEV_BAD_KNOTS);
      }
      const int a = tid < nx ? 0 : (tid < nx + ny ? 1 : (tid < nx + ny + nz ? 2 : -1));
      if (a >= 0) {
        const int i = a == 0 ? tid : (a == 1 ? tid - nx : tid - nx - ny);
        const float* t = kn + a * kKnotMax;
        const float u = sample_param(i, s_n[a]);
        const int s = find_span(t, s_p[a], s_C[a], u);
        float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
        basis_funs<MFA_MAX_DEGREE>(t, s_p[a], s, u, N, dN);
        for (int r = 0; r <= s_p[a]; ++r) sm[L.A[a] + i * CP + s - s_p[a] + r] = N[r];
      }
    }
    __syncthreads();
    if (s_bad) continue;
    if (mode == kGradient) {
      for (int a = 0; a < 3; ++a) {  // M = N^T N
        const float* A = sm + L.A[a];
        float* M = sm + L.M[a];
        const int C = s_C[a], n = s_n[a];
        for (int e = tid; e < C * C; e += blockDim.x) {
          const int r = e / C, c = e - r * C;
          float acc = 0.f;
          for (int i = 0; i < n; ++i) acc = fmaf(A[i * CP + r], A[i * CP + c], acc);
          M[e] = acc;
        }
      }
      for (int e = tid; e < ncps; e += blockDim.x) sm[L.P + e] = prm.cps[cp_off + e];
    }
    float* Y = sm + L.Y;
    for (int e = tid; e < ncps; e += blockDim.x) Y[e] = 0.f;

    const bool vec = vec_ok && (nx % 4 == 0);
    float* Y1 = sm + L.Y1;
    float* Y2 = sm + L.Y2;
    for (int k0 = 0; k0 < nz; k0 += ks) {
      const int kc = min(ks, nz - k0);
      const int rows = kc * ny;
      // x: one sample row per thread, all CP columns in registers
      for (int r = tid; r < rows; r += blockDim.x) {
        const float* xr = X + ((int64_t)k0 * ny + r) * nx;
        float acc[CP];
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = 0.f;
        if (vec) {
          for (int i = 0; i < nx; i += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(xr + i));
            const float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4* ar = reinterpret_cast<const float4*>(Ax + (i + q) * CP);
#pragma unroll
              for (int c4 = 0; c4 < Q4; ++c4) {
                const float4 w = ar[c4];
                acc[4 * c4 + 0] = fmaf(xs[q], w.x, acc[4 * c4 + 0]);
                acc[4 * c4 + 1] = fmaf(xs[q], w.y, acc[4 * c4 + 1]);
                acc[4 * c4 + 2] = fmaf(xs[q], w.z, acc[4 * c4 + 2]);
                acc[4 * c4 + 3] = fmaf(xs[q], w.w, acc[4 * c4 + 3]);
              }
            }
          }
        } else {
          for (int i = 0; i < nx; ++i) {
            const float xv = __ldg(xr + i);
            const float4* ar = reinterpret_cast<const float4*>(Ax + i * CP);
#pragma unroll
            for (int c4 = 0; c4 < Q4; ++c4) {
              const float4 w = ar[c4];
              acc[4 * c4 + 0] = fmaf(xv, w.x, acc[4 * c4 + 0]);
              acc[4 * c4 + 1] = fmaf(xv, w.y, acc[4 * c4 + 1]);
              acc[4 * c4 + 2] = fmaf(xv, w.z, acc[4 * c4 + 2]);
              acc[4 * c4 + 3] = fmaf(xv, w.w, acc[4 * c4 + 3]);
            }
          }
        }
        float4* yr = reinterpret_cast<float4*>(Y1 + r * CPs);
#pragma unroll
        for (int c4 = 0; c4 < Q4; ++c4)
          yr[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
      }
      __syncthreads();
      // y: Y2[kl][b][a] = sum_j Y1[(kl, j)][a] Ay[j][b], 4 values of b per thread
      {
        const int nb4 = (Cy + 3) / 4;
        for (int e = tid; e < kc * nb4 * Cx; e += blockDim.x) {
          const int a = e % Cx, t = e / Cx, b4 = t % nb4, kl = t / nb4;
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          const float* y1 = Y1 + kl * ny * CPs + a;
          for (int j = 0; j < ny; ++j) {
            const float yv = y1[j * CPs];
            const float4 w = *reinterpret_cast<const float4*>(Ay + j * CP + 4 * b4);
            acc.x = fmaf(yv, w.x, acc.x);
            acc.y = fmaf(yv, w.y, acc.y);
            acc.z = fmaf(yv, w.z, acc.z);
            acc.w = fmaf(yv, w.w, acc.w);
          }
          const float av[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int bb = 4 * b4 + q;
            if (bb < Cy) Y2[(kl * Cy + bb) * Cx + a] = av[q];
          }
        }
      }
      __syncthreads();
      // z: Y[c][b][a] += sum_kl Y2[kl][b][a] Az[k0 + kl][c], 4 values of c per thread
      {
        const int nc4 = (Cz + 3) / 4;
        for (int e = tid; e < nc4 * plane; e += blockDim.x) {
          const int ab = e % plane, c4 = e / plane;
          float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int kl = 0; kl < kc; ++kl) {
            const float yv = Y2[kl * plane + ab];
            const float4 w = *reinterpret_cast<const float4*>(Az + (k0 + kl) * CP + 4 * c4);
            acc.x = fmaf(yv, w.x, acc.x);
            acc.y = fmaf(yv, w.y, acc.y);
            acc.z = fmaf(yv, w.z, acc.z);
            acc.w = fmaf(yv, w.w, acc.w);
          }
          const float av[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = 4 * c4 + q;
            if (c < Cz) Y[c * plane + ab] += av[q];
          }
        }
      }
      __syncthreads();
    }

    // ---- epilogues ----
    if (mode == kAdjoint) {
      for (int e = tid; e < ncps; e += blockDim.x) prm.out[cp_off + e] = Y[e];
      continue;
    }
    if (mode == kGradient) {
      float* P = sm + L.P;
      float* Z = sm + L.Z;
      const float* Mx = sm + L.M[0];
      const float* My = sm + L.M[1];
      const float* Mz = sm + L.M[2];
      for (int e = tid; e < ncps; e += blockDim.x) {  // Z = P x_1 M_x
        const int a = e % Cx, cb = e / Cx;
        float acc = 0.f;
        for (int q = 0; q < Cx; ++q) acc = fmaf(P[cb * Cx + q], Mx[q * Cx + a], acc);
        Z[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < ncps; e += blockDim.x) {  // P <- Z x_2 M_y
        const int a = e % Cx, bb = (e / Cx) % Cy, c = e / plane;
        float acc = 0.f;
        for (int q = 0; q < Cy; ++q) acc = fmaf(Z[(c * Cy + q) * Cx + a], My[q * Cy + bb], acc);
        P[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < ncps; e += blockDim.x) {  // G = P x_3 M_z - N^T D
        const int ab = e % plane, c = e / plane;
        float acc = 0.f;
        for (int q = 0; q < Cz; ++q) acc = fmaf(P[q * plane + ab], Mz[q * Cz + c], acc);
        prm.out[cp_off + e] = acc - Y[e];
      }
      continue;
    }
    // kFit
    for (int e = tid; e < ncps; e += blockDim.x) prm.out[cp_off + e] = Y[e];
    if (!prm.rmse) continue;
    // RMSE: banded value decode of the fitted model against the samples. Each thread sums its
    // squared errors in FP32 with Kahan compensation; the per-thread sums are reduced in FP64
    // (FP64 per voxel would run at the low FP64 rate of this GPU).
    {
      const TabEntry* tx = reinterpret_cast<const TabEntry*>(sm + L.tab[0]);
      const TabEntry* ty = reinterpret_cast<const TabEntry*>(sm + L.tab[1]);
      const TabEntry* tz = reinterpret_cast<const TabEntry*>(sm + L.tab[2]);
      const int pxx = s_p[0], pyy = s_p[1], pzz = s_p[2];
      float ksum = 0.f, kcomp = 0.f;
      for (int k0 = 0; k0 < nz; k0 += ks) {
        const int kc = min(ks, nz - k0);
        for (int e = tid; e < plane * kc; e += blockDim.x) {  // T0 -> Y2
          const int kl = e / plane, ab = e - kl * plane;
          const TabEntry te = tz[k0 + kl];
          float acc = 0.f;
          for (int d = 0; d <= pzz; ++d) acc = fmaf(Y[(te.off + d) * plane + ab], te.N[d], acc);
          Y2[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < Cx * ny * kc; e += blockDim.x) {  // U0 -> Y1
          const int a = e % Cx, r = e / Cx, j = r % ny, kl = r / ny;
          const TabEntry te = ty[j];
          float acc = 0.f;
          for (int d = 0; d <= pyy; ++d) acc = fmaf(Y2[(kl * Cy + te.off + d) * Cx + a], te.N[d], acc);
          Y1[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < nx * ny * kc; e += blockDim.x) {
          const int i = e % nx, r = e / nx;
          const TabEntry te = tx[i];
          float f = 0.f;
          for (int d = 0; d <= pxx; ++d) f = fmaf(Y1[r * Cx + te.off + d], te.N[d], f);
          const float diff = f - X[(int64_t)k0 * nx * ny + e];
          const float y = diff * diff - kcomp;
          const float t = ksum + y;
          kcomp = (t - ksum) - y;
          ksum = t;
        }
        __syncthreads();
      }
      double sq = (double)ksum - (double)kcomp;
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if ((tid & 31) == 0) s_red[tid >> 5] = sq;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += s_red[w];
        prm.rmse[s_item] = sqrt(tot / ((double)nx * ny * nz));
      }
    }
  }
}

template <int CP>
cudaError_t launch_c3(mfa_ctx* ctx, const ContractParams& prm, const C3Smem& L, int ks, int vec_ok,
                      cudaStream_t stream) {
  auto kern = contract3_kernel<CP>;
  const size_t smem = (size_t)L.total * 4;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(ctx->num_sms * occ, prm.nblocks));
  kern<<<grid, kThreads, smem, stream>>>(prm, L, ks, vec_ok);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

int contract3(mfa_ctx* ctx, ContractParams prm, cudaStream_t stream) {
  const int CP = round4(prm.maxC);
  const bool rmse = prm.rmse != nullptr;
  int ks = std::min(8, prm.maxN);
  C3Smem L = c3_layout(prm.mode, CP, prm.maxC, prm.maxN, ks, rmse);
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = c3_layout(prm.mode, CP, prm.maxC, prm.maxN, ks, rmse);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  const int vec_ok = (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) && (prm.slot_stride % 4 == 0);
  if (cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  cudaError_t e;
  switch (CP) {
    case 4: e = launch_c3<4>(ctx, prm, L, ks, vec_ok, stream); break;
    case 8: e = launch_c3<8>(ctx, prm, L, ks, vec_ok, stream); break;
    case 12: e = launch_c3<12>(ctx, prm, L, ks, vec_ok, stream); break;
    case 16: e = launch_c3<16>(ctx, prm, L, ks, vec_ok, stream); break;
    case 20: e = launch_c3<20>(ctx, prm, L, ks, vec_ok, stream); break;
    case 24: e = launch_c3<24>(ctx, prm, L, ks, vec_ok, stream); break;
    case 28: e = launch_c3<28>(ctx, prm, L, ks, vec_ok, stream); break;
    case 32: e = launch_c3<32>(ctx, prm, L, ks, vec_ok, stream); break;
    default: return MFA_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
