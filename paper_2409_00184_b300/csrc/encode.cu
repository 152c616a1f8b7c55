// Least-squares micro-model fit (the model(NCP, degree) call of Algorithm 1) and its RMSE.
//
// With samples on a regular grid the design matrix is N_z (x) N_y (x) N_x, so the least-squares
// control points are P = D x_1 N_x^+ x_2 N_y^+ x_3 N_z^+ with N^+ = (N^T N)^{-1} N^T per axis.
//   class kernel (FP64): one CTA per distinct axis class (knots, p, C, n): collocation matrix N,
//     M = N^T N, Cholesky M = L L^T (pivots checked), N^+ by two triangular solves per sample,
//     stored transposed (n x C) in FP32, plus the FP32 span/basis table the RMSE pass decodes with.
//   fit kernel (FP32): one CTA per block (persistent queue), z-slabs of the sample grid through
//     shared memory: dense x-, y- and z-contractions with N_x^+, N_y^+, N_z^+; then, optionally, a
//     banded value decode of the fitted model against the samples with the squared error summed
//     in FP64 (Table 1's RMSE).
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

constexpr int kThreads = 256;
constexpr int kKnotMax = MFA_MAX_NCP + MFA_MAX_DEGREE + 1;

struct EncClass {
  int p, C, n;
  int pinv_off;  // floats into the pseudo-inverse pool: n x C, [i][a]
  int tab_off;   // entries into the basis-table pool: n entries
  int pad;
  float t[kKnotMax];
};

struct EncItem {
  int cls[3];
  int slot;
  int64_t cp_off;
};

// Basis-table entry for the RMSE decode: first nonzero index and the p+1 values.
struct TabEntry {
  int off;
  float N[MFA_MAX_DEGREE + 1];
};

__global__ void __launch_bounds__(kThreads) encode_class_kernel(const EncClass* classes, float* pinv,
                                                                TabEntry* tabs, uint32_t* status) {
  __shared__ double s_t[kKnotMax];
  __shared__ double s_N[MFA_MAX_NSAMP * MFA_MAX_NCP];  // [i][c]
  __shared__ double s_L[MFA_MAX_NCP * MFA_MAX_NCP];    // M, then its Cholesky factor (lower)
  __shared__ int s_fail;
  const EncClass& k = classes[blockIdx.x];
  const int p = k.p, C = k.C, n = k.n, tid = threadIdx.x;
  if (tid == 0) s_fail = 0;
  for (int i = tid; i < C + p + 1; i += blockDim.x) s_t[i] = (double)k.t[i];
  for (int e = tid; e < n * C; e += blockDim.x) s_N[e] = 0.0;
  __syncthreads();
  if (tid < n) {
    // FP32 sample parameter (as every kernel sees it), widened; basis in FP64 and in FP32
    const float uf = sample_param(tid, n);
    const double u = (double)uf;
    const int s = find_span<double>(s_t, p, C, u);
    double N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
    basis_funs<MFA_MAX_DEGREE, double>(s_t, p, s, u, N, dN);
    for (int r = 0; r <= p; ++r) s_N[tid * C + s - p + r] = N[r];
    const int sf = find_span<float>(k.t, p, C, uf);
    float Nf[MFA_MAX_DEGREE + 1], dNf[MFA_MAX_DEGREE + 1];
    basis_funs<MFA_MAX_DEGREE, float>(k.t, p, sf, uf, Nf, dNf);
    TabEntry te;
    te.off = sf - p;
    for (int r = 0; r <= MFA_MAX_DEGREE; ++r) te.N[r] = Nf[r];
    tabs[k.tab_off + tid] = te;
  }
  __syncthreads();
  // M = N^T N (lower triangle, FP64)
  for (int e = tid; e < C * C; e += blockDim.x) {
    const int r = e / C, c = e % C;
    if (c <= r) {
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += s_N[i * C + r] * s_N[i * C + c];
      s_L[r * C + c] = acc;
    }
  }
  __syncthreads();
  // Cholesky, column by column
  for (int j = 0; j < C; ++j) {
    if (tid == 0) {
      double d = s_L[j * C + j];
      for (int q = 0; q < j; ++q) d -= s_L[j * C + q] * s_L[j * C + q];
      if (!(d > 0.0)) { s_fail = 1; d = 1.0; }
      s_L[j * C + j] = sqrt(d);
    }
    __syncthreads();
    for (int r = j + 1 + tid; r < C; r += blockDim.x) {
      double v = s_L[r * C + j];
      for (int q = 0; q < j; ++q) v -= s_L[r * C + q] * s_L[j * C + q];
      s_L[r * C + j] = v / s_L[j * C + j];
    }
    __syncthreads();
  }
  if (tid == 0 && s_fail) flag(status, MFA_DEV_NOT_SPD);
  // N^+ column i solves M x = N[i][:]: forward with L, backward with L^T
  if (tid < n) {
    double x[MFA_MAX_NCP];
    for (int r = 0; r < C; ++r) {
      double v = s_N[tid * C + r];
      for (int q = 0; q < r; ++q) v -= s_L[r * C + q] * x[q];
      x[r] = v / s_L[r * C + r];
    }
    for (int r = C - 1; r >= 0; --r) {
      double v = x[r];
      for (int q = r + 1; q < C; ++q) v -= s_L[q * C + r] * x[q];
      x[r] = v / s_L[r * C + r];
    }
    for (int r = 0; r < C; ++r) pinv[k.pinv_off + tid * C + r] = (float)x[r];
  }
}

struct FitSmem {
  int pinv[3], tab[3], P, D, W1, W2, total;  // offsets in 4-byte words
};

FitSmem fit_layout(int maxC, int maxN, int ks) {
  FitSmem L;
  int o = 0;
  for (int a = 0; a < 3; ++a) { L.pinv[a] = o; o += maxN * maxC; }
  for (int a = 0; a < 3; ++a) { L.tab[a] = o; o += maxN * (int)(sizeof(TabEntry) / 4); }
  o = (o + 3) & ~3;
  L.P = o;  o += maxC * maxC * maxC;
  L.D = o;  o += maxN * maxN * ks;
  L.W1 = o; o += maxN * maxC * ks;  // [kl][j][a]; U0 of the RMSE decode
  L.W2 = o; o += maxC * maxC * ks;  // [kl][b][a]; T0 of the RMSE decode
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(kThreads)
encode_fit_kernel(const EncItem* items, int nblocks, const EncClass* classes, const float* pinv,
                  const TabEntry* tabs, const float* data, int64_t slot_stride, float* cps, double* rmse,
                  uint32_t* counter, FitSmem L, int ks) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item;
  __shared__ double s_red[kThreads / 32];
  const int tid = threadIdx.x;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(counter, 1u);
    __syncthreads();
    const int b = s_item;
    if (b >= nblocks) break;
    const EncItem it = items[b];
    const EncClass& cx = classes[it.cls[0]];
    const EncClass& cy = classes[it.cls[1]];
    const EncClass& cz = classes[it.cls[2]];
    const int Cx = cx.C, Cy = cy.C, Cz = cz.C, nx = cx.n, ny = cy.n, nz = cz.n;
    const EncClass* cl[3] = {&cx, &cy, &cz};
    for (int a = 0; a < 3; ++a) {
      const int len = cl[a]->C * cl[a]->n;
      for (int e = tid; e < len; e += blockDim.x) sm[L.pinv[a] + e] = pinv[cl[a]->pinv_off + e];
      TabEntry* tb = reinterpret_cast<TabEntry*>(sm + L.tab[a]);
      for (int e = tid; e < cl[a]->n; e += blockDim.x) tb[e] = tabs[cl[a]->tab_off + e];
    }
    float* s_P = sm + L.P;
    float* s_D = sm + L.D;
    float* s_W1 = sm + L.W1;
    float* s_W2 = sm + L.W2;
    const float* Px = sm + L.pinv[0];
    const float* Py = sm + L.pinv[1];
    const float* Pz = sm + L.pinv[2];
    const int ncps = Cx * Cy * Cz, plane = Cx * Cy;
    for (int e = tid; e < ncps; e += blockDim.x) s_P[e] = 0.f;
    const float* src = data + (int64_t)it.slot * slot_stride;
    __syncthreads();
    for (int k0 = 0; k0 < nz; k0 += ks) {
      const int kc = min(ks, nz - k0);
      for (int e = tid; e < nx * ny * kc; e += blockDim.x) s_D[e] = src[(int64_t)k0 * nx * ny + e];
      __syncthreads();
      for (int e = tid; e < Cx * ny * kc; e += blockDim.x) {  // x: W1[kl][j][a] = sum_i Px[i][a] D[kl][j][i]
        const int a = e % Cx, r = e / Cx;
        const float* drow = s_D + r * nx;
        float acc = 0.f;
        for (int i = 0; i < nx; ++i) acc = fmaf(Px[i * Cx + a], drow[i], acc);
        s_W1[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < plane * kc; e += blockDim.x) {  // y: W2[kl][b][a] = sum_j Py[j][b] W1[kl][j][a]
        const int a = e % Cx, r = e / Cx, bb = r % Cy, kl = r / Cy;
        float acc = 0.f;
        for (int j = 0; j < ny; ++j) acc = fmaf(Py[j * Cy + bb], s_W1[(kl * ny + j) * Cx + a], acc);
        s_W2[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < ncps; e += blockDim.x) {  // z: P[c][b][a] += sum_kl Pz[k0+kl][c] W2[kl][b][a]
        const int ab = e % plane, c = e / plane;
        float acc = s_P[e];
        for (int kl = 0; kl < kc; ++kl) acc = fmaf(Pz[(k0 + kl) * Cz + c], s_W2[kl * plane + ab], acc);
        s_P[e] = acc;
      }
      __syncthreads();
    }
    for (int e = tid; e < ncps; e += blockDim.x) cps[it.cp_off + e] = s_P[e];
    if (!rmse) continue;
    // RMSE: banded value decode of the fitted model against the samples, squares summed in FP64
    const TabEntry* tx = reinterpret_cast<const TabEntry*>(sm + L.tab[0]);
    const TabEntry* ty = reinterpret_cast<const TabEntry*>(sm + L.tab[1]);
    const TabEntry* tz = reinterpret_cast<const TabEntry*>(sm + L.tab[2]);
    double sq = 0.0;
    for (int k0 = 0; k0 < nz; k0 += ks) {
      const int kc = min(ks, nz - k0);
      for (int e = tid; e < plane * kc; e += blockDim.x) {
        const int kl = e / plane, ab = e - kl * plane;
        const TabEntry te = tz[k0 + kl];
        float acc = 0.f;
        for (int d = 0; d <= cz.p; ++d) acc = fmaf(s_P[(te.off + d) * plane + ab], te.N[d], acc);
        s_W2[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < Cx * ny * kc; e += blockDim.x) {
        const int a = e % Cx, r = e / Cx, j = r % ny, kl = r / ny;
        const TabEntry te = ty[j];
        float acc = 0.f;
        for (int d = 0; d <= cy.p; ++d) acc = fmaf(s_W2[(kl * Cy + te.off + d) * Cx + a], te.N[d], acc);
        s_W1[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < nx * ny * kc; e += blockDim.x) {
        const int i = e % nx, r = e / nx;
        const TabEntry te = tx[i];
        float f = 0.f;
        for (int d = 0; d <= cx.p; ++d) f = fmaf(s_W1[r * Cx + te.off + d], te.N[d], f);
        const double diff = (double)f - (double)src[(int64_t)k0 * nx * ny + e];
        sq += diff * diff;
      }
      __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = sq;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += s_red[w];
      rmse[b] = sqrt(tot / ((double)nx * ny * nz));
    }
  }
}

bool host_knots_ok(const float* t, int p, int C) {
  for (int i = 0; i + 1 < C + p + 1; ++i)
    if (!(t[i] <= t[i + 1])) return false;
  return t[p] < t[C];
}

}  // namespace
}  // namespace mfa

using namespace mfa;

struct mfa_encode_plan {
  mfa_ctx* ctx = nullptr;
  int nblocks = 0, nclasses = 0, maxC = 0, maxN = 0;
  int max_slot = -1;
  int64_t max_vox = 0;
  EncItem* d_items = nullptr;
  EncClass* d_classes = nullptr;
  float* d_pinv = nullptr;
  TabEntry* d_tabs = nullptr;
};

extern "C" {

int mfa_encode_plan_create(mfa_ctx* ctx, mfa_encode_plan** out, const mfa_block_desc* h_desc, int32_t nblocks,
                           const float* h_knots, int64_t knots_len, int64_t cps_len) {
  if (!ctx || !out || nblocks < 1 || !h_desc || !h_knots || knots_len < 1 || cps_len < 1) return MFA_ERR_INVALID_ARG;
  if (nblocks >= (1 << 30)) return MFA_ERR_CAPACITY;
  *out = nullptr;
  std::vector<EncItem> items(nblocks);
  std::vector<EncClass> classes;
  std::map<std::vector<float>, int> index;  // key: p, C, n, knots...
  mfa_encode_plan* plan = new (std::nothrow) mfa_encode_plan();
  if (!plan) return MFA_ERR_CUDA;
  int pinv_len = 0, tab_len = 0;
  for (int b = 0; b < nblocks; ++b) {
    const mfa_block_desc& d = h_desc[b];
    int64_t ncps = 1, vox = 1;
    for (int a = 0; a < 3; ++a) {
      const int p = d.degree[a], C = d.ncp[a], n = d.nsamp[a];
      if (p < 1 || p > MFA_MAX_DEGREE || C < p + 1 || C > MFA_MAX_NCP || n < 2 || n > MFA_MAX_NSAMP || C > n ||
          d.knot_off[a] < 0 || d.knot_off[a] + C + p + 1 > knots_len) {
        delete plan;
        return MFA_ERR_INVALID_ARG;
      }
      const float* t = h_knots + d.knot_off[a];
      if (!host_knots_ok(t, p, C)) { delete plan; return MFA_ERR_INVALID_ARG; }
      std::vector<float> key = {(float)p, (float)C, (float)n};
      key.insert(key.end(), t, t + C + p + 1);
      auto it = index.find(key);
      int cls;
      if (it == index.end()) {
        EncClass c;
        std::memset(&c, 0, sizeof(c));
        c.p = p; c.C = C; c.n = n;
        c.pinv_off = pinv_len;
        c.tab_off = tab_len;
        std::memcpy(c.t, t, sizeof(float) * (C + p + 1));
        pinv_len += C * n;
        tab_len += n;
        cls = (int)classes.size();
        classes.push_back(c);
        index.emplace(key, cls);
      } else {
        cls = it->second;
      }
      items[b].cls[a] = cls;
      ncps *= C;
      vox *= n;
      plan->maxC = std::max(plan->maxC, C);
      plan->maxN = std::max(plan->maxN, n);
    }
    if (d.cp_off < 0 || d.cp_off + ncps > cps_len || d.slot < 0) { delete plan; return MFA_ERR_INVALID_ARG; }
    items[b].slot = d.slot;
    items[b].cp_off = d.cp_off;
    plan->max_slot = std::max(plan->max_slot, d.slot);
    plan->max_vox = std::max(plan->max_vox, vox);
  }
  plan->ctx = ctx;
  plan->nblocks = nblocks;
  plan->nclasses = (int)classes.size();
  if (cudaMalloc(&plan->d_items, sizeof(EncItem) * nblocks) != cudaSuccess ||
      cudaMalloc(&plan->d_classes, sizeof(EncClass) * classes.size()) != cudaSuccess ||
      cudaMalloc(&plan->d_pinv, sizeof(float) * pinv_len) != cudaSuccess ||
      cudaMalloc(&plan->d_tabs, sizeof(TabEntry) * tab_len) != cudaSuccess ||
      cudaMemcpy(plan->d_items, items.data(), sizeof(EncItem) * nblocks, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(plan->d_classes, classes.data(), sizeof(EncClass) * classes.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    mfa_encode_plan_destroy(plan);
    return MFA_ERR_CUDA;
  }
  *out = plan;
  return MFA_OK;
}

void mfa_encode_plan_destroy(mfa_encode_plan* plan) {
  if (!plan) return;
  cudaFree(plan->d_items);
  cudaFree(plan->d_classes);
  cudaFree(plan->d_pinv);
  cudaFree(plan->d_tabs);
  delete plan;
}

int mfa_encode_blocks(mfa_ctx* ctx, const mfa_encode_plan* plan, const float* d_data, int64_t slot_stride_voxels,
                      int64_t nslots, float* d_cps_out, double* d_rmse, void* stream) {
  if (!ctx || !plan || plan->ctx != ctx || !d_data || !d_cps_out) return MFA_ERR_INVALID_ARG;
  if (slot_stride_voxels < plan->max_vox || nslots <= plan->max_slot) return MFA_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_data) & 3) || (reinterpret_cast<uintptr_t>(d_cps_out) & 3) ||
      (reinterpret_cast<uintptr_t>(d_rmse) & 7))
    return MFA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  encode_class_kernel<<<plan->nclasses, kThreads, 0, s>>>(plan->d_classes, plan->d_pinv, plan->d_tabs, ctx->d_status);
  ctx->launches++;
  if (cudaGetLastError() != cudaSuccess) return MFA_ERR_CUDA;
  int ks = std::min(8, plan->maxN);
  FitSmem L = fit_layout(plan->maxC, plan->maxN, ks);
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = fit_layout(plan->maxC, plan->maxN, ks);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  const size_t smem = (size_t)L.total * 4;
  if (cudaFuncSetAttribute(encode_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return MFA_ERR_CUDA;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, encode_fit_kernel, kThreads, smem) != cudaSuccess || occ < 1)
    return MFA_ERR_CUDA;
  uint32_t* counter = ctx->d_counters + kEncodeQueue;
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), s) != cudaSuccess) return MFA_ERR_CUDA;
  const int grid = std::max(1, std::min(ctx->num_sms * occ, plan->nblocks));
  encode_fit_kernel<<<grid, kThreads, smem, s>>>(plan->d_items, plan->nblocks, plan->d_classes, plan->d_pinv,
                                                 plan->d_tabs, d_data, slot_stride_voxels, d_cps_out, d_rmse,
                                                 counter, L, ks);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // extern "C"
