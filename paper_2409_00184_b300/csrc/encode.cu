// Least-squares micro-model fit (the model(NCP, degree) call of Algorithm 1) and its RMSE.
//
// With samples on a regular grid the design matrix is N_z (x) N_y (x) N_x, so the least-squares
// control points are P = D x_1 N_x^+ x_2 N_y^+ x_3 N_z^+ with N^+ = (N^T N)^{-1} N^T per axis.
//   plan (host): validates the batch and groups its axes into classes of equal (knots, p, C, n).
//   class kernel (FP64): one CTA per class: collocation matrix N, M = N^T N, Cholesky M = L L^T
//     (pivots checked), N^+ by two triangular solves per sample, stored transposed (n x C) in
//     FP32, plus the FP32 span/basis table the RMSE pass decodes with.
//   fit: the shared three-axis contraction kernel (contract3.cu, mode kFit) applies the three
//     pseudo-inverses to every block and sums the squared fitting error in FP64.
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
  ContractParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.mode = kFit;
  prm.nblocks = plan->nblocks;
  prm.items = plan->d_items;
  prm.classes = plan->d_classes;
  prm.pinv = plan->d_pinv;
  prm.tabs = plan->d_tabs;
  prm.rmse = d_rmse;
  prm.x = d_data;
  prm.slot_stride = slot_stride_voxels;
  prm.nslots = nslots;
  prm.out = d_cps_out;
  prm.status = ctx->d_status;
  prm.counter = ctx->d_counters + kEncodeQueue;
  prm.maxC = plan->maxC;
  prm.maxN = plan->maxN;
  prm.pmax = MFA_MAX_DEGREE;
  return contract3(ctx, prm, s);
}

}  // extern "C"
