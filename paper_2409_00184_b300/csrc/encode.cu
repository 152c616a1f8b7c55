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
// A plan sets its classes up once, when it is created; the allocation-free entry point, which has
// no plan, sets them up on every call.
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

// Host-side analysis of a batch: validation, axis classes of equal (p, C, n, knots), per-block items.
struct BatchAnalysis {
  std::vector<EncItem> items;
  std::vector<EncClass> classes;
  int pinv_len = 0, tab_len = 0, maxC = 0, maxN = 0, max_slot = -1;
  int64_t max_vox = 0;
  bool rows32 = true;  // every block has 32 samples along x
};

int analyze_batch(const mfa_block_desc* h_desc, int nblocks, const float* h_knots, int64_t knots_len,
                  int64_t cps_len, BatchAnalysis& out) {
  out.items.assign(nblocks, EncItem());
  std::map<std::vector<float>, int> index;  // key: p, C, n, knots...
  for (int b = 0; b < nblocks; ++b) {
    const mfa_block_desc& d = h_desc[b];
    int64_t ncps = 1, vox = 1;
    for (int a = 0; a < 3; ++a) {
      const int p = d.degree[a], C = d.ncp[a], n = d.nsamp[a];
      if (p < 1 || p > MFA_MAX_DEGREE || C < p + 1 || C > MFA_MAX_NCP || n < 2 || n > MFA_MAX_NSAMP || C > n ||
          d.knot_off[a] < 0 || d.knot_off[a] + C + p + 1 > knots_len)
        return MFA_ERR_INVALID_ARG;
      const float* t = h_knots + d.knot_off[a];
      if (!host_knots_ok(t, p, C)) return MFA_ERR_INVALID_ARG;
      std::vector<float> key = {(float)p, (float)C, (float)n};
      key.insert(key.end(), t, t + C + p + 1);
      auto it = index.find(key);
      int cls;
      if (it == index.end()) {
        EncClass c;
        std::memset(&c, 0, sizeof(c));
        c.p = p; c.C = C; c.n = n;
        c.pinv_off = out.pinv_len;
        c.tab_off = out.tab_len;
        std::memcpy(c.t, t, sizeof(float) * (C + p + 1));
        out.pinv_len += C * n;
        out.tab_len += n;
        cls = (int)out.classes.size();
        out.classes.push_back(c);
        index.emplace(key, cls);
      } else {
        cls = it->second;
      }
      out.items[b].cls[a] = cls;
      ncps *= C;
      vox *= n;
      out.maxC = std::max(out.maxC, C);
      out.maxN = std::max(out.maxN, n);
    }
    if (d.cp_off < 0 || d.cp_off + ncps > cps_len || d.slot < 0) return MFA_ERR_INVALID_ARG;
    out.rows32 = out.rows32 && d.nsamp[0] == 32;
    out.items[b].slot = d.slot;
    out.items[b].cp_off = d.cp_off;
    out.max_slot = std::max(out.max_slot, d.slot);
    out.max_vox = std::max(out.max_vox, vox);
  }
  return MFA_OK;
}

// Enqueues the FP64 class set-up (pseudo-inverses and basis tables of every class).
int run_classes(mfa_ctx* ctx, int nclasses, const EncClass* classes, float* pinv, TabEntry* tabs, cudaStream_t s) {
  encode_class_kernel<<<nclasses, kThreads, 0, s>>>(classes, pinv, tabs, ctx->d_status);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

// Enqueues the fit for device-resident items/classes/pools (the classes already set up).
int run_fit(mfa_ctx* ctx, int nblocks, int maxC, int maxN, const EncItem* items, const EncClass* classes,
            float* pinv, TabEntry* tabs, const float* data, int64_t slot_stride, int64_t nslots, float* cps_out,
            double* rmse, cudaStream_t s, int rows32) {
  ContractParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.mode = kFit;
  prm.nblocks = nblocks;
  prm.items = items;
  prm.classes = classes;
  prm.pinv = pinv;
  prm.tabs = tabs;
  prm.rmse = rmse;
  prm.x = data;
  prm.slot_stride = slot_stride;
  prm.nslots = nslots;
  prm.out = cps_out;
  prm.status = ctx->d_status;
  prm.counter = ctx->d_counters + kEncodeQueue;
  prm.maxC = maxC;
  prm.maxN = maxN;
  prm.pmax = MFA_MAX_DEGREE;
  prm.rows32 = rows32;
  return contract3(ctx, prm, s);
}

// The fit on the tensor cores (BF16 / split-BF16, no RMSE pass): the same items, classes and pools.
int run_fit_tc(mfa_ctx* ctx, int nblocks, int maxC, int maxN, const EncItem* items, const EncClass* classes,
               float* pinv, const float* data, int64_t slot_stride, int64_t nslots, float* cps_out, int precision,
               cudaStream_t s) {
  ContractParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.mode = kFit;
  prm.nblocks = nblocks;
  prm.items = items;
  prm.classes = classes;
  prm.pinv = pinv;
  prm.x = data;
  prm.slot_stride = slot_stride;
  prm.nslots = nslots;
  prm.out = cps_out;
  prm.status = ctx->d_status;
  prm.counter = ctx->d_counters + kEncodeQueue;
  prm.maxC = maxC;
  prm.maxN = maxN;
  prm.pmax = MFA_MAX_DEGREE;
  return contract_tc(ctx, prm, precision, s);
}

}  // namespace
}  // namespace mfa

using namespace mfa;

struct mfa_encode_plan {
  mfa_ctx* ctx = nullptr;
  int nblocks = 0, nclasses = 0, maxC = 0, maxN = 0, rows32 = 0;
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
  BatchAnalysis an;
  const int rc = analyze_batch(h_desc, nblocks, h_knots, knots_len, cps_len, an);
  if (rc != MFA_OK) return rc;
  mfa_encode_plan* plan = new (std::nothrow) mfa_encode_plan();
  if (!plan) return MFA_ERR_CUDA;
  plan->ctx = ctx;
  plan->nblocks = nblocks;
  plan->nclasses = (int)an.classes.size();
  plan->maxC = an.maxC;
  plan->maxN = an.maxN;
  plan->max_slot = an.max_slot;
  plan->max_vox = an.max_vox;
  plan->rows32 = an.rows32;
  if (cudaMalloc(&plan->d_items, sizeof(EncItem) * nblocks) != cudaSuccess ||
      cudaMalloc(&plan->d_classes, sizeof(EncClass) * an.classes.size()) != cudaSuccess ||
      cudaMalloc(&plan->d_pinv, sizeof(float) * an.pinv_len) != cudaSuccess ||
      cudaMalloc(&plan->d_tabs, sizeof(TabEntry) * an.tab_len) != cudaSuccess ||
      cudaMemcpy(plan->d_items, an.items.data(), sizeof(EncItem) * nblocks, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(plan->d_classes, an.classes.data(), sizeof(EncClass) * an.classes.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    mfa_encode_plan_destroy(plan);
    return MFA_ERR_CUDA;
  }
  // the classes depend only on the plan: set them up once, here
  if (run_classes(ctx, plan->nclasses, plan->d_classes, plan->d_pinv, plan->d_tabs, 0) != MFA_OK ||
      cudaStreamSynchronize(0) != cudaSuccess) {
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
  return run_fit(ctx, plan->nblocks, plan->maxC, plan->maxN, plan->d_items, plan->d_classes, plan->d_pinv,
                 plan->d_tabs, d_data, slot_stride_voxels, nslots, d_cps_out, d_rmse,
                 static_cast<cudaStream_t>(stream), plan->rows32);
}

int mfa_encode_blocks_ex(mfa_ctx* ctx, const mfa_encode_plan* plan, const float* d_data, int64_t slot_stride_voxels,
                         int64_t nslots, float* d_cps_out, double* d_rmse, int32_t precision, void* stream) {
  if (precision == MFA_PREC_FP32)
    return mfa_encode_blocks(ctx, plan, d_data, slot_stride_voxels, nslots, d_cps_out, d_rmse, stream);
  if (precision != MFA_PREC_BF16 && precision != MFA_PREC_SPLIT_BF16 && precision != MFA_PREC_FP16)
    return MFA_ERR_INVALID_ARG;
  if (!ctx || !plan || plan->ctx != ctx || !d_data || !d_cps_out) return MFA_ERR_INVALID_ARG;
  if (slot_stride_voxels < plan->max_vox || nslots <= plan->max_slot) return MFA_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_data) & 3) || (reinterpret_cast<uintptr_t>(d_cps_out) & 3))
    return MFA_ERR_INVALID_ARG;
  if (precision == MFA_PREC_FP16 || d_rmse) return MFA_ERR_UNSUPPORTED;
  return run_fit_tc(ctx, plan->nblocks, plan->maxC, plan->maxN, plan->d_items, plan->d_classes, plan->d_pinv, d_data,
                    slot_stride_voxels, nslots, d_cps_out, precision, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---- allocation-free encode -----------------------------------------------------------------
// One fixed device array serves as the encode's scratch (status word, queue counter, class table,
// block items, pseudo-inverses, basis tables) for callers that cannot allocate device memory.
// It exists once per device that loads the library and lives until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;
static __device__ __align__(256) unsigned char g_encode_scratch[kNoAllocScratchBytes];

namespace {
// Device address of g_encode_scratch on the current device. In host code the array's name is
// only a host-side stand-in, so the address comes from cudaGetSymbolAddress. It is looked up on
// every call (the lookup is cheap): after a device reset the module is loaded again and the
// array's address may change, so a stored address could go stale.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_encode_scratch) != cudaSuccess || !p) return MFA_ERR_CUDA;
  *out = static_cast<unsigned char*>(p);
  return MFA_OK;
}
}  // namespace

extern "C" int mfa_encode_blocks_noalloc(const mfa_block_desc* h_desc, int32_t nblocks, const float* h_knots,
                                         int64_t knots_len, const float* d_data, int64_t slot_stride_voxels,
                                         int64_t nslots, float* d_cps_out, int64_t cps_len, double* d_rmse,
                                         void* stream) {
  if (!h_desc || !h_knots || !d_data || !d_cps_out || nblocks < 1 || knots_len < 1 || cps_len < 1)
    return MFA_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_data) & 3) || (reinterpret_cast<uintptr_t>(d_cps_out) & 3) ||
      (reinterpret_cast<uintptr_t>(d_rmse) & 7))
    return MFA_ERR_INVALID_ARG;
  if (nblocks >= (1 << 30)) return MFA_ERR_CAPACITY;
  BatchAnalysis an;
  int rc = analyze_batch(h_desc, nblocks, h_knots, knots_len, cps_len, an);
  if (rc != MFA_OK) return rc;
  if (slot_stride_voxels < an.max_vox || nslots <= an.max_slot) return MFA_ERR_INVALID_ARG;

  // scratch layout: [0, 256) status word and queue counters, then the tables, 256-byte aligned
  size_t off = 256;
  auto take = [&off](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return o;
  };
  const size_t o_cls = take(sizeof(EncClass) * an.classes.size());
  const size_t o_items = take(sizeof(EncItem) * an.items.size());
  const size_t o_pinv = take(sizeof(float) * an.pinv_len);
  const size_t o_tabs = take(sizeof(TabEntry) * an.tab_len);
  if (off > kNoAllocScratchBytes) return MFA_ERR_CAPACITY;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MFA_ERR_CUDA;
  unsigned char* base = nullptr;
  rc = scratch_address(&base);
  if (rc != MFA_OK) return rc;
  mfa_ctx local;  // host-side view for the launchers; its device pointers point into the scratch
  local.device = dev;
  if (cudaDeviceGetAttribute(&local.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MFA_ERR_CUDA;
  local.d_status = reinterpret_cast<uint32_t*>(base);
  local.d_counters = reinterpret_cast<uint32_t*>(base + 16);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the status word and counters start at zero
  if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess ||
      cudaMemcpyAsync(base + o_cls, an.classes.data(), sizeof(EncClass) * an.classes.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + o_items, an.items.data(), sizeof(EncItem) * an.items.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return MFA_ERR_CUDA;
  rc = run_classes(&local, (int)an.classes.size(), reinterpret_cast<const EncClass*>(base + o_cls),
                   reinterpret_cast<float*>(base + o_pinv), reinterpret_cast<TabEntry*>(base + o_tabs), s);
  if (rc != MFA_OK) return rc;
  rc = run_fit(&local, nblocks, an.maxC, an.maxN, reinterpret_cast<const EncItem*>(base + o_items),
               reinterpret_cast<const EncClass*>(base + o_cls), reinterpret_cast<float*>(base + o_pinv),
               reinterpret_cast<TabEntry*>(base + o_tabs), d_data, slot_stride_voxels, nslots, d_cps_out, d_rmse, s,
               an.rows32);
  if (rc != MFA_OK) return rc;
  uint32_t status = 0;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpy(&status, base, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MFA_ERR_CUDA;
  return status ? MFA_ERR_DEVICE : MFA_OK;
}
