// C-ABI entry points: context, host-side argument checks, dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "kernels.h"

using namespace mfa;

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool bounds_ok(const mfa_bounds* b) {
  return b && b->max_degree >= 1 && b->max_degree <= MFA_MAX_DEGREE && b->max_ncp >= 2 &&
         b->max_ncp <= MFA_MAX_NCP && b->max_nsamp >= 2 && b->max_nsamp <= MFA_MAX_NSAMP &&
         b->max_ncp >= b->max_degree + 1;
}

}  // namespace

extern "C" {

int mfa_ctx_create(mfa_ctx** out, int device) {
  if (!out) return MFA_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return MFA_ERR_CUDA;
  if (device < 0 || device >= ndev) return MFA_ERR_INVALID_ARG;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return MFA_ERR_CUDA;
  if (prop.major != 10 || prop.minor != 3) return MFA_ERR_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return MFA_ERR_CUDA;
  mfa_ctx* c = new (std::nothrow) mfa_ctx();
  if (!c) return MFA_ERR_CUDA;
  c->device = device;
  c->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->d_counters, kNumCounters * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&c->d_stats, MFA_NUM_STATS * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->d_stats, 0, MFA_NUM_STATS * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(c->d_counters, 0, kNumCounters * sizeof(uint32_t)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(c->d_status);
    cudaFree(c->d_counters);
    cudaFree(c->d_stats);
    delete c;
    return MFA_ERR_CUDA;
  }
  *out = c;
  return MFA_OK;
}

void mfa_ctx_destroy(mfa_ctx* ctx) {
  if (!ctx) return;
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_counters);
  cudaFree(ctx->d_stats);
  cudaFree(ctx->d_touched);
  delete ctx;
}

int mfa_abi_struct_sizes(int32_t* out, int32_t n) {
  const int32_t sizes[5] = {(int32_t)sizeof(mfa_block_desc), (int32_t)sizeof(mfa_bounds),
                            (int32_t)sizeof(mfa_decode_tiling), (int32_t)sizeof(mfa_view),
                            (int32_t)sizeof(mfa_frame_desc)};
  for (int32_t i = 0; out && i < n && i < 5; ++i) out[i] = sizes[i];
  return 5;
}

const char* mfa_status_string(int status) {
  switch (status) {
    case MFA_OK: return "ok";
    case MFA_ERR_INVALID_ARG: return "invalid argument";
    case MFA_ERR_UNSUPPORTED: return "unsupported";
    case MFA_ERR_CUDA: return "CUDA runtime error";
    case MFA_ERR_TIMEOUT: return "bounded device wait timed out";
    case MFA_ERR_CAPACITY: return "request exceeds a library limit";
    case MFA_ERR_DEVICE: return "device status word holds error bits";
    case MFA_ERR_IO: return "model store read or write failed";
    default: return "unknown status";
  }
}

int mfa_ctx_device_status(mfa_ctx* ctx, uint32_t* status, int clear, void* stream) {
  if (!ctx || !status) return MFA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MFA_ERR_CUDA;
  if (cudaMemcpy(status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MFA_ERR_CUDA;
  if (clear && cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess) return MFA_ERR_CUDA;
  return MFA_OK;
}

int64_t mfa_ctx_launch_count(const mfa_ctx* ctx) { return ctx ? ctx->launches : -1; }

int mfa_ctx_read_stats(mfa_ctx* ctx, uint64_t* stats, int nstats, int reset, void* stream) {
  if (!ctx || !stats || nstats < 1 || nstats > MFA_NUM_STATS) return MFA_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return MFA_ERR_CUDA;
  unsigned long long tmp[MFA_NUM_STATS];
  if (cudaMemcpy(tmp, ctx->d_stats, sizeof(tmp), cudaMemcpyDeviceToHost) != cudaSuccess) return MFA_ERR_CUDA;
  for (int i = 0; i < nstats; ++i) stats[i] = tmp[i];
  if (reset && cudaMemset(ctx->d_stats, 0, sizeof(tmp)) != cudaSuccess) return MFA_ERR_CUDA;
  return MFA_OK;
}

static bool same_key(const mfa_bounds& a, const mfa_bounds& b) {
  return a.max_degree == b.max_degree && a.max_ncp == b.max_ncp && a.max_nsamp == b.max_nsamp;
}

int mfa_ctx_set_decode_tiling(mfa_ctx* ctx, const mfa_bounds* key, const mfa_decode_tiling* tiling) {
  if (!ctx || !key || !tiling || !bounds_ok(key) || tiling->ks < 0 || tiling->ctas_per_sm < 0 ||
      tiling->ks > MFA_MAX_NSAMP || tiling->ctas_per_sm > 32)
    return MFA_ERR_INVALID_ARG;
  for (int i = 0; i < ctx->ntilings; ++i)
    if (same_key(ctx->tilings[i].key, *key)) {
      ctx->tilings[i].tiling = *tiling;
      return MFA_OK;
    }
  if (ctx->ntilings >= 64) return MFA_ERR_CAPACITY;
  ctx->tilings[ctx->ntilings].key = *key;
  ctx->tilings[ctx->ntilings].tiling = *tiling;
  ctx->ntilings++;
  return MFA_OK;
}

int mfa_ctx_get_decode_tiling(const mfa_ctx* ctx, const mfa_bounds* key, mfa_decode_tiling* tiling) {
  if (!ctx || !key || !tiling) return MFA_ERR_INVALID_ARG;
  for (int i = 0; i < ctx->ntilings; ++i)
    if (same_key(ctx->tilings[i].key, *key)) {
      *tiling = ctx->tilings[i].tiling;
      return MFA_OK;
    }
  tiling->ks = 0;
  tiling->ctas_per_sm = 0;
  return MFA_ERR_INVALID_ARG;
}

int mfa_copy_to_device(void* d_dst, const void* h_src, int64_t bytes, void* stream) {
  if (!d_dst || !h_src || bytes < 0) return MFA_ERR_INVALID_ARG;
  if (bytes == 0) return MFA_OK;
  return cudaMemcpyAsync(d_dst, h_src, (size_t)bytes, cudaMemcpyHostToDevice, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? MFA_OK
             : MFA_ERR_CUDA;
}

int mfa_copy_to_host(void* h_dst, const void* d_src, int64_t bytes, void* stream) {
  if (!h_dst || !d_src || bytes < 0) return MFA_ERR_INVALID_ARG;
  if (bytes == 0) return MFA_OK;
  return cudaMemcpyAsync(h_dst, d_src, (size_t)bytes, cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? MFA_OK
             : MFA_ERR_CUDA;
}

int64_t mfa_model_bytes(int32_t ncp, int32_t degree) {
  if (ncp < 1 || degree < 0) return -1;
  const int64_t c = ncp;
  return 1 + ((c + degree) * 3 + c * c * c) * 4;
}

}  // extern "C"

namespace {
// mfa_decode_blocks, optionally fused with the comparison to the fitted samples (data != nullptr).
int decode_entry(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks, const int32_t* d_list, int32_t list_len,
                 const int32_t* d_count, const float* d_knots, int64_t knots_len, const float* d_cps, int64_t cps_len,
                 float* d_cache, int64_t slot_stride_voxels, int64_t nslots, const mfa_bounds* bounds,
                 int32_t precision, uint32_t flags, const float* d_data, int64_t data_stride, float* d_residual,
                 double* d_rmse, void* stream) {
  if (!ctx || !bounds_ok(bounds)) return MFA_ERR_INVALID_ARG;
  if (nblocks < 0 || list_len < 0 || knots_len < 0 || cps_len < 0 || slot_stride_voxels < 1 || nslots < 0)
    return MFA_ERR_INVALID_ARG;
  if (flags & ~(MFA_DECODE_VALUE_ONLY | MFA_DECODE_LIST_SLOTS | MFA_DECODE_CUBES | MFA_DECODE_APRON))
    return MFA_ERR_INVALID_ARG;
  if ((flags & MFA_DECODE_CUBES) && (flags & MFA_DECODE_APRON)) return MFA_ERR_INVALID_ARG;
  if ((flags & MFA_DECODE_LIST_SLOTS) && !d_list) return MFA_ERR_INVALID_ARG;
  if (precision < MFA_PREC_FP32 || precision > MFA_PREC_SPLIT_BF16) return MFA_ERR_INVALID_ARG;
  if ((flags & MFA_DECODE_CUBES) && precision != MFA_PREC_FP32) return MFA_ERR_UNSUPPORTED;
  const int items = d_list ? list_len : nblocks;
  if (items == 0 && !d_count) return MFA_OK;
  if (!d_desc || !d_knots || !d_cps || !d_cache || nblocks == 0) return MFA_ERR_INVALID_ARG;
  if (!aligned(d_desc, 8) || !aligned(d_knots, 4) || !aligned(d_cps, 4) || !aligned(d_cache, 16) ||
      (d_list && !aligned(d_list, 4)) || (d_count && !aligned(d_count, 4)))
    return MFA_ERR_INVALID_ARG;
  // work units (item x z-slab) are counted by a 32-bit queue counter
  if ((int64_t)items * MFA_MAX_NSAMP >= (int64_t)1 << 30) return MFA_ERR_CAPACITY;
  DecodeParams prm;
  prm.desc = d_desc;
  prm.nblocks = nblocks;
  prm.list = d_list;
  prm.list_len = list_len;
  prm.count = d_count;
  prm.knots = d_knots;
  prm.knots_len = knots_len;
  prm.cps = d_cps;
  prm.cps_len = cps_len;
  prm.cache = d_cache;
  prm.slot_stride = slot_stride_voxels;
  prm.nslots = nslots;
  prm.bounds = *bounds;
  prm.flags = flags;
  prm.status = ctx->d_status;
  prm.counter = ctx->d_counters + kDecodeQueue;
  prm.ks = 0;
  prm.slabs = 0;
  prm.data = d_data;
  prm.data_stride = data_stride;
  prm.residual = d_residual;
  prm.sq = d_rmse;
  if (precision != MFA_PREC_FP32) return decode_tc(ctx, prm, precision, static_cast<cudaStream_t>(stream));
  DecodeTuning tune;
  mfa_decode_tiling t;
  if (mfa_ctx_get_decode_tiling(ctx, bounds, &t) == MFA_OK) {
    tune.ks = t.ks;
    tune.ctas_per_sm = t.ctas_per_sm;
  }
  return decode_fp32(ctx, prm, tune, static_cast<cudaStream_t>(stream));
}
}  // namespace

extern "C" {

int mfa_decode_blocks(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks,
                      const int32_t* d_list, int32_t list_len, const int32_t* d_count,
                      const float* d_knots, int64_t knots_len, const float* d_cps, int64_t cps_len,
                      float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                      const mfa_bounds* bounds, int32_t precision, uint32_t flags, void* stream) {
  return decode_entry(ctx, d_desc, nblocks, d_list, list_len, d_count, d_knots, knots_len, d_cps, cps_len, d_cache,
                      slot_stride_voxels, nslots, bounds, precision, flags, nullptr, 0, nullptr, nullptr, stream);
}

int mfa_decode_compare_blocks(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks,
                              const int32_t* d_list, int32_t list_len, const int32_t* d_count,
                              const float* d_knots, int64_t knots_len, const float* d_cps, int64_t cps_len,
                              float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                              const mfa_bounds* bounds, uint32_t flags, const float* d_data,
                              int64_t data_slot_stride, float* d_residual, double* d_rmse, void* stream) {
  if (!d_data || data_slot_stride < 1 || !aligned(d_data, 4) || (d_residual && !aligned(d_residual, 4)) ||
      (d_rmse && !aligned(d_rmse, 8)))
    return MFA_ERR_INVALID_ARG;
  return decode_entry(ctx, d_desc, nblocks, d_list, list_len, d_count, d_knots, knots_len, d_cps, cps_len, d_cache,
                      slot_stride_voxels, nslots, bounds, MFA_PREC_FP32, flags, d_data, data_slot_stride, d_residual,
                      d_rmse, stream);
}

int mfa_basis_tables(mfa_ctx* ctx, const mfa_block_desc* d_desc, const float* d_knots, int64_t knots_len,
                     int32_t* d_span, float* d_basis, void* stream) {
  if (!ctx || !d_desc || !d_knots || !d_span || !d_basis || knots_len < 1) return MFA_ERR_INVALID_ARG;
  if (!aligned(d_desc, 8)) return MFA_ERR_INVALID_ARG;
  return basis_tables(ctx, d_desc, d_knots, knots_len, d_span, d_basis, static_cast<cudaStream_t>(stream));
}

int mfa_adjoint_blocks(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks,
                       const float* d_knots, int64_t knots_len,
                       const float* d_residual, int64_t slot_stride_voxels, int64_t nslots,
                       const float* d_cps, float* d_grad_cps, int64_t cps_len,
                       const mfa_bounds* bounds, int32_t precision, void* stream) {
  if (!ctx || !bounds_ok(bounds)) return MFA_ERR_INVALID_ARG;
  if (nblocks < 0 || knots_len < 0 || cps_len < 0 || slot_stride_voxels < 1 || nslots < 0)
    return MFA_ERR_INVALID_ARG;
  if (precision < MFA_PREC_FP32 || precision > MFA_PREC_SPLIT_BF16) return MFA_ERR_INVALID_ARG;
  if (nblocks == 0) return MFA_OK;
  if (nblocks >= (1 << 30)) return MFA_ERR_CAPACITY;
  if (!d_desc || !d_knots || !d_residual || !d_grad_cps) return MFA_ERR_INVALID_ARG;
  if (!aligned(d_desc, 8) || !aligned(d_knots, 4) || !aligned(d_residual, 4) || !aligned(d_grad_cps, 4) ||
      (d_cps && !aligned(d_cps, 4)))
    return MFA_ERR_INVALID_ARG;
  if (precision == MFA_PREC_FP16) return MFA_ERR_UNSUPPORTED;
  AdjointParams prm;
  prm.precision = precision;
  prm.desc = d_desc;
  prm.nblocks = nblocks;
  prm.knots = d_knots;
  prm.knots_len = knots_len;
  prm.residual = d_residual;
  prm.slot_stride = slot_stride_voxels;
  prm.nslots = nslots;
  prm.cps = d_cps;
  prm.grad = d_grad_cps;
  prm.cps_len = cps_len;
  prm.bounds = *bounds;
  prm.status = ctx->d_status;
  prm.counter = ctx->d_counters + kAdjointQueue;
  return adjoint(ctx, prm, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {
// Host checks of the view and the brick grid, and the FP32 camera/march parameters of a ray cast.
// nodes > 0: the volume has `nodes` nodes on every axis (a shared-boundary grid) and the samples carry
// gradients in node units; otherwise brick_dims[a]*brick_n nodes and gradients per brick parameter.
int view_params(mfa::RaycastParams& prm, const int32_t brick_dims[3], int32_t brick_n, const mfa_view* view,
                int64_t nodes = 0) {
  if (view->width < 1 || view->height < 1 || view->width > 16384 || view->height > 16384) return MFA_ERR_INVALID_ARG;
  if (!(view->fov_y_deg > 0.f && view->fov_y_deg < 180.f) || !(view->step_voxels > 0.f) ||
      !(view->vmax > view->vmin))
    return MFA_ERR_INVALID_ARG;

  // Camera frame in FP64, rounded once to FP32 (the per-pixel set-up then runs in FP32).
  const double ex = view->eye[0], ey = view->eye[1], ez = view->eye[2];
  double f[3] = {(double)view->target[0] - ex, (double)view->target[1] - ey, (double)view->target[2] - ez};
  const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fl > 0.0)) return MFA_ERR_INVALID_ARG;
  for (double& v : f) v = v / fl;
  const double u[3] = {view->up[0], view->up[1], view->up[2]};
  double r[3] = {f[1] * u[2] - f[2] * u[1], f[2] * u[0] - f[0] * u[2], f[0] * u[1] - f[1] * u[0]};
  const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  if (!(rl > 0.0)) return MFA_ERR_INVALID_ARG;
  for (double& v : r) v = v / rl;
  const double up[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  const double tan_h = std::tan((double)view->fov_y_deg * M_PI / 360.0);
  const double tan_w = tan_h * view->width / view->height;

  int nmax = 0;
  for (int a = 0; a < 3; ++a) {
    prm.B[a] = brick_dims[a];
    const int N = nodes > 0 ? (int)nodes : brick_dims[a] * brick_n;
    nmax = N > nmax ? N : nmax;
    prm.half[a] = (float)((N - 1) / 2.0);
    prm.gscale[a] = nodes > 0 ? prm.half[a] : (float)((N - 1) / 2.0 / (brick_n - 1));
    prm.eye[a] = view->eye[a];
    prm.fwd[a] = (float)f[a];
    prm.right[a] = (float)r[a];
    prm.up[a] = (float)up[a];
  }
  prm.brick_n = brick_n;
  prm.log2n = -1;
  for (int l = 0; l < 31; ++l)
    if ((1 << l) == brick_n) prm.log2n = l;
  prm.W = view->width;
  prm.H = view->height;
  prm.tan_w = (float)tan_w;
  prm.tan_h = (float)tan_h;
  prm.dt = (float)((double)view->step_voxels * 2.0 / (nmax - 1));
  const double max_samples = 2.0 * std::sqrt(3.0) / prm.dt + 2.0;
  if (!(prm.dt > 0.f) || max_samples > (double)(1 << 24)) return MFA_ERR_INVALID_ARG;
  prm.max_samples = (int)max_samples;
  prm.step_voxels = view->step_voxels;
  prm.opacity_max = view->opacity_max;
  prm.ka = view->ka;
  prm.kd = view->kd;
  prm.ks = view->ks;
  prm.shininess = view->shininess;
  prm.vmin = view->vmin;
  prm.vmax = view->vmax;
  return MFA_OK;
}
}  // namespace

extern "C" {

int mfa_raycast(mfa_ctx* ctx, const float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                const mfa_view* view, const float* d_tf, int32_t tf_n, float* d_image, void* stream) {
  return mfa_raycast_ex(ctx, d_cache, slot_stride_voxels, nslots, d_brick_table, brick_dims, brick_n, view, d_tf,
                        tf_n, d_image, 0u, stream);
}

int mfa_raycast_ex(mfa_ctx* ctx, const float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                   const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                   const mfa_view* view, const float* d_tf, int32_t tf_n, float* d_image, uint32_t flags,
                   void* stream) {
  if (!ctx || !d_cache || !d_brick_table || !brick_dims || !view || !d_tf || !d_image) return MFA_ERR_INVALID_ARG;
  if ((flags & ~(MFA_RAYCAST_CUBES | MFA_RAYCAST_APRON | MFA_RAYCAST_COUNT_SECTORS)) ||
      ((flags & MFA_RAYCAST_CUBES) && (brick_n & 1)))
    return MFA_ERR_INVALID_ARG;
  if ((flags & MFA_RAYCAST_CUBES) && (flags & MFA_RAYCAST_APRON)) return MFA_ERR_INVALID_ARG;
  if (!aligned(d_cache, 16) || !aligned(d_tf, 16) || !aligned(d_image, 16) || !aligned(d_brick_table, 4))
    return MFA_ERR_INVALID_ARG;
  if (brick_n < 2 || slot_stride_voxels < (int64_t)brick_n * brick_n * brick_n || nslots < 0 || tf_n < 2)
    return MFA_ERR_INVALID_ARG;
  if ((flags & MFA_RAYCAST_APRON) &&
      (brick_n > MFA_MAX_NSAMP ||
       slot_stride_voxels < (int64_t)apron_pitch(brick_n) * (brick_n + 1) * (brick_n + 1)))
    return MFA_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (brick_dims[a] < 1 || (int64_t)brick_dims[a] * brick_n > (1 << 20)) return MFA_ERR_INVALID_ARG;
  RaycastParams prm;
  const int vs = view_params(prm, brick_dims, brick_n, view);
  if (vs != MFA_OK) return vs;
  prm.cache = reinterpret_cast<const float4*>(d_cache);
  prm.slot_stride = slot_stride_voxels;
  prm.nslots = nslots;
  prm.table = d_brick_table;
  prm.tf = reinterpret_cast<const float4*>(d_tf);
  prm.tf_n = tf_n;
  prm.image = reinterpret_cast<float4*>(d_image);
  prm.samples = ctx->d_stats + MFA_STAT_RAY_SAMPLES;
  prm.cubes = (flags & MFA_RAYCAST_CUBES) != 0;
  prm.apron = (flags & MFA_RAYCAST_APRON) != 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (flags & MFA_RAYCAST_COUNT_SECTORS) {
    if (prm.log2n < 3 || prm.log2n > 6) return MFA_ERR_UNSUPPORTED;
    const int64_t words = ((nslots * slot_stride_voxels + 1) / 2 + 31) / 32;  // one bit per 32-byte sector
    if (words > ctx->touched_words) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return MFA_ERR_CUDA;
      cudaFree(ctx->d_touched);
      ctx->d_touched = nullptr;
      ctx->touched_words = 0;
      if (cudaMalloc(&ctx->d_touched, (size_t)words * sizeof(uint32_t)) != cudaSuccess) return MFA_ERR_CUDA;
      ctx->touched_words = words;
    }
    if (cudaMemsetAsync(ctx->d_touched, 0, (size_t)words * sizeof(uint32_t), s) != cudaSuccess) return MFA_ERR_CUDA;
    prm.touched = ctx->d_touched;
    prm.sectors = ctx->d_stats + MFA_STAT_RAY_SECTORS;
  }
  return raycast(ctx, prm, s);
}

int mfa_fill_aprons(mfa_ctx* ctx, float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                    const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n, void* stream) {
  if (!ctx || !d_cache || !d_brick_table || !brick_dims) return MFA_ERR_INVALID_ARG;
  if (!aligned(d_cache, 16) || !aligned(d_brick_table, 4)) return MFA_ERR_INVALID_ARG;
  if (brick_n < 2 || brick_n > MFA_MAX_NSAMP || nslots < 0 ||
      slot_stride_voxels < (int64_t)apron_pitch(brick_n) * (brick_n + 1) * (brick_n + 1))
    return MFA_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (brick_dims[a] < 1 || (int64_t)brick_dims[a] * brick_n > (1 << 20)) return MFA_ERR_INVALID_ARG;
  ApronParams prm;
  prm.cache = reinterpret_cast<float4*>(d_cache);
  prm.slot_stride = slot_stride_voxels;
  prm.nslots = nslots;
  prm.table = d_brick_table;
  for (int a = 0; a < 3; ++a) prm.B[a] = brick_dims[a];
  prm.n = brick_n;
  return apron_fill(ctx, prm, static_cast<cudaStream_t>(stream));
}

int mfa_raycast_direct(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks, const float* d_knots,
                       int64_t knots_len, const float* d_cps, int64_t cps_len, const mfa_bounds* bounds,
                       const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                       const mfa_view* view, const float* d_tf, int32_t tf_n, float* d_image, void* stream) {
  if (!ctx || !d_desc || !d_knots || !d_cps || !bounds || !d_brick_table || !brick_dims || !view || !d_tf ||
      !d_image)
    return MFA_ERR_INVALID_ARG;
  if (!aligned(d_desc, 8) || !aligned(d_knots, 4) || !aligned(d_cps, 4) || !aligned(d_tf, 16) ||
      !aligned(d_image, 16) || !aligned(d_brick_table, 4))
    return MFA_ERR_INVALID_ARG;
  if (nblocks < 0 || knots_len < 0 || cps_len < 0 || brick_n < 2 || brick_n > MFA_MAX_NSAMP || tf_n < 2)
    return MFA_ERR_INVALID_ARG;
  if (bounds->max_degree < 1 || bounds->max_degree > MFA_MAX_DEGREE || bounds->max_ncp < 2 ||
      bounds->max_ncp > MFA_MAX_NCP || bounds->max_nsamp < brick_n || bounds->max_nsamp > MFA_MAX_NSAMP)
    return MFA_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if (brick_dims[a] < 1 || (int64_t)brick_dims[a] * brick_n > (1 << 20)) return MFA_ERR_INVALID_ARG;
  RaycastParams prm;
  const int vs = view_params(prm, brick_dims, brick_n, view);
  if (vs != MFA_OK) return vs;
  prm.cache = nullptr;
  prm.slot_stride = 0;
  prm.nslots = 0;
  prm.table = d_brick_table;
  prm.tf = reinterpret_cast<const float4*>(d_tf);
  prm.tf_n = tf_n;
  prm.image = reinterpret_cast<float4*>(d_image);
  prm.samples = ctx->d_stats + MFA_STAT_RAY_SAMPLES;
  DirectModels m;
  m.desc = d_desc;
  m.nblocks = nblocks;
  m.knots = d_knots;
  m.knots_len = knots_len;
  m.cps = d_cps;
  m.cps_len = cps_len;
  m.bounds = *bounds;
  m.status = ctx->d_status;
  return raycast_direct(ctx, prm, m, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

extern "C" int mfa_raycast_lod(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks, const float* d_knots,
                               int64_t knots_len, const float* d_cps, int64_t cps_len, const mfa_bounds* bounds,
                               const int32_t* d_table, int32_t fine_blocks, int32_t n, int32_t levels,
                               const mfa_view* view, const float* d_tf, int32_t tf_n, float* d_image, void* stream) {
  if (!ctx || !d_desc || !d_knots || !d_cps || !bounds || !d_table || !view || !d_tf || !d_image)
    return MFA_ERR_INVALID_ARG;
  if (!aligned(d_desc, 8) || !aligned(d_knots, 4) || !aligned(d_cps, 4) || !aligned(d_tf, 16) ||
      !aligned(d_image, 16) || !aligned(d_table, 4))
    return MFA_ERR_INVALID_ARG;
  if (nblocks < 0 || knots_len < 0 || cps_len < 0 || n < 2 || n > MFA_MAX_NSAMP || tf_n < 2 || levels < 1 ||
      levels > MFA_MAX_LEVELS || fine_blocks < 1 || fine_blocks % (1 << (levels - 1)) != 0 ||
      (int64_t)fine_blocks * (n - 1) + 1 > (1 << 20))
    return MFA_ERR_INVALID_ARG;
  if (bounds->max_degree < 1 || bounds->max_degree > MFA_MAX_DEGREE || bounds->max_ncp < 2 ||
      bounds->max_ncp > MFA_MAX_NCP || bounds->max_nsamp < n || bounds->max_nsamp > MFA_MAX_NSAMP)
    return MFA_ERR_INVALID_ARG;
  LodLevels lv;
  lv.B0 = fine_blocks;
  lv.n = n;
  lv.levels = levels;
  int64_t acc = 0;
  for (int l = 0; l < MFA_MAX_LEVELS; ++l) {
    lv.off[l] = (int)std::min<int64_t>(acc, 0x7fffffff);
    if (l < levels) {
      const int64_t Bl = fine_blocks >> l;
      acc += Bl * Bl * Bl;
    }
  }
  if (acc > 0x7fffffff) return MFA_ERR_CAPACITY;
  const int32_t dims[3] = {fine_blocks, fine_blocks, fine_blocks};
  RaycastParams prm;
  const int vs = view_params(prm, dims, n, view, (int64_t)fine_blocks * (n - 1) + 1);
  if (vs != MFA_OK) return vs;
  prm.cache = nullptr;
  prm.slot_stride = 0;
  prm.nslots = 0;
  prm.table = d_table;
  prm.tf = reinterpret_cast<const float4*>(d_tf);
  prm.tf_n = tf_n;
  prm.image = reinterpret_cast<float4*>(d_image);
  prm.samples = ctx->d_stats + MFA_STAT_RAY_SAMPLES;
  DirectModels m;
  m.desc = d_desc;
  m.nblocks = nblocks;
  m.knots = d_knots;
  m.knots_len = knots_len;
  m.cps = d_cps;
  m.cps_len = cps_len;
  m.bounds = *bounds;
  m.status = ctx->d_status;
  return raycast_lod(ctx, prm, m, lv, static_cast<cudaStream_t>(stream));
}
