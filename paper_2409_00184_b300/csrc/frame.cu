// One rendered frame as a CUDA graph: order the visible blocks by cost, decode them into cache slots
// with the persistent work queue, build the brick table, ray-cast (the per-frame path of Sec. 4.3:
// the visible micro-models of a point of view are decoded and rendered, Algorithm 4).
//
// The graph is captured once with fixed pointers and capacities; before each replay the caller
// writes the frame's visible list and its count into the device buffers the graph reads.
#include <algorithm>
#include <cstring>
#include <new>

#include "common.cuh"
#include "kernels.h"

namespace mfa {
namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kKeys = MFA_MAX_NCP + 1;

// Cost key of list entry b: ascending key = descending max(C_x, C_y, C_z).
__device__ __forceinline__ int cost_key(const mfa_block_desc* desc, int nblocks, int b) {
  if (b < 0 || b >= nblocks) return 0;
  const mfa_block_desc& d = desc[b];
  const int k = max(d.ncp[0], max(d.ncp[1], d.ncp[2]));
  return MFA_MAX_NCP - min(max(k, 0), MFA_MAX_NCP);
}

// Stable counting sort of list[0 .. count) by decreasing cost key max(C_x, C_y, C_z) (largest models
// first, so the persistent queue ends on short items). One CTA; tmp holds `capacity` ints. Each warp
// owns one contiguous chunk of the list: it counts its chunk's keys, a scan over (key, warp) gives every
// warp its first position per key, and the warp then scatters its chunk in order, 32 entries at a time,
// ranking equal keys within a step by lane.
__global__ void __launch_bounds__(kSortThreads) sort_by_cost_kernel(const mfa_block_desc* desc, int nblocks,
                                                                    int32_t* list, int capacity,
                                                                    const int32_t* d_count, int32_t* tmp,
                                                                    uint32_t* status) {
  __shared__ int pos[kSortWarps][kKeys];  // per warp and key: count, then next position
  __shared__ int base[kKeys];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int count = d_count ? *d_count : capacity;
  if (count < 0 || count > capacity) {
    if (tid == 0) flag(status, MFA_DEV_BAD_LIST);
    count = max(0, min(count, capacity));
  }
  for (int e = tid; e < kSortWarps * kKeys; e += kSortThreads) pos[e / kKeys][e % kKeys] = 0;
  __syncthreads();
  const int chunk = (count + kSortWarps - 1) / kSortWarps;
  const int m0 = min(count, warp * chunk), m1 = min(count, m0 + chunk);
  for (int m = m0 + lane; m < m1; m += 32) {
    const int b = list[m];
    tmp[m] = b;
    atomicAdd(&pos[warp][cost_key(desc, nblocks, b)], 1);
  }
  __syncthreads();
  if (tid < kKeys) {  // per key: offsets of the warps' chunks, and the key's total
    int acc = 0;
    for (int w = 0; w < kSortWarps; ++w) {
      const int c = pos[w][tid];
      pos[w][tid] = acc;
      acc += c;
    }
    base[tid] = acc;
  }
  __syncthreads();
  if (tid == 0) {  // first position of every key: exclusive scan of the totals in key order
    int acc = 0;
    for (int k = 0; k < kKeys; ++k) {
      const int c = base[k];
      base[k] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int e = tid; e < kSortWarps * kKeys; e += kSortThreads) pos[e / kKeys][e % kKeys] += base[e % kKeys];
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  for (int mb = m0; mb < m1; mb += 32) {
    const int m = mb + lane;
    const bool valid = m < m1;
    const int b = valid ? tmp[m] : -1;
    const int k = valid ? cost_key(desc, nblocks, b) : kKeys;  // kKeys: no entry
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    if (valid) list[pos[warp][k] + __popc(peers & below)] = b;
    __syncwarp();
    if (valid && (peers >> lane) == 1u) pos[warp][k] += __popc(peers);  // the highest lane of each key
    __syncwarp();
  }
}

// table[b] = position of block b in the decoded list (its cache slot), -1 for blocks not decoded.
__global__ void brick_table_kernel(const int32_t* list, int capacity, const int32_t* d_count, int nblocks,
                                   int32_t* table) {
  int count = d_count ? *d_count : capacity;
  count = max(0, min(count, capacity));
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblocks; b += gridDim.x * blockDim.x) table[b] = -1;
  __syncthreads();  // (grid is one CTA: see launch) clears before the scatter
  for (int m = threadIdx.x; m < count; m += blockDim.x) {
    const int b = list[m];
    if (b >= 0 && b < nblocks) table[b] = m;
  }
}

}  // namespace
}  // namespace mfa

using namespace mfa;

struct mfa_frame_graph {
  mfa_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t* d_tmp = nullptr;
  int64_t kernels = 0;  // kernel nodes per replay
};

extern "C" {

int mfa_frame_graph_create(mfa_ctx* ctx, mfa_frame_graph** out, const mfa_frame_desc* fd) {
  if (!ctx || !out || !fd) return MFA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!fd->d_desc || !fd->d_list || !fd->d_count || !fd->d_knots || !fd->d_cps || !fd->d_cache ||
      fd->nblocks < 1 || fd->list_capacity < 1 || fd->slot_stride_voxels < 1)
    return MFA_ERR_INVALID_ARG;
  if (fd->flags & ~(MFA_FRAME_SORT_BY_COST | MFA_FRAME_RAYCAST | MFA_FRAME_CUBES | MFA_FRAME_APRON))
    return MFA_ERR_INVALID_ARG;
  const bool rc = (fd->flags & MFA_FRAME_RAYCAST) != 0;
  const bool cubes = (fd->flags & MFA_FRAME_CUBES) != 0;
  const bool apron = (fd->flags & MFA_FRAME_APRON) != 0;
  if (cubes && apron) return MFA_ERR_INVALID_ARG;
  if (fd->precision < MFA_PREC_FP32 || fd->precision > MFA_PREC_SPLIT_BF16) return MFA_ERR_INVALID_ARG;
  if (rc && (!fd->d_brick_table || !fd->view || !fd->d_tf || !fd->d_image)) return MFA_ERR_INVALID_ARG;
  if (rc && (int64_t)fd->brick_dims[0] * fd->brick_dims[1] * fd->brick_dims[2] != fd->nblocks)
    return MFA_ERR_INVALID_ARG;
  mfa_frame_graph* g = new (std::nothrow) mfa_frame_graph();
  if (!g) return MFA_ERR_CUDA;
  g->ctx = ctx;
  if (cudaMalloc(&g->d_tmp, sizeof(int32_t) * fd->list_capacity) != cudaSuccess) {
    delete g;
    return MFA_ERR_CUDA;
  }
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    mfa_frame_graph_destroy(g);
    return MFA_ERR_CUDA;
  }
  int status = MFA_OK;
  const int64_t launches0 = ctx->launches;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) status = MFA_ERR_CUDA;
  if (status == MFA_OK && (fd->flags & MFA_FRAME_SORT_BY_COST)) {
    sort_by_cost_kernel<<<1, kSortThreads, 0, s>>>(fd->d_desc, fd->nblocks, fd->d_list, fd->list_capacity,
                                                   fd->d_count, g->d_tmp, ctx->d_status);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) status = MFA_ERR_CUDA;
  }
  if (status == MFA_OK)
    status = mfa_decode_blocks(ctx, fd->d_desc, fd->nblocks, fd->d_list, fd->list_capacity, fd->d_count,
                               fd->d_knots, fd->knots_len, fd->d_cps, fd->cps_len, fd->d_cache,
                               fd->slot_stride_voxels, fd->list_capacity, &fd->bounds, fd->precision,
                               MFA_DECODE_LIST_SLOTS | (cubes ? MFA_DECODE_CUBES : 0u) | (apron ? MFA_DECODE_APRON : 0u), s);
  if (status == MFA_OK && rc) {
    brick_table_kernel<<<1, 1024, 0, s>>>(fd->d_list, fd->list_capacity, fd->d_count, fd->nblocks,
                                          fd->d_brick_table);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) status = MFA_ERR_CUDA;
    if (status == MFA_OK && apron)
      status = mfa_fill_aprons(ctx, fd->d_cache, fd->slot_stride_voxels, fd->list_capacity, fd->d_brick_table,
                               fd->brick_dims, fd->brick_n, s);
    if (status == MFA_OK)
      status = mfa_raycast_ex(ctx, fd->d_cache, fd->slot_stride_voxels, fd->list_capacity, fd->d_brick_table,
                              fd->brick_dims, fd->brick_n, fd->view, fd->d_tf, fd->tf_n, fd->d_image,
                              cubes ? MFA_RAYCAST_CUBES : apron ? MFA_RAYCAST_APRON : 0u, s);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  g->kernels = ctx->launches - launches0;
  ctx->launches = launches0;  // captured, not launched
  if (status == MFA_OK && (ec != cudaSuccess || !graph)) status = MFA_ERR_CUDA;
  g->graph = graph;
  if (status == MFA_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) status = MFA_ERR_CUDA;
  cudaStreamDestroy(s);
  if (status != MFA_OK) {
    mfa_frame_graph_destroy(g);
    return status;
  }
  *out = g;
  return MFA_OK;
}

int mfa_frame_graph_launch(mfa_frame_graph* g, void* stream) {
  if (!g || !g->exec) return MFA_ERR_INVALID_ARG;
  if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return MFA_ERR_CUDA;
  g->ctx->launches += g->kernels;
  return MFA_OK;
}

void mfa_frame_graph_destroy(mfa_frame_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  cudaFree(g->d_tmp);
  delete g;
}

}  // extern "C"
