// Internal launch interfaces between the C-ABI layer and the kernel files (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mfa.h"

struct mfa_ctx;

namespace mfa {

constexpr int kDecodeThreads = 256;
constexpr size_t kMaxDynSmem = 227 * 1024;

struct DecodeParams {
  const mfa_block_desc* desc;
  int nblocks;
  const int32_t* list;
  int list_len;
  const int32_t* count;
  const float* knots;
  int64_t knots_len;
  const float* cps;
  int64_t cps_len;
  float* cache;
  int64_t slot_stride;
  int64_t nslots;
  mfa_bounds bounds;
  uint32_t flags;
  uint32_t* status;
  uint32_t* counter;
  int ks;     // z-planes per work unit
  int slabs;  // work units per block = ceil(max_nsamp / ks)
};

struct DecodeTuning {
  int ks = 0;    // 0 = default
  int grid = 0;  // 0 = one wave of resident CTAs
};

int decode_fp32(mfa_ctx* ctx, DecodeParams prm, const DecodeTuning& tune, cudaStream_t stream);

int basis_tables(mfa_ctx* ctx, const mfa_block_desc* d_desc, const float* d_knots, int64_t knots_len,
                 int32_t* d_span, float* d_basis, cudaStream_t stream);

struct RaycastParams {
  const float4* cache;
  int64_t slot_stride;
  int64_t nslots;
  const int32_t* table;
  int B[3];
  int brick_n;
  const float4* tf;
  int tf_n;
  float4* image;
  int W, H;
  // camera frame (host FP64 rounded to FP32)
  float eye[3], fwd[3], right[3], up[3];
  float tan_w, tan_h;
  float dt;            // world-space step
  int max_samples;     // upper bound on samples per ray (the box diagonal over dt, plus slack)
  float half[3];       // (N_a - 1)/2: world -> voxel scale
  float gscale[3];     // (N_a - 1)/(2 (brick_n - 1)): parametric -> world gradient scale
  float step_voxels, opacity_max, ka, kd, ks, shininess, vmin, vmax;
};

int raycast(mfa_ctx* ctx, const RaycastParams& prm, cudaStream_t stream);

struct AdjointParams {
  const mfa_block_desc* desc;
  int nblocks;
  const float* knots;
  int64_t knots_len;
  const float* residual;
  int64_t slot_stride;
  int64_t nslots;
  const float* cps;  // non-null: residual = decode(cps) - residual
  float* grad;
  int64_t cps_len;
  mfa_bounds bounds;
  uint32_t* status;
  uint32_t* counter;
};

int adjoint(mfa_ctx* ctx, const AdjointParams& prm, cudaStream_t stream);

}  // namespace mfa
