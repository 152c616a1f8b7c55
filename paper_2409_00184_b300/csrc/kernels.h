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
  int ks;     // z-planes per slab
  int group;  // slabs per work unit
  // decode fused with the comparison to the fitted samples (FP32 path; data == nullptr: plain decode)
  const float* data = nullptr;  // sample grids, slot-addressed (data_stride floats per slot)
  int64_t data_stride = 0;
  float* residual = nullptr;    // nullable: f - D per voxel, same addressing as data
  double* sq = nullptr;         // nullable: per item, sum of squared differences, then (finished) the RMSE
  int slabs;  // work units per block = ceil(max_nsamp / (ks * group))
};

struct DecodeTuning {
  int ks = 0;           // 0 = default
  int ctas_per_sm = 0;  // 0 = as many as fit
};

int decode_fp32(mfa_ctx* ctx, DecodeParams prm, const DecodeTuning& tune, cudaStream_t stream);

// Tensor-core decode (BF16, FP16, split-BF16) over sub-cubes whose bands lie within 16 control points per axis.
int decode_tc(mfa_ctx* ctx, DecodeParams prm, int precision, cudaStream_t stream);

int basis_tables(mfa_ctx* ctx, const mfa_block_desc* d_desc, const float* d_knots, int64_t knots_len,
                 int32_t* d_span, float* d_basis, cudaStream_t stream);

struct RaycastParams {
  const float4* cache;
  int64_t slot_stride;
  int64_t nslots;
  const int32_t* table;
  int B[3];
  int brick_n;
  int log2n;  // log2(brick_n) when brick_n is a power of two, else -1
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
  unsigned long long* samples;  // marched samples are added here (one atomic per warp)
  bool cubes = false;           // cache bricks in the cube layout (MFA_RAYCAST_CUBES)
  bool apron = false;           // cache bricks with a one-voxel apron (MFA_RAYCAST_APRON)
  uint32_t* touched = nullptr;  // non-null: sector bitmap of the cache (MFA_RAYCAST_COUNT_SECTORS)
  unsigned long long* sectors = nullptr;  // distinct sectors of the bitmap are added here
};

int raycast(mfa_ctx* ctx, const RaycastParams& prm, cudaStream_t stream);

// Apron planes of every brick of a brick table (MFA_DECODE_APRON layout: bricks of n^3 voxels in slots of
// n + 1 planes of n + 1 rows of apron_pitch(n) voxels).
struct ApronParams {
  float4* cache;
  int64_t slot_stride;
  int64_t nslots;
  const int32_t* table;
  int B[3];
  int n;
};

int apron_fill(mfa_ctx* ctx, const ApronParams& prm, cudaStream_t stream);

// Micro-models queried per sample by the direct ray caster (prm.table holds block indices).
struct DirectModels {
  const mfa_block_desc* desc;
  int nblocks;
  const float* knots;
  int64_t knots_len;
  const float* cps;
  int64_t cps_len;
  mfa_bounds bounds;
  uint32_t* status;
};

int raycast_direct(mfa_ctx* ctx, const RaycastParams& prm, const DirectModels& models, cudaStream_t stream);

// Levels of a multi-resolution volume of shared-boundary micro-blocks (mfa_lod_select, mfa_raycast_lod).
struct LodLevels {
  int B0;      // finest blocks per axis
  int n;       // samples per block and axis
  int levels;
  int off[MFA_MAX_LEVELS];  // first global id of every level
};

// Algorithm 4 with per-sample queries of the models prm.table selects per finest block (global ids).
int raycast_lod(mfa_ctx* ctx, const RaycastParams& prm, const DirectModels& models, const LodLevels& lv,
                cudaStream_t stream);

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
  int precision = MFA_PREC_FP32;  // FP32: CUDA-core kernels; BF16 / split-BF16: the tensor-core contraction
};

int adjoint(mfa_ctx* ctx, const AdjointParams& prm, cudaStream_t stream);

// ---- least-squares encode: per-class tables built by the plan, consumed by the contraction ----
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

// Basis-table entry: first nonzero basis index at a sample and the p+1 values there.
struct TabEntry {
  int off;
  float N[MFA_MAX_DEGREE + 1];
};

// Transposed three-axis contraction Y[c][b][a] = sum X[k][j][i] Ax[i][a] Ay[j][b] Az[k][c] per block.
enum ContractMode { kFit = 0, kAdjoint = 1, kGradient = 2 };

struct ContractParams {
  int mode;
  int nblocks;
  // kFit: items + classes + pools from an encode plan
  const EncItem* items;
  const EncClass* classes;
  const float* pinv;
  const TabEntry* tabs;
  double* rmse;          // kFit, nullable
  // kAdjoint / kGradient: descriptors and knots
  const mfa_block_desc* desc;
  const float* knots;
  int64_t knots_len;
  mfa_bounds bounds;
  const float* cps;      // kGradient: control points P
  // all modes
  const float* x;        // sample grids (slot-addressed)
  int64_t slot_stride;
  int64_t nslots;
  float* out;            // control-point-shaped output
  int64_t cps_len;
  uint32_t* status;
  uint32_t* counter;
  int maxC, maxN, pmax;
  int rows32;            // blocks (mostly) have 32-sample x-rows: use the TMA kernel when aligned
};

// Returns MFA_ERR_CAPACITY (without launching) when the block shapes do not fit shared memory.
int contract3(mfa_ctx* ctx, ContractParams prm, cudaStream_t stream);

// The fit (without RMSE) and the adjoint on the tensor cores in BF16 or split-BF16 (precision MFA_PREC_BF16 /
// MFA_PREC_SPLIT_BF16): 32 samples and at most 16 control points per axis, 16-byte-aligned sample grids with a
// slot stride that is a multiple of 4 floats; MFA_ERR_UNSUPPORTED (nothing launched) for any other call. A
// block of another shape in the batch sets MFA_DEV_BAD_DESC and is skipped.
int contract_tc(mfa_ctx* ctx, const ContractParams& prm, int precision, cudaStream_t stream);

}  // namespace mfa
