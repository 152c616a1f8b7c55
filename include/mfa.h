/*
 * mfa.h - C ABI of the B300 micro-model library (Adaptive-FAM hot path, arxiv 2409.00184).
 *
 * A micro-model (Sec. 4.2, Fig. "Micro-model storage layout") is one micro-block of a
 * volume encoded as a clamped trivariate tensor-product B-spline: per axis a degree p,
 * a control-point count C (the paper's NCP) and a knot vector of C + p + 1 values, plus
 * C_x*C_y*C_z control points. The library
 *
 *   - decodes batches of micro-models into a device voxel cache of value and gradient
 *     (the queries valueMicroModel / gradientMicroModel of Algorithm 4, evaluated on
 *     each block's regular sample grid instead of per ray sample),
 *   - ray-casts that cache front to back with early termination (Algorithm 4),
 *   - fits micro-models to sample blocks by least squares (the model(NCP, degree) call
 *     of Algorithm 1), and
 *   - applies the transposed decode (adjoint) that turns that fit into a gradient method.
 *
 * Conventions for every entry point
 *   - Plain C types only. "d_" pointers are CUDA device pointers the CALLER allocates and
 *     owns; "h_" pointers are host memory. The library allocates device memory only in
 *     mfa_ctx_create and mfa_encode_plan_create, and frees it in the matching destroy.
 *   - `stream` is a cudaStream_t (0 = legacy default stream). Calls enqueue work on it
 *     and return without synchronising, except mfa_ctx_device_status (documented there).
 *   - Return value: MFA_OK (0) or a negative MFA_ERR_* code. Arguments are checked on the
 *     host before anything is enqueued; nothing is enqueued when a call fails.
 *   - Checks that need device data (descriptor contents, knot order, list entries) run
 *     in the kernels: a block that fails them is skipped (its output is left untouched)
 *     and a bit is OR-ed into the context's device status word (MFA_DEV_* below), which
 *     mfa_ctx_device_status reads.
 *   - A context is not thread-safe; use one per host thread (or serialise calls).
 *
 * Layouts
 *   - knots: float32; a block's axis-a vector is knots[knot_off[a] .. knot_off[a]+C_a+p_a].
 *   - control points: float32, cps[cp_off + a + C_x*(b + C_y*c)] = P_abc (x fastest).
 *   - sample grid of a block: n_x*n_y*n_z samples at parameters u_i = i/(n-1) (FP32
 *     quotient), stored [z][y][x] (x fastest) in the block's slot:
 *     base + slot*slot_stride_voxels.
 *   - decoded cache voxel: 4 floats (f, df/du, df/dv, df/dw); gradients are with respect
 *     to the block parameters u, v, w in [0, 1] (divide by n-1 for per-voxel units).
 *     Voxels of a slot are [z][y][x] (x fastest), or with MFA_DECODE_CUBES (blocks with even
 *     n per axis) in 2x2x2-voxel cubes: voxel (x, y, z) at 8*(((z/2)*(n_y/2) + y/2)*(n_x/2) + x/2)
 *     + 4*(z%2) + 2*(y%2) + x%2, so the 8 voxels of a cube (128 bytes of float4) share a cache
 *     line; a block with an odd n sets MFA_DEV_BAD_DESC and is skipped. With MFA_DECODE_APRON
 *     the slot holds A_x(n_y+1)(n_z+1) voxels with A_x = n_x+1 rounded up to even, voxel (x, y, z)
 *     at ((z*(n_y+1) + y)*A_x + x): for an even n_x and an even slot stride every row starts on a
 *     32-byte sector. The decode writes x < n_x,
 *     y < n_y, z < n_z; mfa_fill_aprons writes the planes x = n_x, y = n_y, z = n_z from the
 *     neighbouring bricks and zeros the padding columns n_x < x < A_x (a block whose apron volume
 *     exceeds slot_stride_voxels sets MFA_DEV_BAD_RANGE and is skipped).
 */
#ifndef MFA_H
#define MFA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (return values) -------------------------------------------------- */
#define MFA_OK               0
#define MFA_ERR_INVALID_ARG -1   /* null/misaligned pointer, size out of range, bad enum */
#define MFA_ERR_UNSUPPORTED -2   /* valid request this build does not implement          */
#define MFA_ERR_CUDA        -3   /* a CUDA runtime call failed (launch, copy, malloc)    */
#define MFA_ERR_TIMEOUT     -4   /* a bounded device wait gave up (see MFA_DEV_TIMEOUT)   */
#define MFA_ERR_CAPACITY    -5   /* request exceeds a fixed library limit                */
#define MFA_ERR_DEVICE      -6   /* the device status word holds error bits              */
#define MFA_ERR_IO          -7   /* a model store could not be written or read           */

/* ---- device status word bits (mfa_ctx_device_status) -------------------------------- */
#define MFA_DEV_BAD_DESC   0x1u  /* degree/ncp/nsamp outside the launch bounds or limits */
#define MFA_DEV_BAD_KNOTS  0x2u  /* knot vector decreasing, or t_p >= t_C (empty domain) */
#define MFA_DEV_BAD_RANGE  0x4u  /* knot/cp offset or slot outside the stated lengths    */
#define MFA_DEV_BAD_LIST   0x8u  /* a list entry outside [0, nblocks), or count > length */
#define MFA_DEV_TIMEOUT    0x10u /* a bounded wait (mbarrier/TMA/MMA) gave up            */
#define MFA_DEV_NOT_SPD    0x20u /* an N^T N Cholesky pivot was not positive (C > n?)    */

/* ---- precisions of the decode contractions ------------------------------------------ */
#define MFA_PREC_FP32        0   /* FP32 FMA on the CUDA cores, banded (p+1 terms)       */
#define MFA_PREC_BF16        1   /* tensor cores, BF16 operands, FP32 accumulation       */
#define MFA_PREC_FP16        2   /* tensor cores, FP16 operands, FP32 accumulation       */
#define MFA_PREC_SPLIT_BF16  3   /* tensor cores, hi+lo BF16 split (3 products), FP32 acc */

/* ---- decode flags ------------------------------------------------------------------- */
#define MFA_DECODE_VALUE_ONLY  0x1u /* write f only: 1 float per voxel instead of 4       */
#define MFA_DECODE_LIST_SLOTS  0x2u /* with a list: item m goes to slot m (not desc.slot) */
#define MFA_DECODE_CUBES       0x4u /* cache voxels in the cube layout (see Layouts); FP32 only */
#define MFA_DECODE_APRON       0x8u /* cache voxels with a one-voxel apron (see Layouts)            */

/* ---- fixed limits -------------------------------------------------------------------- */
#define MFA_MAX_DEGREE 3
#define MFA_MAX_NCP    32
#define MFA_MAX_NSAMP  64

/* One micro-block (72 bytes, 8-byte aligned). Axis order everywhere is x, y, z. */
typedef struct {
  int32_t degree[3];   /* p per axis, 1 <= p <= MFA_MAX_DEGREE                         */
  int32_t ncp[3];      /* C per axis (the paper's NCP), p+1 <= C <= MFA_MAX_NCP          */
  int32_t nsamp[3];    /* n per axis, 2 <= n <= MFA_MAX_NSAMP                            */
  int32_t slot;        /* slot of the block's sample grid / cache entry                  */
  int64_t knot_off[3]; /* first knot of each axis in the knots array                     */
  int64_t cp_off;      /* first control point in the cps array                           */
} mfa_block_desc;

/* Upper bounds of a batch, stated by the caller; they size shared memory and select the
 * kernel instance. Every block must satisfy degree <= max_degree, ncp <= max_ncp and
 * nsamp <= max_nsamp on every axis (else MFA_DEV_BAD_DESC and the block is skipped). */
typedef struct {
  int32_t max_degree;
  int32_t max_ncp;
  int32_t max_nsamp;
} mfa_bounds;

typedef struct mfa_ctx mfa_ctx;

/* Create a context on CUDA device `device`: queries the device, allocates the device
 * status word and work-queue counters. Returns MFA_ERR_UNSUPPORTED on a device that is
 * not compute capability 10.3 (this library is built for sm_103a only). */
int  mfa_ctx_create(mfa_ctx** out, int device);
void mfa_ctx_destroy(mfa_ctx* ctx);
const char* mfa_status_string(int status);
/* Sizes in bytes of the structs this header declares, for bindings that mirror them:
 * out[0] mfa_block_desc, out[1] mfa_bounds, out[2] mfa_decode_tiling, out[3] mfa_view,
 * out[4] mfa_frame_desc. Writes the first min(n, 5) of them (none when out is NULL) and returns
 * 5, the number of structs. Host only: needs no device and no context. */
int mfa_abi_struct_sizes(int32_t* out, int32_t n);

/* Synchronise `stream`, copy the device status word to *status and, if `clear`, reset
 * it to 0. Returns MFA_OK, or MFA_ERR_CUDA if the stream reported an error. */
int mfa_ctx_device_status(mfa_ctx* ctx, uint32_t* status, int clear, void* stream);

/* Number of kernels this context launched since creation (all entry points). */
int64_t mfa_ctx_launch_count(const mfa_ctx* ctx);

/* Device statistics kept by the context (64-bit counters, summed over launches). */
#define MFA_STAT_RAY_SAMPLES 0   /* samples marched by mfa_raycast (after early termination) */
#define MFA_STAT_RAY_SECTORS 1   /* distinct 32-byte cache sectors read by a ray cast with
                                    MFA_RAYCAST_COUNT_SECTORS (summed over such launches) */
#define MFA_NUM_STATS        2
/* Synchronises `stream` and copies the first `nstats` counters to stats[]; resets them if `reset`. */
int mfa_ctx_read_stats(mfa_ctx* ctx, uint64_t* stats, int nstats, int reset, void* stream);

/* Tile shape of the FP32 decode for one batch class: `ks` z-planes per work unit and at most
 * `ctas_per_sm` resident CTAs of the persistent grid (0 = library default for either field).
 * A context holds up to 64 entries keyed by (max_degree, max_ncp, max_nsamp) of the call's
 * mfa_bounds; mfa_decode_blocks uses the matching entry, else the defaults. Setting an entry
 * again replaces it; ks is clamped to max_nsamp and lowered when shared memory requires it.
 * Used by the autotuner (paper_2409_00184_b300/autotune.py), which times candidate shapes. */
typedef struct {
  int32_t ks;
  int32_t ctas_per_sm;
} mfa_decode_tiling;
int mfa_ctx_set_decode_tiling(mfa_ctx* ctx, const mfa_bounds* key, const mfa_decode_tiling* tiling);
int mfa_ctx_get_decode_tiling(const mfa_ctx* ctx, const mfa_bounds* key, mfa_decode_tiling* tiling);

/* Eq. 2: the size in bytes of one micro-model file, 1 + ((NCP + degree)*3 + NCP^3)*4.
 * Returns -1 for NCP < 1 or degree < 0. */
int64_t mfa_model_bytes(int32_t ncp, int32_t degree);

/* Host <-> device copies of caller-owned buffers on `stream`, for callers whose sample grids and images
 * live in host memory (the paper's pipeline moves the visible micro-models to the GPU and the frame back,
 * Sec. 4.3): mfa_copy_to_device copies `bytes` from host h_src to device d_dst, mfa_copy_to_host from
 * device d_src to host h_dst. Asynchronous with respect to the host when the host buffer is page-locked
 * (otherwise the copy completes before the call returns). MFA_ERR_INVALID_ARG for null pointers or
 * bytes < 0 (0 bytes: nothing is enqueued), MFA_ERR_CUDA if the copy cannot be enqueued. */
int mfa_copy_to_device(void* d_dst, const void* h_src, int64_t bytes, void* stream);
int mfa_copy_to_host(void* h_dst, const void* d_src, int64_t bytes, void* stream);

/* ---- decode (Algorithm 4's value and gradient queries, batched on sample grids) ----- */
/* Decodes blocks into the cache: for each selected block b and sample (i, j, k),
 *   f   = sum_{a,b,c} N_a(u_i) N_b(v_j) N_c(w_k) P_abc,  and f_u, f_v, f_w with N' in the
 * corresponding factor. Selection: if d_list is NULL every block 0..nblocks-1 is decoded;
 * otherwise the items d_list[0 .. count) where count = *d_count (device int32, read by
 * the kernel, so the call can be replayed from a CUDA graph) or list_len if d_count is
 * NULL; count must be <= list_len (a larger or negative *d_count sets MFA_DEV_BAD_LIST and is
 * clamped to 0 .. list_len; a count of 0 decodes nothing; with no blocks, or an empty list and
 * no d_count, nothing is enqueued). Destination: slot desc.slot, or slot m for item m
 * with MFA_DECODE_LIST_SLOTS. Output per voxel: 4 floats (f, f_u, f_v, f_w), or 1 float
 * with MFA_DECODE_VALUE_ONLY, at d_cache + (slot*slot_stride_voxels + voxel)*width.
 * d_cache must be 16-byte aligned. knots_len / cps_len are the array lengths (floats),
 * used for the range checks. precision: MFA_PREC_FP32 (any supported shape) or, on the tensor
 * cores, MFA_PREC_BF16 / MFA_PREC_FP16 / MFA_PREC_SPLIT_BF16 (row or apron layout, with or
 * without VALUE_ONLY; the cube layout returns MFA_ERR_UNSUPPORTED). The tensor-core decode takes a block in sub-cubes of 32
 * samples per axis, or 16 on an axis with more than 16 control points; every sub-cube's samples
 * must have their nonzero basis functions within 16 consecutive control points per axis. That
 * holds for every block with at most 16 control points per axis, and for uniform knots with up
 * to 24 control points when n >= 32. A sub-cube that breaks it sets MFA_DEV_BAD_DESC and is not
 * written. */
int mfa_decode_blocks(mfa_ctx* ctx,
                      const mfa_block_desc* d_desc, int32_t nblocks,
                      const int32_t* d_list, int32_t list_len, const int32_t* d_count,
                      const float* d_knots, int64_t knots_len,
                      const float* d_cps, int64_t cps_len,
                      float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                      const mfa_bounds* bounds, int32_t precision, uint32_t flags,
                      void* stream);

/* The FP32 decode fused with the comparison to the samples the models were fitted to (the
 * residual of the least-squares fit of Algorithm 1's model() and Table 1's RMSE), in one pass:
 * selection, destination, flags and cache output as mfa_decode_blocks with MFA_PREC_FP32; and for every
 * decoded voxel r = f - D, with D at d_data + slot*data_slot_stride + voxel (FP32, [z][y][x] per slot,
 * slot = the block's destination slot; a block with more voxels than data_slot_stride sets
 * MFA_DEV_BAD_RANGE and is skipped).
 *   d_residual (nullable): r written with the same addressing as d_data.
 *   d_rmse (nullable, FP64, one per selected item: list position, or block index without a list):
 *     sqrt(mean r^2) over the block's voxels; squares are summed per thread in FP32 (Kahan) and
 *     across threads in FP64. NaN for an item whose block failed its checks. The call zeroes d_rmse
 *     before the decode and finishes it with one more kernel (d_rmse needs max(list_len, nblocks)
 *     entries). */
int mfa_decode_compare_blocks(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks,
                              const int32_t* d_list, int32_t list_len, const int32_t* d_count,
                              const float* d_knots, int64_t knots_len, const float* d_cps, int64_t cps_len,
                              float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                              const mfa_bounds* bounds, uint32_t flags, const float* d_data,
                              int64_t data_slot_stride, float* d_residual, double* d_rmse, void* stream);

/* Fills per-axis basis tables for one block, for testing the span search and the
 * Cox-de Boor recurrence on their own: for each axis a and sample i, span[a*MAXN + i]
 * (int32) and N, N' at the p+1 nonzero functions, basis[((a*MAXN + i)*2 + {0,1})*4 + r]
 * (float32, r < p+1; unused entries 0), MAXN = MFA_MAX_NSAMP. d_desc points at one
 * descriptor. */
int mfa_basis_tables(mfa_ctx* ctx, const mfa_block_desc* d_desc,
                     const float* d_knots, int64_t knots_len,
                     int32_t* d_span, float* d_basis, void* stream);

/* ---- adjoint (transposed decode) ----------------------------------------------------- */
/* For each block b: dP_abc = sum_{i,j,k} R_b[k][j][i] N_a(u_i) N_b(v_j) N_c(w_k), with R_b
 * the block's residual grid at d_residual + slot*slot_stride_voxels (1 float per sample).
 * Written to d_grad_cps at the block's cp_off (same layout as the control points);
 * overwrites, does not accumulate. With d_cps non-NULL the residual is formed in the
 * kernel instead: R = decode_value(d_cps) - d_residual (d_residual then holds the data
 * samples D), which is the gradient of 0.5*||decode(P) - D||^2.
 * precision: MFA_PREC_FP32 (CUDA cores, any supported shape), or MFA_PREC_BF16 /
 * MFA_PREC_SPLIT_BF16 on the tensor cores (BF16 operands, split-BF16 A*B ~ Ahi*Bhi + Ahi*Blo +
 * Alo*Bhi, FP32 accumulation) for bounds with max_nsamp = 32 and max_ncp <= 16, d_cps NULL,
 * d_residual 16-byte aligned and slot_stride_voxels a multiple of 4 (otherwise, and for
 * MFA_PREC_FP16, MFA_ERR_UNSUPPORTED and nothing is enqueued); a block of another shape in such a
 * batch sets MFA_DEV_BAD_DESC and is skipped. */
int mfa_adjoint_blocks(mfa_ctx* ctx,
                       const mfa_block_desc* d_desc, int32_t nblocks,
                       const float* d_knots, int64_t knots_len,
                       const float* d_residual, int64_t slot_stride_voxels, int64_t nslots,
                       const float* d_cps, float* d_grad_cps, int64_t cps_len,
                       const mfa_bounds* bounds, int32_t precision, void* stream);

/* Camera and shading of a ray cast (Algorithm 4), see mfa_raycast. */
typedef struct {
  float eye[3], target[3], up[3];
  float fov_y_deg;
  int32_t width, height;
  float step_voxels;   /* sample spacing in voxels of the longest axis (1 = one per voxel) */
  float opacity_max;   /* early termination once accumulated opacity exceeds this          */
  float ka, kd, ks, shininess;  /* headlight Blinn-Phong coefficients                     */
  float vmin, vmax;    /* value range mapped onto the transfer function                   */
} mfa_view;

/* ---- one frame as a CUDA graph (the per-POV decode + render of Sec. 4.3, Algorithm 4) - */
#define MFA_FRAME_SORT_BY_COST 0x1u /* order the visible list by decreasing max(C) first     */
#define MFA_FRAME_RAYCAST      0x2u /* build the brick table and ray-cast after the decode   */
#define MFA_FRAME_CUBES        0x4u /* decode into (and ray-cast from) the cube layout        */
#define MFA_FRAME_APRON        0x8u /* decode into the apron layout; with MFA_FRAME_RAYCAST   */
                                    /* also fill the aprons and ray-cast with them, which     */
                                    /* needs slot_stride_voxels >= A(n+1)^2, A = n+1 rounded  */
                                    /* up to even, n = brick_n (else creation returns         */
                                    /* MFA_ERR_INVALID_ARG); not with MFA_FRAME_CUBES         */

/* Everything a frame reads; pointers and sizes are fixed when the graph is captured. Per frame
 * the caller writes the visible block ids into d_list[0 .. *d_count) (device memory, count <=
 * list_capacity) and replays the graph. Decoded block m of the (ordered) list goes to cache slot
 * m (the cache holds list_capacity slots of slot_stride_voxels float4). With MFA_FRAME_RAYCAST the
 * blocks are the bricks of a Bx*By*Bz volume (nblocks = Bx*By*Bz, brick id z-major) of brick_n^3
 * samples each; the graph rewrites d_brick_table (nblocks int32: list position or -1) and renders
 * into d_image as mfa_raycast does. precision: MFA_PREC_* of the captured decode (0, a zeroed
 * descriptor, is FP32); the tensor-core precisions take the row or the apron layout and the
 * shapes mfa_decode_blocks gives them (otherwise creation returns MFA_ERR_UNSUPPORTED). */
typedef struct {
  const mfa_block_desc* d_desc;
  int32_t nblocks;
  int32_t* d_list;            /* list_capacity int32, reordered in place by SORT_BY_COST */
  int32_t list_capacity;
  const int32_t* d_count;     /* device int32: the frame's number of visible blocks */
  const float* d_knots;
  int64_t knots_len;
  const float* d_cps;
  int64_t cps_len;
  float* d_cache;
  int64_t slot_stride_voxels;
  mfa_bounds bounds;
  uint32_t flags;             /* MFA_FRAME_* */
  /* ray cast (MFA_FRAME_RAYCAST only) */
  int32_t* d_brick_table;
  int32_t brick_dims[3];
  int32_t brick_n;
  const mfa_view* view;
  const float* d_tf;
  int32_t tf_n;
  float* d_image;
  int32_t precision;          /* MFA_PREC_* of the decode */
} mfa_frame_desc;

typedef struct mfa_frame_graph mfa_frame_graph;
/* Captures the frame's kernels (cost ordering, persistent decode with the device-side count,
 * brick table, ray cast) into a CUDA graph on a private stream and instantiates it. Allocates a
 * list_capacity int32 scratch for the ordering. The mfa_view is read at capture time. */
int  mfa_frame_graph_create(mfa_ctx* ctx, mfa_frame_graph** out, const mfa_frame_desc* frame);
/* Replays the captured frame on `stream`. */
int  mfa_frame_graph_launch(mfa_frame_graph* graph, void* stream);
void mfa_frame_graph_destroy(mfa_frame_graph* graph);

/* ---- least-squares encode (Algorithm 1's model(NCP, degree)) ------------------------- */
/* A plan validates a batch on the host, copies its descriptors and knots to the device
 * and groups the axes into classes of equal (knots, p, C, n). Creating it also computes, per
 * class, M = N^T N and its Cholesky factor in FP64 and the pseudo-inverse (N^T N)^-1 N^T
 * (on the legacy default stream, synchronised before the call returns; a class whose M fails
 * the pivot check sets MFA_DEV_NOT_SPD in the context status). Executing the plan fits every
 * block: P = D x_1 N_x^+ x_2 N_y^+ x_3 N_z^+ (the exact least-squares solution of the
 * Kronecker system), and optionally its RMSE over the samples in FP64 (Table 1's error
 * metric). Requires p+1 <= C <= n per axis. */
typedef struct mfa_encode_plan mfa_encode_plan;
int  mfa_encode_plan_create(mfa_ctx* ctx, mfa_encode_plan** out,
                            const mfa_block_desc* h_desc, int32_t nblocks,
                            const float* h_knots, int64_t knots_len, int64_t cps_len);
/* Frees the plan's device tables with cudaFree, which waits for the device's pending work first, so a plan
 * may be destroyed right after the fits that use it have been enqueued (at the cost of that wait). */
void mfa_encode_plan_destroy(mfa_encode_plan* plan);
int  mfa_encode_blocks(mfa_ctx* ctx, const mfa_encode_plan* plan,
                       const float* d_data, int64_t slot_stride_voxels, int64_t nslots,
                       float* d_cps_out, double* d_rmse /* nullable, one per block */,
                       void* stream);

/* mfa_encode_blocks in a chosen arithmetic (the same least-squares fit of Algorithm 1's model()).
 * MFA_PREC_FP32: mfa_encode_blocks. MFA_PREC_BF16 / MFA_PREC_SPLIT_BF16: the three pseudo-inverse
 * contractions P = D x_1 Px x_2 Py x_3 Pz run on the tensor cores with BF16 operands (split-BF16:
 * A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi, each stage's FP32 result split again) and FP32 accumulation; the
 * pseudo-inverses are the plan's (FP64-built, stored FP32). For plans whose blocks all have 32 samples
 * and at most 16 control points per axis, with d_rmse NULL, d_data 16-byte aligned and
 * slot_stride_voxels a multiple of 4; otherwise (and for MFA_PREC_FP16) MFA_ERR_UNSUPPORTED and nothing
 * is enqueued. Other checks as mfa_encode_blocks. */
int  mfa_encode_blocks_ex(mfa_ctx* ctx, const mfa_encode_plan* plan,
                          const float* d_data, int64_t slot_stride_voxels, int64_t nslots,
                          float* d_cps_out, double* d_rmse, int32_t precision, void* stream);

/* In-level adaptive encoding, Eq. 4 (Sec. 4.2.2): NCP* = the smallest NCP whose error is below the
 * bound e. d_errors holds, candidate-major, one error per (candidate, block):
 * d_errors[c*nblocks + b] = Error(h_ncp[c]) of block b, e.g. the RMSE that mfa_encode_blocks
 * wrote for a batch fitted with h_ncp[c] control points per axis. For every block,
 * d_ncp_out[b] = min { h_ncp[c] : d_errors[c*nblocks + b] < bound } over all candidates (the
 * exhaustive search of Eq. 4, whatever the order of the candidates), or -1 when no candidate
 * meets the bound; a NaN error never meets it. h_ncp (host, ncand entries) must be positive.
 * Device buffers: d_errors (FP64, ncand*nblocks, 8-byte aligned), d_ncp_out (int32, nblocks).
 * Returns MFA_ERR_INVALID_ARG for a null ctx or h_ncp, ncand < 1 or > 64, nblocks < 0, a
 * non-positive candidate or a NaN bound, and (when nblocks > 0) null or misaligned device
 * buffers; nblocks = 0 enqueues nothing and accepts null device buffers. */
int mfa_select_ncp(mfa_ctx* ctx, const double* d_errors, int32_t ncand, const int32_t* h_ncp,
                   int64_t nblocks, double bound, int32_t* d_ncp_out, void* stream);

/* Multi-resolution partition (Sec. 4.2 and Algorithm 1): the micro-blocks of one level of detail.
 * d_field holds dims[0] x dims[1] x dims[2] FP32 samples, [z][y][x] (x fastest). Level `stride`
 * (1, 2, 4, ...) cuts the field into blocks of n*stride samples per axis (dims[a] must be a
 * multiple of n*stride) and keeps every stride-th sample of each, so every micro-block has n^3
 * samples. Block (bx, by, bz) has id (bz*By + by)*Bx + bx with B_a = dims[a]/(n*stride); its
 * sample (i, j, k) is field[(bz*n + k)*stride][(by*n + j)*stride][(bx*n + i)*stride].
 * d_ids (nullable) lists the nblocks block ids to gather, else ids 0..nblocks-1 are gathered;
 * entry e goes to slot e of d_out (slot_stride >= n^3 floats per slot). Device buffers 4-byte
 * aligned. Returns MFA_ERR_INVALID_ARG for null pointers, n < 2 or > MFA_MAX_NSAMP, stride < 1,
 * dims not multiples of n*stride, nblocks < 0 or, without d_ids, more than the level's blocks;
 * a listed id outside the level sets MFA_DEV_BAD_LIST and its slot is left untouched. */
int mfa_lod_gather(mfa_ctx* ctx, const float* d_field, const int32_t dims[3], int32_t n, int32_t stride,
                   const int32_t* d_ids, int32_t nblocks, float* d_out, int64_t slot_stride, void* stream);

/* mfa_lod_gather with flags. MFA_LOD_SHARED_BOUNDARY: the blocks of a level share their boundary
 * samples (Sec. 4.2: neighbouring blocks share one sample on the boundary in x, y and z, which keeps
 * the micro-models C0 across blocks): block (bx, by, bz) spans (n-1)*stride intervals from node
 * (bx, by, bz)*(n-1)*stride, its last samples being the next block's first, and each dims[a] - 1 must
 * be a positive multiple of (n-1)*stride (else MFA_ERR_INVALID_ARG). Without the flag, as
 * mfa_lod_gather. Unknown flags: MFA_ERR_INVALID_ARG. */
#define MFA_LOD_SHARED_BOUNDARY 0x1u
int mfa_lod_gather_ex(mfa_ctx* ctx, const float* d_field, const int32_t dims[3], int32_t n, int32_t stride,
                      const int32_t* d_ids, int32_t nblocks, float* d_out, int64_t slot_stride, uint32_t flags,
                      void* stream);

/* ---- levels of detail chosen by distance (Sec. 5.1.3) and rendered by model queries ------------ */
/* A multi-resolution volume of `levels` levels of shared-boundary micro-blocks with n samples per axis
 * (MFA_LOD_SHARED_BOUNDARY): level l = 0 (finest) .. levels-1 has B_l = fine_blocks / 2^l blocks per
 * axis, each spanning (n-1)*2^l intervals of the finest grid of N = fine_blocks*(n-1) + 1 nodes per axis,
 * which maps onto [-1, 1]^3. Global block ids list level 0 first, each level z-major:
 * id = off_l + (bz*B_l + by)*B_l + bx with off_l the number of blocks of the finer levels. */
#define MFA_MAX_LEVELS 8

/* For a point of view `eye` (world coordinates), the level of detail of every part of the volume by the
 * distance from the eye to the block centroids (Sec. 5.1.3: four ranges [0, 0.8], [0.8, 1.6], [1.6, 2.4],
 * [2.4, inf), the nearest taking the finest level): walking from the coarsest level down, a block of
 * level l >= 1 is taken when its centroid lies at distance >= ranges[l-1], else its eight children are
 * examined; level 0 is taken where no coarser block was. The distance test is decided in FP32, one
 * rounded operation at a time: c_a = (2*g0_a + E)/(N - 1) - 1 with g0 the block's first node and E its
 * extent in finest nodes, d^2 = ((c_x - e_x)^2 + (c_y - e_y)^2) + (c_z - e_z)^2 against ranges[l-1]^2.
 * Writes d_table[(fz*B0 + fy)*B0 + fx] = the global id of the block covering finest block (fx, fy, fz),
 * B0 = fine_blocks (int32, B0^3 entries, caller-owned). ranges: levels-1 host floats (NULL when levels
 * is 1). MFA_ERR_INVALID_ARG for null or misaligned pointers, n outside [2, MFA_MAX_NSAMP], levels
 * outside [1, MFA_MAX_LEVELS], fine_blocks not a multiple of 2^(levels-1), a negative or non-finite
 * range or eye coordinate, or a grid of 2^23 finest intervals or more. */
int mfa_lod_select(mfa_ctx* ctx, const float eye[3], int32_t fine_blocks, int32_t n, int32_t levels,
                   const float* ranges, int32_t* d_table, void* stream);

/* Algorithm 4 over a multi-resolution volume with per-sample queries of the selected micro-models
 * (valueMicroModel / gradientMicroModel of Sec. 4.3.3 on the blocks mfa_lod_select chose): the camera,
 * marching, transfer function, shading, compositing and early termination of mfa_raycast, on the
 * finest grid of N = fine_blocks*(n-1) + 1 nodes per axis (one sample per finest node spacing at
 * step_voxels 1). A sample at finest-node coordinates g lies in finest block min(floor(g/(n-1)),
 * fine_blocks - 1) per axis; d_table gives the global id of the block that covers it (its level l,
 * first node g0 and extent E = (n-1)*2^l follow from the id), and the sample is that model's value and
 * gradient at u = (g - g0)/E clamped to [0, 1] (gradient / E in node units). d_desc[id] describes block
 * id: n samples per axis (else MFA_DEV_BAD_DESC and the block reads as zero), degree, NCP, knots and
 * control points as for mfa_decode_blocks; nblocks must cover every id of the levels. Other arguments
 * and checks as mfa_raycast_direct. */
int mfa_raycast_lod(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks, const float* d_knots,
                    int64_t knots_len, const float* d_cps, int64_t cps_len, const mfa_bounds* bounds,
                    const int32_t* d_table, int32_t fine_blocks, int32_t n, int32_t levels, const mfa_view* view,
                    const float* d_tf, int32_t tf_n, float* d_image, void* stream);

/* Allocation-free least-squares encode. The paper has no counterpart to this entry point: it
 * exists for callers that cannot call cudaMalloc - a process whose device memory is reserved
 * by another runtime's memory pool, so that a fresh allocation fails or has to wait for that
 * pool, or a per-frame loop that must not stall, which cudaMalloc and cudaFree can do because
 * they may synchronise the device. It fits the same least-squares control points and RMSE as
 * mfa_encode_plan_create + mfa_encode_blocks, without a context or a plan and without allocating:
 * its scratch (status word, queue counter, class table, block items, pseudo-inverses and basis
 * tables) lives in one fixed 2 MiB device array compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *   - The batch's scratch need, 256 bytes + 168 per axis class + 24 per block + 4*C*n per axis
 *     class (pseudo-inverse) + 20*n per axis class (basis table), each part rounded up to 256
 *     bytes, must fit the 2 MiB; a larger batch returns MFA_ERR_CAPACITY and enqueues nothing.
 *   - Every call looks up the array's device address on the current device (cudaGetSymbolAddress).
 *   - The call copies the host descriptors into the array, enqueues the fit on `stream` and then
 *     synchronises `stream` and copies the status word back synchronously, so it must not be called
 *     while any stream on the device is being captured into a CUDA graph.
 *   - It returns MFA_ERR_DEVICE if a device-side check failed, else MFA_OK. Which check failed (the
 *     MFA_DEV_* bits, e.g. MFA_DEV_NOT_SPD) is not returned; a caller that needs it runs the same
 *     batch through a context (mfa_encode_plan_create, mfa_encode_blocks, mfa_ctx_device_status).
 *   - Every call uses the same array; it clears the status word and counter itself. Calls whose
 *     work overlaps on the GPU (other threads, other streams) race on the array: serialise them.
 * Arguments as for mfa_encode_plan_create (h_desc, nblocks, h_knots, knots_len, cps_len) and
 * mfa_encode_blocks (d_data, slot_stride_voxels, nslots, d_cps_out, d_rmse); the current CUDA
 * device is used. */
int mfa_encode_blocks_noalloc(const mfa_block_desc* h_desc, int32_t nblocks,
                              const float* h_knots, int64_t knots_len,
                              const float* d_data, int64_t slot_stride_voxels, int64_t nslots,
                              float* d_cps_out, int64_t cps_len, double* d_rmse, void* stream);

/* ---- failure-detection self-test --------------------------------------------------- */
/* Test hook; the paper has no counterpart. Launches one CTA whose thread 0 initialises an
 * mbarrier that nothing ever arrives on and waits for it with the library's bounded wait,
 * limited to `polls` polls (1 .. 2^20; each poll is a try_wait plus a short sleep). The wait
 * must give up: the kernel then ORs MFA_DEV_TIMEOUT into the context's status word and
 * returns, exactly as the TMA and tensor-core kernels do when a copy or MMA never completes.
 * No copy or MMA is in flight, so nothing is left running. Returns MFA_ERR_INVALID_ARG for
 * a null ctx or `polls` out of range. */
int mfa_selftest_wait_timeout(mfa_ctx* ctx, int32_t polls, void* stream);

/* ---- ray casting (Algorithm 4) -------------------------------------------------------- */


/* Renders width*height premultiplied RGBA floats (row 0 at the top) into d_image from a
 * decoded cache of bricks of brick_n^3 voxels. d_brick_table[(bz*By + by)*Bx + bx] is the
 * slot of brick (bx, by, bz) or -1 if absent (its nodes read as zero); brick_dims =
 * {Bx, By, Bz}. The volume of B_a*brick_n nodes per axis maps onto [-1, 1]^3. The
 * transfer function is tf_n RGBA float entries over [vmin, vmax]. MFA_ERR_INVALID_ARG for null
 * pointers, d_cache / d_tf / d_image not 16-byte aligned, brick_n < 2, slot_stride_voxels below
 * brick_n^3, brick_dims[a] < 1 or brick_dims[a]*brick_n > 2^20, tf_n < 2, an image side outside
 * 1 .. 16384, a field of view outside (0, 180) degrees, step_voxels <= 0, vmax <= vmin, eye equal to
 * target or up parallel to the view direction, or a step so small that a ray would exceed 2^24
 * samples; MFA_ERR_CAPACITY for tf_n > 1024. */
int mfa_raycast(mfa_ctx* ctx,
                const float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                const mfa_view* view, const float* d_tf, int32_t tf_n,
                float* d_image, void* stream);

/* mfa_raycast with flags. MFA_RAYCAST_CUBES: the cache bricks are in the cube layout that
 * MFA_DECODE_CUBES writes (brick_n must be even; MFA_ERR_INVALID_ARG otherwise). The image is
 * the same, bit for bit, as mfa_raycast's over the same voxels in the [z][y][x] layout: only
 * the addresses of the eight corner loads change. Unknown flags: MFA_ERR_INVALID_ARG. */
#define MFA_RAYCAST_CUBES 0x1u
/* MFA_RAYCAST_APRON: the cache bricks carry the one-voxel apron that MFA_DECODE_APRON and
 * mfa_fill_aprons produce (brick_n <= MFA_MAX_NSAMP and slot_stride_voxels >= A(brick_n+1)^2 with
 * A = brick_n+1 rounded up to even, else MFA_ERR_INVALID_ARG); every cell of a present brick then
 * reads its eight corners from its own slot. Same image, bit for bit, as mfa_raycast over the same
 * voxels. */
#define MFA_RAYCAST_APRON 0x2u
/* MFA_RAYCAST_COUNT_SECTORS: a measuring variant of the same ray cast (same image, bit for bit) that
 * also records every 32-byte sector of d_cache its corner loads read, and adds the number of distinct
 * sectors to MFA_STAT_RAY_SECTORS: the cache bytes the ray cast must read at least once (its
 * algorithmic bytes from memory). It is much slower (one atomic per corner load) and is meant for
 * measurement, not rendering. The context allocates a bitmap of one bit per sector of the cache
 * (nslots * slot_stride_voxels / 2 bits) on first use and keeps it until destroyed. Power-of-two
 * brick_n from 8 to 64 only (the persistent queue kernel), else MFA_ERR_UNSUPPORTED. */
#define MFA_RAYCAST_COUNT_SECTORS 0x4u
int mfa_raycast_ex(mfa_ctx* ctx,
                   const float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                   const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                   const mfa_view* view, const float* d_tf, int32_t tf_n,
                   float* d_image, uint32_t flags, void* stream);

/* Writes the apron of every brick of d_brick_table (layout of MFA_DECODE_APRON, bricks of brick_n^3
 * voxels in slots of at least A(brick_n+1)^2, A = brick_n+1 rounded up to even): voxel
 * (x, y, z) of brick (bx, by, bz) with
 * x, y or z equal to brick_n (and x, y, z <= brick_n) becomes voxel (x mod brick_n, y mod brick_n,
 * z mod brick_n) of brick (bx + [x = n], by + [y = n], bz + [z = n]), or zero when that brick lies
 * outside the volume or is absent (-1); the padding voxels brick_n < x < A become zero. Reads interior
 * voxels only and writes apron and padding voxels only, 4 floats each. Bricks with slot -1 are
 * skipped. Returns MFA_ERR_INVALID_ARG for null or misaligned pointers, brick_n outside
 * 2 .. MFA_MAX_NSAMP, a slot stride below A(brick_n+1)^2 or bad brick_dims. */
int mfa_fill_aprons(mfa_ctx* ctx, float* d_cache, int64_t slot_stride_voxels, int64_t nslots,
                    const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n, void* stream);

/* Algorithm 4 with per-sample queries of the micro-models instead of a decoded cache: the same rays,
 * transfer function, shading and compositing as mfa_raycast, but every sample evaluates the value
 * and parametric gradient of the B-spline model of its brick (the paper's valueMicroModel and
 * gradientMicroModel). d_brick_table[(bz*By + by)*Bx + bx] is the block index (into d_desc) of
 * brick (bx, by, bz), or -1 if absent (reads as zero). Every block must have brick_n samples per
 * axis: its model covers nodes b*brick_n .. b*brick_n + brick_n - 1 of the brick grid (parameter
 * u = (g - b*brick_n)/(brick_n - 1)); in the one-node gap before the next brick the sample is the
 * linear blend, along that axis, of the two models at their common boundary (multilinear where
 * gaps of several axes meet), as trilinear interpolation of a decoded cache would be there.
 * Descriptors, knots and control points as for mfa_decode_blocks (bounds: the batch's maxima,
 * max_nsamp >= brick_n); a block that fails its checks reads as absent and sets its status bit.
 * Samples marched add to MFA_STAT_RAY_SAMPLES. The view, transfer function, image and brick grid are
 * checked as in mfa_raycast (slot strides aside), and the model arrays as in mfa_decode_blocks. */
int mfa_raycast_direct(mfa_ctx* ctx, const mfa_block_desc* d_desc, int32_t nblocks, const float* d_knots,
                       int64_t knots_len, const float* d_cps, int64_t cps_len, const mfa_bounds* bounds,
                       const int32_t* d_brick_table, const int32_t brick_dims[3], int32_t brick_n,
                       const mfa_view* view, const float* d_tf, int32_t tf_n, float* d_image, void* stream);

/* ---- out-of-core model storage and caching (Sec. 4.3: Algorithms 2 and 3) ------------- */
/* Storage: micro-models in the byte layout whose size is Eq. 2, 1 + ((NCP + degree)*3 + NCP^3)*4:
 * one byte holding the degree, then for each axis x, y, z the first NCP + degree knots as float32
 * (the last knot of a clamped vector repeats the one before it and is implied), then the NCP^3
 * control points as float32, x fastest. Only isotropic models (equal NCP and degree on the three
 * axes) have this layout. A store file holds a header ("MFAPACK1", uint32 count, uint32 0), an index
 * of count entries (uint64 byte offset, uint32 NCP, uint32 degree) and the models back to back.
 * mfa_store_write writes blocks 0..nblocks-1 of a host batch (descriptors, knots, control points as
 * for mfa_decode_blocks) to `path`; MFA_ERR_INVALID_ARG for an anisotropic or inconsistent block,
 * MFA_ERR_IO when the file cannot be written. */
int mfa_store_write(const char* path, const mfa_block_desc* h_desc, int32_t nblocks, const float* h_knots,
                    int64_t knots_len, const float* h_cps, int64_t cps_len);

/* An LRU cache of up to `capacity` micro-models of a store, in host memory (page-locked when
 * `pinned` is non-zero, which needs a CUDA device; pageable otherwise). It reads models from the
 * store file on demand (one positioned read per model). Not thread-safe except for the prefetch
 * thread it owns. */
typedef struct mfa_model_cache mfa_model_cache;
int  mfa_cache_create(mfa_model_cache** out, const char* path, int32_t capacity, int32_t pinned);
void mfa_cache_destroy(mfa_model_cache* cache);
/* Number of models in the store and the largest model's NCP and degree (any pointer may be null). */
int  mfa_cache_info(const mfa_model_cache* cache, int32_t* count, int32_t* max_ncp, int32_t* max_degree);
/* Algorithm 2, caching for one point of view: for every listed model, in order, a hit marks it most
 * recently used; a miss loads it from storage into a free entry or into the least recently used
 * one. All n models must fit (n <= capacity; repeated ids count once). h_stats (nullable, 4 int64):
 * hits, misses, bytes read from storage, elapsed nanoseconds. MFA_ERR_INVALID_ARG for an id
 * outside the store or n > capacity, MFA_ERR_IO when a read fails. */
int  mfa_cache_lookup(mfa_model_cache* cache, const int32_t* h_ids, int32_t n, int64_t* h_stats);
/* Copies the listed models (already in the cache: call mfa_cache_lookup first) to the device as one
 * batch: d_desc[i] describes model h_ids[i] with slot i and `nsamp` samples per axis, its knots (all
 * NCP + degree + 1 per axis) and control points packed into d_knots / d_cps (capacities in floats).
 * h_lens (2 int64): the knot and control-point counts written; h_bounds: the batch's bounds. The
 * packing goes through the cache's host staging buffers and three cudaMemcpyAsync on `stream`; the
 * next upload waits for these copies before it reuses the staging. MFA_ERR_CAPACITY when the
 * device buffers are too small, MFA_ERR_INVALID_ARG for a model that is not cached. */
int  mfa_cache_upload(mfa_model_cache* cache, const int32_t* h_ids, int32_t n, int32_t nsamp,
                      mfa_block_desc* d_desc, float* d_knots, int64_t knots_cap, float* d_cps, int64_t cps_cap,
                      int64_t* h_lens, mfa_bounds* h_bounds, void* stream);
/* Algorithm 3, prefetching for the next point of view: a background thread loads the listed models
 * that are not cached (LRU replacement as above) until the list ends or mfa_cache_prefetch_stop is
 * called (rendering done). The cache must not be used by other calls in between. stop joins the
 * thread; h_stats (nullable, 2 int64): models loaded, bytes read. */
int  mfa_cache_prefetch_start(mfa_model_cache* cache, const int32_t* h_ids, int32_t n);
int  mfa_cache_prefetch_stop(mfa_model_cache* cache, int64_t* h_stats);

#ifdef __cplusplus
}
#endif

#endif /* MFA_H */
