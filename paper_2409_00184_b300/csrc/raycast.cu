// Front-to-back direct volume rendering over the decoded value+gradient cache (Algorithm 4).
//
// Per ray: an FP32 set-up written with explicitly rounded operations (no FMA contraction) decides
// the integers fixed before marching (hit or miss, number of samples), so they are reproducible bit
// for bit. Per sample: node-centred trilinear (f, f_u, f_v, f_w) from the bricked cache (absent
// bricks read as zero), transfer-function lookup, headlight shading from the gradient, compositing
// C += (1-A) a c, A += (1-A) a, and termination once A > O_max.
//
// Two kernels share that arithmetic:
//  * raycast_queue_kernel<L> (bricks of 2^L voxels, the usual case): persistent warps, each taking
//    4x8-pixel tiles from a global queue (one atomic per tile) until the image is done, so SMs do not
//    sit idle behind long tiles at the end of the launch. The lanes of a warp march neighbouring rays
//    in step, which keeps their corner loads on shared cache lines (the kernel is bound by L1
//    wavefronts: eight 16-byte corner gathers and two transfer-function entries per sample). The
//    brick slot of the next sample is fetched one sample ahead, so the table lookup is off the path
//    of the corner loads, whose offsets are compile-time constants.
//  * raycast_tile_kernel (any brick size): one thread per pixel, 16x16-pixel tiles per CTA.
//  * raycast_direct_kernel: the same rays and compositing, but every sample queries the micro-models
//    themselves (value and parametric gradient of the B-spline, Algorithm 4's value and gradient
//    queries) instead of a decoded cache. Brick b's model covers nodes b n .. b n + n - 1 (parameter
//    u = (g - b n)/(n - 1)); in the one-node gap before brick b + 1 the sample is the linear blend,
//    along that axis, of the two models at their boundary, multilinear where gaps of several axes meet.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace mfa {

constexpr int kTile = 16;
constexpr int kMaxTf = 1024;
constexpr int kQueueThreads = 256;
constexpr int kTileW = 8, kTileH = 4;  // pixels of one warp tile

// Pixel of lane `lane` inside its warp tile: each quarter-warp (8 lanes, one L1 wavefront of float4
// loads when they share a line) takes a 4 x 2 block, the four blocks side by side in two columns. A
// model of the distinct 128-byte lines per quarter-warp over the step's rays gives 3.97 wavefronts per
// sample for this map against 4.13 for 4 x 8 tiles of 4 x 2 blocks and 4.86 for 8 x 1 rows.
__device__ __forceinline__ int tile_dx(int lane) { return (lane & 3) + ((lane >> 4) << 2); }
__device__ __forceinline__ int tile_dy(int lane) { return (lane >> 2) & 3; }

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float w) {
  // a + w (b - a) per channel, as packed float2 pairs (the same roundings as the scalar form)
  const float2 ww = make_float2(w, w);
  const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
  const float2 d0 = __fadd2_rn(make_float2(b.x, b.y), make_float2(-a.x, -a.y));
  const float2 d1 = __fadd2_rn(make_float2(b.z, b.w), make_float2(-a.z, -a.w));
  const float2 r0 = __ffma2_rn(ww, d0, a0), r1 = __ffma2_rn(ww, d1, a1);
  return make_float4(r0.x, r0.y, r1.x, r1.y);
}

// FP32 ray set-up of pixel (px, py): unit direction d and entry distance t0; returns the number of
// samples K (0 for a ray that misses the [-1, 1]^3 box).
__device__ __forceinline__ int ray_setup(const RaycastParams& prm, int px, int py, float d[3], float& t0) {
  const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * px + 1), (float)prm.W), 1.0f), prm.tan_w);
  const float sy = __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * py + 1), (float)prm.H)), prm.tan_h);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    d[a] = __fadd_rn(__fadd_rn(prm.fwd[a], __fmul_rn(sx, prm.right[a])), __fmul_rn(sy, prm.up[a]));
  const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                         __fmul_rn(d[2], d[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = __fdiv_rn(d[a], len);
  t0 = 0.f;
  float t1 = __int_as_float(0x7f800000);
  bool miss = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0.f) {
      const float ta = __fdiv_rn(__fsub_rn(-1.0f, prm.eye[a]), d[a]);
      const float tb = __fdiv_rn(__fsub_rn(1.0f, prm.eye[a]), d[a]);
      t0 = fmaxf(t0, fminf(ta, tb));
      t1 = fminf(t1, fmaxf(ta, tb));
    } else if (prm.eye[a] < -1.0f || prm.eye[a] > 1.0f) {
      miss = true;
    }
  }
  if (miss || !(t1 > t0)) return 0;
  const float q = __fdiv_rn(__fsub_rn(t1, t0), prm.dt);
  // a chord of [-1,1]^3 is at most 2*sqrt(3) long: q beyond max_samples cannot occur for finite
  // inputs; the clamp keeps the loop bounded whatever the inputs are
  return q < (float)prm.max_samples ? max(0, (int)ceilf(__fsub_rn(q, 0.5f))) : 0;
}

// Transfer function, shading and compositing of one interpolated sample s = (f, f_u, f_v, f_w).
// Returns true once the accumulated opacity exceeds O_max.
__device__ __forceinline__ bool composite(const RaycastParams& prm, const float4* s_tf, float4 s, const float d[3],
                                          float inv_range, float tfs, float& cr, float& cg, float& cb, float& A) {
  const float x = fminf(fmaxf((s.x - prm.vmin) * inv_range, 0.f), 1.f) * tfs;
  const int i0 = min((int)x, prm.tf_n - 2);
  const float4 rgba = lerp4(s_tf[i0], s_tf[i0 + 1], x - (float)i0);
  float a = rgba.w;
  if (prm.step_voxels != 1.0f) a = 1.0f - __powf(1.0f - a, prm.step_voxels);
  // headlight shading from the world-space gradient
  const float g0 = s.y * prm.gscale[0], g1 = s.z * prm.gscale[1], g2 = s.w * prm.gscale[2];
  const float gl2 = g0 * g0 + g1 * g1 + g2 * g2;
  float shade = 1.0f, spec = 0.0f;
  if (gl2 >= 1e-16f) {
    const float nd = fminf(fabsf(g0 * d[0] + g1 * d[1] + g2 * d[2]) * rsqrtf(gl2), 1.0f);
    shade = prm.ka + prm.kd * nd;
    spec = nd > 0.f ? prm.ks * __powf(nd, prm.shininess) : 0.f;
  }
  const float w = (1.0f - A) * a;
  cr = fmaf(w, fmaf(rgba.x, shade, spec), cr);
  cg = fmaf(w, fmaf(rgba.y, shade, spec), cg);
  cb = fmaf(w, fmaf(rgba.z, shade, spec), cb);
  A += w;
  return A > prm.opacity_max;
}

__device__ __forceinline__ float4 trilinear(const float4 (&c)[2][2][2], float wx, float wy, float wz) {
  return lerp4(lerp4(lerp4(c[0][0][0], c[0][0][1], wx), lerp4(c[0][1][0], c[0][1][1], wx), wy),
               lerp4(lerp4(c[1][0][0], c[1][0][1], wx), lerp4(c[1][1][0], c[1][1][1], wx), wy), wz);
}

// Index of brick-local voxel (x, y, z) in its slot: [z][y][x] (rows of n; with an apron rows of
// apron_pitch(n) and planes of n + 1 rows), or the cube layout.
__device__ __forceinline__ int brick_voxel(bool cubes, bool apron, int n, int x, int y, int z) {
  if (cubes) return cube_index(x, y, z, n, n);
  if (apron) return (z * (n + 1) + y) * apron_pitch(n) + x;
  return (z * n + y) * n + x;
}

// The eight corners of the cell at voxel (ix, iy, iz) when it spans two bricks on some axis (or the
// brick size is not a power of two): one table lookup per corner.
template <int LAYOUT>  // 0: [z][y][x], 1: cubes, 2: apron, -1: as prm says
__device__ __forceinline__ void corners_general(const RaycastParams& prm, int n, int ix, int iy, int iz,
                                                float4 (&c)[2][2][2]) {
  const bool cubes = LAYOUT < 0 ? prm.cubes : LAYOUT == 1;
  const bool apron = LAYOUT < 0 ? prm.apron : LAYOUT == 2;
  const int bx0 = ix / n, by0 = iy / n, bz0 = iz / n;
  const int lx0 = ix - bx0 * n, ly0 = iy - by0 * n, lz0 = iz - bz0 * n;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const bool ox = dx && lx0 == n - 1, oy = dy && ly0 == n - 1, oz = dz && lz0 == n - 1;
        const int bx = bx0 + ox, by = by0 + oy, bz = bz0 + oz;
        const int lx = ox ? 0 : lx0 + dx, ly = oy ? 0 : ly0 + dy, lz = oz ? 0 : lz0 + dz;
        const int slot = __ldg(prm.table + (bz * prm.B[1] + by) * prm.B[0] + bx);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (slot >= 0 && slot < prm.nslots)
          v = __ldg(prm.cache + (int64_t)slot * prm.slot_stride + brick_voxel(cubes, apron, n, lx, ly, lz));
        c[dz][dy][dx] = v;
      }
}

// One corner load of the queue kernel. The measuring instance (TOUCH) also sets the bit of the 32-byte
// cache sector it reads in prm.touched.
template <bool TOUCH>
__device__ __forceinline__ float4 load_corner(const RaycastParams& prm, const float4* p) {
  if (TOUCH) {
    const int64_t sec = (p - prm.cache) >> 1;  // two float4 per sector
    atomicOr(prm.touched + (sec >> 5), 1u << (sec & 31));
  }
  return __ldg(p);
}

// The eight corners of a cell that spans two bricks on some axis, for bricks of 2^L voxels: per axis the
// brick step (0 or 1) and local coordinate of the two corner planes are formed once with shifts and
// masks; every corner then costs one table lookup and one load.
template <int L, int LAYOUT, bool TOUCH>  // 0: [z][y][x], 1: cubes, 2: apron (rows of apron_pitch(2^L), planes of 2^L + 1)
__device__ __forceinline__ void corners_seam(const RaycastParams& prm, int ix, int iy, int iz, float4 (&c)[2][2][2]) {
  constexpr int n = 1 << L, P = n + 1, PX = apron_pitch(n);
  const int lx = ix & (n - 1), ly = iy & (n - 1), lz = iz & (n - 1);
  const int sx = lx == n - 1, sy = ly == n - 1, sz = lz == n - 1;  // the +1 plane lies in the next brick
  const int lxd[2] = {lx, sx ? 0 : lx + 1}, lyd[2] = {ly, sy ? 0 : ly + 1}, lzd[2] = {lz, sz ? 0 : lz + 1};
  const int t0 = ((iz >> L) * prm.B[1] + (iy >> L)) * prm.B[0] + (ix >> L);
  const int tx[2] = {0, sx}, ty[2] = {0, sy * prm.B[0]}, tz[2] = {0, sz * prm.B[0] * prm.B[1]};
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int dx = e & 1, dy = (e >> 1) & 1, dz = e >> 2;
    const int slot = __ldg(prm.table + t0 + tz[dz] + ty[dy] + tx[dx]);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (slot >= 0 && slot < prm.nslots) {
      const int vox = LAYOUT == 1   ? cube_index(lxd[dx], lyd[dy], lzd[dz], n, n)
                      : LAYOUT == 2 ? (lzd[dz] * P + lyd[dy]) * PX + lxd[dx]
                                    : (((lzd[dz] << L) + lyd[dy]) << L) + lxd[dx];
      v = load_corner<TOUCH>(prm, prm.cache + (int64_t)slot * prm.slot_stride + vox);
    }
    c[dz][dy][dx] = v;
  }
}

// Adds the warp's marched samples to the statistics counter (lane = linear thread index mod 32).
__device__ __forceinline__ void count_marched(const RaycastParams& prm, unsigned long long m, int lane) {
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if (lane == 0 && prm.samples) atomicAdd(prm.samples, m);
}

__global__ void __launch_bounds__(kTile * kTile, 4) raycast_tile_kernel(RaycastParams prm) {
  __shared__ float4 s_tf[kMaxTf];
  const int tid = threadIdx.y * kTile + threadIdx.x;
  for (int e = tid; e < prm.tf_n; e += kTile * kTile) s_tf[e] = prm.tf[e];
  __syncthreads();
  const int px = blockIdx.x * kTile + threadIdx.x;
  const int py = blockIdx.y * kTile + threadIdx.y;
  int marched = 0;
  if (px < prm.W && py < prm.H) {
    float d[3], t0;
    const int K = ray_setup(prm, px, py, d, t0);
    const int n = prm.brick_n;
    const int Nx = prm.B[0] * n, Ny = prm.B[1] * n, Nz = prm.B[2] * n;
    const float inv_range = 1.0f / (prm.vmax - prm.vmin);
    const float tfs = (float)(prm.tf_n - 1);
    float cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f;
    for (int k = 0; k < K; ++k) {
      const float t = fmaf((float)k + 0.5f, prm.dt, t0);
      const float gx = fminf(fmaxf((fmaf(t, d[0], prm.eye[0]) + 1.0f) * prm.half[0], 0.f), (float)(Nx - 1));
      const float gy = fminf(fmaxf((fmaf(t, d[1], prm.eye[1]) + 1.0f) * prm.half[1], 0.f), (float)(Ny - 1));
      const float gz = fminf(fmaxf((fmaf(t, d[2], prm.eye[2]) + 1.0f) * prm.half[2], 0.f), (float)(Nz - 1));
      const int ix = min((int)gx, Nx - 2), iy = min((int)gy, Ny - 2), iz = min((int)gz, Nz - 2);
      const int bx0 = ix / n, by0 = iy / n, bz0 = iz / n;
      const int lx0 = ix - bx0 * n, ly0 = iy - by0 * n, lz0 = iz - bz0 * n;
      float4 c[2][2][2];
      const bool inside = lx0 < n - 1 && ly0 < n - 1 && lz0 < n - 1;
      const int slot0 = prm.apron || inside ? __ldg(prm.table + (bz0 * prm.B[1] + by0) * prm.B[0] + bx0) : -1;
      // an apron keeps every cell of a present brick in that brick; an absent brick has no apron
      if (inside || (prm.apron && slot0 >= 0 && slot0 < prm.nslots)) {
        const int slot = slot0;
        if (slot >= 0 && slot < prm.nslots) {
          const float4* sb = prm.cache + (int64_t)slot * prm.slot_stride;
#pragma unroll
          for (int e = 0; e < 8; ++e)
            c[e >> 2][(e >> 1) & 1][e & 1] =
                __ldg(sb + brick_voxel(prm.cubes, prm.apron, n, lx0 + (e & 1), ly0 + ((e >> 1) & 1), lz0 + (e >> 2)));
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) c[e >> 2][(e >> 1) & 1][e & 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
        corners_general<-1>(prm, n, ix, iy, iz, c);
      }
      const float4 s = trilinear(c, gx - (float)ix, gy - (float)iy, gz - (float)iz);
      marched = k + 1;
      if (composite(prm, s_tf, s, d, inv_range, tfs, cr, cg, cb, A)) break;
    }
    prm.image[(int64_t)py * prm.W + px] = make_float4(cr, cg, cb, A);
  }
  count_marched(prm, (unsigned long long)marched, tid & 31);
}

// LAYOUT of the cache bricks: 0 [z][y][x], 1 cubes, 2 [z][y][x] with a one-voxel apron (pitch 2^L + 1).
// TOUCH: the measuring instance that records the cache sectors it reads (MFA_RAYCAST_COUNT_SECTORS).
template <int L, int LAYOUT, bool TOUCH>
__global__ void __launch_bounds__(kQueueThreads, 3) raycast_queue_kernel(RaycastParams prm, uint32_t* counter) {
  constexpr bool CUBES = LAYOUT == 1, APRON = LAYOUT == 2;
  constexpr int P = (1 << L) + 1, PX = apron_pitch(1 << L);  // apron: rows per plane, row pitch
  constexpr int n = 1 << L, n2 = n * n;
  extern __shared__ float4 s_tf[];  // tf_n entries
  for (int e = threadIdx.x; e < prm.tf_n; e += kQueueThreads) s_tf[e] = prm.tf[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tiles_x = (prm.W + kTileW - 1) / kTileW;
  const int ntiles = tiles_x * ((prm.H + kTileH - 1) / kTileH);
  const int Nx = prm.B[0] * n, Ny = prm.B[1] * n, Nz = prm.B[2] * n;
  const float inv_range = 1.0f / (prm.vmax - prm.vmin);
  const float tfs = (float)(prm.tf_n - 1);
  unsigned long long marched = 0;

  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    const int px = (tile % tiles_x) * kTileW + tile_dx(lane);
    const int py = (tile / tiles_x) * kTileH + tile_dy(lane);
    if (px < prm.W && py < prm.H) {  // lanes of a ragged edge tile idle until the warp's next tile
      float d[3], t0;
      const int K = ray_setup(prm, px, py, d, t0);
      // voxel position of sample k: g = ((t0 + (k + 1/2) dt) d + eye + 1) * half, as gb + k * dg
      float gb[3], dg[3];
      const float ts = fmaf(0.5f, prm.dt, t0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gb[a] = (fmaf(ts, d[a], prm.eye[a]) + 1.0f) * prm.half[a];
        dg[a] = prm.dt * d[a] * prm.half[a];
      }
      // cell of sample kk: lower corner, weights, and (when all eight corners lie in one brick) its slot
      auto locate = [&](int kk, int& ix, int& iy, int& iz, float& wx, float& wy, float& wz, int& slot) {
        const float kf = (float)kk;
        const float gx = fminf(fmaxf(fmaf(kf, dg[0], gb[0]), 0.f), (float)(Nx - 1));
        const float gy = fminf(fmaxf(fmaf(kf, dg[1], gb[1]), 0.f), (float)(Ny - 1));
        const float gz = fminf(fmaxf(fmaf(kf, dg[2], gb[2]), 0.f), (float)(Nz - 1));
        ix = min((int)gx, Nx - 2);
        iy = min((int)gy, Ny - 2);
        iz = min((int)gz, Nz - 2);
        wx = gx - (float)ix;
        wy = gy - (float)iy;
        wz = gz - (float)iz;
        // with an apron every cell lies in its lower corner's brick
        const bool one = APRON || ((ix & (n - 1)) < n - 1 && (iy & (n - 1)) < n - 1 && (iz & (n - 1)) < n - 1);
        slot = -2;  // -2: spans bricks
        if (one) slot = __ldg(prm.table + ((iz >> L) * prm.B[1] + (iy >> L)) * prm.B[0] + (ix >> L));
      };
      float cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f;
      int ix = 0, iy = 0, iz = 0, slot = -1;
      float wx = 0.f, wy = 0.f, wz = 0.f;
      if (K > 0) locate(0, ix, iy, iz, wx, wy, wz, slot);
      int k = 0;
      while (k < K) {
        float4 c[2][2][2];
        if (!APRON && slot == -2) {
          corners_seam<L, LAYOUT, TOUCH>(prm, ix, iy, iz, c);
        } else if (slot >= 0 && slot < prm.nslots && APRON) {
          const float4* base = prm.cache + (int64_t)slot * prm.slot_stride +
                               ((iz & (n - 1)) * P + (iy & (n - 1))) * PX + (ix & (n - 1));
#pragma unroll
          for (int e = 0; e < 8; ++e)
            c[e >> 2][(e >> 1) & 1][e & 1] = load_corner<TOUCH>(prm, base + (e >> 2) * P * PX + ((e >> 1) & 1) * PX + (e & 1));
        } else if (APRON && (((ix & (n - 1)) == n - 1) | ((iy & (n - 1)) == n - 1) | ((iz & (n - 1)) == n - 1))) {
          // an absent brick has no apron: a seam cell reads the neighbouring bricks' corners directly
          corners_seam<L, LAYOUT, TOUCH>(prm, ix, iy, iz, c);
        } else if (slot >= 0 && slot < prm.nslots && CUBES) {
          // cube layout: the two x, y and z corner planes of the cell
          const int lx = ix & (n - 1), ly = iy & (n - 1), lz = iz & (n - 1);
          const int ox[2] = {((lx >> 1) << 3) + (lx & 1), (((lx + 1) >> 1) << 3) + ((lx + 1) & 1)};
          const int oy[2] = {((ly >> 1) << (L + 2)) + ((ly & 1) << 1), (((ly + 1) >> 1) << (L + 2)) + (((ly + 1) & 1) << 1)};
          const int oz[2] = {((lz >> 1) << (2 * L + 1)) + ((lz & 1) << 2),
                             (((lz + 1) >> 1) << (2 * L + 1)) + (((lz + 1) & 1) << 2)};
          const float4* sb = prm.cache + (int64_t)slot * prm.slot_stride;
#pragma unroll
          for (int e = 0; e < 8; ++e)
            c[e >> 2][(e >> 1) & 1][e & 1] = load_corner<TOUCH>(prm, sb + oz[e >> 2] + oy[(e >> 1) & 1] + ox[e & 1]);
        } else if (slot >= 0 && slot < prm.nslots) {
          const float4* base = prm.cache + (int64_t)slot * prm.slot_stride +
                               ((((iz & (n - 1)) << L) + (iy & (n - 1))) << L) + (ix & (n - 1));
#pragma unroll
          for (int e = 0; e < 8; ++e)
            c[e >> 2][(e >> 1) & 1][e & 1] = load_corner<TOUCH>(prm, base + (e >> 2) * n2 + ((e >> 1) & 1) * n + (e & 1));
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) c[e >> 2][(e >> 1) & 1][e & 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float4 s = trilinear(c, wx, wy, wz);
        ++k;
        // the next sample's cell (and brick slot) is located while this sample is shaded
        if (k < K) locate(k, ix, iy, iz, wx, wy, wz, slot);
        if (composite(prm, s_tf, s, d, inv_range, tfs, cr, cg, cb, A)) break;
      }
      prm.image[(int64_t)py * prm.W + px] = make_float4(cr, cg, cb, A);
      marched += (unsigned long long)k;
    }
  }
  count_marched(prm, marched, lane);
}

// Adds the number of set bits of words[0 .. nwords) to *out.
__global__ void count_bits_kernel(const uint32_t* __restrict__ words, int64_t nwords, unsigned long long* out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
    c += __popc(words[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

template <int L, bool TOUCH>
auto queue_kernel(const RaycastParams& prm) {
  return prm.apron ? raycast_queue_kernel<L, 2, TOUCH>
                   : prm.cubes ? raycast_queue_kernel<L, 1, TOUCH> : raycast_queue_kernel<L, 0, TOUCH>;
}

template <int L>
int launch_queue(mfa_ctx* ctx, const RaycastParams& prm, cudaStream_t stream) {
  const size_t smem = (size_t)prm.tf_n * sizeof(float4);
  auto kern = prm.touched ? queue_kernel<L, true>(prm) : queue_kernel<L, false>(prm);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kQueueThreads, smem) != cudaSuccess)
    return MFA_ERR_CUDA;
  uint32_t* counter = ctx->d_counters + kRaycastQueue;
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  kern<<<ctx->num_sms * (per_sm > 0 ? per_sm : 1), kQueueThreads, smem, stream>>>(prm, counter);
  if (prm.touched) {
    const int64_t words = ((prm.nslots * prm.slot_stride + 1) / 2 + 31) / 32;
    count_bits_kernel<<<ctx->num_sms * 4, 256, 0, stream>>>(prm.touched, words, prm.sectors);
    ctx->launches++;
  }
  return MFA_OK;
}

// ---- direct query of the micro-models ----

struct ModelGeom {
  int block;  // -1: none loaded
  bool ok;
  int p[3], C[3];
  int64_t koff[3], cpoff;
};

// Loads and checks block `block`'s descriptor and knots (once per change of block along a ray).
__device__ __forceinline__ void load_model(const DirectModels& m, int brick_n, int block, ModelGeom& g) {
  g.block = block;
  g.ok = false;
  if (block < 0 || block >= m.nblocks) return;
  BlockGeom bg;
  const uint32_t bad = load_desc(m.desc + block, m.bounds, m.knots_len, m.cps_len, 1, INT64_MAX, bg, false);
  if (bad) { flag(m.status, bad); return; }
  for (int a = 0; a < 3; ++a) {
    if (bg.n[a] != brick_n) { flag(m.status, MFA_DEV_BAD_DESC); return; }
    if (!knots_ok(m.knots + bg.knot_off[a], bg.p[a], bg.C[a])) { flag(m.status, MFA_DEV_BAD_KNOTS); return; }
    g.p[a] = bg.p[a];
    g.C[a] = bg.C[a];
    g.koff[a] = bg.knot_off[a];
  }
  g.cpoff = bg.cp_off;
  g.ok = true;
}

// (f, f_u, f_v, f_w) of one model at parameters (u, v, w): basis of degree p and its derivative per axis,
// then the (p+1)^3 control points of the span.
__device__ __forceinline__ float4 eval_model(const DirectModels& m, const ModelGeom& g, float u, float v, float w) {
  const float prm3[3] = {u, v, w};
  float N[3][MFA_MAX_DEGREE + 1], dN[3][MFA_MAX_DEGREE + 1];
  int off[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* t = m.knots + g.koff[a];
    const int s = find_span(t, g.p[a], g.C[a], prm3[a]);
    basis_funs<MFA_MAX_DEGREE>(t, g.p[a], s, prm3[a], N[a], dN[a]);
    off[a] = s - g.p[a];
  }
  const int Cx = g.C[0], Cy = g.C[1];
  float f = 0.f, fu = 0.f, fv = 0.f, fw = 0.f;
#pragma unroll
  for (int c = 0; c <= MFA_MAX_DEGREE; ++c) {
    if (c > g.p[2]) break;
#pragma unroll
    for (int b = 0; b <= MFA_MAX_DEGREE; ++b) {
      if (b > g.p[1]) break;
      const float* row = m.cps + g.cpoff + ((int64_t)(off[2] + c) * Cy + off[1] + b) * Cx + off[0];
      float sa = 0.f, sda = 0.f;
#pragma unroll
      for (int a = 0; a <= MFA_MAX_DEGREE; ++a) {
        if (a > g.p[0]) break;
        const float P = __ldg(row + a);
        sa = fmaf(N[0][a], P, sa);
        sda = fmaf(dN[0][a], P, sda);
      }
      const float nbc = N[1][b] * N[2][c];
      f = fmaf(nbc, sa, f);
      fu = fmaf(nbc, sda, fu);
      fv = fmaf(dN[1][b] * N[2][c], sa, fv);
      fw = fmaf(N[1][b] * dN[2][c], sa, fw);
    }
  }
  return make_float4(f, fu, fv, fw);
}

__device__ __forceinline__ float4 sample_direct(const RaycastParams& prm, const DirectModels& m, const float (&gv)[3],
                                                ModelGeom& cur) {
  const int n = prm.brick_n;
  const float inv = 1.0f / (float)(n - 1);
  int b[3];
  float u[3], w[3];
  bool gap[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b[a] = min((int)(gv[a] / (float)n), prm.B[a] - 1);
    const float local = gv[a] - (float)(b[a] * n);
    gap[a] = local > (float)(n - 1);
    u[a] = gap[a] ? 1.0f : local * inv;
    w[a] = gap[a] ? local - (float)(n - 1) : 0.f;
  }
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int combo = 0; combo < 8; ++combo) {
    bool use = true;
    float wt = 1.f;
    int bb[3];
    float uu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int side = (combo >> a) & 1;
      if (side && !gap[a]) use = false;
      bb[a] = b[a] + side;
      uu[a] = gap[a] ? (side ? 0.f : 1.f) : u[a];
      wt *= gap[a] ? (side ? w[a] : 1.f - w[a]) : 1.f;
    }
    if (!use) continue;
    const int block = __ldg(prm.table + ((int64_t)bb[2] * prm.B[1] + bb[1]) * prm.B[0] + bb[0]);
    if (block < 0) continue;
    if (block != cur.block) load_model(m, n, block, cur);
    if (!cur.ok) continue;
    const float4 v = eval_model(m, cur, uu[0], uu[1], uu[2]);
    acc.x = fmaf(wt, v.x, acc.x);
    acc.y = fmaf(wt, v.y, acc.y);
    acc.z = fmaf(wt, v.z, acc.z);
    acc.w = fmaf(wt, v.w, acc.w);
  }
  return acc;
}

__global__ void __launch_bounds__(kQueueThreads) raycast_direct_kernel(RaycastParams prm, DirectModels models,
                                                                       uint32_t* counter) {
  extern __shared__ float4 s_tf[];  // tf_n entries
  for (int e = threadIdx.x; e < prm.tf_n; e += kQueueThreads) s_tf[e] = prm.tf[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tiles_x = (prm.W + kTileW - 1) / kTileW;
  const int ntiles = tiles_x * ((prm.H + kTileH - 1) / kTileH);
  const int n = prm.brick_n;
  const float Nmax[3] = {(float)(prm.B[0] * n - 1), (float)(prm.B[1] * n - 1), (float)(prm.B[2] * n - 1)};
  const float inv_range = 1.0f / (prm.vmax - prm.vmin);
  const float tfs = (float)(prm.tf_n - 1);
  unsigned long long marched = 0;
  ModelGeom cur;
  cur.block = -1;
  cur.ok = false;

  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    const int px = (tile % tiles_x) * kTileW + tile_dx(lane);
    const int py = (tile / tiles_x) * kTileH + tile_dy(lane);
    if (px < prm.W && py < prm.H) {
      float d[3], t0;
      const int K = ray_setup(prm, px, py, d, t0);
      float gb[3], dg[3];
      const float ts = fmaf(0.5f, prm.dt, t0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gb[a] = (fmaf(ts, d[a], prm.eye[a]) + 1.0f) * prm.half[a];
        dg[a] = prm.dt * d[a] * prm.half[a];
      }
      float cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f;
      int k = 0;
      while (k < K) {
        const float kf = (float)k;
        float gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a] = fminf(fmaxf(fmaf(kf, dg[a], gb[a]), 0.f), Nmax[a]);
        const float4 s = sample_direct(prm, models, gv, cur);
        ++k;
        if (composite(prm, s_tf, s, d, inv_range, tfs, cr, cg, cb, A)) break;
      }
      prm.image[(int64_t)py * prm.W + px] = make_float4(cr, cg, cb, A);
      marched += (unsigned long long)k;
    }
  }
  count_marched(prm, marched, lane);
}

// The selected model's (f, df/dg) at finest-node coordinates gv (node-unit gradient) of a multi-resolution
// volume: the finest block holding gv, the global id the table gives it, and that block's level, first
// node and extent, from which u = (g - g0)/E.
__device__ __forceinline__ float4 sample_lod(const RaycastParams& prm, const DirectModels& m, const LodLevels& lv,
                                             const float (&gv)[3], ModelGeom& cur) {
  const int nm1 = lv.n - 1;
  int fb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) fb[a] = min((int)(gv[a] / (float)nm1), lv.B0 - 1);
  const int id = __ldg(prm.table + ((int64_t)fb[2] * lv.B0 + fb[1]) * lv.B0 + fb[0]);
  if (id < 0 || id >= m.nblocks) {
    flag(m.status, MFA_DEV_BAD_LIST);
    return make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int l = 0;
  while (l + 1 < lv.levels && id >= lv.off[l + 1]) ++l;
  const int local = id - lv.off[l], Bl = lv.B0 >> l, E = nm1 << l;
  const int b[3] = {local % Bl, (local / Bl) % Bl, local / (Bl * Bl)};
  float u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = fminf(fmaxf((gv[a] - (float)(b[a] * E)) / (float)E, 0.f), 1.f);
  if (id != cur.block) load_model(m, lv.n, id, cur);
  if (!cur.ok) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 v = eval_model(m, cur, u[0], u[1], u[2]);
  const float inv = 1.0f / (float)E;
  return make_float4(v.x, v.y * inv, v.z * inv, v.w * inv);
}

__global__ void __launch_bounds__(kQueueThreads) raycast_lod_kernel(RaycastParams prm, DirectModels models,
                                                                    LodLevels lv, uint32_t* counter) {
  extern __shared__ float4 s_tf[];  // tf_n entries
  for (int e = threadIdx.x; e < prm.tf_n; e += kQueueThreads) s_tf[e] = prm.tf[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tiles_x = (prm.W + kTileW - 1) / kTileW;
  const int ntiles = tiles_x * ((prm.H + kTileH - 1) / kTileH);
  const float Nmax = (float)(lv.B0 * (lv.n - 1));
  const float inv_range = 1.0f / (prm.vmax - prm.vmin);
  const float tfs = (float)(prm.tf_n - 1);
  unsigned long long marched = 0;
  ModelGeom cur;
  cur.block = -1;
  cur.ok = false;

  for (;;) {
    int tile = 0;
    if (lane == 0) tile = (int)atomicAdd(counter, 1u);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= ntiles) break;
    const int px = (tile % tiles_x) * kTileW + tile_dx(lane);
    const int py = (tile / tiles_x) * kTileH + tile_dy(lane);
    if (px < prm.W && py < prm.H) {
      float d[3], t0;
      const int K = ray_setup(prm, px, py, d, t0);
      float gb[3], dg[3];
      const float ts = fmaf(0.5f, prm.dt, t0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gb[a] = (fmaf(ts, d[a], prm.eye[a]) + 1.0f) * prm.half[a];
        dg[a] = prm.dt * d[a] * prm.half[a];
      }
      float cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f;
      int k = 0;
      while (k < K) {
        const float kf = (float)k;
        float gv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gv[a] = fminf(fmaxf(fmaf(kf, dg[a], gb[a]), 0.f), Nmax);
        const float4 s = sample_lod(prm, models, lv, gv, cur);
        ++k;
        if (composite(prm, s_tf, s, d, inv_range, tfs, cr, cg, cb, A)) break;
      }
      prm.image[(int64_t)py * prm.W + px] = make_float4(cr, cg, cb, A);
      marched += (unsigned long long)k;
    }
  }
  count_marched(prm, marched, lane);
}

int raycast_lod(mfa_ctx* ctx, const RaycastParams& prm, const DirectModels& models, const LodLevels& lv,
                cudaStream_t stream) {
  if (prm.tf_n > kMaxTf) return MFA_ERR_CAPACITY;
  const size_t smem = (size_t)prm.tf_n * sizeof(float4);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raycast_lod_kernel, kQueueThreads, smem) != cudaSuccess)
    return MFA_ERR_CUDA;
  uint32_t* counter = ctx->d_counters + kRaycastQueue;
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  raycast_lod_kernel<<<ctx->num_sms * (per_sm > 0 ? per_sm : 1), kQueueThreads, smem, stream>>>(prm, models, lv,
                                                                                                 counter);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

int raycast_direct(mfa_ctx* ctx, const RaycastParams& prm, const DirectModels& models, cudaStream_t stream) {
  if (prm.tf_n > kMaxTf) return MFA_ERR_CAPACITY;
  const size_t smem = (size_t)prm.tf_n * sizeof(float4);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, raycast_direct_kernel, kQueueThreads, smem) !=
      cudaSuccess)
    return MFA_ERR_CUDA;
  uint32_t* counter = ctx->d_counters + kRaycastQueue;
  if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  raycast_direct_kernel<<<ctx->num_sms * (per_sm > 0 ? per_sm : 1), kQueueThreads, smem, stream>>>(prm, models,
                                                                                                    counter);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

int raycast(mfa_ctx* ctx, const RaycastParams& prm, cudaStream_t stream) {
  if (prm.tf_n > kMaxTf) return MFA_ERR_CAPACITY;
  int st = MFA_OK;
  switch (prm.log2n) {
    case 3: st = launch_queue<3>(ctx, prm, stream); break;
    case 4: st = launch_queue<4>(ctx, prm, stream); break;
    case 5: st = launch_queue<5>(ctx, prm, stream); break;
    case 6: st = launch_queue<6>(ctx, prm, stream); break;
    default: {
      dim3 block(kTile, kTile);
      dim3 grid((prm.W + kTile - 1) / kTile, (prm.H + kTile - 1) / kTile);
      raycast_tile_kernel<<<grid, block, 0, stream>>>(prm);
    }
  }
  if (st != MFA_OK) return st;
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
