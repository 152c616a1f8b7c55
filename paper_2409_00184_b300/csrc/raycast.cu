// Front-to-back direct volume rendering over the decoded value+gradient cache (Algorithm 4).
//
// One thread per pixel, 16x16-pixel tiles per CTA for coherent cache reads. The integers decided
// before marching (hit or miss, number of samples) come from an FP32 set-up written with
// explicitly rounded operations (no FMA contraction), so they are reproducible bit for bit.
// Each sample: node-centred trilinear (f, f_u, f_v, f_w) from the bricked cache (absent bricks
// read as zero), transfer-function lookup, headlight shading from the gradient, compositing
// C += (1-A) a c, A += (1-A) a, and termination once A > O_max.
#include "common.cuh"
#include "kernels.h"

namespace mfa {

constexpr int kTile = 16;
constexpr int kMaxTf = 1024;

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float w) {
  return make_float4(fmaf(w, b.x - a.x, a.x), fmaf(w, b.y - a.y, a.y), fmaf(w, b.z - a.z, a.z),
                     fmaf(w, b.w - a.w, a.w));
}

__global__ void __launch_bounds__(kTile * kTile, 4) raycast_kernel(RaycastParams prm) {
  __shared__ float4 s_tf[kMaxTf];
  const int tid = threadIdx.y * kTile + threadIdx.x;
  for (int e = tid; e < prm.tf_n; e += kTile * kTile) s_tf[e] = prm.tf[e];
  __syncthreads();
  const int px = blockIdx.x * kTile + threadIdx.x;
  const int py = blockIdx.y * kTile + threadIdx.y;
  const bool inside = px < prm.W && py < prm.H;

  int marched = 0;
  if (inside) {
  // ---- FP32 ray set-up, every operation rounded on its own ----
  const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * px + 1), (float)prm.W), 1.0f), prm.tan_w);
  const float sy = __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * py + 1), (float)prm.H)), prm.tan_h);
  float d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    d[a] = __fadd_rn(__fadd_rn(prm.fwd[a], __fmul_rn(sx, prm.right[a])), __fmul_rn(sy, prm.up[a]));
  const float len = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])),
                                         __fmul_rn(d[2], d[2])));
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = __fdiv_rn(d[a], len);
  float t0 = 0.f, t1 = __int_as_float(0x7f800000);
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
  int K = 0;
  if (!miss && t1 > t0) {
    const float q = __fdiv_rn(__fsub_rn(t1, t0), prm.dt);
    // a chord of [-1,1]^3 is at most 2*sqrt(3) long: q beyond max_samples cannot occur for finite
    // inputs; the clamp keeps the loop bounded whatever the inputs are
    K = q < (float)prm.max_samples ? max(0, (int)ceilf(__fsub_rn(q, 0.5f))) : 0;
  }

  // ---- march ----
  const int n = prm.brick_n;
  const int sh = prm.log2n;  // >= 0: power-of-two bricks (shift/mask addressing)
  const int Nx = prm.B[0] * n, Ny = prm.B[1] * n, Nz = prm.B[2] * n;
  const float inv_range = 1.0f / (prm.vmax - prm.vmin);
  const float tfs = (float)(prm.tf_n - 1);
  const int n2 = n * n;
  float cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f;
  for (int k = 0; k < K; ++k) {
    const float t = fmaf((float)k + 0.5f, prm.dt, t0);
    const float gx = fminf(fmaxf((fmaf(t, d[0], prm.eye[0]) + 1.0f) * prm.half[0], 0.f), (float)(Nx - 1));
    const float gy = fminf(fmaxf((fmaf(t, d[1], prm.eye[1]) + 1.0f) * prm.half[1], 0.f), (float)(Ny - 1));
    const float gz = fminf(fmaxf((fmaf(t, d[2], prm.eye[2]) + 1.0f) * prm.half[2], 0.f), (float)(Nz - 1));
    const int ix = min((int)gx, Nx - 2), iy = min((int)gy, Ny - 2), iz = min((int)gz, Nz - 2);
    const float wx = gx - (float)ix, wy = gy - (float)iy, wz = gz - (float)iz;
    // brick and local index of the two corner layers on each axis
    int bx0, by0, bz0, lx0, ly0, lz0;
    if (sh >= 0) {
      bx0 = ix >> sh; by0 = iy >> sh; bz0 = iz >> sh;
      lx0 = ix & (n - 1); ly0 = iy & (n - 1); lz0 = iz & (n - 1);
    } else {
      bx0 = ix / n; by0 = iy / n; bz0 = iz / n;
      lx0 = ix - bx0 * n; ly0 = iy - by0 * n; lz0 = iz - bz0 * n;
    }
    float4 c[2][2][2];
    if (lx0 < n - 1 && ly0 < n - 1 && lz0 < n - 1) {
      // all eight corners in one brick: one table lookup
      const int slot = __ldg(prm.table + (bz0 * prm.B[1] + by0) * prm.B[0] + bx0);
      if (slot >= 0 && slot < prm.nslots) {
        const float4* base = prm.cache + (int64_t)slot * prm.slot_stride + (lz0 * n + ly0) * n + lx0;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
          for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) c[dz][dy][dx] = __ldg(base + dz * n2 + dy * n + dx);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) c[e >> 2][(e >> 1) & 1][e & 1] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
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
              v = __ldg(prm.cache + (int64_t)slot * prm.slot_stride + (lz * n + ly) * n + lx);
            c[dz][dy][dx] = v;
          }
    }
    const float4 s = lerp4(lerp4(lerp4(c[0][0][0], c[0][0][1], wx), lerp4(c[0][1][0], c[0][1][1], wx), wy),
                           lerp4(lerp4(c[1][0][0], c[1][0][1], wx), lerp4(c[1][1][0], c[1][1][1], wx), wy), wz);
    // transfer function
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
    if (A > prm.opacity_max) { marched = k + 1; break; }
    marched = k + 1;
  }
  prm.image[(int64_t)py * prm.W + px] = make_float4(cr, cg, cb, A);
  }
  // marched-sample count for the roofline: warp sum, one atomic per warp
  unsigned long long m = (unsigned long long)marched;
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  if ((threadIdx.x & 31) == 0 && prm.samples) atomicAdd(prm.samples, m);
}

int raycast(mfa_ctx* ctx, const RaycastParams& prm, cudaStream_t stream) {
  if (prm.tf_n > kMaxTf) return MFA_ERR_CAPACITY;
  dim3 block(kTile, kTile);
  dim3 grid((prm.W + kTile - 1) / kTile, (prm.H + kTile - 1) / kTile);
  raycast_kernel<<<grid, block, 0, stream>>>(prm);
  ctx->launches++;
  return cudaGetLastError() == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
