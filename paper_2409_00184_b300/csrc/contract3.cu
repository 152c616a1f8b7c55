// Transposed three-axis contraction of per-block sample grids, shared by the least-squares fit and
// the adjoint:
//     Y[c][b][a] = sum_{k,j,i} X[k][j][i] Ax[i][a] Ay[j][b] Az[k][c]
//   kFit:      A = (N^T N)^{-1} N^T per axis (from the encode plan) -> least-squares control points,
//              then optionally the RMSE of the fitted model over the samples (Table 1's metric);
//   kAdjoint:  A = N (collocation matrix, built from the knots in the CTA) -> N^T R;
//   kGradient: G = N^T (decode(P) - D), the gradient of 0.5*||decode(P) - D||^2: each slab of samples is
//              replaced in shared memory by its residual (a banded value decode of P minus the samples)
//              before the contraction, so the cancellation happens per sample, at the data's scale.
//              TMA kernel only; other shapes use the banded adjoint kernel.
// One CTA per block; the grid streams through in z-slabs of ks planes:
//   x:  Y1[(k,j)][a] = sum_i X[k][j][i] Ax[i][a]   thread per sample row, all columns in registers,
//                                                  Ax rows broadcast from shared memory
//   y:  Y2[k][b][a]  = sum_j Y1[(k,j)][a] Ay[j][b]  4 columns b per thread
//   z:  Y[c][b][a]  += sum_k Y2[k][b][a] Az[k][c]   4 columns c per thread
// Two kernels share these stages. The TMA kernel (rows of 32 samples) loads each slab with one
// cp.async.bulk.tensor into a 128-byte-swizzled shared buffer, double-buffered on mbarriers, and
// prefetches the next (block, slab) of its static schedule while it computes the current one; the
// swizzle makes the thread-per-row 16-byte reads bank-conflict-free. The queue kernel (any row
// length) reads rows from global memory with 16-byte loads and takes blocks from an atomic queue.
#include <algorithm>
#include <cstring>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace mfa {
namespace {

constexpr int kThreads = 256;
constexpr int kTmaRow = 32;  // samples per row on the TMA path (128 bytes)

struct C3Smem {
  int A[3], off[3], tab[3], knots, Y1, Y2, Y, P, X, total;  // offsets in 4-byte words
  int us;  // gradient: row stride of the decoded U rows kept in Y1 (odd: per-thread rows, no bank conflicts)
};

struct C3Geom {
  int p[3], C[3], n[3], cls[3];
  int slot, valid, bad;
  int64_t cpoff, koff[3];
};

int round4(int v) { return (v + 3) & ~3; }

C3Smem c3_layout(int mode, int CP, int maxC, int maxN, int ks, bool rmse, int xbuf_words) {
  const int CPs = (CP % 8 == 0) ? CP + 4 : CP;
  C3Smem L;
  int o = 0;
  for (int a = 0; a < 3; ++a) { L.A[a] = o; o += maxN * CP; }
  L.us = CP + 1;
  for (int a = 0; a < 3; ++a) { L.off[a] = o; if (mode == kGradient) o += maxN; }
  for (int a = 0; a < 3; ++a) {
    L.tab[a] = o;
    if ((mode == kFit && rmse) || mode == kGradient) o += maxN * (int)(sizeof(TabEntry) / 4);
  }
  L.knots = o; if (mode != kFit) o += 3 * kKnotMax;
  o = round4(o);
  L.Y1 = o; o += ks * maxN * std::max(CPs, L.us);
  L.Y2 = o; o += round4(ks * maxC * maxC);
  L.Y = o;  o += round4(maxC * maxC * maxC);
  L.P = o;  if (mode == kGradient) o += round4(maxC * maxC * maxC);
  L.X = o;  if (xbuf_words) o += 256 + 2 * xbuf_words;  // two slab buffers + slack for 1024-byte alignment
  L.total = o;
  return L;
}

// Geometry of block `item` (one thread): from the plan's items/classes (kFit) or a checked descriptor.
__device__ void c3_fetch(const ContractParams& prm, int item, C3Geom& g) {
  g.valid = item < prm.nblocks;
  g.bad = 0;
  if (!g.valid) return;
  if (prm.mode == kFit) {
    const EncItem it = prm.items[item];
    for (int a = 0; a < 3; ++a) {
      const EncClass& c = prm.classes[it.cls[a]];
      g.p[a] = c.p; g.C[a] = c.C; g.n[a] = c.n; g.cls[a] = it.cls[a];
    }
    g.slot = it.slot;
    g.cpoff = it.cp_off;
  } else {
    BlockGeom bg;
    const uint32_t bad = load_desc(prm.desc + item, prm.bounds, prm.knots_len, prm.cps_len, prm.nslots,
                                   prm.slot_stride, bg);
    if (bad) {
      flag(prm.status, bad);
      g.bad = 1;
      return;
    }
    for (int a = 0; a < 3; ++a) { g.p[a] = bg.p[a]; g.C[a] = bg.C[a]; g.n[a] = bg.n[a]; g.koff[a] = bg.knot_off[a]; }
    g.slot = bg.slot;
    g.cpoff = bg.cp_off;
  }
}

// Builds the three n x CP matrices (zero-padded columns), the RMSE tables (kFit), the span offsets
// and P (kGradient), zeroes Y. Ends with a barrier; sets *s_bad when a knot vector is invalid.
template <int CP, int MODE>
__device__ void c3_setup(const ContractParams& prm, const C3Smem& L, float* sm, const C3Geom& g, int* s_bad) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int ncps = g.C[0] * g.C[1] * g.C[2];
  if (MODE == kFit) {
    for (int a = 0; a < 3; ++a) {
      const EncClass& c = prm.classes[g.cls[a]];
      float* A = sm + L.A[a];
      for (int e = tid; e < c.n * CP; e += nthr) {
        const int i = e / CP, col = e - i * CP;
        A[e] = col < c.C ? prm.pinv[c.pinv_off + i * c.C + col] : 0.f;
      }
      if (prm.rmse) {
        TabEntry* tb = reinterpret_cast<TabEntry*>(sm + L.tab[a]);
        for (int e = tid; e < c.n; e += nthr) tb[e] = prm.tabs[c.tab_off + e];
      }
    }
  } else {
    float* kn = sm + L.knots;
    for (int a = 0; a < 3; ++a) {  // every maxN row zeroed: padded sample rows must contribute nothing
      for (int i = tid; i < g.C[a] + g.p[a] + 1; i += nthr) kn[a * kKnotMax + i] = prm.knots[g.koff[a] + i];
      for (int e = tid; e < prm.maxN * CP; e += nthr) sm[L.A[a] + e] = 0.f;
      if (MODE == kGradient) {  // entries past n[a] stay zero: offset 0, zero band
        for (int i = tid; i < prm.maxN; i += nthr) reinterpret_cast<int*>(sm + L.off[a])[i] = 0;
        for (int e = tid; e < prm.maxN * (int)(sizeof(TabEntry) / 4); e += nthr) sm[L.tab[a] + e] = 0.f;
      }
    }
    __syncthreads();
    if (tid < 3 && !knots_ok(kn + tid * kKnotMax, g.p[tid], g.C[tid])) {
      atomicOr(s_bad, 1);
      flag(prm.status, MFA_DEV_BAD_KNOTS);
    }
    const int a = tid < nx ? 0 : (tid < nx + ny ? 1 : (tid < nx + ny + nz ? 2 : -1));
    if (a >= 0) {
      const int i = a == 0 ? tid : (a == 1 ? tid - nx : tid - nx - ny);
      const float* t = kn + a * kKnotMax;
      const float u = sample_param(i, g.n[a]);
      const int s = find_span(t, g.p[a], g.C[a], u);
      float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
      basis_funs<MFA_MAX_DEGREE>(t, g.p[a], s, u, N, dN);
      for (int r = 0; r <= g.p[a]; ++r) sm[L.A[a] + i * CP + s - g.p[a] + r] = N[r];
      if (MODE == kGradient) {
        reinterpret_cast<int*>(sm + L.off[a])[i] = s - g.p[a];
        TabEntry te;  // band of sample i (N[r] is zero for r > p)
        te.off = s - g.p[a];
        for (int r = 0; r <= MFA_MAX_DEGREE; ++r) te.N[r] = N[r];
        reinterpret_cast<TabEntry*>(sm + L.tab[a])[i] = te;
      }
    }
  }
  __syncthreads();
  if (MODE == kGradient)
    for (int e = tid; e < ncps; e += nthr) sm[L.P + e] = prm.cps[g.cpoff + e];
  for (int e = tid; e < ncps; e += nthr) sm[L.Y + e] = 0.f;
  __syncthreads();
}

template <int CP>
__device__ __forceinline__ void fma_row4(float (&acc)[CP], const float* Ax, int i, const float4 v) {
  const float xs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4* ar = reinterpret_cast<const float4*>(Ax + (i + q) * CP);
#pragma unroll
    for (int c4 = 0; c4 < CP / 4; ++c4) {
      const float4 w = ar[c4];
      acc[4 * c4 + 0] = fmaf(xs[q], w.x, acc[4 * c4 + 0]);
      acc[4 * c4 + 1] = fmaf(xs[q], w.y, acc[4 * c4 + 1]);
      acc[4 * c4 + 2] = fmaf(xs[q], w.z, acc[4 * c4 + 2]);
      acc[4 * c4 + 3] = fmaf(xs[q], w.w, acc[4 * c4 + 3]);
    }
  }
}

template <int CP>
__device__ __forceinline__ void store_row(float* Y1, int r, const float (&acc)[CP]) {
  constexpr int CPs = (CP % 8 == 0) ? CP + 4 : CP;
  float4* yr = reinterpret_cast<float4*>(Y1 + r * CPs);
#pragma unroll
  for (int c4 = 0; c4 < CP / 4; ++c4)
    yr[c4] = make_float4(acc[4 * c4], acc[4 * c4 + 1], acc[4 * c4 + 2], acc[4 * c4 + 3]);
}

// Stage x from global memory (any row length; 16-byte loads when rows allow).
template <int CP>
__device__ void c3_stage_x_global(const float* X, const float* Ax, float* Y1, int k0, int kc, int nx, int ny,
                                  bool vec) {
  const int rows = kc * ny;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    const float* xr = X + ((int64_t)k0 * ny + r) * nx;
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;
    if (vec) {
      for (int i = 0; i < nx; i += 4) fma_row4<CP>(acc, Ax, i, __ldg(reinterpret_cast<const float4*>(xr + i)));
    } else {
      for (int i = 0; i < nx; ++i) {
        const float xv = __ldg(xr + i);
        const float4* ar = reinterpret_cast<const float4*>(Ax + i * CP);
#pragma unroll
        for (int c4 = 0; c4 < CP / 4; ++c4) {
          const float4 w = ar[c4];
          acc[4 * c4 + 0] = fmaf(xv, w.x, acc[4 * c4 + 0]);
          acc[4 * c4 + 1] = fmaf(xv, w.y, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(xv, w.z, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(xv, w.w, acc[4 * c4 + 3]);
        }
      }
    }
    store_row<CP>(Y1, r, acc);
  }
}

// Stage x from a 128-byte-swizzled shared slab of 32-sample rows: logical 16-byte chunk c of row r
// sits at chunk c ^ (r & 7).
template <int CP>
__device__ void c3_stage_x_smem(const float4* xb, const float* Ax, float* Y1, int rows) {
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;
    const float4* row = xb + r * 8;
    const int sw = r & 7;
#pragma unroll
    for (int c = 0; c < 8; ++c) fma_row4<CP>(acc, Ax, 4 * c, row[c ^ sw]);
    store_row<CP>(Y1, r, acc);
  }
}

template <int CP>
__device__ void c3_stage_yz(const C3Smem& L, float* sm, const C3Geom& g, int k0, int kc) {
  constexpr int CPs = (CP % 8 == 0) ? CP + 4 : CP;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2], ny = g.n[1];
  const int plane = Cx * Cy;
  const float* Y1 = sm + L.Y1;
  float* Y2 = sm + L.Y2;
  float* Y = sm + L.Y;
  const float* Ay = sm + L.A[1];
  const float* Az = sm + L.A[2];
  // y: thread per (kl, a), every b in registers: Y2[kl][b][a] = sum_j Y1[(kl, j)][a] Ay[j][b]
  for (int e = tid; e < kc * Cx; e += nthr) {
    const int kl = e / Cx, a = e - kl * Cx;
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;
    const float* y1 = Y1 + kl * ny * CPs + a;
    for (int j = 0; j < ny; ++j) {
      const float yv = y1[j * CPs];
      const float4* ar = reinterpret_cast<const float4*>(Ay + j * CP);
#pragma unroll
      for (int c4 = 0; c4 < CP / 4; ++c4) {
        const float4 w = ar[c4];
        acc[4 * c4 + 0] = fmaf(yv, w.x, acc[4 * c4 + 0]);
        acc[4 * c4 + 1] = fmaf(yv, w.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(yv, w.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(yv, w.w, acc[4 * c4 + 3]);
      }
    }
#pragma unroll
    for (int bb = 0; bb < CP; ++bb)
      if (bb < Cy) Y2[(kl * Cy + bb) * Cx + a] = acc[bb];
  }
  __syncthreads();
  // z: thread per (b, a), every c in registers: Y[c][b][a] += sum_kl Y2[kl][b][a] Az[k0 + kl][c]
  for (int ab = tid; ab < plane; ab += nthr) {
    float acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = 0.f;
    for (int kl = 0; kl < kc; ++kl) {
      const float yv = Y2[kl * plane + ab];
      const float4* ar = reinterpret_cast<const float4*>(Az + (k0 + kl) * CP);
#pragma unroll
      for (int c4 = 0; c4 < CP / 4; ++c4) {
        const float4 w = ar[c4];
        acc[4 * c4 + 0] = fmaf(yv, w.x, acc[4 * c4 + 0]);
        acc[4 * c4 + 1] = fmaf(yv, w.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(yv, w.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(yv, w.w, acc[4 * c4 + 3]);
      }
    }
#pragma unroll
    for (int c = 0; c < CP; ++c)
      if (c < Cz) Y[c * plane + ab] += acc[c];
  }
  __syncthreads();
}

// Writes the block's result Y; for the fit also the RMSE of
// the fitted model (banded value decode vs the samples; per-thread FP32 Kahan sums reduced in FP64).
template <int CP, int MODE>
__device__ void c3_epilogue(const ContractParams& prm, const C3Smem& L, float* sm, const C3Geom& g, int item,
                            const float* X, int ks, double* s_red) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Cx = g.C[0], Cy = g.C[1], Cz = g.C[2];
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int plane = Cx * Cy, ncps = plane * Cz;
  const float* Y = sm + L.Y;
  if (MODE != kFit) {  // adjoint N^T R, or gradient N^T (decode(P) - D)
    for (int e = tid; e < ncps; e += nthr) prm.out[g.cpoff + e] = Y[e];
    return;
  }
  for (int e = tid; e < ncps; e += nthr) prm.out[g.cpoff + e] = Y[e];
  if (!prm.rmse) return;
  const TabEntry* tx = reinterpret_cast<const TabEntry*>(sm + L.tab[0]);
  const TabEntry* ty = reinterpret_cast<const TabEntry*>(sm + L.tab[1]);
  const TabEntry* tz = reinterpret_cast<const TabEntry*>(sm + L.tab[2]);
  float* Y1 = sm + L.Y1;
  float* Y2 = sm + L.Y2;
  float ksum = 0.f, kcomp = 0.f;
  for (int k0 = 0; k0 < nz; k0 += ks) {
    const int kc = min(ks, nz - k0);
    for (int e = tid; e < plane * kc; e += nthr) {  // T0 -> Y2
      const int kl = e / plane, ab = e - kl * plane;
      const TabEntry te = tz[k0 + kl];
      float acc = 0.f;
      _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[2]) acc = fmaf(Y[(te.off + d) * plane + ab], te.N[d], acc);
      Y2[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < Cx * ny * kc; e += nthr) {  // U0 -> Y1
      const int a = e % Cx, r = e / Cx, j = r % ny, kl = r / ny;
      const TabEntry te = ty[j];
      float acc = 0.f;
      _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[1]) acc = fmaf(Y2[(kl * Cy + te.off + d) * Cx + a], te.N[d], acc);
      Y1[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < nx * ny * kc; e += nthr) {
      const int i = e % nx, r = e / nx;
      const TabEntry te = tx[i];
      float f = 0.f;
      _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[0]) f = fmaf(Y1[r * Cx + te.off + d], te.N[d], f);
      const float diff = f - __ldg(X + (int64_t)k0 * nx * ny + e);
      const float y = diff * diff - kcomp;
      const float t = ksum + y;
      kcomp = (t - ksum) - y;
      ksum = t;
    }
    __syncthreads();
  }
  double sq = (double)ksum - (double)kcomp;
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = sq;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(nthr / 32); ++w) tot += s_red[w];
    prm.rmse[item] = sqrt(tot / ((double)nx * ny * nz));
  }
}

// Banded value decode of one z-slab inside the contraction kernel, on rows of 32 samples in the
// 128-byte-swizzled slab buffer (logical 16-byte chunk c of row r at chunk c ^ (r & 7)):
//   stage z  T[kl][b][a]  = sum_d Q[o_k + d][b][a] N_z[k][d]      (-> Y2; flat over (kl, b, a))
//   stage y  U[(kl,j)][a] = sum_d T[kl][o_j + d][a] N_y[j][d]      (-> rows of Y1, stride ys; a thread
//                                                                 keeps one column a and steps over rows)
//   stage x  f[(kl,j)][i] = sum_d U[(kl,j)][o_i + d] N_x[i][d]     (a thread owns sample i)
// kResidual (gradient): Q = P, and the buffer's samples D become r = f - D in place.
// kRmse (fit): Q = the fitted control points, (f - D)^2 goes into the thread's Kahan sum.
enum SlabDecode { kResidual = 0, kRmse = 1 };

template <int MODE, bool SHORT_ROWS>
__device__ void c3_value_decode_slab(const C3Smem& L, float* sm, const C3Geom& g, const float* Q, float4* xb,
                                     int k0, int kc, int ys, float& ksum, float& kcomp) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int Cx = g.C[0], Cy = g.C[1], ny = g.n[1];
  const int plane = Cx * Cy;
  float* Y1 = sm + L.Y1;
  float* Y2 = sm + L.Y2;
  const TabEntry* tx = reinterpret_cast<const TabEntry*>(sm + L.tab[0]);
  const TabEntry* ty = reinterpret_cast<const TabEntry*>(sm + L.tab[1]);
  const TabEntry* tz = reinterpret_cast<const TabEntry*>(sm + L.tab[2]);
  {  // stage z, flat index e = kl*plane + ab with incremental (kl, ab)
    int kl = tid / plane, ab = tid - (tid / plane) * plane;
    for (int e = tid; e < kc * plane; e += nthr) {
      const TabEntry te = tz[k0 + kl];
      float acc = 0.f;
      _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[2]) acc = fmaf(Q[(te.off + d) * plane + ab], te.N[d], acc);
      Y2[e] = acc;
      ab += nthr;
      while (ab >= plane) { ab -= plane; ++kl; }
    }
  }
  __syncthreads();
  {  // stage y: thread keeps column a; rows r = (kl, j) advance by `step`
    const int step = nthr / Cx, grp = tid / Cx;
    if (grp < step) {
      const int a = tid - grp * Cx;
      int kl = grp / ny, j = grp - (grp / ny) * ny;
      for (int r = grp; r < kc * ny; r += step) {
        const TabEntry te = ty[j];
        const float* tp = Y2 + (kl * Cy + te.off) * Cx + a;
        float u = 0.f;
        _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[1]) u = fmaf(tp[d * Cx], te.N[d], u);
        Y1[r * ys + a] = u;
        j += step;
        while (j >= ny) { j -= ny; ++kl; }
      }
    }
  }
  __syncthreads();
  // stage x: thread owns sample i of 32-sample rows; rows r0, r0 + nthr/32, ...; with SHORT_ROWS the
  // samples i >= nx (zero padding of shorter rows) are left as they are
  const int i = tid & 31;
  if (!SHORT_ROWS || i < g.n[0]) {
    const int rstep = nthr >> 5;
    const TabEntry te = tx[i];
    float* xf = reinterpret_cast<float*>(xb);
    for (int r = tid >> 5; r < kc * ny; r += rstep) {
      const float* ur = Y1 + r * ys + te.off;
      float f = 0.f;
      _Pragma("unroll") for (int d = 0; d <= MFA_MAX_DEGREE; ++d) if (d <= g.p[0]) f = fmaf(ur[d], te.N[d], f);
      const int idx = r * 32 + (((i >> 2) ^ (r & 7)) << 2) + (i & 3);
      if (MODE == kResidual) {
        xf[idx] = f - xf[idx];
      } else {
        const float diff = f - xf[idx];
        const float y = diff * diff - kcomp;
        const float t = ksum + y;
        kcomp = (t - ksum) - y;
        ksum = t;
      }
    }
  }
  __syncthreads();
}

// Queue kernel: blocks from an atomic counter, rows read from global memory.
template <int CP, int MODE>
__global__ void __launch_bounds__(kThreads) contract3_kernel(ContractParams prm, C3Smem L, int ks, int vec_ok) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item, s_bad;
  __shared__ C3Geom s_g;
  __shared__ double s_red[kThreads / 32];
  const int tid = threadIdx.x;
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_item = atomicAdd(prm.counter, 1u);
      s_bad = 0;
      c3_fetch(prm, s_item, s_g);
    }
    __syncthreads();
    if (!s_g.valid) break;
    if (s_g.bad) continue;
    const C3Geom& g = s_g;
    c3_setup<CP, MODE>(prm, L, sm, g, &s_bad);
    if (s_bad) continue;
    const float* X = prm.x + (int64_t)g.slot * prm.slot_stride;
    const bool vec = vec_ok && (g.n[0] % 4 == 0);
    for (int k0 = 0; k0 < g.n[2]; k0 += ks) {
      const int kc = min(ks, g.n[2] - k0);
      c3_stage_x_global<CP>(X, sm + L.A[0], sm + L.Y1, k0, kc, g.n[0], g.n[1], vec);
      __syncthreads();
      c3_stage_yz<CP>(L, sm, g, k0, kc);
    }
    c3_epilogue<CP, MODE>(prm, L, sm, g, s_item, X, ks, s_red);
  }
}

// TMA kernel: static schedule (blocks blockIdx.x, +gridDim.x, ...), slab loads double-buffered.
template <int CP, int MODE>
__global__ void __launch_bounds__(kThreads)
contract3_tma_kernel(ContractParams prm, C3Smem L, int ks, int box_rows, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ C3Geom s_g[2];
  __shared__ int s_bad;
  __shared__ double s_red[kThreads / 32];
  const int tid = threadIdx.x;
  float4* xbuf = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(sm + L.X) + 1023) & ~uintptr_t(1023));
  const int buf_f4 = box_rows * (kTmaRow / 4);
  const uint32_t box_bytes = (uint32_t)box_rows * kTmaRow * 4;
  const int64_t rows_per_slot = prm.slot_stride / kTmaRow;

  if (tid == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
    c3_fetch(prm, blockIdx.x, s_g[0]);
  }
  __syncthreads();

  uint32_t q_issue = 0, q_cons = 0;  // slabs issued / consumed by this CTA (same in every thread)
  int cur = 0;
  int item = blockIdx.x;
  auto tma_ok = [&](const C3Geom& g) {
    return g.valid && !g.bad && g.n[0] == kTmaRow && (int64_t)ks * g.n[1] <= box_rows;
  };
  if (tid == 0 && MODE == kGradient && s_g[0].valid && !s_g[0].bad && s_g[0].n[0] > kTmaRow)
    flag(prm.status, MFA_DEV_BAD_DESC);
  auto issue = [&](const C3Geom& g, int k0) {  // one thread
    const int b = q_issue & 1;
    mbar_arrive_expect_tx(&s_bar[b], box_bytes);
    const int64_t row = (int64_t)g.slot * rows_per_slot + (int64_t)k0 * g.n[1];
    tma_load_2d(xbuf + b * buf_f4, &xmap, &s_bar[b], 0, (int)row);
  };
  if (tma_ok(s_g[0])) {
    if (tid == 0) issue(s_g[0], 0);
    ++q_issue;
  }

  while (s_g[cur].valid) {
    const int nitem = item + gridDim.x;
    if (tid == 0) {
      s_bad = 0;
      c3_fetch(prm, nitem, s_g[cur ^ 1]);
    }
    __syncthreads();
    const C3Geom& g = s_g[cur];
    const C3Geom& gn = s_g[cur ^ 1];
    const bool use_tma = tma_ok(g);
    if (!g.bad) c3_setup<CP, MODE>(prm, L, sm, g, &s_bad);
    const bool skip = g.bad || s_bad;
    const float* X = prm.x + (int64_t)g.slot * prm.slot_stride;
    const int nz = g.valid && !g.bad ? g.n[2] : 0;
    const int nslab = (nz + ks - 1) / ks;
    // units of this block: the contraction's slabs, then (fit with RMSE, TMA rows) the residual slabs
    const bool rmse_pass = MODE == kFit && prm.rmse && use_tma;
    const int nunits = nslab * (rmse_pass ? 2 : 1);
    float ksum = 0.f, kcomp = 0.f;
    for (int u = 0; u < nunits; ++u) {
      const int pass = u >= nslab, s = pass ? u - nslab : u;
      const int k0 = s * ks, kc = min(ks, nz - k0);
      // prefetch the next unit of the schedule into the other buffer
      if (u + 1 < nunits) {
        if (use_tma) {
          if (tid == 0) issue(g, ((u + 1) % nslab) * ks);
          ++q_issue;
        }
      } else if (tma_ok(gn)) {
        if (tid == 0) issue(gn, 0);
        ++q_issue;
      }
      if (use_tma) {
        const int b = q_cons & 1;
        const bool ok = mbar_wait_bounded(&s_bar[b], (q_cons >> 1) & 1);
        ++q_cons;
        if (__syncthreads_or(!ok)) {
          if (tid == 0) {
            flag(prm.status, MFA_DEV_TIMEOUT);
            for (uint32_t q = q_cons; q < q_issue; ++q) mbar_wait_bounded(&s_bar[q & 1], (q >> 1) & 1);
          }
          __syncthreads();
          return;
        }
        if (!skip) {
          if (pass == 0) {
            if (MODE == kGradient)
              c3_value_decode_slab<kResidual, false>(L, sm, g, sm + L.P, xbuf + b * buf_f4, k0, kc, L.us, ksum,
                                                     kcomp);
            c3_stage_x_smem<CP>(xbuf + b * buf_f4, sm + L.A[0], sm + L.Y1, kc * g.n[1]);
          } else {
            c3_value_decode_slab<kRmse, false>(L, sm, g, sm + L.Y, xbuf + b * buf_f4, k0, kc, L.us, ksum, kcomp);
          }
        }
      } else if (!skip && MODE == kGradient) {
        // rows shorter than 32 samples: fill the buffer no TMA copy is using, zero-padded and swizzled
        float4* xb = xbuf + (q_issue & 1) * buf_f4;
        float* xf = reinterpret_cast<float*>(xb);
        const int nx = g.n[0], rows = kc * g.n[1];
        for (int e = tid; e < rows * kTmaRow; e += blockDim.x) {
          const int r = e >> 5, i = e & 31;
          const float v = i < nx ? X[((int64_t)k0 * g.n[1] + r) * nx + i] : 0.f;
          xf[r * kTmaRow + (((i >> 2) ^ (r & 7)) << 2) + (i & 3)] = v;
        }
        __syncthreads();
        c3_value_decode_slab<kResidual, true>(L, sm, g, sm + L.P, xb, k0, kc, L.us, ksum, kcomp);
        c3_stage_x_smem<CP>(xb, sm + L.A[0], sm + L.Y1, rows);
      } else if (!skip) {
        c3_stage_x_global<CP>(X, sm + L.A[0], sm + L.Y1, k0, kc, g.n[0], g.n[1],
                              (g.n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) &&
                                  (prm.slot_stride % 4 == 0));
      }
      __syncthreads();
      if (!skip && pass == 0) c3_stage_yz<CP>(L, sm, g, k0, kc);
    }
    if (nslab == 0 && tma_ok(gn)) {  // no slab of this block carried the next block's prefetch
      if (tid == 0) issue(gn, 0);
      ++q_issue;
    }
    if (!skip && nslab > 0) {
      if (rmse_pass) {
        const int ncps = g.C[0] * g.C[1] * g.C[2];
        for (int e = tid; e < ncps; e += blockDim.x) prm.out[g.cpoff + e] = sm[L.Y + e];
        double sq = (double)ksum - (double)kcomp;
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = sq;
        __syncthreads();
        if (tid == 0) {
          double tot = 0.0;
          for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += s_red[w];
          prm.rmse[item] = sqrt(tot / ((double)g.n[0] * g.n[1] * g.n[2]));
        }
      } else {
        c3_epilogue<CP, MODE>(prm, L, sm, g, item, X, ks, s_red);
      }
    }
    __syncthreads();
    cur ^= 1;
    item = nitem;
  }
}

template <int CP>
cudaError_t launch_c3(mfa_ctx* ctx, const ContractParams& prm, const C3Smem& L, int ks, int vec_ok,
                      const CUtensorMap* xmap, int box_rows, cudaStream_t stream) {
  const size_t smem = (size_t)L.total * 4;
  int occ = 0;
  cudaError_t e;
  if (xmap) {
    auto kern = prm.mode == kFit ? contract3_tma_kernel<CP, kFit>
                                 : (prm.mode == kAdjoint ? contract3_tma_kernel<CP, kAdjoint> : contract3_tma_kernel<CP, kGradient>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(ctx->num_sms * occ, prm.nblocks));
    kern<<<grid, kThreads, smem, stream>>>(prm, L, ks, box_rows, *xmap);
  } else {
    if (prm.mode == kGradient) return cudaErrorInvalidValue;  // the gradient needs the TMA path
    auto kern = prm.mode == kFit ? contract3_kernel<CP, kFit> : contract3_kernel<CP, kAdjoint>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int grid = std::max(1, std::min(ctx->num_sms * occ, prm.nblocks));
    kern<<<grid, kThreads, smem, stream>>>(prm, L, ks, vec_ok);
  }
  ctx->launches++;
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map over the sample grids viewed as rows of 32 floats: box = 32 x box_rows, 128-byte swizzle.
bool make_row_map(CUtensorMap* map, const float* x, int64_t nslots, int64_t slot_stride, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int64_t rows = nslots * slot_stride / kTmaRow;
  if (rows < 1 || rows >= (int64_t(1) << 31)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kTmaRow, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kTmaRow * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kTmaRow, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int contract3(mfa_ctx* ctx, ContractParams prm, cudaStream_t stream) {
  const int CP = round4(prm.maxC);
  const bool rmse = prm.rmse != nullptr;
  // TMA path: rows of 32 samples (caller's hint), 16-byte aligned grids whose slots hold whole rows
  const bool tma = prm.rows32 && (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) && (prm.slot_stride % kTmaRow == 0);
  int ks = std::min(8, prm.maxN);
  if (tma) ks = std::max(1, std::min(ks, 256 / prm.maxN));
  auto layout = [&](int k) { return c3_layout(prm.mode, CP, prm.maxC, prm.maxN, k, rmse, tma ? k * prm.maxN * kTmaRow : 0); };
  C3Smem L = layout(ks);
  while ((size_t)L.total * 4 > kMaxDynSmem && ks > 1) {
    ks = std::max(1, ks / 2);
    L = layout(ks);
  }
  if ((size_t)L.total * 4 > kMaxDynSmem) return MFA_ERR_CAPACITY;
  if (prm.mode == kGradient && !tma) return MFA_ERR_UNSUPPORTED;
  CUtensorMap map;
  const int box_rows = ks * prm.maxN;
  const bool use_map = tma && make_row_map(&map, prm.x, prm.nslots, prm.slot_stride, box_rows);
  if (!use_map && prm.mode == kGradient) return MFA_ERR_UNSUPPORTED;
  if (!use_map) L = c3_layout(prm.mode, CP, prm.maxC, prm.maxN, ks, rmse, 0);
  const int vec_ok = (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) && (prm.slot_stride % 4 == 0);
  if (!use_map && cudaMemsetAsync(prm.counter, 0, sizeof(uint32_t), stream) != cudaSuccess) return MFA_ERR_CUDA;
  const CUtensorMap* mp = use_map ? &map : nullptr;
  cudaError_t e;
  switch (CP) {
    case 4: e = launch_c3<4>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 8: e = launch_c3<8>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 12: e = launch_c3<12>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 16: e = launch_c3<16>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 20: e = launch_c3<20>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 24: e = launch_c3<24>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 28: e = launch_c3<28>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    case 32: e = launch_c3<32>(ctx, prm, L, ks, vec_ok, mp, box_rows, stream); break;
    default: return MFA_ERR_INVALID_ARG;
  }
  return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

}  // namespace mfa
