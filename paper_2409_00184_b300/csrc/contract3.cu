// Transposed three-axis contraction of per-block sample grids, shared by the least-squares fit and
// the adjoint:
//     Y[c][b][a] = sum_{k,j,i} X[k][j][i] Ax[i][a] Ay[j][b] Az[k][c]
//   kFit:      A = (N^T N)^{-1} N^T per axis (from the encode plan) -> least-squares control points,
//              then optionally the RMSE of the fitted model over the samples (Table 1's metric);
//   kAdjoint:  A = N (collocation matrix, its band built from the knots in the CTA) -> N^T R;
//   kGradient: G = N^T (decode(P) - D), the gradient of 0.5*||decode(P) - D||^2: each slab of samples is
//              replaced in shared memory by its residual (a banded value decode of P minus the samples)
//              before the contraction, so the cancellation happens per sample, at the data's scale.
//              TMA kernel only; other shapes use the banded adjoint kernel.
// One CTA per block; the grid streams through in z-slabs of ks planes:
//   x:  Y1[(k,j)][a] = sum_i X[k][j][i] Ax[i][a]   thread per sample row
//   y:  Y2[k][b][a]  = sum_j Y1[(k,j)][a] Ay[j][b]  thread per (k, a)
//   z:  Y[c][b][a]  += sum_k Y2[k][b][a] Az[k][c]   thread per (b, a)
// The fit's A (the pseudo-inverse) is dense: a thread keeps all columns of its output in registers
// and reads the rows of A as shared-memory broadcasts. The adjoint's and the gradient's A = N has
// q = p + 1 nonzeros per sample: those modes keep only the q partial sums of the sample's band and
// write each column once the band has passed it (a quarter of the dense products at C = 12).
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
  int A[3], bandN[3], bandO[3], adv, off[3], tab[3], knots, Y1, Y2, Y, P, X, total;  // offsets in 4-byte words
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
  for (int a = 0; a < 3; ++a) { L.A[a] = o; if (mode == kFit) o += maxN * CP; }
  // adjoint and gradient: banded basis per axis and sample (q values as a float4, band offset s - p)
  for (int a = 0; a < 3; ++a) { L.bandN[a] = o; if (mode != kFit) o += 4 * maxN; }
  for (int a = 0; a < 3; ++a) { L.bandO[a] = o; if (mode != kFit) o += maxN; }
  o = round4(o);
  // per axis: 64-bit mask of the samples where the band moves on by one column, then a flag word
  // (1: the band starts at column 0 and never moves by more than one column per sample)
  L.adv = o; if (mode != kFit) o += 12;
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
    for (int a = 0; a < 3; ++a) {
      for (int i = tid; i < g.C[a] + g.p[a] + 1; i += nthr) kn[a * kKnotMax + i] = prm.knots[g.koff[a] + i];
      // band entries past n[a] (zero padding of shorter rows): zero weights, offset C - 1 (the band
      // only moves forward, so those entries close every remaining column and add nothing)
      for (int i = g.n[a] + tid; i < prm.maxN; i += nthr) {
        reinterpret_cast<float4*>(sm + L.bandN[a])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<int*>(sm + L.bandO[a])[i] = g.C[a] - 1;
      }
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
      reinterpret_cast<float4*>(sm + L.bandN[a])[i] = make_float4(N[0], N[1], N[2], N[3]);
      reinterpret_cast<int*>(sm + L.bandO[a])[i] = s - g.p[a];
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
  if (MODE != kFit && tid < 3) {
    const int* bO = reinterpret_cast<const int*>(sm + L.bandO[tid]);
    unsigned long long m = 0ull;
    int simple = bO[0] == 0;
    for (int i = 1; i < g.n[tid]; ++i) {
      const int step = bO[i] - bO[i - 1];
      if (step == 1) m |= 1ull << i;
      else if (step != 0) simple = 0;
    }
    reinterpret_cast<unsigned long long*>(sm + L.adv)[tid] = m;
    reinterpret_cast<int*>(sm + L.adv)[6 + tid] = simple;
  }
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

// ---- banded transposed stages (adjoint and gradient: A = N, q = p + 1 nonzeros per sample) ----
// A sample's band covers the columns o_i .. o_i + q - 1, and o_i never decreases with i. A thread
// walks its samples in order with the q partial sums of the current band in registers; when the band
// moves on, the column it leaves is complete and is written out (ACC: added to the output). Every
// thread of a stage walks the same sample sequence, so the band moves are uniform across a warp.
// The usual case (band from column 0, at most one column per sample) reads the moves from a bit mask
// held in a register, so no branch waits on a shared-memory load; other knot vectors take the
// general walk over the stored offsets.
template <int Q, bool ACC>
__device__ __forceinline__ void band_emit(float (&w)[Q], int& o, float* __restrict__ out, int stride) {
  if (ACC) out[o * stride] += w[0]; else out[o * stride] = w[0];
#pragma unroll
  for (int d = 0; d + 1 < Q; ++d) w[d] = w[d + 1];
  w[Q - 1] = 0.f;
  ++o;
}

template <int Q, bool ACC>
__device__ __forceinline__ void band_advance(float (&w)[Q], int& o, int to, float* __restrict__ out, int stride) {
  while (o < to) band_emit<Q, ACC>(w, o, out, stride);
}

template <int Q>
__device__ __forceinline__ void band_fma(float (&w)[Q], const float4 nw, float x) {
  w[0] = fmaf(nw.x, x, w[0]);
  w[1] = fmaf(nw.y, x, w[1]);
  w[2] = fmaf(nw.z, x, w[2]);
  if (Q > 3) w[Q > 3 ? 3 : 0] = fmaf(nw.w, x, w[Q > 3 ? 3 : 0]);
}

struct Band {
  const float4* __restrict__ N;  // q basis values per sample (zero past q)
  const int* __restrict__ off;   // first column of the sample's band
  unsigned long long adv;        // SIMPLE walk: bit i set when the band moves on at sample i
};

__device__ __forceinline__ Band c3_band(const C3Smem& L, const float* sm, int a) {
  Band b;
  b.N = reinterpret_cast<const float4*>(sm + L.bandN[a]);
  b.off = reinterpret_cast<const int*>(sm + L.bandO[a]);
  b.adv = reinterpret_cast<const unsigned long long*>(sm + L.adv)[a];
  return b;
}

__device__ __forceinline__ bool c3_band_simple(const C3Smem& L, const float* sm, int a) {
  return reinterpret_cast<const int*>(sm + L.adv)[6 + a] != 0;
}

// moves the band to sample i's columns
template <int Q, bool SIMPLE, bool ACC>
__device__ __forceinline__ void band_to(const Band& bd, int i, float (&w)[Q], int& o, float* __restrict__ out,
                                        int stride) {
  if (SIMPLE) {
    if ((bd.adv >> i) & 1ull) band_emit<Q, ACC>(w, o, out, stride);
  } else {
    band_advance<Q, ACC>(w, o, bd.off[i], out, stride);
  }
}

// x^T: V[r][a] = sum_i N_a(u_i) X[r][i], thread per row of 32 samples of the swizzled slab buffer.
template <int Q, bool SIMPLE>
__device__ void c3_stage_xT_smem(const float4* __restrict__ xb, const Band bd, int C, float* __restrict__ Y1, int ys,
                                 int rows) {
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    float w[Q];
#pragma unroll
    for (int d = 0; d < Q; ++d) w[d] = 0.f;
    int o = 0;
    float* yr = Y1 + r * ys;
    const float4* row = xb + r * 8;
    const int sw = r & 7;
#pragma unroll 2
    for (int c = 0; c < 8; ++c) {
      const float4 v = row[c ^ sw];
      const float xs[4] = {v.x, v.y, v.z, v.w};
      float4 nw[4];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) nw[q4] = bd.N[4 * c + q4];
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        band_to<Q, SIMPLE, false>(bd, 4 * c + q4, w, o, yr, 1);
        band_fma<Q>(w, nw[q4], xs[q4]);
      }
    }
    band_advance<Q, false>(w, o, C, yr, 1);
  }
}

// x^T from global memory (rows of any length nx).
template <int Q>
__device__ void c3_stage_xT_global(const float* X, const Band bd, int C, float* __restrict__ Y1, int ys, int k0,
                                   int kc, int nx, int ny) {
  for (int r = threadIdx.x; r < kc * ny; r += blockDim.x) {
    const float* xr = X + ((int64_t)k0 * ny + r) * nx;
    float w[Q];
#pragma unroll
    for (int d = 0; d < Q; ++d) w[d] = 0.f;
    int o = 0;
    float* yr = Y1 + r * ys;
    for (int i = 0; i < nx; ++i) {
      band_advance<Q, false>(w, o, bd.off[i], yr, 1);
      band_fma<Q>(w, bd.N[i], __ldg(xr + i));
    }
    band_advance<Q, false>(w, o, C, yr, 1);
  }
}

//   W[kl][b][a]  = sum_j N_b(v_j) V[(kl, j)][a]        thread per (kl, a)
template <int Q, bool SIMPLE>
__device__ void c3_stage_yT(const float* __restrict__ Y1, int ys, const Band bd, float* __restrict__ Y2, int kc,
                            int Cx, int Cy, int ny) {
  const int plane = Cx * Cy;
  for (int e = threadIdx.x; e < kc * Cx; e += blockDim.x) {
    const int kl = e / Cx, a = e - kl * Cx;
    const float* y1 = Y1 + kl * ny * ys + a;
    float* y2 = Y2 + kl * plane + a;
    float w[Q];
#pragma unroll
    for (int d = 0; d < Q; ++d) w[d] = 0.f;
    int o = 0;
#pragma unroll 4
    for (int j = 0; j < ny; ++j) {
      const float v = y1[j * ys];
      const float4 nw = bd.N[j];
      band_to<Q, SIMPLE, false>(bd, j, w, o, y2, Cx);
      band_fma<Q>(w, nw, v);
    }
    band_advance<Q, false>(w, o, Cy, y2, Cx);
  }
}

//   Y[c][b][a]  += sum_kl N_c(w_{k0+kl}) W[kl][b][a]    thread per (b, a); the band of the slab's first
//                                                       plane opens the window, columns are added to Y
template <int Q, bool SIMPLE>
__device__ void c3_stage_zT(const float* __restrict__ Y2, const Band bd, float* __restrict__ Y, int k0, int kc,
                            int plane, int Cz) {
  for (int ab = threadIdx.x; ab < plane; ab += blockDim.x) {
    float w[Q];
#pragma unroll
    for (int d = 0; d < Q; ++d) w[d] = 0.f;
    int o = bd.off[k0];
    for (int kl = 0; kl < kc; ++kl) {
      const float v = Y2[kl * plane + ab];
      const float4 nw = bd.N[k0 + kl];
      if (kl > 0) band_to<Q, SIMPLE, true>(bd, k0 + kl, w, o, Y + ab, plane);
      band_fma<Q>(w, nw, v);
    }
#pragma unroll
    for (int d = 0; d < Q; ++d)
      if (o + d < Cz) Y[(o + d) * plane + ab] += w[d];
  }
}

// Dispatch on the band width (q = 3 covers degrees 1 and 2) and on the walk.
template <int Q>
__device__ __forceinline__ void c3_banded_x_smem_q(const C3Smem& L, float* sm, const C3Geom& g, const float4* xb,
                                                   int rows) {
  const Band bd = c3_band(L, sm, 0);
  if (c3_band_simple(L, sm, 0)) c3_stage_xT_smem<Q, true>(xb, bd, g.C[0], sm + L.Y1, L.us, rows);
  else c3_stage_xT_smem<Q, false>(xb, bd, g.C[0], sm + L.Y1, L.us, rows);
}

__device__ __forceinline__ void c3_banded_x_smem(const C3Smem& L, float* sm, const C3Geom& g, const float4* xb,
                                                 int rows) {
  if (g.p[0] <= 2) c3_banded_x_smem_q<3>(L, sm, g, xb, rows);
  else c3_banded_x_smem_q<4>(L, sm, g, xb, rows);
}

__device__ __forceinline__ void c3_banded_x_global(const C3Smem& L, float* sm, const C3Geom& g, const float* X,
                                                   int k0, int kc) {
  const Band bd = c3_band(L, sm, 0);
  if (g.p[0] <= 2) c3_stage_xT_global<3>(X, bd, g.C[0], sm + L.Y1, L.us, k0, kc, g.n[0], g.n[1]);
  else c3_stage_xT_global<4>(X, bd, g.C[0], sm + L.Y1, L.us, k0, kc, g.n[0], g.n[1]);
}

template <int Q>
__device__ __forceinline__ void c3_banded_y_q(const C3Smem& L, float* sm, const C3Geom& g, int kc) {
  const Band bd = c3_band(L, sm, 1);
  if (c3_band_simple(L, sm, 1)) c3_stage_yT<Q, true>(sm + L.Y1, L.us, bd, sm + L.Y2, kc, g.C[0], g.C[1], g.n[1]);
  else c3_stage_yT<Q, false>(sm + L.Y1, L.us, bd, sm + L.Y2, kc, g.C[0], g.C[1], g.n[1]);
}

template <int Q>
__device__ __forceinline__ void c3_banded_z_q(const C3Smem& L, float* sm, const C3Geom& g, int k0, int kc) {
  const Band bd = c3_band(L, sm, 2);
  const int plane = g.C[0] * g.C[1];
  if (c3_band_simple(L, sm, 2)) c3_stage_zT<Q, true>(sm + L.Y2, bd, sm + L.Y, k0, kc, plane, g.C[2]);
  else c3_stage_zT<Q, false>(sm + L.Y2, bd, sm + L.Y, k0, kc, plane, g.C[2]);
}

// y^T then z^T of one slab
__device__ __forceinline__ void c3_banded_yz(const C3Smem& L, float* sm, const C3Geom& g, int k0, int kc) {
  if (g.p[1] <= 2) c3_banded_y_q<3>(L, sm, g, kc); else c3_banded_y_q<4>(L, sm, g, kc);
  __syncthreads();
  if (g.p[2] <= 2) c3_banded_z_q<3>(L, sm, g, k0, kc); else c3_banded_z_q<4>(L, sm, g, k0, kc);
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
  for (int e = tid; e < ncps; e += nthr) prm.out[g.cpoff + e] = Y[e];
  // the adjoint N^T R and the gradient N^T (decode(P) - D) end here; the fit may add its RMSE
  if (MODE != kFit || !prm.rmse) return;
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
      if (MODE == kFit) c3_stage_x_global<CP>(X, sm + L.A[0], sm + L.Y1, k0, kc, g.n[0], g.n[1], vec);
      else c3_banded_x_global(L, sm, g, X, k0, kc);
      __syncthreads();
      if (MODE == kFit) c3_stage_yz<CP>(L, sm, g, k0, kc);
      else c3_banded_yz(L, sm, g, k0, kc);
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
            if (MODE == kFit) c3_stage_x_smem<CP>(xbuf + b * buf_f4, sm + L.A[0], sm + L.Y1, kc * g.n[1]);
            else c3_banded_x_smem(L, sm, g, xbuf + b * buf_f4, kc * g.n[1]);
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
        c3_banded_x_smem(L, sm, g, xb, rows);
      } else if (!skip) {
        if (MODE == kFit)
          c3_stage_x_global<CP>(X, sm + L.A[0], sm + L.Y1, k0, kc, g.n[0], g.n[1],
                                (g.n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) &&
                                    (prm.slot_stride % 4 == 0));
        else
          c3_banded_x_global(L, sm, g, X, k0, kc);
      }
      __syncthreads();
      if (!skip && pass == 0) {
        if (MODE == kFit) c3_stage_yz<CP>(L, sm, g, k0, kc);
        else c3_banded_yz(L, sm, g, k0, kc);
      }
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

// ---- z-first streaming kernel (fit without its RMSE pass, adjoint; n <= 32 per axis, C <= 16) ----
// The sample planes stream through a ring of TMA slabs and are contracted over z on arrival:
//   z:  T[c][j][i] = sum_k Az[k][c] X[k][j][i]     thread per 4 neighbouring (j, i) columns, all C rows
//                                                   of its columns in registers; the plane's Az row is
//                                                   one broadcast for every thread, so the stage is
//                                                   almost only FMAs
//   y:  U[c][b][i] = sum_j Ay[j][b] T[c][j][i]     thread per (c, i), all b in registers
//   x:  Y[c][b][a] = sum_i Ax[i][a] U[c][b][i]     thread per (c, b), all a in registers
// One CTA per SM, two warp groups working on consecutive blocks of the CTA's static schedule:
//  * the z group (warps 0-7) streams block after block through the z stage; its thread 0 keeps the
//    TMA ring up to R slabs ahead, into the next block once that block's set-up is published (the
//    producer reads the geometry from the set-up, so it never waits on a descriptor load);
//  * the y/x group (warps 8-15) finishes the previous block (y and x stages, output) and sets up the
//    block three ahead of it: its geometry is fetched before the wait for T, its A matrices are built
//    after the x stage, and only when the block's class (fit) or degree, C, n and knot vectors
//    (adjoint) differ from those of the block the buffer held before.
// Geometry and A rotate through four buffers (block n in buffer n % 4), so the geometry of the next
// block is published well before the producer needs it; T is handed from the z group
// (which keeps its sums in registers until a block's last plane) to the y/x group and back on
// mbarriers (T full, T free, set-up ready), so neither group waits for the other's stages and the
// samples keep streaming while a block is finished. Slabs are 8 planes (32 KB) where shared memory
// allows: the streaming rate grows with the bytes per copy. Every wait is bounded (MFA_DEV_TIMEOUT).
// Blocks whose x-rows or y-columns are shorter than 32 are copied into their T buffer (not yet in
// use), zero-padded, instead of loaded by TMA; the zero rows of A make the padding contribute nothing.
constexpr int kZfPlane = 1024;   // samples of a 32 x 32 plane
constexpr int kZfMaxRing = 16;
constexpr int kZfGroup = 256;    // z group: 8 consumer warps
constexpr int kZfYx = 224;       // y/x group: 7 warps
constexpr int kZfThreads = kZfGroup + 32 + kZfYx;  // + the producer warp: 512 threads
constexpr int kBarZ = 1, kBarYX = 2;  // named barriers of the two groups

constexpr int kZfSets = 4;  // set-up buffers (geometry, A, knots)

struct ZfSmem {
  int A[kZfSets][3], knots[kZfSets], T, U, ring, ks, R, total;  // offsets in 4-byte words; ks planes per slab
};

ZfSmem zf_layout(int mode, int CP, int ks, int R) {
  ZfSmem L;
  int o = 0;
  for (int p = 0; p < kZfSets; ++p)
    for (int a = 0; a < 3; ++a) { L.A[p][a] = o; o += 32 * CP; }
  for (int p = 0; p < kZfSets; ++p) { L.knots[p] = o; if (mode != kFit) o += 3 * kKnotMax; }
  o = round4(o);
  L.T = o; o += CP * kZfPlane;
  L.U = o; o += round4(CP * CP * 33);
  L.ring = o; o += 252 + R * ks * kZfPlane;  // slack for 1024-byte alignment
  L.ks = ks;
  L.R = R;
  L.total = o;
  return L;
}

__device__ __forceinline__ void group_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// true in every thread of the group if `pred` holds in any of them
__device__ __forceinline__ bool group_any(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred q, o;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred o, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, o;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Zero-padded A matrices of a block (32 rows x CP columns per axis) into A[.][a]: the fit's
// pseudo-inverses from the plan, or the adjoint's collocation matrices from the knots. Run by the y/x
// group (t = thread of the group); ends with the group's barrier.
template <int CP, int MODE>
__device__ void zf_setup(const ContractParams& prm, const int* A, float* kn, float* sm, const C3Geom& g, int t,
                         int* s_bad) {
  for (int e = t; e < 3 * 32 * CP; e += kZfYx) sm[A[0] + e] = 0.f;
  if (MODE != kFit)
    for (int a = 0; a < 3; ++a)
      for (int i = t; i < g.C[a] + g.p[a] + 1; i += kZfYx) kn[a * kKnotMax + i] = prm.knots[g.koff[a] + i];
  group_sync(kBarYX, kZfYx);
  if (MODE == kFit) {
    for (int a = 0; a < 3; ++a) {
      const EncClass& c = prm.classes[g.cls[a]];
      for (int e = t; e < c.n * c.C; e += kZfYx) {
        const int i = e / c.C, col = e - i * c.C;
        sm[A[a] + i * CP + col] = prm.pinv[c.pinv_off + e];
      }
    }
  } else {
    if (t < 3 && !knots_ok(kn + t * kKnotMax, g.p[t], g.C[t])) {
      atomicOr(s_bad, 1);
      flag(prm.status, MFA_DEV_BAD_KNOTS);
    }
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int a = t < nx ? 0 : (t < nx + ny ? 1 : (t < nx + ny + nz ? 2 : -1));
    if (a >= 0) {
      const int i = a == 0 ? t : (a == 1 ? t - nx : t - nx - ny);
      const float* kt = kn + a * kKnotMax;
      const float u = sample_param(i, g.n[a]);
      const int s = find_span(kt, g.p[a], g.C[a], u);
      float N[MFA_MAX_DEGREE + 1], dN[MFA_MAX_DEGREE + 1];
      basis_funs<MFA_MAX_DEGREE>(kt, g.p[a], s, u, N, dN);
      for (int r = 0; r <= g.p[a]; ++r) sm[A[a] + i * CP + s - g.p[a] + r] = N[r];
    }
  }
  group_sync(kBarYX, kZfYx);
}

// z stage over the kc planes of one slab (rows of 32 in the 128-byte-swizzled layout): thread t of
// the z group owns samples i = 4(t & 7) .. +3 of row j = t >> 3 in every plane. The FMAs run as packed
// float2 pairs (two round-to-nearest FMAs per instruction; the same results as scalar fmaf).
template <int CP>
__device__ __forceinline__ void zf_stage_z(const float4* buf, const float* Az, int k0, int kc, float2 (&acc)[CP][2]) {
  const int j = threadIdx.x >> 3, ch = threadIdx.x & 7;
#pragma unroll 2
  for (int kl = 0; kl < kc; ++kl) {
    const float4 v = buf[(kl * 32 + j) * 8 + (ch ^ (j & 7))];
    const float2 vlo = make_float2(v.x, v.y), vhi = make_float2(v.z, v.w);
    const float4* w4 = reinterpret_cast<const float4*>(Az + (k0 + kl) * CP);
#pragma unroll
    for (int c4 = 0; c4 < CP / 4; ++c4) {
      const float4 w = w4[c4];
      const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 ww = make_float2(ws[q], ws[q]);
        acc[4 * c4 + q][0] = __ffma2_rn(ww, vlo, acc[4 * c4 + q][0]);
        acc[4 * c4 + q][1] = __ffma2_rn(ww, vhi, acc[4 * c4 + q][1]);
      }
    }
  }
}

// y stage: columns e = t and t + 256 of T (c = e >> 5, i = e & 31) in one pass over j; the results
// stay in registers until the group has read all of T, then overwrite it as U.
template <int CP>
__device__ __forceinline__ void zf_y_fma(float2 (&acc)[CP / 2], const float* Ay, int j, float v) {
  const float4* w4 = reinterpret_cast<const float4*>(Ay + j * CP);
  const float2 vv = make_float2(v, v);
#pragma unroll
  for (int b4 = 0; b4 < CP / 4; ++b4) {
    const float4 w = w4[b4];
    acc[2 * b4 + 0] = __ffma2_rn(make_float2(w.x, w.y), vv, acc[2 * b4 + 0]);
    acc[2 * b4 + 1] = __ffma2_rn(make_float2(w.z, w.w), vv, acc[2 * b4 + 1]);
  }
}

template <int CP>
__device__ void zf_stage_y(const float* T, const float* Ay, float* U, int Cy, int Cz, int ny, int t) {
  // columns e (c = e >> 5, i = e & 31) in pairs e, e + kZfYx sharing the loads of Ay; a pair's second
  // column exists or not for a whole warp (Cz * 32 is a multiple of 32)
  for (int e0 = t; e0 < Cz * 32; e0 += 2 * kZfYx) {
    const int e1 = e0 + kZfYx;
    const bool h1 = e1 < Cz * 32;
    float2 a0[CP / 2], a1[CP / 2];
#pragma unroll
    for (int b = 0; b < CP / 2; ++b) a0[b] = a1[b] = make_float2(0.f, 0.f);
    const float* t0 = T + (e0 >> 5) * kZfPlane + (e0 & 31);
    const float* t1 = T + (e1 >> 5) * kZfPlane + (e1 & 31);
    if (h1) {
#pragma unroll 4
      for (int j = 0; j < ny; ++j) {
        const float v0 = t0[j * 32], v1 = t1[j * 32];
        zf_y_fma<CP>(a0, Ay, j, v0);
        zf_y_fma<CP>(a1, Ay, j, v1);
      }
    } else {
#pragma unroll 4
      for (int j = 0; j < ny; ++j) zf_y_fma<CP>(a0, Ay, j, t0[j * 32]);
    }
#pragma unroll
    for (int b = 0; b < CP; ++b)
      if (b < Cy) {
        U[((e0 >> 5) * Cy + b) * 33 + (e0 & 31)] = (b & 1) ? a0[b >> 1].y : a0[b >> 1].x;
        if (h1) U[((e1 >> 5) * Cy + b) * 33 + (e1 & 31)] = (b & 1) ? a1[b >> 1].y : a1[b >> 1].x;
      }
  }
}

template <int CP>
__device__ void zf_stage_x(const float* U, const float* Ax, float* out, int Cx, int Cy, int Cz, int nx, int t) {
  for (int q = t; q < Cz * Cy; q += kZfYx) {
    float2 acc[CP / 2];
#pragma unroll
    for (int a = 0; a < CP / 2; ++a) acc[a] = make_float2(0.f, 0.f);
    const float* ur = U + q * 33;
#pragma unroll 4
    for (int i = 0; i < nx; ++i) zf_y_fma<CP>(acc, Ax, i, ur[i]);
    float* o = out + (int64_t)q * Cx;
#pragma unroll
    for (int a = 0; a < CP; ++a)
      if (a < Cx) o[a] = (a & 1) ? acc[a >> 1].y : acc[a >> 1].x;
  }
}

template <int CP, int MODE>
__global__ void __launch_bounds__(kZfThreads, 1)
contract3_zf_kernel(ContractParams prm, ZfSmem L, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(16) float sm[];
  __shared__ __align__(8) uint64_t s_full[kZfMaxRing], s_empty[kZfMaxRing];
  __shared__ __align__(8) uint64_t s_tfull, s_tfree, s_ready[kZfSets];
  __shared__ C3Geom s_g[kZfSets], s_built[kZfSets];  // geometry of the buffer's block / of its A matrices
  __shared__ int s_bad[kZfSets], s_rebuild[kZfSets], s_has[kZfSets];  // s_rebuild: 0 keep, 1 build, 2 copy
  __shared__ int s_zabort;  // a z warp gave up waiting for a slab
  const int tid = threadIdx.x;
  const int R = L.R, ks = L.ks;
  float4* ring = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(sm + L.ring) + 1023) & ~uintptr_t(1023));
  const int slab_f4 = ks * kZfPlane / 4;
  const uint32_t slab_bytes = (uint32_t)ks * kZfPlane * 4;
  auto tma_block = [](const C3Geom& g) { return g.valid && !g.bad && g.n[0] == 32 && g.n[1] == 32; };

  if (tid == 0) {
    for (int r = 0; r < R; ++r) {
      mbar_init(&s_full[r], 1);
      mbar_init(&s_empty[r], kZfGroup / 32);  // one arrival per z warp
    }
    mbar_init(&s_tfull, kZfGroup);
    mbar_init(&s_tfree, 1);
    for (int p = 0; p < kZfSets; ++p) {
      mbar_init(&s_ready[p], 1);
      s_has[p] = 0;
    }
    s_zabort = 0;
    fence_mbar_init();
  }
  __syncthreads();  // the last CTA-wide barrier: from here on each role synchronises on its own

  if (tid < kZfGroup) {
    // ------------------------------ z group (consumers) ------------------------------
    const int lane = tid & 31;
    uint32_t consumed = 0;  // the same sequence in every warp of the group
    auto fail = [&]() {
      if (tid == 0) flag(prm.status, MFA_DEV_TIMEOUT);
    };
    for (int n = 0;; ++n) {
      const int p = n % kZfSets;
      // set-up of block n (geometry, A)
      if (group_any(kBarZ, kZfGroup, !mbar_wait_bounded(&s_ready[p], (n / kZfSets) & 1))) { fail(); return; }
      const C3Geom g = s_g[p];
      if (!g.valid) break;
      const bool skip = g.bad || s_bad[p];
      const bool tmab = tma_block(g);
      const int nz = g.bad ? 0 : g.n[2];
      const float* Az = sm + L.A[p][2];
      float* T = sm + L.T;
      // T is this block's once the y/x group is done with block n - 1 (hand-filled blocks stage their
      // planes in it, so they take it first)
      bool own_t = n == 0;
      auto take_t = [&]() {
        if (own_t) return true;
        own_t = true;
        return !group_any(kBarZ, kZfGroup, !mbar_wait_bounded(&s_tfree, (n - 1) & 1));
      };
      if (!tmab && nz > 0 && !take_t()) { fail(); return; }
      float2 acc[CP][2];
#pragma unroll
      for (int c = 0; c < CP; ++c) acc[c][0] = acc[c][1] = make_float2(0.f, 0.f);
      if (tmab) {
        // each warp consumes the ring at its own pace and hands every slab back on its empty barrier
        for (int k0 = 0; k0 < nz; k0 += ks) {
          const uint32_t slot = consumed % R;
          const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&s_full[slot], (consumed / R) & 1));
          ++consumed;
          if (!got) {  // the block's remaining slabs are abandoned; the group leaves below
            if (lane == 0) atomicExch(&s_zabort, 1);
            break;
          }
          if (!skip) zf_stage_z<CP>(ring + slot * slab_f4, Az, k0, min(ks, nz - k0), acc);
          __syncwarp();
          if (lane == 0) mbar_arrive(&s_empty[slot]);
        }
        if (group_any(kBarZ, kZfGroup, s_zabort != 0)) { fail(); return; }
      } else {
        const int step = min(ks, CP);  // a hand-filled slab must fit T (CP planes)
        const float* X = prm.x + (int64_t)g.slot * prm.slot_stride;
        const int nx = g.n[0], ny = g.n[1];
        for (int k0 = 0; k0 < nz; k0 += step) {
          const int kc = min(step, nz - k0);
          for (int e = tid; e < kc * kZfPlane; e += kZfGroup) {
            const int row = e >> 5, i = e & 31, kl = row >> 5, j = row & 31;
            const float v = (i < nx && j < ny) ? X[((int64_t)(k0 + kl) * ny + j) * nx + i] : 0.f;
            T[row * 32 + (((i >> 2) ^ (row & 7)) << 2) + (i & 3)] = v;
          }
          group_sync(kBarZ, kZfGroup);
          if (!skip) zf_stage_z<CP>(reinterpret_cast<const float4*>(T), Az, k0, kc, acc);
          group_sync(kBarZ, kZfGroup);
        }
      }
      if (!take_t()) { fail(); return; }
      if (!skip && nz > 0) {
        const int j = tid >> 3, i0 = (tid & 7) * 4;
#pragma unroll
        for (int c = 0; c < CP; ++c)
          if (c < g.C[2])
            *reinterpret_cast<float4*>(T + c * kZfPlane + j * 32 + i0) =
                make_float4(acc[c][0].x, acc[c][0].y, acc[c][1].x, acc[c][1].y);
      }
      mbar_arrive(&s_tfull);  // every thread of the group: T holds block n's z stage
    }
  } else if (tid < kZfGroup + 32) {
    // ------------------------------ producer warp ------------------------------
    // Lane 0 issues the TMA slabs of the CTA's blocks in order, each into the ring slot the z warps
    // have handed back. A block's geometry comes from its published set-up (never overwritten before
    // the z group has consumed the block, so a register copy taken after the wait stays valid).
    if (tid != kZfGroup) return;
    const int64_t rows_per_slot = prm.slot_stride / 32;
    uint32_t issued = 0;
    // the CTA must not end with a copy in flight: before leaving, the producer waits (bounded) until its
    // last R copies have landed; a copy's phase, once complete, stays complete until the slot is reused
    auto land = [&]() {
      for (uint32_t q = issued > (uint32_t)R ? issued - R : 0; q < issued; ++q)
        mbar_wait_bounded(&s_full[q % R], (q / R) & 1);
    };
    auto drain = [&]() {  // a wait gave up: report, let the copies in flight land, leave
      flag(prm.status, MFA_DEV_TIMEOUT);
      land();
    };
    for (int m = 0;; ++m) {
      const int pp = m % kZfSets;
      if (!mbar_wait_bounded(&s_ready[pp], (m / kZfSets) & 1)) { drain(); return; }
      const C3Geom& pg = s_g[pp];
      if (!pg.valid) break;
      if (!tma_block(pg)) continue;
      const int64_t row0 = (int64_t)pg.slot * rows_per_slot;
      const int nzp = pg.n[2];
      for (int k0 = 0; k0 < nzp; k0 += ks) {
        const uint32_t slot = issued % R;
        if (issued >= (uint32_t)R && !mbar_wait_bounded(&s_empty[slot], ((issued / R) - 1) & 1)) {
          drain();
          return;
        }
        mbar_arrive_expect_tx(&s_full[slot], slab_bytes);
        tma_load_2d(ring + slot * slab_f4, &xmap, &s_full[slot], 0, (int)(row0 + (int64_t)k0 * 32));
        ++issued;
      }
    }
    land();
  } else {
    // ------------------------------ y/x group ------------------------------
    const int t = tid - kZfGroup - 32;
    // one thread: geometry of block m into buffer m % 4, and how its A comes about: kept
    // (the buffer's previous block had the same class, or degree, C, n and knots), copied from the
    // buffer of block m - 1 (the same key), or built
    auto same_key = [](const C3Geom& g, const C3Geom& h) {
      bool same = true;
      for (int a = 0; a < 3 && same; ++a)
        same = MODE == kFit ? g.cls[a] == h.cls[a]
                            : (g.p[a] == h.p[a] && g.C[a] == h.C[a] && g.n[a] == h.n[a] && g.koff[a] == h.koff[a]);
      return same;
    };
    auto fetch = [&](int m) {
      const int b = m % kZfSets, bp = (m + kZfSets - 1) % kZfSets;
      c3_fetch(prm, blockIdx.x + m * (int)gridDim.x, s_g[b]);
      const C3Geom& g = s_g[b];
      int how = 0;
      if (g.valid && !g.bad && !(s_has[b] && same_key(g, s_built[b])))
        how = (m > 0 && s_has[bp] && same_key(g, s_built[bp])) ? 2 : 1;
      s_rebuild[b] = how;
      if (how == 1) s_bad[b] = 0;
      if (how == 2) s_bad[b] = s_bad[bp];
    };
    auto build = [&](int m) {  // the group: A of block m when needed, then publish the set-up
      const int b = m % kZfSets, bp = (m + kZfSets - 1) % kZfSets;
      group_sync(kBarYX, kZfYx);
      const int how = s_rebuild[b];
      if (how == 1) {
        zf_setup<CP, MODE>(prm, L.A[b], sm + L.knots[b], sm, s_g[b], t, &s_bad[b]);
      } else if (how == 2) {  // buffer bp holds block m - 1's A (rebuilt only after this one)
        for (int e = t; e < 3 * 32 * CP; e += kZfYx) sm[L.A[b][0] + e] = sm[L.A[bp][0] + e];
        group_sync(kBarYX, kZfYx);
      }
      if (how && t == 0) {
        s_built[b] = s_g[b];
        s_has[b] = 1;
      }
      if (t == 0) mbar_arrive(&s_ready[b]);
    };
    for (int m = 0; m < kZfSets - 1; ++m) {
      if (t == 0) fetch(m);
      build(m);
    }
    // the fetch for block n + 3 runs on the group's last warp during the x stage, which has the fewest
    // rows there (none for C <= 12); it writes the buffer of block n - 1, which every role is done with
    const int fetcher = kZfYx - 32;
    for (int n = 0;; ++n) {
      const int b = n % kZfSets;
      const C3Geom g = s_g[b];
      if (!g.valid) break;
      const bool ok = mbar_wait_bounded(&s_tfull, n & 1);
      if (group_any(kBarYX, kZfYx, !ok)) {
        if (t == 0) flag(prm.status, MFA_DEV_TIMEOUT);
        return;
      }
      const bool work = !g.bad && !s_bad[b] && g.n[2] > 0;
      if (work) zf_stage_y<CP>(sm + L.T, sm + L.A[b][1], sm + L.U, g.C[1], g.C[2], g.n[1], t);
      group_sync(kBarYX, kZfYx);
      if (t == 0) mbar_arrive(&s_tfree);  // T may take block n + 1
      if (t == fetcher) fetch(n + kZfSets - 1);
      if (work) zf_stage_x<CP>(sm + L.U, sm + L.A[b][0], prm.out + g.cpoff, g.C[0], g.C[1], g.C[2], g.n[0], t);
      build(n + kZfSets - 1);
    }
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

template <int CP>
cudaError_t launch_zf(mfa_ctx* ctx, const ContractParams& prm, const ZfSmem& L, const CUtensorMap& xmap,
                      cudaStream_t stream) {
  const size_t smem = (size_t)L.total * 4;
  auto kern = prm.mode == kFit ? contract3_zf_kernel<CP, kFit> : contract3_zf_kernel<CP, kAdjoint>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kZfThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(ctx->num_sms * occ, prm.nblocks));
  kern<<<grid, kZfThreads, smem, stream>>>(prm, L, xmap);
  ctx->launches++;
  return cudaGetLastError();
}

// The driver's tensor-map encoder, looked up once. The function-local static is initialised exactly once
// even when several threads make their first call at the same time (entry points without a context, such
// as the allocation-free encode, can be called from any thread).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
  }();
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

// The z-first kernel: the fit without its RMSE pass and the adjoint, for grids of at most 32 samples per
// axis and at most 16 control points per axis, on 16-byte-aligned sample grids whose slots hold whole
// rows of 32; one CTA per SM with the deepest ring that fits. Returns MFA_ERR_UNSUPPORTED when the call
// does not qualify.
static int contract3_zfirst(mfa_ctx* ctx, const ContractParams& prm, cudaStream_t stream) {
  const int CP = round4(prm.maxC);
  const bool qualifies = (prm.mode == kAdjoint || (prm.mode == kFit && prm.rmse == nullptr)) && CP <= 16 &&
                         prm.maxN <= 32 && (reinterpret_cast<uintptr_t>(prm.x) % 16 == 0) &&
                         (prm.slot_stride % 32 == 0);
  if (!qualifies) return MFA_ERR_UNSUPPORTED;
  // slab planes and ring depth: the largest slab with at least three in the ring, else with two
  auto depth = [&](int ks) {
    int R = 0;
    for (int r = kZfMaxRing; r >= 2 && !R; --r)
      if ((size_t)zf_layout(prm.mode, CP, ks, r).total * 4 + 2048 <= kMaxDynSmem) R = r;  // room for static smem
    return R;
  };
  int ks = 0, R = 0;
  for (int need = 3; need >= 2 && !ks; --need)
    for (int k : {8, 4, 2})
      if (!ks && depth(k) >= need) { ks = k; R = depth(k); }
  if (!ks) return MFA_ERR_UNSUPPORTED;
  const ZfSmem L = zf_layout(prm.mode, CP, ks, R);
  CUtensorMap map;
  if (!make_row_map(&map, prm.x, prm.nslots, prm.slot_stride, ks * 32)) return MFA_ERR_UNSUPPORTED;
  cudaError_t e;
  switch (CP) {
    case 4: e = launch_zf<4>(ctx, prm, L, map, stream); break;
    case 8: e = launch_zf<8>(ctx, prm, L, map, stream); break;
    case 12: e = launch_zf<12>(ctx, prm, L, map, stream); break;
    case 16: e = launch_zf<16>(ctx, prm, L, map, stream); break;
    default: return MFA_ERR_UNSUPPORTED;
  }
  return e == cudaSuccess ? MFA_OK : MFA_ERR_CUDA;
}

int contract3(mfa_ctx* ctx, ContractParams prm, cudaStream_t stream) {
  {
    const int rc = contract3_zfirst(ctx, prm, stream);
    if (rc != MFA_ERR_UNSUPPORTED) return rc;
  }
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
