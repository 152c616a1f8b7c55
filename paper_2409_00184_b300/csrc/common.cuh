// Internal definitions shared by the library's CUDA sources (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mfa.h"

struct mfa_tiling_entry {
  mfa_bounds key;
  mfa_decode_tiling tiling;
};

struct mfa_ctx {
  int device = 0;
  int num_sms = 0;
  uint32_t* d_status = nullptr;   // device status word (MFA_DEV_* bits)
  uint32_t* d_counters = nullptr; // work-queue counters, one per concurrent launch kind
  unsigned long long* d_stats = nullptr;  // device statistics (MFA_STAT_*)
  uint32_t* d_touched = nullptr;  // sector bitmap of MFA_RAYCAST_COUNT_SECTORS, grown on demand
  int64_t touched_words = 0;
  int64_t launches = 0;           // kernels enqueued through this context
  int ntilings = 0;
  mfa_tiling_entry tilings[64];   // decode tile shapes keyed by batch bounds (autotuner)
};

namespace mfa {

enum Counter { kDecodeQueue = 0, kAdjointQueue = 1, kEncodeQueue = 2, kRaycastQueue = 3, kNumCounters = 4 };

// Validated per-block geometry, decoded from an mfa_block_desc inside a kernel.
struct BlockGeom {
  int p[3], C[3], n[3];
  int slot;
  int64_t knot_off[3];
  int64_t cp_off;
};

// Reads and checks one descriptor against the launch bounds and array lengths (the slot field
// only when check_slot). Returns 0 or the MFA_DEV_* bit that failed.
__device__ __forceinline__ uint32_t load_desc(const mfa_block_desc* d, const mfa_bounds& bd,
                                              int64_t knots_len, int64_t cps_len,
                                              int64_t nslots, int64_t slot_stride,
                                              BlockGeom& g, bool check_slot = true) {
  for (int a = 0; a < 3; ++a) {
    g.p[a] = d->degree[a];
    g.C[a] = d->ncp[a];
    g.n[a] = d->nsamp[a];
    g.knot_off[a] = d->knot_off[a];
  }
  g.slot = d->slot;
  g.cp_off = d->cp_off;
  int64_t vox = 1, ncps = 1;
  for (int a = 0; a < 3; ++a) {
    if (g.p[a] < 1 || g.p[a] > bd.max_degree || g.C[a] < g.p[a] + 1 || g.C[a] > bd.max_ncp ||
        g.n[a] < 2 || g.n[a] > bd.max_nsamp)
      return MFA_DEV_BAD_DESC;
    if (g.knot_off[a] < 0 || g.knot_off[a] + g.C[a] + g.p[a] + 1 > knots_len) return MFA_DEV_BAD_RANGE;
    vox *= g.n[a];
    ncps *= g.C[a];
  }
  if (g.cp_off < 0 || g.cp_off + ncps > cps_len) return MFA_DEV_BAD_RANGE;
  if (vox > slot_stride) return MFA_DEV_BAD_RANGE;
  if (check_slot && (g.slot < 0 || g.slot >= nslots)) return MFA_DEV_BAD_RANGE;
  return 0;
}

// Knot vector sanity for one axis (non-decreasing, non-empty parameter domain).
__device__ __forceinline__ bool knots_ok(const float* t, int p, int C) {
  for (int i = 0; i + 1 < C + p + 1; ++i)
    if (!(t[i] <= t[i + 1])) return false;
  return t[p] < t[C];
}

// Index of voxel (x, y, z) of an nx x ny x nz cache brick in the cube layout (MFA_DECODE_CUBES; even
// n per axis): 2x2x2-voxel cubes in [z/2][y/2][x/2] order, the 8 voxels of a cube in [z&1][y&1][x&1]
// order, so one cube of float4 voxels fills one 128-byte line.
__device__ __forceinline__ int cube_index(int x, int y, int z, int nx, int ny) {
  return ((((z >> 1) * (ny >> 1) + (y >> 1)) * (nx >> 1) + (x >> 1)) << 3) | ((z & 1) << 2) | ((y & 1) << 1) | (x & 1);
}

// Row pitch of a brick of n voxels per row in the apron layout (MFA_DECODE_APRON): n + 1 voxels rounded up
// to even, so that rows of float4 voxels start on 32-byte sectors (for an even slot stride) and the apron
// column x = n with its padding fills whole sectors.
__host__ __device__ constexpr int apron_pitch(int n) { return (n + 2) & ~1; }

// Sample parameter u_i = i/(n-1), rounded once (IEEE division).
__device__ __forceinline__ float sample_param(int i, int n) {
  return __fdiv_rn((float)i, (float)(n - 1));
}

// Span s with t_s <= u < t_{s+1}, p <= s <= C-1; u >= t_C gives the last span C-1.
template <typename T>
__device__ __forceinline__ int find_span(const T* t, int p, int C, T u) {
  if (u >= t[C]) return C - 1;
  int lo = p, hi = C;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (u < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// The p+1 nonzero B-spline basis values N_{s-p+r,p}(u) and derivatives, r = 0..p, at span s,
// by the triangular form of the Cox-de Boor recurrence (each degree built from the previous
// one with the left/right knot distances). Entries r > p are set to 0. PMAX >= p.
template <int PMAX, typename T>
__device__ __forceinline__ void basis_funs(const T* t, int p, int s, T u, T (&N)[PMAX + 1], T (&dN)[PMAX + 1]) {
  T left[PMAX + 1], right[PMAX + 1], cur[PMAX + 1], low[PMAX + 1];
#pragma unroll
  for (int r = 0; r <= PMAX; ++r) { cur[r] = T(0); low[r] = T(0); left[r] = T(0); right[r] = T(0); }
  cur[0] = T(1);
  if (p == 1) low[0] = T(1);
#pragma unroll
  for (int k = 1; k <= PMAX; ++k) {
    if (k <= p) {
      left[k] = u - t[s + 1 - k];
      right[k] = t[s + k] - u;
      T saved = T(0);
#pragma unroll
      for (int r = 0; r < k; ++r) {
        T den = right[r + 1] + left[k - r];
        T tmp = den != T(0) ? cur[r] / den : T(0);
        cur[r] = saved + right[r + 1] * tmp;
        saved = left[k - r] * tmp;
      }
      cur[k] = saved;
      if (k == p - 1) {
#pragma unroll
        for (int r = 0; r <= PMAX; ++r) low[r] = cur[r];
      }
    }
  }
  // low[r] = N_{s-p+1+r, p-1}(u), r = 0..p-1. N'_{i,p} = p (N_{i,p-1}/(t_{i+p}-t_i)
  //                                                   - N_{i+1,p-1}/(t_{i+p+1}-t_{i+1})).
#pragma unroll
  for (int r = 0; r <= PMAX; ++r) {
    N[r] = (r <= p) ? cur[r] : T(0);
    T d = T(0);
    if (r <= p) {
      const int i = s - p + r;
      if (r >= 1) {
        T den = t[i + p] - t[i];
        if (den != T(0)) d += low[r - 1] / den;
      }
      if (r <= p - 1) {
        T den = t[i + p + 1] - t[i + 1];
        if (den != T(0)) d -= low[r] / den;
      }
      d *= (T)p;
    }
    dN[r] = d;
  }
}

__device__ __forceinline__ void flag(uint32_t* status, uint32_t bits) {
  if (bits) atomicOr(status, bits);
}

}  // namespace mfa
