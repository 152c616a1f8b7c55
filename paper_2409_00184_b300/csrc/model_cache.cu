// Out-of-core micro-model storage and caching (Sec. 4.3: Algorithm 2 caching, Algorithm 3 prefetching).
//
// Storage: one file of micro-models, each in the byte layout whose size is Eq. 2 (degree byte, the
// first NCP + degree knots per axis, NCP^3 control points), behind a small header and an index.
// Cache: an LRU set of models held in host memory (page-locked when asked), loaded from the file by
// positioned reads; a visible list is then packed into descriptors, knots and control points and
// copied to the device in three transfers. A prefetch thread loads the models predicted for the next
// point of view while the current one renders, until it is told that rendering is done.
#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "mfa.h"

namespace {

constexpr char kMagic[8] = {'M', 'F', 'A', 'P', 'A', 'C', 'K', '1'};

struct IndexEntry {
  uint64_t offset;
  uint32_t ncp;
  uint32_t degree;
};
static_assert(sizeof(IndexEntry) == 16, "index entry layout");

int64_t model_bytes_eq2(int64_t ncp, int64_t degree) { return 1 + ((ncp + degree) * 3 + ncp * ncp * ncp) * 4; }

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

bool read_at(int fd, void* dst, size_t bytes, uint64_t offset) {
  unsigned char* p = static_cast<unsigned char*>(dst);
  while (bytes > 0) {
    const ssize_t r = pread(fd, p, bytes, (off_t)offset);
    if (r <= 0) return false;
    p += r;
    bytes -= (size_t)r;
    offset += (uint64_t)r;
  }
  return true;
}

}  // namespace

struct mfa_model_cache {
  int fd = -1;
  std::vector<IndexEntry> index;
  int32_t capacity = 0;
  int64_t slot_bytes = 0;  // largest model in the store
  bool pinned = false;
  unsigned char* slots = nullptr;  // capacity x slot_bytes raw models
  std::list<int32_t> lru;          // front = most recently used
  struct Entry {
    std::list<int32_t>::iterator it;
    int32_t slot;
  };
  std::unordered_map<int32_t, Entry> map;
  std::vector<int32_t> free_slots;
  std::mutex mu;
  // upload staging
  std::vector<unsigned char> stage_pageable;
  unsigned char* stage = nullptr;
  size_t stage_bytes = 0;
  cudaEvent_t copied = nullptr;
  bool copy_pending = false;
  // prefetch
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<int64_t> pf_loaded{0}, pf_bytes{0};

  // Loads model `id` into the cache (caller holds mu, id not cached); false on a read error.
  bool load(int32_t id, int64_t* bytes_read) {
    int32_t slot;
    if (!free_slots.empty()) {
      slot = free_slots.back();
      free_slots.pop_back();
    } else {
      const int32_t victim = lru.back();
      lru.pop_back();
      slot = map[victim].slot;
      map.erase(victim);
    }
    const IndexEntry& e = index[id];
    const int64_t bytes = model_bytes_eq2(e.ncp, e.degree);
    if (!read_at(fd, slots + (int64_t)slot * slot_bytes, (size_t)bytes, e.offset)) {
      free_slots.push_back(slot);
      return false;
    }
    lru.push_front(id);
    map[id] = Entry{lru.begin(), slot};
    if (bytes_read) *bytes_read += bytes;
    return true;
  }
};

extern "C" {

int mfa_store_write(const char* path, const mfa_block_desc* h_desc, int32_t nblocks, const float* h_knots,
                    int64_t knots_len, const float* h_cps, int64_t cps_len) {
  if (!path || nblocks < 0 || (nblocks > 0 && (!h_desc || !h_knots || !h_cps))) return MFA_ERR_INVALID_ARG;
  std::vector<IndexEntry> index((size_t)nblocks);
  uint64_t off = sizeof(kMagic) + 8 + (uint64_t)nblocks * sizeof(IndexEntry);
  for (int32_t b = 0; b < nblocks; ++b) {
    const mfa_block_desc& d = h_desc[b];
    const int32_t C = d.ncp[0], p = d.degree[0];
    for (int a = 0; a < 3; ++a) {
      if (d.ncp[a] != C || d.degree[a] != p) return MFA_ERR_INVALID_ARG;  // the layout is isotropic
      if (d.knot_off[a] < 0 || d.knot_off[a] + C + p + 1 > knots_len) return MFA_ERR_INVALID_ARG;
    }
    if (p < 1 || p > MFA_MAX_DEGREE || C < p + 1 || C > MFA_MAX_NCP) return MFA_ERR_INVALID_ARG;
    if (d.cp_off < 0 || d.cp_off + (int64_t)C * C * C > cps_len) return MFA_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)  // clamped end: the implied last knot equals the one before it
      if (h_knots[d.knot_off[a] + C + p] != h_knots[d.knot_off[a] + C + p - 1]) return MFA_ERR_INVALID_ARG;
    index[b] = IndexEntry{off, (uint32_t)C, (uint32_t)p};
    off += (uint64_t)model_bytes_eq2(C, p);
  }
  FILE* f = std::fopen(path, "wb");
  if (!f) return MFA_ERR_IO;
  bool ok = std::fwrite(kMagic, 1, sizeof(kMagic), f) == sizeof(kMagic);
  const uint32_t head[2] = {(uint32_t)nblocks, 0u};
  ok = ok && std::fwrite(head, sizeof(uint32_t), 2, f) == 2;
  ok = ok && (nblocks == 0 || std::fwrite(index.data(), sizeof(IndexEntry), index.size(), f) == index.size());
  std::vector<unsigned char> buf;
  for (int32_t b = 0; ok && b < nblocks; ++b) {
    const mfa_block_desc& d = h_desc[b];
    const int32_t C = d.ncp[0], p = d.degree[0];
    buf.assign((size_t)model_bytes_eq2(C, p), 0);
    buf[0] = (unsigned char)p;
    size_t o = 1;
    for (int a = 0; a < 3; ++a) {
      std::memcpy(buf.data() + o, h_knots + d.knot_off[a], sizeof(float) * (size_t)(C + p));
      o += sizeof(float) * (size_t)(C + p);
    }
    std::memcpy(buf.data() + o, h_cps + d.cp_off, sizeof(float) * (size_t)C * C * C);
    ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MFA_OK : MFA_ERR_IO;
}

int mfa_cache_create(mfa_model_cache** out, const char* path, int32_t capacity, int32_t pinned) {
  if (!out || !path || capacity < 1) return MFA_ERR_INVALID_ARG;
  *out = nullptr;
  mfa_model_cache* c = new (std::nothrow) mfa_model_cache();
  if (!c) return MFA_ERR_CAPACITY;
  c->fd = open(path, O_RDONLY);
  char magic[8];
  uint32_t head[2];
  if (c->fd < 0 || !read_at(c->fd, magic, 8, 0) || std::memcmp(magic, kMagic, 8) != 0 ||
      !read_at(c->fd, head, 8, 8)) {
    mfa_cache_destroy(c);
    return MFA_ERR_IO;
  }
  c->index.resize(head[0]);
  if (head[0] > 0 && !read_at(c->fd, c->index.data(), sizeof(IndexEntry) * head[0], 16)) {
    mfa_cache_destroy(c);
    return MFA_ERR_IO;
  }
  int64_t largest = 1;
  for (const IndexEntry& e : c->index) {
    if (e.degree < 1 || e.degree > MFA_MAX_DEGREE || e.ncp < e.degree + 1 || e.ncp > MFA_MAX_NCP) {
      mfa_cache_destroy(c);
      return MFA_ERR_IO;
    }
    largest = std::max(largest, model_bytes_eq2(e.ncp, e.degree));
  }
  c->capacity = capacity;
  c->slot_bytes = (largest + 15) & ~int64_t(15);
  c->pinned = pinned != 0;
  const size_t bytes = (size_t)capacity * (size_t)c->slot_bytes;
  if (c->pinned) {
    if (cudaHostAlloc(reinterpret_cast<void**>(&c->slots), bytes, cudaHostAllocDefault) != cudaSuccess) {
      c->slots = nullptr;
      mfa_cache_destroy(c);
      return MFA_ERR_CUDA;
    }
  } else {
    c->slots = static_cast<unsigned char*>(std::malloc(bytes));
    if (!c->slots) {
      mfa_cache_destroy(c);
      return MFA_ERR_CAPACITY;
    }
  }
  c->free_slots.reserve((size_t)capacity);
  for (int32_t s = capacity - 1; s >= 0; --s) c->free_slots.push_back(s);
  *out = c;
  return MFA_OK;
}

void mfa_cache_destroy(mfa_model_cache* c) {
  if (!c) return;
  c->stop = true;
  if (c->worker.joinable()) c->worker.join();
  if (c->copied) {
    cudaEventSynchronize(c->copied);
    cudaEventDestroy(c->copied);
  }
  if (c->slots) {
    if (c->pinned) cudaFreeHost(c->slots);
    else std::free(c->slots);
  }
  if (c->stage && c->pinned) cudaFreeHost(c->stage);
  if (c->fd >= 0) close(c->fd);
  delete c;
}

int mfa_cache_info(const mfa_model_cache* c, int32_t* count, int32_t* max_ncp, int32_t* max_degree) {
  if (!c) return MFA_ERR_INVALID_ARG;
  int32_t mc = 0, md = 0;
  for (const IndexEntry& e : c->index) {
    mc = std::max(mc, (int32_t)e.ncp);
    md = std::max(md, (int32_t)e.degree);
  }
  if (count) *count = (int32_t)c->index.size();
  if (max_ncp) *max_ncp = mc;
  if (max_degree) *max_degree = md;
  return MFA_OK;
}

int mfa_cache_lookup(mfa_model_cache* c, const int32_t* h_ids, int32_t n, int64_t* h_stats) {
  if (!c || n < 0 || (n > 0 && !h_ids) || n > c->capacity) return MFA_ERR_INVALID_ARG;
  if (c->worker.joinable()) return MFA_ERR_INVALID_ARG;  // prefetching: stop it first
  for (int32_t i = 0; i < n; ++i)
    if (h_ids[i] < 0 || h_ids[i] >= (int32_t)c->index.size()) return MFA_ERR_INVALID_ARG;
  const int64_t t0 = now_ns();
  int64_t hits = 0, misses = 0, bytes = 0;
  std::lock_guard<std::mutex> lock(c->mu);
  for (int32_t i = 0; i < n; ++i) {
    const int32_t id = h_ids[i];
    auto it = c->map.find(id);
    if (it != c->map.end()) {  // hit: most recently used
      c->lru.splice(c->lru.begin(), c->lru, it->second.it);
      ++hits;
    } else {
      if (!c->load(id, &bytes)) return MFA_ERR_IO;
      ++misses;
    }
  }
  if (h_stats) {
    h_stats[0] = hits;
    h_stats[1] = misses;
    h_stats[2] = bytes;
    h_stats[3] = now_ns() - t0;
  }
  return MFA_OK;
}

int mfa_cache_upload(mfa_model_cache* c, const int32_t* h_ids, int32_t n, int32_t nsamp, mfa_block_desc* d_desc,
                     float* d_knots, int64_t knots_cap, float* d_cps, int64_t cps_cap, int64_t* h_lens,
                     mfa_bounds* h_bounds, void* stream) {
  if (!c || n < 0 || (n > 0 && (!h_ids || !d_desc || !d_knots || !d_cps)) || !h_lens || !h_bounds)
    return MFA_ERR_INVALID_ARG;
  if (nsamp < 2 || nsamp > MFA_MAX_NSAMP || c->worker.joinable()) return MFA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(c->mu);
  int64_t nk = 0, ncp = 0;
  int32_t maxC = 2, maxP = 1;
  for (int32_t i = 0; i < n; ++i) {
    if (h_ids[i] < 0 || h_ids[i] >= (int32_t)c->index.size() || !c->map.count(h_ids[i])) return MFA_ERR_INVALID_ARG;
    const IndexEntry& e = c->index[h_ids[i]];
    nk += 3 * (int64_t)(e.ncp + e.degree + 1);
    ncp += (int64_t)e.ncp * e.ncp * e.ncp;
    maxC = std::max(maxC, (int32_t)e.ncp);
    maxP = std::max(maxP, (int32_t)e.degree);
  }
  if (nk > knots_cap || ncp > cps_cap) return MFA_ERR_CAPACITY;
  const size_t desc_bytes = sizeof(mfa_block_desc) * (size_t)n;
  const size_t need = desc_bytes + sizeof(float) * (size_t)(nk + ncp) + 64;
  if (c->copy_pending) {  // the previous upload's copies still read the staging
    if (cudaEventSynchronize(c->copied) != cudaSuccess) return MFA_ERR_CUDA;
    c->copy_pending = false;
  }
  if (need > c->stage_bytes) {
    if (c->pinned) {
      if (c->stage) cudaFreeHost(c->stage);
      c->stage = nullptr;
      if (cudaHostAlloc(reinterpret_cast<void**>(&c->stage), need, cudaHostAllocDefault) != cudaSuccess) {
        c->stage = nullptr;
        c->stage_bytes = 0;
        return MFA_ERR_CUDA;
      }
    } else {
      c->stage_pageable.resize(need);
      c->stage = c->stage_pageable.data();
    }
    c->stage_bytes = need;
  }
  mfa_block_desc* desc = reinterpret_cast<mfa_block_desc*>(c->stage);
  float* knots = reinterpret_cast<float*>(c->stage + desc_bytes);
  float* cps = knots + nk;
  int64_t ko = 0, co = 0;
  for (int32_t i = 0; i < n; ++i) {
    const IndexEntry& e = c->index[h_ids[i]];
    const int32_t C = (int32_t)e.ncp, p = (int32_t)e.degree;
    const unsigned char* m = c->slots + (int64_t)c->map[h_ids[i]].slot * c->slot_bytes;
    mfa_block_desc d;
    std::memset(&d, 0, sizeof(d));
    size_t o = 1;
    for (int a = 0; a < 3; ++a) {
      d.degree[a] = p;
      d.ncp[a] = C;
      d.nsamp[a] = nsamp;
      d.knot_off[a] = ko;
      std::memcpy(knots + ko, m + o, sizeof(float) * (size_t)(C + p));
      knots[ko + C + p] = knots[ko + C + p - 1];  // the implied clamped end
      ko += C + p + 1;
      o += sizeof(float) * (size_t)(C + p);
    }
    d.slot = i;
    d.cp_off = co;
    std::memcpy(cps + co, m + o, sizeof(float) * (size_t)C * C * C);
    co += (int64_t)C * C * C;
    desc[i] = d;
  }
  h_lens[0] = nk;
  h_lens[1] = ncp;
  h_bounds->max_degree = maxP;
  h_bounds->max_ncp = maxC;
  h_bounds->max_nsamp = nsamp;
  if (n == 0) return MFA_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(d_desc, desc, desc_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_knots, knots, sizeof(float) * (size_t)nk, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_cps, cps, sizeof(float) * (size_t)ncp, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MFA_ERR_CUDA;
  if (!c->copied && cudaEventCreateWithFlags(&c->copied, cudaEventDisableTiming) != cudaSuccess) {
    c->copied = nullptr;
    return MFA_ERR_CUDA;
  }
  if (cudaEventRecord(c->copied, s) != cudaSuccess) return MFA_ERR_CUDA;
  c->copy_pending = true;
  return MFA_OK;
}

int mfa_cache_prefetch_start(mfa_model_cache* c, const int32_t* h_ids, int32_t n) {
  if (!c || n < 0 || (n > 0 && !h_ids) || c->worker.joinable()) return MFA_ERR_INVALID_ARG;
  std::vector<int32_t> ids;
  ids.reserve((size_t)n);
  for (int32_t i = 0; i < n; ++i)
    if (h_ids[i] >= 0 && h_ids[i] < (int32_t)c->index.size()) ids.push_back(h_ids[i]);
  c->stop = false;
  c->pf_loaded = 0;
  c->pf_bytes = 0;
  c->worker = std::thread([c, ids]() {
    for (int32_t id : ids) {
      if (c->stop.load(std::memory_order_relaxed)) break;  // rendering finished: stop prefetching
      std::lock_guard<std::mutex> lock(c->mu);
      if (c->map.count(id)) continue;
      int64_t bytes = 0;
      if (!c->load(id, &bytes)) break;
      c->pf_loaded += 1;
      c->pf_bytes += bytes;
    }
  });
  return MFA_OK;
}

int mfa_cache_prefetch_stop(mfa_model_cache* c, int64_t* h_stats) {
  if (!c) return MFA_ERR_INVALID_ARG;
  c->stop = true;
  if (c->worker.joinable()) c->worker.join();
  if (h_stats) {
    h_stats[0] = c->pf_loaded;
    h_stats[1] = c->pf_bytes;
  }
  return MFA_OK;
}

}  // extern "C"
