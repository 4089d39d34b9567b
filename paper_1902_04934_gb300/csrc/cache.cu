// Process-wide cache of the device and pinned host buffers that handles own.  A handle is made and
// destroyed per intrinsic point, and cudaMalloc / cudaFree / cudaMallocHost cost tens to hundreds of
// microseconds each, which adds up next to a few-millisecond marginalisation.  Freed buffers stay
// in the cache, keyed by device and size, and serve later requests of the same size (up to twice
// it); callers return a buffer only when no work in flight uses it.  The cache gives memory back to
// CUDA when an allocation fails for lack of memory, and on rift_release_cached_memory().
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <unordered_map>

#include "rift_device.cuh"
#include "rift_internal.h"

namespace {

struct Key {
  int device;
  size_t size;
  bool operator<(const Key &o) const { return device != o.device ? device < o.device : size < o.size; }
};

struct Cache {
  std::mutex mu;
  std::multimap<Key, void *> free_dev, free_host;
  std::unordered_map<void *, Key> live_dev, live_host;
  // requests served (device, pinned host) and the CUDA allocations they needed
  unsigned long long n_req_dev = 0, n_req_host = 0, n_malloc_dev = 0, n_malloc_host = 0;
};

Cache &cache() {
  static Cache *c = new Cache;   // never destroyed: buffers may be returned during process teardown
  return *c;
}

size_t rounded(size_t n) { return ((n ? n : 1) + 511) & ~size_t(511); }

// The smallest cached block of the device that holds k.size bytes (and not more than twice that);
// k becomes the block's own key.
void *take(std::multimap<Key, void *> &pool, Key &k) {
  auto it = pool.lower_bound(k);
  if (it == pool.end() || it->first.device != k.device || it->first.size > 2 * k.size) return nullptr;
  void *p = it->second;
  k = it->first;
  pool.erase(it);
  return p;
}

void release_locked(Cache &c) {
  for (auto &kv : c.free_dev) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first.device);
    cudaFree(kv.second);
    cudaSetDevice(cur);
  }
  c.free_dev.clear();
  for (auto &kv : c.free_host) cudaFreeHost(kv.second);
  c.free_host.clear();
}

cudaError_t alloc(void **p, size_t n, bool host) {
  *p = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  Key k{host ? -1 : dev, rounded(n)};
  (host ? c.n_req_host : c.n_req_dev) += 1;
  void *q = take(host ? c.free_host : c.free_dev, k);
  if (!q) {
    (host ? c.n_malloc_host : c.n_malloc_dev) += 1;
    e = host ? cudaMallocHost(&q, k.size) : cudaMalloc(&q, k.size);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();   // the failed call's error is not sticky; clear it before retrying
      release_locked(c);
      e = host ? cudaMallocHost(&q, k.size) : cudaMalloc(&q, k.size);
    }
    if (e != cudaSuccess) return e;
  }
  (host ? c.live_host : c.live_dev)[q] = k;
  *p = q;
  return cudaSuccess;
}

void give_back(void *p, bool host) {
  if (!p) return;
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  auto &live = host ? c.live_host : c.live_dev;
  auto it = live.find(p);
  if (it == live.end()) {   // not from the cache
    if (host) cudaFreeHost(p); else cudaFree(p);
    return;
  }
  (host ? c.free_host : c.free_dev).emplace(it->second, p);
  live.erase(it);
}

}  // namespace

cudaError_t cache_dev_alloc(void **p, size_t n) { return alloc(p, n, false); }
cudaError_t cache_host_alloc(void **p, size_t n) { return alloc(p, n, true); }
void cache_dev_free(void *p) { give_back(p, false); }
void cache_host_free(void *p) { give_back(p, true); }

extern "C" void rift_release_cached_memory(void) {
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  release_locked(c);
}

extern "C" void rift_cache_counters(unsigned long long out[4]) {
  if (!out) return;
  Cache &c = cache();
  std::lock_guard<std::mutex> lock(c.mu);
  out[0] = c.n_req_dev;
  out[1] = c.n_req_host;
  out[2] = c.n_malloc_dev;
  out[3] = c.n_malloc_host;
}
