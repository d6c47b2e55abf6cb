// Process-wide cache of device and pinned host blocks.
//
// A factorization allocates its working pools, its upload arena, the W store
// and the operator in blocks of tens to hundreds of megabytes; cudaMalloc and
// cudaFree of such blocks cost a large part of a millisecond each, and a
// factorization of the same problem asks for the same sizes again.  Freed
// blocks are kept here (per device, by rounded size) and handed out again;
// spaqr_release_cached_memory() returns them to the driver.
//
// A block is returned to the cache only after cudaDeviceSynchronize() -- the
// guarantee cudaFree gives: no kernel still in flight can touch a block that
// the cache hands out again.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "internal.h"

namespace spaqr {

namespace {

struct Cache {
  std::mutex mu;
  // (device, rounded bytes) -> free blocks; device -1 for pinned host blocks
  std::multimap<std::pair<int, size_t>, void*> free_;
  std::unordered_map<void*, std::pair<int, size_t>> live_;
  size_t cached = 0;
};

Cache& cache() {
  static Cache* c = new Cache();  // never destroyed: blocks may be freed during process exit
  return *c;
}

// sizes are rounded so that repeated requests of nearly the same size meet:
// powers of two up to 1 MiB, multiples of 2 MiB above
size_t rounded(size_t bytes) {
  if (bytes <= 4096) return 4096;
  if (bytes <= (size_t(1) << 20)) {
    size_t s = 4096;
    while (s < bytes) s <<= 1;
    return s;
  }
  const size_t g = size_t(2) << 20;
  return (bytes + g - 1) / g * g;
}

// a cached block of at least `size` bytes and at most 5/4 of it, or nullptr
void* take(Cache& c, int dev, size_t size) {
  auto it = c.free_.lower_bound({dev, size});
  if (it == c.free_.end() || it->first.first != dev || it->first.second > size + size / 4) return nullptr;
  void* p = it->second;
  const size_t s = it->first.second;
  c.free_.erase(it);
  c.cached -= s;
  c.live_[p] = {dev, s};
  return p;
}

void drop_all(Cache& c, int dev_only, bool all_devices) {
  for (auto it = c.free_.begin(); it != c.free_.end();) {
    const int dev = it->first.first;
    if (!all_devices && dev != dev_only) {
      ++it;
      continue;
    }
    if (dev < 0)
      cudaFreeHost(it->second);
    else
      cudaFree(it->second);
    c.cached -= it->first.second;
    it = c.free_.erase(it);
  }
}

}  // namespace

cudaError_t dmalloc(void** p, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t size = rounded(bytes);
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  if ((*p = take(c, dev, size))) return cudaSuccess;
  e = cudaMalloc(p, size);
  if (e == cudaErrorMemoryAllocation) {  // give the cached blocks of this device back and retry
    cudaGetLastError();
    drop_all(c, dev, false);
    e = cudaMalloc(p, size);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c.live_[*p] = {dev, size};
  return cudaSuccess;
}

void dfree(void* p) {
  if (!p) return;
  Cache& c = cache();
  std::pair<int, size_t> key;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.live_.find(p);
    if (it == c.live_.end()) {  // not from dmalloc
      cudaFree(p);
      return;
    }
    key = it->second;
    c.live_.erase(it);
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (key.first != cur) cudaSetDevice(key.first);
  const bool idle = cudaDeviceSynchronize() == cudaSuccess;
  if (key.first != cur) cudaSetDevice(cur);
  if (!idle) {  // a failed context: hand the block back to the driver
    cudaGetLastError();
    cudaFree(p);
    return;
  }
  std::lock_guard<std::mutex> lk(c.mu);
  c.free_.insert({key, p});
  c.cached += key.second;
}

cudaError_t hmalloc(void** p, size_t bytes) {
  const size_t size = rounded(bytes);
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  if ((*p = take(c, -1, size))) return cudaSuccess;
  const cudaError_t e = cudaMallocHost(p, size);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  c.live_[*p] = {-1, size};
  return cudaSuccess;
}

void hfree(void* p) {
  if (!p) return;
  Cache& c = cache();
  std::pair<int, size_t> key;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.live_.find(p);
    if (it == c.live_.end()) {
      cudaFreeHost(p);
      return;
    }
    key = it->second;
    c.live_.erase(it);
  }
  // the guarantee cudaFreeHost gives: no copy still in flight reads the block
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(p);
    return;
  }
  std::lock_guard<std::mutex> lk(c.mu);
  c.free_.insert({key, p});
  c.cached += key.second;
}

void release_cached_memory() {
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  cudaDeviceSynchronize();
  drop_all(c, 0, true);
}

size_t cached_bytes() {
  Cache& c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  return c.cached;
}

}  // namespace spaqr
