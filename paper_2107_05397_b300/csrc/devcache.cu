// Process-wide cache of large device blocks.
//
// A context's work buffers at 50,000 samples are tens of GB (the 20 GB
// output stage, 18 GB of counts, 15 GB of partial sums, ...); freeing them
// takes tens of milliseconds and allocating them again a few more, per
// context.  Blocks of at least
// kMinCached bytes that a context frees are kept here instead, per device,
// and a later allocation of about the same size takes one back.  The cache
// holds at most a cap of bytes per device (default: half the device's
// memory; unifrac_set_memory_cache), unifrac_release_cached_memory frees
// everything it holds, and an allocation that fails releases the device's
// cache and tries once more.
//
// Callers hand a block back only when no device work can still use it (the
// contexts synchronise the device first), so a block taken from the cache is
// idle.  Its contents are whatever the last user left: nothing in the
// library reads device memory it did not write.
#include <algorithm>
#include <map>
#include <mutex>
#include <unordered_map>

#include "ufb_internal.cuh"

namespace ufb {
namespace {

constexpr size_t kMinCached = size_t(64) << 20;  // smaller blocks go straight to the driver
constexpr size_t kGranule = size_t(2) << 20;

struct DeviceCache {
  std::multimap<size_t, void *> free_blocks;  // size -> block
  size_t cached = 0;                          // bytes in free_blocks
  int64_t cap = -1;                           // -1: not yet set (half the device's memory)
};

std::mutex g_mu;
std::map<int, DeviceCache> g_dev;
std::unordered_map<void *, size_t> g_live;  // blocks handed out, with their real size

size_t round_up(size_t bytes) { return (bytes + kGranule - 1) / kGranule * kGranule; }

DeviceCache &cache_of(int dev) {
  DeviceCache &c = g_dev[dev];
  if (c.cap < 0) {
    size_t free_b = 0, total_b = 0;
    c.cap = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess ? (int64_t)(total_b / 2) : 0;
  }
  return c;
}

void release_locked(DeviceCache &c) {
  for (auto &kv : c.free_blocks) cudaFree(kv.second);
  c.free_blocks.clear();
  c.cached = 0;
}

}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes < kMinCached) return dev_malloc_retry(p, bytes);
  const size_t want = round_up(bytes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceCache &c = cache_of(dev);
    auto it = c.free_blocks.lower_bound(want);
    if (it != c.free_blocks.end() && it->first <= want + want / 8) {
      *p = it->second;
      g_live[*p] = it->first;
      c.cached -= it->first;
      c.free_blocks.erase(it);
      return cudaSuccess;
    }
  }
  e = cudaMalloc(p, want);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_mu);
      release_locked(cache_of(dev));
    }
    e = cudaMalloc(p, want);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_live[*p] = want;
  return cudaSuccess;
}

cudaError_t dev_malloc_retry(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    int dev = 0;
    cudaGetDevice(&dev);
    {
      std::lock_guard<std::mutex> lk(g_mu);
      release_locked(cache_of(dev));
    }
    e = cudaMalloc(p, bytes);
  }
  return e;
}

void dev_free(void *p) {
  if (!p) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) {  // a small block, straight from the driver
    cudaFree(p);
    return;
  }
  const size_t size = it->second;
  g_live.erase(it);
  DeviceCache &c = cache_of(dev);
  // over the cap: the largest cached blocks go first (they cost most to keep)
  while (!c.free_blocks.empty() && (int64_t)(c.cached + size) > c.cap) {
    auto last = std::prev(c.free_blocks.end());
    cudaFree(last->second);
    c.cached -= last->first;
    c.free_blocks.erase(last);
  }
  if ((int64_t)(c.cached + size) > c.cap) {
    cudaFree(p);
    return;
  }
  c.free_blocks.emplace(size, p);
  c.cached += size;
}

}  // namespace ufb

extern "C" {

int unifrac_release_cached_memory(int device) {
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return UNIFRAC_E_CUDA;
  std::lock_guard<std::mutex> lk(ufb::g_mu);
  for (auto &kv : ufb::g_dev) {
    if (device >= 0 && kv.first != device) continue;
    if (kv.first != prev && cudaSetDevice(kv.first) != cudaSuccess) continue;
    ufb::release_locked(kv.second);
  }
  cudaSetDevice(prev);
  return UNIFRAC_OK;
}

int unifrac_set_memory_cache(int device, int64_t max_bytes) {
  if (max_bytes < -1) return UNIFRAC_E_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return UNIFRAC_E_CUDA;
  if (device < 0) device = prev;
  if (device != prev && cudaSetDevice(device) != cudaSuccess) return UNIFRAC_E_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(ufb::g_mu);
    ufb::DeviceCache &c = ufb::g_dev[device];
    if (max_bytes == -1) {
      c.cap = -1;
      ufb::cache_of(device);  // back to half the device's memory
    } else {
      c.cap = max_bytes;
    }
    while (!c.free_blocks.empty() && (int64_t)c.cached > c.cap) {
      auto last = std::prev(c.free_blocks.end());
      cudaFree(last->second);
      c.cached -= last->first;
      c.free_blocks.erase(last);
    }
  }
  if (device != prev) cudaSetDevice(prev);
  return UNIFRAC_OK;
}

int unifrac_cached_memory(int device, int64_t *bytes) {
  if (!bytes) return UNIFRAC_E_INVALID_ARG;
  int prev = 0;
  if (device < 0) {
    if (cudaGetDevice(&prev) != cudaSuccess) return UNIFRAC_E_CUDA;
    device = prev;
  }
  std::lock_guard<std::mutex> lk(ufb::g_mu);
  auto it = ufb::g_dev.find(device);
  *bytes = it == ufb::g_dev.end() ? 0 : (int64_t)it->second.cached;
  return UNIFRAC_OK;
}

}  // extern "C"
