// Per-device cache of released device blocks, keyed by exact size.  The cache
// holds at most DFJK_CACHE_BYTES (environment, default 96 GiB) per device;
// beyond that released blocks are freed.  An allocation that fails first
// empties the cache and retries.
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "pool.cuh"

namespace dfjk {

namespace {
struct DevCache {
  std::multimap<size_t, void *> blocks;
  size_t bytes = 0;
};
std::mutex g_mu;
std::map<int, DevCache> g_cache;

size_t cache_limit() {
  static size_t lim = [] {
    const char *s = std::getenv("DFJK_CACHE_BYTES");
    return s ? (size_t)std::strtoull(s, nullptr, 10) : ((size_t)96 << 30);
  }();
  return lim;
}

int current_device() {
  int d = 0;
  DFJK_CUDA_CHECK(cudaGetDevice(&d));
  return d;
}

void trim_locked(DevCache &c) {
  for (auto &kv : c.blocks) cudaFree(kv.second);
  c.blocks.clear();
  c.bytes = 0;
}
}  // namespace

void *pool_alloc(size_t bytes) {
  if (bytes == 0) return nullptr;
  const int dev = current_device();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DevCache &c = g_cache[dev];
    auto it = c.blocks.find(bytes);
    if (it != c.blocks.end()) {
      void *p = it->second;
      c.blocks.erase(it);
      c.bytes -= bytes;
      return p;
    }
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    {
      std::lock_guard<std::mutex> lk(g_mu);
      trim_locked(g_cache[dev]);
    }
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{DFJK_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
    }
  }
  return p;
}

void pool_free(void *p, size_t bytes) {
  if (!p) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaFree(p);
    return;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  DevCache &c = g_cache[dev];
  if (c.bytes + bytes > cache_limit()) {
    cudaFree(p);
    return;
  }
  c.blocks.emplace(bytes, p);
  c.bytes += bytes;
}

void pool_trim() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  trim_locked(g_cache[dev]);
}

size_t pool_cached_bytes() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_mu);
  return g_cache[dev].bytes;
}

}  // namespace dfjk

extern "C" int dfjk_trim_cache(void) {
  try {
    dfjk::pool_trim();
    return DFJK_OK;
  } catch (const dfjk::Error &e) {
    dfjk::set_error(e.msg);
    return e.code;
  }
}
