// arena.cpp — host arenas: pinned, mapped host memory handed out block by
// block (Algorithm 1's allocation requests served from one buffer).  A tree
// built in an arena needs no marshal: its blocks already sit in memory the
// GPU can read and write, so the deep copy and the copy back move them with
// the move kernel directly, whatever their size.
#include <algorithm>
#include <mutex>
#include <vector>

#include "internal.hpp"

struct dc_host_arena_s {
  uint8_t* base = nullptr;
  uint8_t* dev = nullptr;
  uint64_t bytes = 0, used = 0;
  std::mutex m;
};

namespace {
std::mutex g_mu;
std::vector<dc_host_arena_s*> g_arenas;
}  // namespace

bool dc::in_host_arena(const void* host, uint64_t bytes, uint64_t* dev) {
  const uint8_t* h = static_cast<const uint8_t*>(host);
  std::lock_guard<std::mutex> g(g_mu);
  for (auto* a : g_arenas)
    if (h >= a->base && bytes <= a->bytes && h - a->base <= (ptrdiff_t)(a->bytes - bytes)) {
      if (dev) *dev = (uint64_t)(uintptr_t)(a->dev + (h - a->base));
      return true;
    }
  return false;
}

extern "C" {

dc_status dc_host_arena_create(uint64_t bytes, dc_host_arena_t* out) {
  if (!out || bytes == 0) return dc::fail(DC_EINVAL, "bad argument");
  *out = nullptr;
  auto* a = new (std::nothrow) dc_host_arena_s;
  if (!a) return dc::fail(DC_ENOMEM, "out of host memory");
  a->bytes = dc::round_up(bytes, 256);
  cudaError_t e = dc::host_alloc((void**)&a->base, a->bytes, cudaHostAllocMapped);
  if (e != cudaSuccess) {
    delete a;
    return dc::fail(DC_ENOMEM, "host arena of %llu bytes: %s", (unsigned long long)bytes, cudaGetErrorString(e));
  }
  if ((e = cudaHostGetDevicePointer((void**)&a->dev, a->base, 0)) != cudaSuccess) {
    cudaFreeHost(a->base);
    delete a;
    return dc::cuda_fail(e, "cudaHostGetDevicePointer");
  }
  {
    std::lock_guard<std::mutex> g(g_mu);
    g_arenas.push_back(a);
  }
  *out = a;
  return DC_OK;
}

void* dc_host_arena_alloc(dc_host_arena_t a, uint64_t bytes, uint64_t align) {
  if (!a) return nullptr;
  if (align < 16) align = 16;
  if (align & (align - 1)) return nullptr;
  std::lock_guard<std::mutex> g(a->m);
  const uint64_t at = dc::round_up(a->used, align);
  if (at > a->bytes || bytes > a->bytes - at) return nullptr;
  a->used = at + std::max<uint64_t>(bytes, 1);
  return a->base + at;
}

dc_status dc_host_arena_used(dc_host_arena_t a, uint64_t* used) {
  if (!a || !used) return dc::fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(a->m);
  *used = a->used;
  return DC_OK;
}

dc_status dc_host_arena_reset(dc_host_arena_t a) {
  if (!a) return dc::fail(DC_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(a->m);
  a->used = 0;
  return DC_OK;
}

dc_status dc_host_arena_destroy(dc_host_arena_t a) {
  if (!a) return DC_OK;
  {
    std::lock_guard<std::mutex> g(g_mu);
    g_arenas.erase(std::remove(g_arenas.begin(), g_arenas.end(), a), g_arenas.end());
  }
  cudaFreeHost(a->base);
  delete a;
  return DC_OK;
}

}  // extern "C"
