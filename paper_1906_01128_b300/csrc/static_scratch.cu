// static_scratch.cu — dc_relocate_static: the relocation kernel run with its
// scratch (block records, struct-block offsets, tile offsets, control words)
// taken from one fixed array in device memory instead of from a buffer the
// caller sized and allocated.  Nothing here allocates: no cudaMalloc,
// cudaHostAlloc or cudaFree, and no allocating library call.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.hpp"

using namespace dc;

namespace {

constexpr uint64_t MAX_BLOCKS = DC_STATIC_MAX_BLOCKS;
constexpr uint64_t MAX_TILES = 64;  // tile words reserved; enough for any tile of >= 1024 blocks
static_assert(MAX_BLOCKS <= MAX_TILES * RELOC_TILE, "tile words cover every tile");
constexpr uint64_t al256(uint64_t x) { return (x + 255) / 256 * 256; }
// byte layout of the array
constexpr uint64_t OFF_REC = 0;                                   // 16 B per block
constexpr uint64_t OFF_SOFF = al256(OFF_REC + 16 * MAX_BLOCKS);   // 8 B per struct block
constexpr uint64_t OFF_STATUS = al256(OFF_SOFF + 8 * MAX_BLOCKS); // 8 B per tile: tile base offsets
constexpr uint64_t OFF_READY = al256(OFF_STATUS + 8 * MAX_TILES); // 4 B per tile (unused)
constexpr uint64_t OFF_CTRL = al256(OFF_READY + 4 * MAX_TILES);   // control words
constexpr uint64_t SCRATCH_BYTES = al256(OFF_CTRL + 4 * CTRL_WORDS);
static_assert(SCRATCH_BYTES == DC_STATIC_SCRATCH_BYTES, "dc.h states the array's size");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
uint8_t* g_addr[MAX_DEVICES];  // device address of g_scratch, per device ordinal
int g_sms[MAX_DEVICES];

// Look the array up once per device, with that device current.  In host code
// `g_scratch` names a host-side stand-in, never the device memory itself.
dc_status scratch_for(int dev, uint8_t** addr, int* sms) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* a = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&a, g_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_addr[dev] = static_cast<uint8_t*>(a);
    g_sms[dev] = n;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return DC_OK;
}

}  // namespace

extern "C" dc_status dc_relocate_static(dc_plan_t p, void* dev_data, uint64_t data_bytes, uint32_t* dev_status,
                                        dc_stream_t stream) {
  if (!p || !dev_data) return fail(DC_EINVAL, "NULL argument");
  if ((uintptr_t)dev_data % 16) return fail(DC_EINVAL, "device data region must be 16-byte aligned");
  if (data_bytes < p->data_bytes)
    return fail(DC_EINVAL, "device data region holds %llu bytes, the plan's is %llu", (unsigned long long)data_bytes,
                (unsigned long long)p->data_bytes);
  const uint64_t nb = p->blocks.size();
  if (nb > MAX_BLOCKS)
    return fail(DC_EBUDGET, "the plan has %llu blocks; dc_relocate_static handles at most %llu (use dc_relocate)",
                (unsigned long long)nb, (unsigned long long)MAX_BLOCKS);
  int dev = 0;
  DC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(DC_EINVAL, "device ordinal %d out of range", dev);
  uint8_t* s = nullptr;
  int sms = 0;
  dc_status st = scratch_for(dev, &s, &sms);
  if (st) return st;
  cudaStream_t cs = stream;
  // the array keeps the previous call's contents: the error word must start
  // at zero, and this plan's tables replace the last call's
  DC_CUDA(cudaMemsetAsync(s + OFF_CTRL, 0, SCRATCH_BYTES - OFF_CTRL, cs));
  DC_CUDA(cudaMemcpyAsync(s + OFF_REC, p->rec.data(), nb * sizeof(BlockRec), cudaMemcpyHostToDevice, cs));
  DC_CUDA(cudaMemcpyAsync(s + OFF_SOFF, p->struct_off.data(), p->struct_off.size() * 8, cudaMemcpyHostToDevice, cs));
  DC_CUDA(cudaMemcpyAsync(s + OFF_STATUS, p->tile_base.data(), p->tile_base.size() * 8, cudaMemcpyHostToDevice, cs));
  RelocArgs a;
  a.arena = static_cast<uint8_t*>(dev_data);
  a.data_bytes = p->data_bytes;
  a.rec = reinterpret_cast<const BlockRec*>(s + OFF_REC);
  a.hostp = nullptr;  // no slot check in this variant
  a.soff = reinterpret_cast<const uint64_t*>(s + OFF_SOFF);
  a.tile_base = reinterpret_cast<const uint64_t*>(s + OFF_STATUS);
  a.ctrl = reinterpret_cast<uint32_t*>(s + OFF_CTRL);
  a.nblocks = (uint32_t)nb;
  a.nstruct_blocks = (uint32_t)p->nstruct_blocks;
  a.ntiles = (uint32_t)((nb + RELOC_TILE - 1) / RELOC_TILE);
  a.verify = 0;
  DC_CUDA(launch_relocate(a, cs, sms));
  if (dev_status)
    DC_CUDA(cudaMemcpyAsync(dev_status, s + OFF_CTRL + CTRL_ERR * 4, 4, cudaMemcpyDeviceToDevice, cs));
  return DC_OK;
}
