// static_scratch.cu — dc_relocate_static: the relocation kernel run with its
// scratch (relocation records, lane groups, tile table, control words) taken
// from one fixed array in device memory instead of from a buffer the caller
// sized and allocated.  Nothing here allocates: no cudaMalloc,
// cudaHostAlloc or cudaFree, and no allocating library call.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.hpp"

using namespace dc;

namespace {

constexpr uint64_t MAX_BLOCKS = DC_STATIC_MAX_BLOCKS;  // records: at most one per block
constexpr uint64_t MAX_SEGS = DC_STATIC_MAX_BLOCKS;    // a lane group holds at least one record
constexpr uint64_t MAX_TILES = DC_STATIC_MAX_TILES;    // relocation tiles that hold a pointer slot
constexpr uint64_t al256(uint64_t x) { return (x + 255) / 256 * 256; }
// byte layout of the array
constexpr uint64_t OFF_REC = 0;                                              // 8 B per record
constexpr uint64_t OFF_SEG = al256(OFF_REC + sizeof(RelocRec) * (MAX_BLOCKS + 2));  // 16 B per group + 1
constexpr uint64_t OFF_TILE = al256(OFF_SEG + sizeof(RelocSeg) * (MAX_SEGS + 1));  // 16 B per tile
constexpr uint64_t OFF_CTRL = al256(OFF_TILE + sizeof(RelocTile) * MAX_TILES);      // control words
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
  const uint64_t ntiles = p->rtiles.size(), nseg = p->rseg.size() - 1, nrec = p->rrec.size();
  if (ntiles > MAX_TILES)
    return fail(DC_EBUDGET, "the plan has pointer slots in %llu relocation tiles of %u bytes; dc_relocate_static "
                "handles at most %llu (use dc_relocate)", (unsigned long long)ntiles, RELOC_SPAN,
                (unsigned long long)MAX_TILES);
  if (nseg > MAX_SEGS || nrec > MAX_BLOCKS) return fail(DC_EINVAL, "internal: relocation tables exceed the array");
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
  if (nrec) DC_CUDA(cudaMemcpyAsync(s + OFF_REC, p->rrec.data(), nrec * sizeof(RelocRec), cudaMemcpyHostToDevice, cs));
  DC_CUDA(cudaMemcpyAsync(s + OFF_SEG, p->rseg.data(), p->rseg.size() * sizeof(RelocSeg), cudaMemcpyHostToDevice, cs));
  if (ntiles)
    DC_CUDA(cudaMemcpyAsync(s + OFF_TILE, p->rtiles.data(), ntiles * sizeof(RelocTile), cudaMemcpyHostToDevice, cs));
  RelocArgs a;
  a.arena = static_cast<uint8_t*>(dev_data);
  a.data_bytes = p->data_bytes;
  a.struct_bytes = p->struct_bytes;
  a.rec = reinterpret_cast<const RelocRec*>(s + OFF_REC);
  a.seg = reinterpret_cast<const RelocSeg*>(s + OFF_SEG);
  a.tiles = reinterpret_cast<const RelocTile*>(s + OFF_TILE);
  a.rec_host = nullptr;  // no slot check in this variant
  a.rec_off = nullptr;
  a.ctrl = reinterpret_cast<uint32_t*>(s + OFF_CTRL);
  a.nrec = (uint32_t)nrec;
  a.nseg = (uint32_t)nseg;
  a.ntiles = (uint32_t)ntiles;
  a.verify = 0;
  a.scan = 0;  // the offsets the plan assigned
  a.unit_shift = p->unit_shift;
  DC_CUDA(launch_relocate(a, cs, sms));
  if (dev_status)
    DC_CUDA(cudaMemcpyAsync(dev_status, s + OFF_CTRL + CTRL_ERR * 4, 4, cudaMemcpyDeviceToDevice, cs));
  return DC_OK;
}
