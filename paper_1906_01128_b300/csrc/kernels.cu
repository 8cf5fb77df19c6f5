// kernels.cu — device side of the deep-copy hot path (sm_103a).
//
//   relocate_kernel  Fig 2 step d / Algorithm 1's attach loop: one pass over
//                    the struct lane in RELOC_SPAN-byte tiles.  A tile stages
//                    its struct bytes in shared memory, writes into each of
//                    its slots the device address of the block it points at
//                    (the arena base + the slot's lane group base + the
//                    target's offset in the group: the record's, or a
//                    prefix sum of sizes with DC_PLAN_DEVICE_SCAN), and
//                    stores the tile back: whole coalesced sectors instead
//                    of one 8-byte store per pointer.
//   leaf_tma_kernel  the leaf update through resolved effective addresses
//                    (Sec. 3): x += 0.5*y or x *= scale over (x, y, n)
//                    segments, no pointer loads; x and y come into shared
//                    memory by 1-D bulk copies, half a tile at a time in
//                    three stages (the default for dc_update_leaves).
//   leaf_kernel      the same update by direct 16-byte vector loads
//                    (DC_LEAF_TMA=0).
//   fused_kernel     relocation tiles, then the leaf update's half tiles from
//                    an atomic counter, staged by bulk copies in the
//                    relocation's two stages (dc_relocate_update).
//   chase_kernel     the same update with every element walking its pointer
//                    chain from the root (Listing 2's loop body), with loads
//                    that may not be hoisted out of the element loop.
//   move_kernel      moves whole blocks between mapped host pages and the
//                    arena in 16-byte units (the deep copy's transfer and the
//                    copy back, one launch for every block instead of one DMA
//                    per block).
//   place_kernel     span staging's placement: every staged block from its
//                    place among the host spans moved to the device to its
//                    arena offset, one descriptor per block piece.
//   stream_kernel    the fused step: reads x and y of the selected structs from
//                    host memory (mapped caller pages or the mapped pinned
//                    arena), applies the leaf update, writes x and y into the
//                    arena and x straight back to the host, in one pass.
//   walk_kernel      one thread follows a chain and reports the address.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.hpp"

namespace dc {

namespace {

// ---- 1-D bulk copies (TMA) and mbarriers ------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared, completing `bytes` of the barrier's transaction count
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// At most `limit` try_wait rounds for the barrier's phase `parity`; false if
// the phase has not completed by then (a limit of 0 gives up without trying).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t n = 0; n < limit; n++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- relocation ----------------------------------------------------------------

constexpr uint32_t RSTAGES = 2;

// One pipeline stage: a tile's struct bytes, its records (from an even
// index, so the copy starts on 16 bytes) and its lane groups.
struct __align__(16) RelocStage {
  uint4 img[RELOC_SPAN / 16];
  uint2 rec[RELOC_MAXREC + 2];
  RelocSeg grp[RELOC_MAXGROUPS + 1];
};
struct __align__(16) RelocSmem {
  RelocStage st[RSTAGES];
  uint64_t bar[RSTAGES];
  uint4 hdr[RSTAGES];  // the staged tile: (t, r0, r1, ng); t = NONE ends the CTA's tiles
};

__device__ __forceinline__ uint32_t warp_incl_scan32(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= (uint32_t)d) v += o;
  }
  return v;
}

// One staged tile's slots from offset records (the default): a slot's target
// lies at its lane group's base plus the record's 32-bit offset, both in the
// plan's record units (16 bytes, or 4 with DC_PLAN_PACK_SMALL).  Record j goes to thread j % THREADS: conflict-free shared
// loads, and a warp's slot writes land in a few hundred consecutive bytes.
template <uint32_t THREADS, bool VERIFY>
__device__ __forceinline__ void reloc_apply_offsets(const RelocArgs& a, RelocStage& S, uint32_t r0, uint32_t nr,
                                                    uint32_t ng, uint32_t sh, uint32_t n8, uint64_t base) {
  constexpr uint32_t ITEMS = RELOC_MAXREC / THREADS;
  const uint32_t tid = threadIdx.x;
  uint2 r[ITEMS];
#pragma unroll
  for (uint32_t i = 0; i < ITEMS; i++) {
    const uint32_t j = tid + i * THREADS;
    r[i] = j < nr ? S.rec[sh + j] : make_uint2(0, 0);
  }
  uint64_t* img64 = reinterpret_cast<uint64_t*>(S.img);
#pragma unroll
  for (uint32_t i = 0; i < ITEMS; i++) {
    const uint32_t j = tid + i * THREADS;
    if (j >= nr) continue;
    const uint32_t w = r[i].y & 0xFFFFu, g = r[i].y >> 16;  // slot word in the tile, lane group
    if (w >= n8 || g >= ng) {
      atomicOr(&a.ctrl[CTRL_ERR], ERR_BOUNDS);
      continue;
    }
    const uint64_t off = (S.grp[g].base + r[i].x) << a.unit_shift;
    uint64_t* sp = img64 + w;
    if (VERIFY) {
      const uint32_t ri = r0 + j;
      if (*sp != __ldg(&a.rec_host[ri]) || off != __ldg(&a.rec_off[ri])) atomicOr(&a.ctrl[CTRL_ERR], ERR_VERIFY);
    }
    *sp = base + off;
  }
}

// One staged tile's slots from scan records (DC_PLAN_DEVICE_SCAN): the
// records are cut into slices of 32, slice k to warp k % NW, and each warp
// scans its slice with shuffles, segmented at the heads (a slice's first
// record, and a lane group's first).  A head holds its own offset from its
// group's base; any other record holds the size of the record before it, so a
// target's offset is the sum from its segment's head to itself: the inclusive
// prefix minus the exclusive prefix at the head (32-bit: a group's offsets stay
// below 2^32 units, so the difference is exact modulo 2^32).  The slices are
// independent, so the tile needs no barrier beyond the offset form's, and
// record j goes to thread j % THREADS as there.
template <uint32_t THREADS, bool VERIFY>
__device__ __forceinline__ void reloc_apply_scan(const RelocArgs& a, RelocStage& S, uint32_t r0, uint32_t nr,
                                                 uint32_t ng, uint32_t sh, uint32_t n8, uint64_t base) {
  constexpr uint32_t NW = THREADS / 32, ITEMS = RELOC_MAXREC / THREADS;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t* img64 = reinterpret_cast<uint64_t*>(S.img);
#pragma unroll
  for (uint32_t i = 0; i < ITEMS; i++) {
    const uint32_t j0 = (i * NW + warp) * 32;  // the slice's first record
    if (j0 >= nr) break;                        // uniform across the warp
    const uint32_t j = j0 + lane;
    const uint2 rr = j < nr ? S.rec[sh + j] : make_uint2(0, 0);
    // lane 0 starts the slice: a head whatever its record says
    const uint32_t heads = __ballot_sync(0xffffffffu, (rr.y & SCAN_HEAD) != 0) | 1u;
    const uint32_t incl = warp_incl_scan32(rr.x, lane);
    const uint32_t head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));  // the last head at or below
    const uint32_t off32 = incl - __shfl_sync(0xffffffffu, incl - rr.x, head);
    if (j >= nr) continue;
    const uint32_t w = rr.y & (SCAN_HEAD - 1), g = rr.y >> 16;
    if (w >= n8 || g >= ng) {
      atomicOr(&a.ctrl[CTRL_ERR], ERR_BOUNDS);
      continue;
    }
    const uint64_t off = (S.grp[g].base + off32) << a.unit_shift;
    uint64_t* sp = img64 + w;
    if (VERIFY) {
      const uint32_t ri = r0 + j;
      if (*sp != __ldg(&a.rec_host[ri]) || off != __ldg(&a.rec_off[ri])) atomicOr(&a.ctrl[CTRL_ERR], ERR_VERIFY);
    }
    *sp = base + off;
  }
}

// The producer (thread 0) fills stage s with listed tile i of the CTA (or
// marks the CTA's tiles done, i = NONE), after checking the tile's header
// against the tables; a header that fails is recorded and its stage skipped.
__device__ __forceinline__ void issue_tile(const RelocArgs& a, RelocSmem& sm, uint32_t s, uint32_t i, uint4 h) {
  RelocStage& S = sm.st[s];
  if (i == NONE) {
    sm.hdr[s] = make_uint4(NONE, 0, 0, 0);
    mbar_arrive_tx(&sm.bar[s], 0);
    return;
  }
  const uint32_t t = h.x, r0 = h.y, g0 = h.z, nr = h.w & 0xFFFFu, ng = h.w >> 16;
  const uint64_t lo = (uint64_t)t * RELOC_SPAN, hi = min(a.struct_bytes, lo + RELOC_SPAN);
  if (nr == 0 || nr > RELOC_MAXREC || (uint64_t)r0 + nr > a.nrec || ng == 0 || ng > RELOC_MAXGROUPS ||
      (uint64_t)g0 + ng > a.nseg || lo >= hi || (hi - lo) % 16 || hi > a.data_bytes) {
    atomicOr(&a.ctrl[CTRL_ERR], ERR_BOUNDS);
    sm.hdr[s] = make_uint4(t, r0, r0, 0);  // nothing to do in this stage
    mbar_arrive_tx(&sm.bar[s], 0);
    return;
  }
  const uint32_t ra = r0 & ~1u, rb = (r0 + nr + 1) & ~1u;  // even bounds: 16-byte aligned (the table has 2 spare)
  const uint32_t b_img = (uint32_t)(hi - lo), b_rec = (rb - ra) * 8, b_grp = (ng + 1) * 16;
  sm.hdr[s] = make_uint4(t, r0, r0 + nr, ng);
  mbar_arrive_tx(&sm.bar[s], b_img + b_rec + b_grp);
  bulk_load(S.img, a.arena + lo, b_img, &sm.bar[s]);
  bulk_load(S.rec, a.rec + ra, b_rec, &sm.bar[s]);
  bulk_load(S.grp, a.seg + g0, b_grp, &sm.bar[s]);
}

// Every listed relocation tile i = blockIdx.x + k * gridDim.x, through a
// two-stage pipeline: while the CTA rewrites the slots of one staged tile,
// the bulk copies of the next are in flight, and the producer has the header
// after that in a register.  A stage is refilled one step after its store,
// just after the next stage's wait.  A slot's target lies at its lane group's base
// plus its offset in the group (both in record units): the record's own
// offset, or with DC_PLAN_DEVICE_SCAN a prefix sum of the records' sizes.  The
// rewritten staged tile goes back by one bulk store.  The loop's exits are
// uniform across the CTA; every wait has an iteration limit.
template <uint32_t THREADS, bool VERIFY, bool SCAN>
__device__ __forceinline__ void reloc_tiles(const RelocArgs& a, RelocSmem& sm) {
  constexpr uint32_t ITEMS = RELOC_MAXREC / THREADS;
  static_assert(ITEMS * THREADS == RELOC_MAXREC, "tile shape");
  const uint32_t tid = threadIdx.x;
  uint32_t* err = &a.ctrl[CTRL_ERR];
  if (blockIdx.x >= a.ntiles) return;
  const uint4* hdrs = reinterpret_cast<const uint4*>(a.tiles);
  uint32_t in = NONE;  // the producer's next listed tile and its header
  uint4 hn = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (uint32_t s = 0; s < RSTAGES; s++) mbar_init(&sm.bar[s]);
    mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t i = blockIdx.x;
    for (uint32_t s = 0; s < RSTAGES; s++, i += gridDim.x) {
      const bool have = i < a.ntiles;
      issue_tile(a, sm, s, have ? i : NONE, have ? __ldg(hdrs + i) : hn);
    }
    in = i < a.ntiles ? i : NONE;
    if (in != NONE) hn = __ldg(hdrs + in);
  }
  const uint64_t base = reinterpret_cast<uint64_t>(a.arena);
  uint32_t pend = NONE;  // (producer) the stage stored at the end of the last step, not yet refilled
  for (uint32_t k = 0;; k++) {
    const uint32_t s = k % RSTAGES, parity = (k / RSTAGES) & 1;
    const bool late = !mbar_wait(&sm.bar[s], parity, a.wait_limit);
    if (__syncthreads_or(late)) {
      if (tid == 0) {  // give the copies in flight another bounded wait before leaving
        atomicOr(err, ERR_TIMEOUT);
        for (uint32_t q = 0; q < RSTAGES; q++) {
          const uint32_t kq = k + q;
          if (kq % RSTAGES != pend) mbar_wait(&sm.bar[kq % RSTAGES], (kq / RSTAGES) & 1, WAIT_LIMIT);
        }
      }
      break;
    }
    // The stage stored at the end of the last step is refilled here, once every
    // thread has seen this step's stage complete: its bulk store has had the
    // whole wait to read it, so the producer rarely waits here, and the other
    // warps no longer wait for the store and the refill at a barrier.
    if (tid == 0 && pend != NONE) {
      bulk_wait_read();
      issue_tile(a, sm, pend, in, hn);
      if (in != NONE) {
        in += gridDim.x;
        in = in < a.ntiles ? in : NONE;
        if (in != NONE) hn = __ldg(hdrs + in);  // used at the next refill
      }
      pend = NONE;
    }
    const uint4 h = sm.hdr[s];
    if (h.x == NONE) break;  // uniform: every thread reads the same header
    RelocStage& S = sm.st[s];
    const uint32_t t = h.x, r0 = h.y, nr = h.z - h.y, ng = h.w, sh = r0 & 1u;
    const uint64_t lo = (uint64_t)t * RELOC_SPAN, hi = min(a.struct_bytes, lo + RELOC_SPAN);
    if (nr) {  // uniform
      const uint32_t n8 = (uint32_t)((hi - lo) / 8);
      if (SCAN)
        reloc_apply_scan<THREADS, VERIFY>(a, S, r0, nr, ng, sh, n8, base);
      else
        reloc_apply_offsets<THREADS, VERIFY>(a, S, r0, nr, ng, sh, n8, base);
      fence_async_smem();  // the slot writes are seen by the bulk store
    }
    __syncthreads();  // nobody reads stage s any more
    if (tid == 0) {
      if (nr) bulk_store(a.arena + lo, S.img, (uint32_t)(hi - lo));
      pend = s;  // refilled after the next step's wait
    }
  }
  if (tid == 0) bulk_wait_all();
  __syncthreads();  // shared memory may be reused
}

template <bool VERIFY, bool SCAN>
__global__ void __launch_bounds__(RELOC_THREADS) relocate_kernel(RelocArgs a) {
  __shared__ RelocSmem sm;
  reloc_tiles<RELOC_THREADS, VERIFY, SCAN>(a, sm);
}

// ---- leaf update over resolved segments -------------------------------------

template <typename T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
  static constexpr int N = 4;
};
template <>
struct V16<double> {
  using type = double2;
  static constexpr int N = 2;
};

__device__ __forceinline__ float op_axpy(float x, float y) { return __fadd_rn(x, __fmul_rn(0.5f, y)); }
__device__ __forceinline__ double op_axpy(double x, double y) { return __dadd_rn(x, __dmul_rn(0.5, y)); }
__device__ __forceinline__ float op_scale(float x, float s) { return __fmul_rn(x, s); }
__device__ __forceinline__ double op_scale(double x, double s) { return __dmul_rn(x, s); }

template <typename T, int KIND>
__device__ __forceinline__ T apply(T x, T y, T s) {
  return KIND == DC_OP_AXPY_HALF ? op_axpy(x, y) : op_scale(x, s);
}

// last s in [lo, hi] with key(s) <= u
template <typename F>
__device__ __forceinline__ uint32_t search(uint32_t lo, uint32_t hi, uint64_t u, F key) {
  while (lo < hi) {
    uint32_t mid = (lo + hi + 1) >> 1;
    if (key(mid) <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float4 ldcs(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ldcs(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ void stcs(float4* p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void stcs(double2* p, double2 v) { __stcs(p, v); }

// One tile of LEAF_TILE 16-byte units, done by a CTA of THREADS threads
// (LEAF_TILE / THREADS units each).  No barriers.
template <typename T, int KIND, uint32_t THREADS>
__device__ __forceinline__ void leaf_tile(const LeafArgs& a, uint64_t t) {
  using VT = typename V16<T>::type;
  constexpr int EPU = V16<T>::N;
  constexpr uint32_t UNROLL = LEAF_TILE / THREADS;
  const T sc = (T)a.scale;
  const Segment* seg = a.seg;
  auto ub = [&](uint32_t s) { return __ldg(&seg[s].ubeg); };
  const uint64_t u0 = t * LEAF_TILE;
  // the tile's segments are [lo, hi]; most tiles lie inside one segment
  const uint32_t lo = __ldg(&a.tile_seg[t]), hi = __ldg(&a.tile_seg[t + 1]);
  VT xv[UNROLL], yv[UNROLL];
  VT* xp[UNROLL];
  const VT* yp[UNROLL];
  uint32_t tail[UNROLL];  // elements of this unit; EPU = a full vector
#pragma unroll
  for (uint32_t k = 0; k < UNROLL; k++) {
    const uint64_t u = u0 + threadIdx.x + k * THREADS;
    tail[k] = 0;
    xp[k] = nullptr;
    yp[k] = nullptr;
    if (u >= a.units) continue;
    const uint32_t s = lo == hi ? lo : search(lo, hi, u, ub);
    const Segment g = seg[s];
    const uint64_t e0 = (u - g.ubeg) * EPU;
    xp[k] = reinterpret_cast<VT*>(g.x + e0 * sizeof(T));
    yp[k] = reinterpret_cast<const VT*>(g.y + e0 * sizeof(T));
    const uint64_t left = g.n - e0;
    tail[k] = left >= (uint64_t)EPU ? EPU : (uint32_t)left;
  }
#pragma unroll
  for (uint32_t k = 0; k < UNROLL; k++) {
    if (tail[k] == EPU) {
      xv[k] = ldcs(xp[k]);
      if (KIND == DC_OP_AXPY_HALF) yv[k] = ldcs(yp[k]);
    }
  }
#pragma unroll
  for (uint32_t k = 0; k < UNROLL; k++) {
    if (tail[k] == EPU) {
      T* x = reinterpret_cast<T*>(&xv[k]);
      const T* y = reinterpret_cast<const T*>(&yv[k]);
#pragma unroll
      for (int i = 0; i < EPU; i++) x[i] = apply<T, KIND>(x[i], KIND == DC_OP_AXPY_HALF ? y[i] : T(0), sc);
      stcs(xp[k], xv[k]);
    } else if (tail[k]) {
      T* x = reinterpret_cast<T*>(xp[k]);
      const T* y = reinterpret_cast<const T*>(yp[k]);
      for (uint32_t i = 0; i < tail[k]; i++) x[i] = apply<T, KIND>(x[i], KIND == DC_OP_AXPY_HALF ? y[i] : T(0), sc);
    }
  }
}

// With many tiles per CTA (`dynamic`), tiles come from an atomic counter in the
// plan's control words, since tiles take uneven times (those that straddle
// segments search for theirs); the last CTA to finish resets it for the next
// launch (launches on one stream never overlap).  With a few tiles per CTA
// there is little to balance, and CTA b takes tiles b, b + grid, ... without
// the per-tile atomic and barriers.
template <typename T, int KIND>
__global__ void __launch_bounds__(LEAF_THREADS) leaf_kernel(LeafArgs a, int dynamic) {
  const uint64_t ntiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  if (!dynamic) {  // uniform across the grid
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) leaf_tile<T, KIND, LEAF_THREADS>(a, t);
    return;
  }
  __shared__ unsigned long long s_t;
  unsigned long long* next = reinterpret_cast<unsigned long long*>(&a.ctrl[CTRL_NEXT]);
  for (;;) {
    if (threadIdx.x == 0) s_t = atomicAdd(next, 1ull);
    __syncthreads();
    const uint64_t t = s_t;
    __syncthreads();
    if (t >= ntiles) break;
    leaf_tile<T, KIND, LEAF_THREADS>(a, t);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.ctrl[CTRL_DONE], 1u) == gridDim.x - 1) {
      atomicExch(next, 0ull);
      atomicExch(&a.ctrl[CTRL_DONE], 0u);
    }
  }
}

// ---- leaf update with its operands staged by 1-D bulk copies -----------------

constexpr uint32_t LSTAGES = 3;                    // sub-tiles in flight per CTA
constexpr uint32_t LSUB = LEAF_TILE / 2;           // 16-byte units per sub-tile (half a leaf tile)
constexpr size_t LSUB_BYTES = (size_t)LSUB * 16;  // 8 KiB per operand

// Dynamic shared memory of leaf_tma_kernel: per stage one sub-tile of x (and of
// y for AXPY_HALF), then the stage headers and barriers.
template <int KIND>
constexpr size_t leaf_tma_smem() {
  return LSTAGES * (KIND == DC_OP_AXPY_HALF ? 2 : 1) * LSUB_BYTES + LSTAGES * (8 + 32);
}

// The table entries a sub-tile's copies need: its leaf tile's segment range
// and, when that is one segment, the segment.  The producer loads them in two
// steps a refill ahead: the range at one refill, the segment (whose index the
// range gives) at the start of the next iteration, so that no load on the
// refill path waits for another.
struct LeafNext {
  uint32_t lo, hi;
  Segment g;
};
__device__ __forceinline__ void leaf_next_range(const LeafArgs& a, uint64_t w, uint64_t nsub, LeafNext* n) {
  n->lo = n->hi = NONE;
  if (w >= nsub) return;
  n->lo = __ldg(&a.tile_seg[w / 2]);
  n->hi = __ldg(&a.tile_seg[w / 2 + 1]);
}
__device__ __forceinline__ void leaf_next_seg(const LeafArgs& a, LeafNext* n) {
  if (n->lo < a.nseg) n->g = a.seg[n->lo];  // used only when lo == hi < nseg
}

// The producer (thread 0) stages sub-tile w (units [w, w+1) * LSUB, in leaf
// tile w / 2) in stage s.  A leaf tile inside one segment comes by bulk copies
// (its x and y units are contiguous and 16-byte aligned, the last one inside
// its block's padding); a tile across segments, or in a segment off a 16-byte
// boundary, goes to the direct path,
// whole, from its first half (its second half is then empty); w past the end
// marks the end.  hdr[2s] = (w, mode, units), hdr[2s+1] = the destination of
// the sub-tile's first unit and the elements left from it.
// (xd, yd: the stage's 8 KiB buffers for x and y; hdr: its two header slots.)
template <int KIND>
__device__ __forceinline__ void leaf_issue(const LeafArgs& a, uint4* xd, uint4* yd, uint64_t* bar, uint4* hdr,
                                           uint64_t w, uint64_t nsub, const LeafNext& n) {
  constexpr uint32_t NB = KIND == DC_OP_AXPY_HALF ? 2 : 1;
  if (w >= nsub) {
    hdr[0] = make_uint4(NONE, NONE, 0, 0);
    mbar_arrive_tx(bar, 0);
    return;
  }
  const uint64_t u0 = w * LSUB, u1 = min(u0 + LSUB, a.units);
  // across segments, or in a segment that does not start on 16 bytes (a
  // packed arena's short head): the direct path takes the whole tile once
  if (n.lo != n.hi || n.lo >= a.nseg || ((n.g.x | (KIND == DC_OP_AXPY_HALF ? n.g.y : 0)) & 15)) {
    hdr[0] = make_uint4((uint32_t)w, (uint32_t)(w >> 32), (w & 1) ? 3u : 0u, 0);
    mbar_arrive_tx(bar, 0);
    return;
  }
  const Segment& g = n.g;
  const uint32_t bytes = (uint32_t)((u1 - u0) * 16);
  const uint64_t x0 = g.x + (u0 - g.ubeg) * 16, left = g.n - (u0 - g.ubeg) * (16 / (a.f64 ? 8 : 4));
  hdr[0] = make_uint4((uint32_t)w, (uint32_t)(w >> 32), 1, (uint32_t)(u1 - u0));
  hdr[1] = make_uint4((uint32_t)x0, (uint32_t)(x0 >> 32), (uint32_t)left, (uint32_t)(left >> 32));
  mbar_arrive_tx(bar, NB * bytes);
  bulk_load(xd, reinterpret_cast<const void*>(g.x + (u0 - g.ubeg) * 16), bytes, bar);
  if (KIND == DC_OP_AXPY_HALF) bulk_load(yd, reinterpret_cast<const void*>(g.y + (u0 - g.ubeg) * 16), bytes, bar);
}

// One staged sub-tile's update (header h, h2 as leaf_issue wrote them): mode 0
// runs the whole leaf tile by direct loads, mode 1 the staged units, mode 3
// nothing.  x goes back by 16-byte stores; a segment's last elements are read
// from the staged copy, so the register vectors take static indices only.
template <typename T, int KIND, uint32_t THREADS>
__device__ __forceinline__ void leaf_staged_apply(const LeafArgs& a, const uint4* xbuf, const uint4* ybuf, uint4 h,
                                                  uint4 h2) {
  using VT = typename V16<T>::type;
  constexpr int EPU = V16<T>::N;
  constexpr uint32_t UNROLL = LSUB / THREADS;
  static_assert(UNROLL * THREADS == LSUB, "sub-tile shape");
  const uint32_t tid = threadIdx.x;
  const T sc = (T)a.scale;
  const uint64_t w = (uint64_t)h.x | ((uint64_t)h.y << 32);
  if (h.z == 0) {
    leaf_tile<T, KIND, THREADS>(a, w / 2);  // the whole leaf tile, by direct loads
    return;
  }
  if (h.z != 1) return;  // the second half of a tile the direct path took whole
  const uint64_t x0 = (uint64_t)h2.x | ((uint64_t)h2.y << 32), left0 = (uint64_t)h2.z | ((uint64_t)h2.w << 32);
  const VT* xs = reinterpret_cast<const VT*>(xbuf);
  const VT* ys = reinterpret_cast<const VT*>(KIND == DC_OP_AXPY_HALF ? ybuf : xbuf);
#pragma unroll
  for (uint32_t i = 0; i < UNROLL; i++) {
    const uint32_t j = tid + i * THREADS;
    if (j >= h.w) break;
    const uint64_t e0 = (uint64_t)j * EPU;  // from the sub-tile's first element
    const uint64_t left = left0 - e0;
    if (left >= (uint64_t)EPU) {
      VT xv = xs[j];
      const VT yv = ys[j];
      T* x = reinterpret_cast<T*>(&xv);  // static indices only: the vector stays in registers
      const T* y = reinterpret_cast<const T*>(&yv);
#pragma unroll
      for (int q = 0; q < EPU; q++) x[q] = apply<T, KIND>(x[q], KIND == DC_OP_AXPY_HALF ? y[q] : T(0), sc);
      stcs(reinterpret_cast<VT*>(x0 + e0 * sizeof(T)), xv);
    } else {  // the segment's last elements, read from the staged copy
      const T* xsm = reinterpret_cast<const T*>(xs + j);
      const T* ysm = reinterpret_cast<const T*>(ys + j);
      T* xd = reinterpret_cast<T*>(x0 + e0 * sizeof(T));
      for (uint32_t q = 0; q < (uint32_t)left; q++)
        xd[q] = apply<T, KIND>(xsm[q], KIND == DC_OP_AXPY_HALF ? ysm[q] : T(0), sc);
    }
  }
}

// The leaf update with x and y brought into shared memory by 1-D bulk copies
// (the tensor-memory-access engine), in half tiles of 8 KiB per operand with
// LSTAGES of them in flight per CTA: while the CTA updates one, the copies of
// the next two are under way.  The update runs in registers and x goes back
// by coalesced 16-byte stores.  Sub-tiles w = blockIdx.x + k * gridDim.x.
// Every wait has an iteration limit.
template <typename T, int KIND, uint32_t THREADS>
__global__ void __launch_bounds__(THREADS, 3) leaf_tma_kernel(LeafArgs a) {
  constexpr uint32_t NB = KIND == DC_OP_AXPY_HALF ? 2 : 1;
  extern __shared__ __align__(128) uint8_t dsm[];
  uint4* buf = reinterpret_cast<uint4*>(dsm);
  uint4* hdr = reinterpret_cast<uint4*>(dsm + LSTAGES * NB * LSUB_BYTES);  // 16-byte aligned, 2 per stage
  uint64_t* bar = reinterpret_cast<uint64_t*>(hdr + 2 * LSTAGES);
  const uint32_t tid = threadIdx.x;
  const uint64_t nsub = (a.units + LSUB - 1) / LSUB;
  if (blockIdx.x >= nsub) return;
  auto xbuf = [&](uint32_t s) { return buf + (size_t)s * NB * LSUB; };
  auto ybuf = [&](uint32_t s) { return buf + ((size_t)s * NB + (NB - 1)) * LSUB; };
  if (tid == 0) {
    for (uint32_t s = 0; s < LSTAGES; s++) mbar_init(&bar[s]);
    mbar_init_fence();
  }
  __syncthreads();
  uint64_t wn = blockIdx.x;  // the producer's next sub-tile, and its table entries
  LeafNext nx{NONE, NONE, {0, 0, 0, 0}};
  if (tid == 0) {
    for (uint32_t s = 0; s < LSTAGES; s++, wn += gridDim.x) {
      leaf_next_range(a, wn, nsub, &nx);
      leaf_next_seg(a, &nx);
      leaf_issue<KIND>(a, xbuf(s), ybuf(s), &bar[s], &hdr[2 * s], wn, nsub, nx);
    }
    leaf_next_range(a, wn, nsub, &nx);
  }
  for (uint32_t k = 0;; k++) {
    const uint32_t s = k % LSTAGES, parity = (k / LSTAGES) & 1;
    if (tid == 0) leaf_next_seg(a, &nx);  // the range arrived during the last iteration
    const bool late = !mbar_wait(&bar[s], parity, a.wait_limit);
    if (__syncthreads_or(late)) {
      if (tid == 0) {  // give the copies in flight another bounded wait before leaving
        atomicOr(&a.ctrl[CTRL_ERR], ERR_TIMEOUT);
        for (uint32_t q = 0; q < LSTAGES; q++) {
          const uint32_t kq = k + q;
          mbar_wait(&bar[kq % LSTAGES], (kq / LSTAGES) & 1, WAIT_LIMIT);
        }
      }
      break;
    }
    const uint4 h = hdr[2 * s];
    if (h.x == NONE && h.y == NONE) break;  // uniform
    leaf_staged_apply<T, KIND, THREADS>(a, xbuf(s), ybuf(s), h, hdr[2 * s + 1]);
    __syncthreads();  // nobody reads stage s any more
    if (tid == 0) {
      leaf_issue<KIND>(a, xbuf(s), ybuf(s), &bar[s], &hdr[2 * s], wn, nsub, nx);
      if (wn < nsub) wn += gridDim.x;
      leaf_next_range(a, wn, nsub, &nx);  // its segment is loaded next iteration
    }
  }
}

// Relocation and leaf update in one persistent launch.  The two touch disjoint
// bytes (the leaf update works through addresses resolved on the host and
// never reads a pointer; the relocation writes only pointer slots), so no
// grid-wide barrier separates them and one launch over a forest replaces two
// per structure.  Every CTA first runs its share of the relocation tiles
// (reloc_tiles: tile blockIdx.x + k * gridDim.x).
// After its relocation tiles, a CTA takes half tiles of the leaf update from a
// counter (so the CTAs that relocated take fewer) and stages them in its two
// relocation stages by bulk copies: x in a stage's struct buffer, y in its
// record buffer (8 KiB each).  Thread 0 grabs sub-tile indices two refills
// ahead, loads their segment range one refill ahead and the segment at the
// start of an iteration, so that no load on the refill path waits for another.
// The last CTA to finish resets the counter for the next launch (launches on
// one stream never overlap).  Every wait has an iteration limit.
template <typename T, int KIND, uint32_t THREADS, bool SCAN>
__global__ void __launch_bounds__(THREADS) fused_kernel(RelocArgs r, LeafArgs l, uint64_t leaf_tiles) {
  static_assert(sizeof(RelocStage::img) >= LSUB_BYTES && sizeof(RelocStage::rec) >= LSUB_BYTES,
                "a relocation stage holds a half tile of x and of y");
  __shared__ RelocSmem sm;
  __shared__ uint64_t lbar[RSTAGES];
  __shared__ uint4 lhdr[2 * RSTAGES];
  (void)leaf_tiles;  // the launch's grid size counts them; the CTAs count half tiles
  if (r.verify)
    reloc_tiles<THREADS, true, SCAN>(r, sm);
  else
    reloc_tiles<THREADS, false, SCAN>(r, sm);
  // The relocation's stages are free: its loop ended with every stage's copies
  // complete and its stores drained (or the CTA had no relocation tile).
  const uint32_t tid = threadIdx.x;
  unsigned long long* next = reinterpret_cast<unsigned long long*>(&r.ctrl[CTRL_NEXT]);
  const uint64_t nsub = (l.units + LSUB - 1) / LSUB;
  auto xbuf = [&](uint32_t s) { return sm.st[s].img; };
  auto ybuf = [&](uint32_t s) { return reinterpret_cast<uint4*>(sm.st[s].rec); };
  if (tid == 0) {
    for (uint32_t s = 0; s < RSTAGES; s++) mbar_init(&lbar[s]);
    mbar_init_fence();
  }
  __syncthreads();
  uint64_t cur = 0, ahead = 0;  // the producer's next two sub-tiles
  LeafNext nx{NONE, NONE, {0, 0, 0, 0}};
  if (tid == 0) {
    for (uint32_t s = 0; s < RSTAGES; s++) {
      const uint64_t w = atomicAdd(next, 1ull);
      leaf_next_range(l, w, nsub, &nx);
      leaf_next_seg(l, &nx);
      leaf_issue<KIND>(l, xbuf(s), ybuf(s), &lbar[s], &lhdr[2 * s], w, nsub, nx);
    }
    cur = atomicAdd(next, 1ull);
    leaf_next_range(l, cur, nsub, &nx);
    ahead = atomicAdd(next, 1ull);
  }
  for (uint32_t k = 0;; k++) {
    const uint32_t s = k % RSTAGES, parity = (k / RSTAGES) & 1;
    if (tid == 0) leaf_next_seg(l, &nx);  // the range arrived during the last iteration
    const bool late = !mbar_wait(&lbar[s], parity, l.wait_limit);
    if (__syncthreads_or(late)) {
      if (tid == 0) {  // give the copies in flight another bounded wait before leaving
        atomicOr(&r.ctrl[CTRL_ERR], ERR_TIMEOUT);
        for (uint32_t q = 0; q < RSTAGES; q++) {
          const uint32_t kq = k + q;
          mbar_wait(&lbar[kq % RSTAGES], (kq / RSTAGES) & 1, WAIT_LIMIT);
        }
      }
      break;
    }
    const uint4 h = lhdr[2 * s];
    // the counter hands each CTA increasing indices: past the end, every later one is too
    if (h.x == NONE && h.y == NONE) break;  // uniform
    leaf_staged_apply<T, KIND, THREADS>(l, xbuf(s), ybuf(s), h, lhdr[2 * s + 1]);
    __syncthreads();  // nobody reads stage s any more
    if (tid == 0) {
      leaf_issue<KIND>(l, xbuf(s), ybuf(s), &lbar[s], &lhdr[2 * s], cur, nsub, nx);
      cur = ahead;
      leaf_next_range(l, cur, nsub, &nx);  // its segment is loaded next iteration
      ahead = atomicAdd(next, 1ull);
    }
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&r.ctrl[CTRL_DONE], 1u) == gridDim.x - 1) {
      atomicExch(next, 0ull);
      atomicExch(&r.ctrl[CTRL_DONE], 0u);
    }
  }
}

// ---- block moves between host and device ------------------------------------

// Copy n (<= 16) bytes with the widest access both addresses allow; never
// touches a byte outside [src, src + n) or [dst, dst + n).
__device__ __forceinline__ void move_partial(uint64_t src, uint64_t dst, uint32_t n) {
  const uint64_t al = src | dst;
  if ((al & 7) == 0 && (n & 7) == 0) {
    for (uint32_t i = 0; i < n; i += 8) *reinterpret_cast<uint64_t*>(dst + i) = *reinterpret_cast<const uint64_t*>(src + i);
  } else if ((al & 3) == 0 && (n & 3) == 0) {
    for (uint32_t i = 0; i < n; i += 4) *reinterpret_cast<uint32_t*>(dst + i) = *reinterpret_cast<const uint32_t*>(src + i);
  } else {
    for (uint32_t i = 0; i < n; i++) *reinterpret_cast<uint8_t*>(dst + i) = *reinterpret_cast<const uint8_t*>(src + i);
  }
}

__global__ void __launch_bounds__(LEAF_THREADS) move_kernel(MoveArgs a) {
  const MoveDesc* d = a.d;
  auto ub = [&](uint32_t i) { return __ldg(&d[i].ubeg); };
  for (uint64_t t = blockIdx.x; t * LEAF_TILE < a.units; t += gridDim.x) {
    const uint64_t u0 = t * LEAF_TILE;
    const uint32_t lo = __ldg(&a.tile_desc[t]), hi = __ldg(&a.tile_desc[t + 1]);
    uint4 v[LEAF_UNROLL];
    uint64_t dst[LEAF_UNROLL];
    bool full[LEAF_UNROLL];
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {  // issue every load first
      const uint64_t u = u0 + threadIdx.x + k * LEAF_THREADS;
      full[k] = false;
      dst[k] = 0;
      if (u >= a.units) continue;
      const uint32_t s = lo == hi ? lo : search(lo, hi, u, ub);
      const MoveDesc g = d[s];
      const uint64_t off = (u - g.ubeg) * 16;
      const uint64_t left = g.bytes - off;
      const uint64_t src = g.src + off;
      dst[k] = g.dst + off;
      if (left >= 16 && ((src | dst[k]) & 15) == 0) {
        v[k] = *reinterpret_cast<const uint4*>(src);
        full[k] = true;
      } else {
        move_partial(src, dst[k], left >= 16 ? 16u : (uint32_t)left);
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++)
      if (full[k]) *reinterpret_cast<uint4*>(dst[k]) = v[k];
  }
}

// ---- span placement: staged blocks from the staging region to the arena ----------

// Bytes [o, o + n) of a piece (o a multiple of 16, n <= 16) from s to d; the
// bytes at or past `valid` are written as zeros.  16-byte vectors when both
// sides allow it (the staging region then holds the whole 16 bytes), else
// 8-, 4- or 1-byte steps over the valid bytes.
__device__ __forceinline__ void place_chunk(const uint8_t* s, uint8_t* d, uint32_t o, uint32_t n, uint32_t valid) {
  const uint64_t al = reinterpret_cast<uint64_t>(s + o) | reinterpret_cast<uint64_t>(d + o);
  if (n == 16 && (al & 15) == 0) {
    uint4 v = *reinterpret_cast<const uint4*>(s + o);
    if (valid < o + 16) {  // zeros after the block's bytes (its slot's padding)
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) {
        const uint32_t b0 = o + 4 * q;  // bytes [b0, b0 + 4) of the piece
        const uint32_t keep = valid <= b0 ? 0u : valid >= b0 + 4 ? 4u : valid - b0;
        w[q] = keep == 4 ? w[q] : keep == 0 ? 0u : (w[q] & ((1u << (8 * keep)) - 1));
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    *reinterpret_cast<uint4*>(d + o) = v;
    return;
  }
  const uint32_t e = o + n, ve = valid < e ? (valid > o ? valid : o) : e;  // [o, ve) copied, [ve, e) zeroed
  uint32_t k = o;
  if ((al & 7) == 0)
    for (; k + 8 <= ve; k += 8) *reinterpret_cast<uint64_t*>(d + k) = *reinterpret_cast<const uint64_t*>(s + k);
  if ((al & 3) == 0)
    for (; k + 4 <= ve; k += 4) *reinterpret_cast<uint32_t*>(d + k) = *reinterpret_cast<const uint32_t*>(s + k);
  for (; k < ve; k++) d[k] = s[k];
  for (; k < e; k++) d[k] = 0;
}

// Word x holding bytes [b, b + 4) of a piece, with the bytes at or past `valid` zeroed.
__device__ __forceinline__ uint32_t keep_below(uint32_t x, uint32_t b, uint32_t valid) {
  return valid >= b + 4 ? x : valid <= b ? 0u : (x & ((1u << (8 * (valid - b))) - 1));
}

// A piece that writes more than 64 bytes, by a whole warp, 16 bytes per lane at
// a time (rare in a span-staged plan, so kept out of line).
__device__ __noinline__ void place_big(const uint8_t* s, uint8_t* d, uint32_t wlen, uint32_t valid, uint32_t lane) {
  for (uint32_t o = lane * 16; o < wlen; o += 32 * 16) place_chunk(s, d, o, min(16u, wlen - o), valid);
}

// A piece that writes at most 64 bytes, by one lane: with both sides on 16
// bytes and whole vectors, every load is issued before the first store (a
// store could alias a later load, so chunk by chunk each load would wait for
// the store before it); else chunk by chunk.
__device__ __forceinline__ void place_small(const uint8_t* s, uint8_t* d, uint32_t wlen, uint32_t valid) {
  const uint64_t al = reinterpret_cast<uint64_t>(s) | reinterpret_cast<uint64_t>(d);
  if ((al & 15) == 0 && (wlen & 15) == 0) {
    uint4 v[4];
#pragma unroll
    for (uint32_t q = 0; q < 4; q++)
      if (16 * q < wlen) v[q] = *reinterpret_cast<const uint4*>(s + 16 * q);
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      if (16 * q < wlen) {
        // zeros after the block's bytes (its slot's padding)
        const uint32_t b0 = 16 * q;
        const uint4 o = make_uint4(keep_below(v[q].x, b0, valid), keep_below(v[q].y, b0 + 4, valid),
                                   keep_below(v[q].z, b0 + 8, valid), keep_below(v[q].w, b0 + 12, valid));
        *reinterpret_cast<uint4*>(d + b0) = o;
      }
    }
    return;
  }
  for (uint32_t o = 0; o < wlen; o += 16) place_chunk(s, d, o, min(16u, wlen - o), valid);
}

// Every piece of the placement table, warp by warp: each lane loads one
// descriptor (16 coalesced bytes, a round ahead) and copies its piece itself when it writes
// at most 64 bytes; larger pieces are copied by the whole warp, one after
// another, 16 bytes per lane.  The pieces are in staging order, so a warp
// reads consecutive bytes, and its writes of small pieces fall in a few runs
// of consecutive slots (one per lane of the arena).
__global__ void __launch_bounds__(LEAF_THREADS) place_kernel(PlaceArgs a) {
  constexpr uint32_t WPB = LEAF_THREADS / 32;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * WPB;
  uint64_t w = (uint64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
  PlaceDesc gn{0, 0};  // the lane's descriptor for the next round, loaded a round ahead
  if (w * 32 + lane < a.nd) gn = a.d[w * 32 + lane];
  for (; w * 32 < a.nd; w += nwarps) {  // uniform per warp
    const uint64_t i = w * 32 + lane, inext = (w + nwarps) * 32 + lane;
    const PlaceDesc g = gn;
    if (inext < a.nd) gn = a.d[inext];
    const uint64_t so = g.src & ((1ull << 60) - 1), dso = g.dst >> 16;
    const uint32_t pad = (uint32_t)(g.src >> 60), wlen = (uint32_t)(g.dst & 0xFFFFu) + 1, len = wlen - pad;
    bool ok = i < a.nd;
    if (ok && (pad >= wlen || so + len > a.stage_bytes || dso + wlen > a.data_bytes)) {
      atomicOr(a.err, ERR_BOUNDS);
      ok = false;
    }
    if (ok && wlen <= 64) place_small(a.stage + so, a.arena + dso, wlen, len);
    uint32_t big = __ballot_sync(0xffffffffu, ok && wlen > 64);
    while (big) {
      const int j = __ffs(big) - 1;
      big &= big - 1;
      const uint64_t bso = __shfl_sync(0xffffffffu, so, j), bdo = __shfl_sync(0xffffffffu, dso, j);
      const uint32_t bw = __shfl_sync(0xffffffffu, wlen, j), bl = __shfl_sync(0xffffffffu, len, j);
      place_big(a.stage + bso, a.arena + bdo, bw, bl, lane);
    }
  }
}

// ---- fused step: host -> update -> arena + host --------------------------------

// Device-visible address of byte `off` of a block whose host copy is split in a
// mapped interior [lo, hi) and the rest, kept in the mapped pinned arena.
__device__ __forceinline__ uint64_t host_side(uint64_t h, uint64_t lo, uint64_t hi, uint64_t idev, uint64_t pin,
                                              uint64_t off) {
  const uint64_t a = h + off;
  return (a >= lo && a < hi) ? idev + (a - lo) : pin + off;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(LEAF_THREADS) stream_kernel(StreamArgs a) {
  using VT = typename V16<T>::type;
  constexpr int EPU = V16<T>::N;
  const T sc = (T)a.scale;
  const StreamSeg* seg = a.seg;
  auto ub = [&](uint32_t s) { return __ldg(&seg[s].ubeg); };
  for (uint64_t t = a.t_begin + blockIdx.x; t < a.t_end && t * LEAF_TILE < a.units; t += gridDim.x) {
    const uint64_t u0 = t * LEAF_TILE;
    const uint32_t lo = __ldg(&a.tile_seg[t]), hi = __ldg(&a.tile_seg[t + 1]);
    VT xv[LEAF_UNROLL], yv[LEAF_UNROLL];
    uint64_t xs[LEAF_UNROLL], xd[LEAF_UNROLL], yd[LEAF_UNROLL];
    uint32_t cnt[LEAF_UNROLL];  // elements of this unit
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {  // issue every host read first
      const uint64_t u = u0 + threadIdx.x + k * LEAF_THREADS;
      cnt[k] = 0;
      if (u >= a.units) continue;
      const uint32_t s = lo == hi ? lo : search(lo, hi, u, ub);
      const StreamSeg& g = seg[s];
      const uint64_t e0 = (u - __ldg(&g.ubeg)) * EPU, off = e0 * sizeof(T);
      const uint64_t left = __ldg(&g.n) - e0;
      cnt[k] = left >= (uint64_t)EPU ? EPU : (uint32_t)left;
      xs[k] = host_side(__ldg(&g.xh), __ldg(&g.xlo), __ldg(&g.xhi), __ldg(&g.xi), __ldg(&g.xp), off);
      xd[k] = __ldg(&g.xd) + off;
      uint64_t ys = 0;
      if (KIND == DC_OP_AXPY_HALF) {
        ys = host_side(__ldg(&g.yh), __ldg(&g.ylo), __ldg(&g.yhi), __ldg(&g.yi), __ldg(&g.yp), off);
        yd[k] = __ldg(&g.yd) + off;
      }
      if (cnt[k] == EPU) {
        xv[k] = *reinterpret_cast<const VT*>(xs[k]);
        if (KIND == DC_OP_AXPY_HALF) yv[k] = *reinterpret_cast<const VT*>(ys);
      } else {
        T* xe = reinterpret_cast<T*>(&xv[k]);
        T* ye = reinterpret_cast<T*>(&yv[k]);
        for (uint32_t i = 0; i < cnt[k]; i++) {
          xe[i] = reinterpret_cast<const T*>(xs[k])[i];
          if (KIND == DC_OP_AXPY_HALF) ye[i] = reinterpret_cast<const T*>(ys)[i];
        }
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {
      if (!cnt[k]) continue;
      T* x = reinterpret_cast<T*>(&xv[k]);
      const T* y = reinterpret_cast<const T*>(&yv[k]);
      if (cnt[k] == EPU) {
        if (KIND == DC_OP_AXPY_HALF) *reinterpret_cast<VT*>(yd[k]) = yv[k];  // the deep copy of y
#pragma unroll
        for (int i = 0; i < EPU; i++) x[i] = apply<T, KIND>(x[i], KIND == DC_OP_AXPY_HALF ? y[i] : T(0), sc);
        *reinterpret_cast<VT*>(xd[k]) = xv[k];  // the arena holds the updated x
        *reinterpret_cast<VT*>(xs[k]) = xv[k];  // and so does the host
      } else {
        for (uint32_t i = 0; i < cnt[k]; i++) {
          if (KIND == DC_OP_AXPY_HALF) reinterpret_cast<T*>(yd[k])[i] = y[i];
          const T v = apply<T, KIND>(x[i], KIND == DC_OP_AXPY_HALF ? y[i] : T(0), sc);
          reinterpret_cast<T*>(xd[k])[i] = v;
          reinterpret_cast<T*>(xs[k])[i] = v;
        }
      }
    }
  }
}

// ---- per-element pointer chase ---------------------------------------------

// A load the compiler must issue every time it appears (no hoisting or reuse).
__device__ __forceinline__ uint64_t chase_ld(uint64_t addr) {
  uint64_t v;
  asm volatile("ld.global.u64 %0, [%1];" : "=l"(v) : "l"(addr));
  return v;
}

constexpr uint32_t CHASE_THREADS = 256;
constexpr uint32_t CHASE_UNROLL = 4;
constexpr uint32_t CHASE_TILE = CHASE_THREADS * CHASE_UNROLL;

template <typename T, int KIND>
__global__ void __launch_bounds__(CHASE_THREADS) chase_kernel(ChaseArgs a) {
  __shared__ uint32_t s_lo, s_hi;
  const T sc = (T)a.scale;
  auto eb = [&](uint32_t s) { return a.seg[s].ebeg; };
  for (uint64_t e0 = (uint64_t)blockIdx.x * CHASE_TILE; e0 < a.elems; e0 += (uint64_t)gridDim.x * CHASE_TILE) {
    if (threadIdx.x == 0) {
      uint64_t last = min(e0 + CHASE_TILE, a.elems) - 1;
      s_lo = search(0, a.nseg - 1, e0, eb);
      s_hi = search(s_lo, a.nseg - 1, last, eb);
    }
    __syncthreads();
    const uint32_t lo = s_lo, hi = s_hi;
    for (uint32_t k = 0; k < CHASE_UNROLL; k++) {
      uint64_t e = e0 + threadIdx.x + k * CHASE_THREADS;
      if (e >= a.elems) break;
      uint32_t s = lo == hi ? lo : search(lo, hi, e, eb);
      const ChaseSeg g = a.seg[s];
      uint64_t i = e - g.ebeg;
      uint64_t p = g.root;
      for (uint32_t st = 0; st < g.nsteps; st++) {
        const ChaseStep cs = a.steps[g.step_first + st];
        p = chase_ld(p + cs.field_off) + cs.index * cs.child_size;
      }
      T* x = reinterpret_cast<T*>(chase_ld(p + a.x_off));
      if (KIND == DC_OP_AXPY_HALF) {
        const T* y = reinterpret_cast<const T*>(chase_ld(p + a.y_off));
        x[i] = op_axpy(x[i], y[i]);
      } else {
        x[i] = op_scale(x[i], sc);
      }
    }
    __syncthreads();
  }
}

__global__ void walk_kernel(uint64_t root, const ChaseStep* steps, uint32_t nsteps, uint64_t final_add,
                            uint64_t* out) {
  uint64_t p = root;
  for (uint32_t st = 0; st < nsteps; st++) p = chase_ld(p + steps[st].field_off) + steps[st].index * steps[st].child_size;
  *out = p + final_add;
}

// Resident CTAs per SM of `kernel` at `threads` threads and `smem` bytes of
// dynamic shared memory, computed once per (kernel, threads, smem); a kernel
// that needs more than the default 48 KiB of dynamic shared memory is allowed
// it on first use.
template <typename K>
int occupancy(K kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_tuple(reinterpret_cast<const void*>(kernel), threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (smem > (48u << 10)) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
  cache.emplace(key, n);
  return n;
}

}  // namespace

cudaError_t launch_relocate(const RelocArgs& args, cudaStream_t s, int sm_count) {
  if (args.ntiles == 0) return cudaSuccess;
  RelocArgs a = args;
  a.wait_limit = first_wait_limit();
  auto go = [&](auto kernel) {
    const int occ = occupancy(kernel, RELOC_THREADS, 0);
    const uint32_t grid = (uint32_t)std::min<uint64_t>(a.ntiles, (uint64_t)sm_count * occ);  // persistent CTAs
    kernel<<<grid, RELOC_THREADS, 0, s>>>(a);
  };
  if (a.scan)
    a.verify ? go(relocate_kernel<true, true>) : go(relocate_kernel<false, true>);
  else
    a.verify ? go(relocate_kernel<true, false>) : go(relocate_kernel<false, false>);
  count_launch();
  return cudaGetLastError();
}

// The leaf update's kernel: leaf_tma_kernel (bulk copies into shared memory)
// unless DC_LEAF_TMA=0, read at every launch, selects leaf_kernel (direct loads).
cudaError_t launch_leaf(const LeafArgs& args, cudaStream_t s, int sm_count) {
  if (args.units == 0 || args.nseg == 0) return cudaSuccess;
  LeafArgs a = args;
  a.wait_limit = first_wait_limit();
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  const char* v = getenv("DC_LEAF_TMA");
  const bool tma = !(v && v[0] == '0');
  if (tma) {
    auto go_tma = [&](auto kernel, size_t smem) {
      const int occ = occupancy(kernel, LEAF_THREADS, smem);
      const uint64_t nsub = (a.units + LSUB - 1) / LSUB;  // the kernel's work items: half tiles
      uint32_t grid = (uint32_t)std::min<uint64_t>(nsub, (uint64_t)sm_count * occ);
      kernel<<<grid, LEAF_THREADS, smem, s>>>(a);
    };
    if (a.f64)
      a.kind == DC_OP_AXPY_HALF
          ? go_tma(leaf_tma_kernel<double, DC_OP_AXPY_HALF, LEAF_THREADS>, leaf_tma_smem<DC_OP_AXPY_HALF>())
          : go_tma(leaf_tma_kernel<double, DC_OP_SCALE, LEAF_THREADS>, leaf_tma_smem<DC_OP_SCALE>());
    else
      a.kind == DC_OP_AXPY_HALF
          ? go_tma(leaf_tma_kernel<float, DC_OP_AXPY_HALF, LEAF_THREADS>, leaf_tma_smem<DC_OP_AXPY_HALF>())
          : go_tma(leaf_tma_kernel<float, DC_OP_SCALE, LEAF_THREADS>, leaf_tma_smem<DC_OP_SCALE>());
    count_launch();
    return cudaGetLastError();
  }
  auto go = [&](auto kernel) {
    const int occ = occupancy(kernel, LEAF_THREADS, 0);
    uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
    kernel<<<grid, LEAF_THREADS, 0, s>>>(a, tiles >= 8ull * grid ? 1 : 0);
  };
  if (a.f64)
    a.kind == DC_OP_AXPY_HALF ? go(leaf_kernel<double, DC_OP_AXPY_HALF>) : go(leaf_kernel<double, DC_OP_SCALE>);
  else
    a.kind == DC_OP_AXPY_HALF ? go(leaf_kernel<float, DC_OP_AXPY_HALF>) : go(leaf_kernel<float, DC_OP_SCALE>);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_chase(const ChaseArgs& a, cudaStream_t s, int sm_count) {
  if (a.elems == 0 || a.nseg == 0) return cudaSuccess;
  uint64_t tiles = (a.elems + CHASE_TILE - 1) / CHASE_TILE;
  auto go = [&](auto kernel) {
    const int occ = occupancy(kernel, CHASE_THREADS, 0);
    uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
    kernel<<<grid, CHASE_THREADS, 0, s>>>(a);
  };
  if (a.f64)
    a.kind == DC_OP_AXPY_HALF ? go(chase_kernel<double, DC_OP_AXPY_HALF>) : go(chase_kernel<double, DC_OP_SCALE>);
  else
    a.kind == DC_OP_AXPY_HALF ? go(chase_kernel<float, DC_OP_AXPY_HALF>) : go(chase_kernel<float, DC_OP_SCALE>);
  count_launch();
  return cudaGetLastError();
}

namespace {
template <typename T, int KIND>
cudaError_t fused_go(const RelocArgs& r, const LeafArgs& l, uint32_t threads, uint32_t ctas_per_sm, int sm_count,
                     cudaStream_t s, int* max_per_sm) {
  const uint64_t leaf_tiles = (l.units + LEAF_TILE - 1) / LEAF_TILE;
  const uint64_t total = (uint64_t)r.ntiles + leaf_tiles;
  auto go = [&](auto kernel, uint32_t nt) -> cudaError_t {
    int occ = occupancy(kernel, (int)nt, 0);
    if (max_per_sm) {
      *max_per_sm = occ;
      return cudaSuccess;
    }
    if (total == 0) return cudaSuccess;
    uint32_t per = ctas_per_sm ? std::min<uint32_t>(ctas_per_sm, (uint32_t)occ) : (uint32_t)occ;
    uint32_t grid = (uint32_t)std::min<uint64_t>(total, (uint64_t)sm_count * per);
    kernel<<<grid, nt, 0, s>>>(r, l, leaf_tiles);
    count_launch();
    return cudaGetLastError();
  };
  if (r.scan) {
    switch (threads) {
      case 128: return go(fused_kernel<T, KIND, 128, true>, 128);
      case 512: return go(fused_kernel<T, KIND, 512, true>, 512);
      default: return go(fused_kernel<T, KIND, 256, true>, 256);
    }
  }
  switch (threads) {
    case 128: return go(fused_kernel<T, KIND, 128, false>, 128);
    case 512: return go(fused_kernel<T, KIND, 512, false>, 512);
    default: return go(fused_kernel<T, KIND, 256, false>, 256);
  }
}
}  // namespace

cudaError_t launch_fused(const RelocArgs& ra, const LeafArgs& la, uint32_t threads, uint32_t ctas_per_sm, int sm_count,
                         cudaStream_t s, int* max_per_sm) {
  RelocArgs r = ra;
  LeafArgs l = la;
  r.wait_limit = l.wait_limit = first_wait_limit();
  if (l.f64)
    return l.kind == DC_OP_AXPY_HALF ? fused_go<double, DC_OP_AXPY_HALF>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm)
                                     : fused_go<double, DC_OP_SCALE>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm);
  return l.kind == DC_OP_AXPY_HALF ? fused_go<float, DC_OP_AXPY_HALF>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm)
                                   : fused_go<float, DC_OP_SCALE>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm);
}

cudaError_t launch_move(const MoveArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nd == 0) return cudaSuccess;
  const int occ = occupancy(move_kernel, LEAF_THREADS, 0);
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
  move_kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_place(const PlaceArgs& a, cudaStream_t s, int sm_count) {
  if (a.nd == 0) return cudaSuccess;
  const int occ = occupancy(place_kernel, LEAF_THREADS, 0);
  const uint64_t blocks = (a.nd + LEAF_THREADS - 1) / LEAF_THREADS;  // one descriptor per thread at a time
  const uint32_t grid = (uint32_t)std::min<uint64_t>(blocks, (uint64_t)sm_count * occ);
  place_kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_stream(const StreamArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nseg == 0 || a.t_end <= a.t_begin) return cudaSuccess;
  const uint64_t tiles = a.t_end - a.t_begin;
  auto go = [&](auto kernel) {
    const int occ = occupancy(kernel, LEAF_THREADS, 0);
    uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
    kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
  };
  if (a.f64)
    a.kind == DC_OP_AXPY_HALF ? go(stream_kernel<double, DC_OP_AXPY_HALF>) : go(stream_kernel<double, DC_OP_SCALE>);
  else
    a.kind == DC_OP_AXPY_HALF ? go(stream_kernel<float, DC_OP_AXPY_HALF>) : go(stream_kernel<float, DC_OP_SCALE>);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_walk(uint64_t root, const ChaseStep* steps, uint32_t nsteps, uint64_t final_add, uint64_t* out,
                        cudaStream_t s) {
  walk_kernel<<<1, 1, 0, s>>>(root, steps, nsteps, final_add, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dc
