// kernels.cu — device side of the deep-copy hot path (sm_103a).
//
//   relocate_kernel  Fig 2 step d / Algorithm 1's attach loop: one pass that
//                    computes every block's arena offset (an exclusive scan of
//                    the 16-byte block sizes with warp shuffles, on top of the
//                    tile's base offset) and rewrites the pointer slot that
//                    refers to each block with the block's device address.
//                    Block records are read as 16-byte vectors.
//   leaf_kernel      the leaf update through resolved effective addresses
//                    (Sec. 3): x += 0.5*y or x *= scale over (x, y, n)
//                    segments, 16-byte vector loads/stores, no pointer loads.
//   chase_kernel     the same update with every element walking its pointer
//                    chain from the root (Listing 2's loop body), with loads
//                    that may not be hoisted out of the element loop.
//   move_kernel      moves whole blocks between mapped host pages and the
//                    arena in 16-byte units (the deep copy's transfer and the
//                    copy back, one launch for every block instead of one DMA
//                    per block).
//   stream_kernel    the fused step: reads x and y of the selected structs from
//                    host memory (mapped caller pages or the mapped pinned
//                    arena), applies the leaf update, writes x and y into the
//                    arena and x straight back to the host, in one pass.
//   walk_kernel      one thread follows a chain and reports the address.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"

namespace dc {

namespace {

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= (uint32_t)d) v += o;
  }
  return v;
}

// One tile of RELOC_TILE blocks, done by a CTA of THREADS threads.  Warp w
// owns blocks [base + w*32*ITEMS, base + (w+1)*32*ITEMS); its lanes read 32
// consecutive 16-byte records per instruction (coalesced).  The block sizes
// are scanned with warp shuffles (slice by slice, carrying the running total),
// then across the tile's warps, on top of the tile's base offset; every
// block's parent slot is then rewritten.  Parents in an earlier tile take
// their offset from the struct-offset table.  Ends with a barrier.
template <uint32_t THREADS>
__device__ __forceinline__ void reloc_tile(const RelocArgs& a, uint32_t t, uint64_t* s_off, uint64_t* s_warp) {
  constexpr uint32_t NW = THREADS / 32;
  constexpr uint32_t ITEMS = RELOC_TILE / THREADS;
  constexpr uint32_t WSPAN = 32 * ITEMS;  // blocks per warp
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* err = &a.ctrl[CTRL_ERR];
  const uint64_t base = (uint64_t)t * RELOC_TILE;
  const uint64_t wbase = base + warp * WSPAN;
  BlockRec r[ITEMS];
#pragma unroll
  for (uint32_t k = 0; k < ITEMS; k++) {
    const uint64_t b = wbase + k * 32 + lane;
    if (b < a.nblocks) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(a.rec) + b);
      r[k] = BlockRec{v.x, v.y, v.z, v.w};
    } else {
      r[k] = BlockRec{0, NONE, 0, 0};
    }
  }
  // exclusive offsets inside the warp's span, slice by slice
  uint64_t ex[ITEMS];
  uint64_t carry = 0;
#pragma unroll
  for (uint32_t k = 0; k < ITEMS; k++) {
    const uint64_t incl = warp_incl_scan(r[k].size16, lane);
    ex[k] = carry + incl - r[k].size16;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) s_warp[warp] = carry;
  __syncthreads();
  uint64_t wpre = 0;  // every warp adds up the totals of the warps before it
#pragma unroll
  for (uint32_t w = 0; w < NW; w++) wpre += w < warp ? s_warp[w] : 0;
  const uint64_t o16 = __ldg(&a.tile_base[t]) + wpre;
#pragma unroll
  for (uint32_t k = 0; k < ITEMS; k++) {
    const uint64_t b = wbase + k * 32 + lane;
    ex[k] = (o16 + ex[k]) * 16;  // byte offset of block b
    s_off[b - base] = ex[k];
    if (a.verify && b < a.nstruct_blocks && __ldg(&a.soff[b]) != ex[k]) atomicOr(err, ERR_VERIFY);
  }
  __syncthreads();
  // rewrite the slot that points at each block (roots have none)
#pragma unroll
  for (uint32_t k = 0; k < ITEMS; k++) {
    const uint64_t b = wbase + k * 32 + lane;
    const uint32_t p = r[k].parent;
    if (b >= a.nblocks || p == NONE) continue;
    if (p >= b || p >= a.nstruct_blocks) {
      atomicOr(err, ERR_BOUNDS);
      continue;
    }
    const uint64_t poff = p >= base ? s_off[p - base] : __ldg(&a.soff[p]);
    const uint64_t slot = poff + r[k].slot_off;
    if (slot + 8 > a.data_bytes || (slot & 7)) {
      atomicOr(err, ERR_BOUNDS);
      continue;
    }
    uint64_t* sp = reinterpret_cast<uint64_t*>(a.arena + slot);
    if (a.verify && *sp != a.hostp[b]) atomicOr(err, ERR_VERIFY);
    *sp = reinterpret_cast<uint64_t>(a.arena) + ex[k];
  }
  __syncthreads();  // s_off and s_warp are reused by the next tile
}

__global__ void __launch_bounds__(RELOC_THREADS) relocate_kernel(RelocArgs a) {
  __shared__ uint64_t s_off[RELOC_TILE];
  __shared__ uint64_t s_warp[RELOC_THREADS / 32];
  for (uint32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) reloc_tile<RELOC_THREADS>(a, t, s_off, s_warp);
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

template <typename T, int KIND>
__global__ void __launch_bounds__(LEAF_THREADS) leaf_kernel(LeafArgs a) {
  for (uint64_t t = blockIdx.x; t * LEAF_TILE < a.units; t += gridDim.x) leaf_tile<T, KIND, LEAF_THREADS>(a, t);
}

// Relocation and leaf update in one persistent launch: work item w < the
// relocation's tile count is a relocation tile, the rest are leaf tiles.  The
// two are independent (the leaf kernel works through addresses resolved on
// the host, the relocation writes only pointer slots), so one launch over a
// forest replaces two per structure.
template <typename T, int KIND, uint32_t THREADS>
__global__ void __launch_bounds__(THREADS) fused_kernel(RelocArgs r, LeafArgs l, uint64_t leaf_tiles) {
  __shared__ uint64_t s_off[RELOC_TILE];
  __shared__ uint64_t s_warp[THREADS / 32];
  const uint64_t total = (uint64_t)r.ntiles + leaf_tiles;
  for (uint64_t w = blockIdx.x; w < total; w += gridDim.x) {
    if (w < r.ntiles)
      reloc_tile<THREADS>(r, (uint32_t)w, s_off, s_warp);
    else
      leaf_tile<T, KIND, THREADS>(l, w - r.ntiles);
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
  for (uint64_t t = blockIdx.x; t * LEAF_TILE < a.units; t += gridDim.x) {
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

template <typename K>
int occupancy(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
  return n;
}

}  // namespace

cudaError_t launch_relocate(const RelocArgs& a, cudaStream_t s, int sm_count) {
  (void)sm_count;
  uint32_t grid = a.ntiles;  // one tile per CTA; the block scheduler overlaps their phases
  if (grid == 0) grid = 1;
  relocate_kernel<<<grid, RELOC_THREADS, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_leaf(const LeafArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nseg == 0) return cudaSuccess;
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  auto go = [&](auto kernel) {
    static int occ = 0;
    if (!occ) occ = occupancy(kernel, LEAF_THREADS, 0);
    uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
    kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
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
    static int occ = 0;
    if (!occ) occ = occupancy(kernel, CHASE_THREADS, 0);
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
  switch (threads) {
    case 128: return go(fused_kernel<T, KIND, 128>, 128);
    case 512: return go(fused_kernel<T, KIND, 512>, 512);
    default: return go(fused_kernel<T, KIND, 256>, 256);
  }
}
}  // namespace

cudaError_t launch_fused(const RelocArgs& r, const LeafArgs& l, uint32_t threads, uint32_t ctas_per_sm, int sm_count,
                         cudaStream_t s, int* max_per_sm) {
  if (l.f64)
    return l.kind == DC_OP_AXPY_HALF ? fused_go<double, DC_OP_AXPY_HALF>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm)
                                     : fused_go<double, DC_OP_SCALE>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm);
  return l.kind == DC_OP_AXPY_HALF ? fused_go<float, DC_OP_AXPY_HALF>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm)
                                   : fused_go<float, DC_OP_SCALE>(r, l, threads, ctas_per_sm, sm_count, s, max_per_sm);
}

cudaError_t launch_move(const MoveArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nd == 0) return cudaSuccess;
  static int occ = occupancy(move_kernel, LEAF_THREADS, 0);
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
  move_kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_stream(const StreamArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nseg == 0) return cudaSuccess;
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  auto go = [&](auto kernel) {
    static int occ = 0;
    if (!occ) occ = occupancy(kernel, LEAF_THREADS, 0);
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
