// kernels.cu — device side of the deep-copy hot path (sm_103a).
//
//   relocate_kernel  Fig 2 step d / Algorithm 1's attach loop: one pass that
//                    computes every block's arena offset (an exclusive scan of
//                    the 16-byte block sizes, warp shuffles inside a tile and
//                    decoupled look-back across tiles) and rewrites the pointer
//                    slot that refers to each block with the block's device
//                    address.  Block records are read as 16-byte vectors.
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
//   walk_kernel      one thread follows a chain and reports the address.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.hpp"

namespace dc {

namespace {

constexpr uint32_t FLAG_AGG = 1, FLAG_PREFIX = 2;
constexpr uint32_t SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// look-back status word: epoch (22 bits) | flag (2 bits) | inclusive/aggregate
// sum of 16-byte units (40 bits)
__device__ __forceinline__ unsigned long long pack(uint32_t epoch, uint32_t flag, uint64_t v) {
  return ((unsigned long long)epoch << 42) | ((unsigned long long)flag << 40) |
         (v & ((1ull << 40) - 1));
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= (uint32_t)d) v += o;
  }
  return v;
}

// Warp 0 of a CTA: publish this tile's aggregate, then look back over the
// predecessors 32 at a time until a tile with an inclusive prefix is found
// (decoupled look-back).  Returns the exclusive prefix (lane 0 publishes the
// inclusive one).  Every wait is bounded; on a timeout the error word is set.
__device__ uint64_t look_back(const RelocArgs& a, uint32_t t, uint64_t tile_sum, uint32_t lane) {
  uint32_t* err = &a.ctrl[CTRL_ERR];
  if (t == 0) {
    if (lane == 0) st_release(&a.status[0], pack(a.epoch, FLAG_PREFIX, tile_sum));
    return 0;
  }
  if (lane == 0) st_release(&a.status[t], pack(a.epoch, FLAG_AGG, tile_sum));
  uint64_t prefix = 0;
  int64_t top = (int64_t)t - 1;  // window: predecessors top, top-1, ..., top-31
  uint32_t spins = 0;
  while (top >= 0) {
    const int64_t j = top - (int64_t)lane;
    uint32_t fl = FLAG_PREFIX;  // before tile 0: an empty prefix
    uint64_t v = 0;
    if (j >= 0) {
      unsigned long long w = ld_acquire(&a.status[j]);
      fl = ((uint32_t)(w >> 42) == a.epoch) ? (uint32_t)(w >> 40) & 3u : 0u;
      v = w & ((1ull << 40) - 1);
    }
    if (__any_sync(0xffffffffu, fl == 0)) {
      if (++spins > SPIN_LIMIT || (ld_relaxed(err) & ERR_TIMEOUT)) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    const uint32_t pmask = __ballot_sync(0xffffffffu, fl == FLAG_PREFIX);
    const uint32_t stop = pmask ? (uint32_t)(__ffs(pmask) - 1) : 31u;  // closest prefix in the window
    uint64_t part = lane <= stop ? v : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    prefix += part;
    if (pmask) break;
    top -= 32;
  }
  if (lane == 0) st_release(&a.status[t], pack(a.epoch, FLAG_PREFIX, prefix + tile_sum));
  return prefix;
}

__global__ void __launch_bounds__(RELOC_THREADS) relocate_kernel(RelocArgs a) {
  constexpr uint32_t NW = RELOC_THREADS / 32;
  __shared__ uint64_t s_off[RELOC_TILE];
  __shared__ uint64_t s_warp[NW];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t s_tile;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* err = &a.ctrl[CTRL_ERR];
  uint32_t ready_tile = NONE;  // last parent tile this thread saw ready

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&a.ctrl[CTRL_TILE], 1u);
    __syncthreads();
    const uint32_t t = s_tile;
    if (t >= a.ntiles) break;
    const uint64_t base = (uint64_t)t * RELOC_TILE;

    // this thread's blocks: base + tid*ITEMS + k (one 16-byte record each)
    BlockRec r[RELOC_ITEMS];
    uint64_t local = 0;
#pragma unroll
    for (uint32_t k = 0; k < RELOC_ITEMS; k++) {
      uint64_t b = base + tid * RELOC_ITEMS + k;
      if (b < a.nblocks) {
        uint4 v = __ldg(reinterpret_cast<const uint4*>(a.rec) + b);
        r[k] = BlockRec{v.x, v.y, v.z, v.w};
      } else {
        r[k] = BlockRec{0, NONE, 0, 0};
      }
      local += r[k].size16;
    }
    // tile-wide exclusive scan of the block sizes
    uint64_t incl = warp_incl_scan(local, lane);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = lane < NW ? s_warp[lane] : 0;
      w = warp_incl_scan(w, lane);
      if (lane < NW) s_warp[lane] = w;
      __syncwarp();
      const uint64_t pre = look_back(a, t, __shfl_sync(0xffffffffu, w, NW - 1), lane);
      if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    const uint64_t excl = (warp ? s_warp[warp - 1] : 0) + incl - local;

    // byte offsets of this thread's blocks; struct blocks publish theirs
    uint64_t o16 = s_prefix + excl;
    uint64_t off[RELOC_ITEMS];
#pragma unroll
    for (uint32_t k = 0; k < RELOC_ITEMS; k++) {
      uint64_t b = base + tid * RELOC_ITEMS + k;
      off[k] = o16 * 16;
      s_off[tid * RELOC_ITEMS + k] = off[k];
      if (b < a.nstruct_blocks) a.soff[b] = off[k];
      o16 += r[k].size16;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(&a.ready[t], a.epoch);
    }

    // rewrite the slot that points at each block (the root has none)
#pragma unroll
    for (uint32_t k = 0; k < RELOC_ITEMS; k++) {
      uint64_t b = base + tid * RELOC_ITEMS + k;
      uint32_t p = r[k].parent;
      if (b >= a.nblocks || p == NONE) continue;
      if (p >= b || p >= a.nstruct_blocks) {
        atomicOr(err, ERR_BOUNDS);
        continue;
      }
      uint64_t poff;
      if (p >= base) {
        poff = s_off[p - base];
      } else {
        const uint32_t pt = p / RELOC_TILE;
        if (pt != ready_tile) {
          uint32_t spins = 0;
          bool ok = true;
          while (ld_acquire(&a.ready[pt]) != a.epoch) {
            if (++spins > SPIN_LIMIT || (ld_relaxed(err) & ERR_TIMEOUT)) {
              atomicOr(err, ERR_TIMEOUT);
              ok = false;
              break;
            }
            __nanosleep(32);
          }
          if (!ok) continue;
          ready_tile = pt;
        }
        poff = *(volatile const uint64_t*)&a.soff[p];
      }
      uint64_t slot = poff + r[k].slot_off;
      if (slot + 8 > a.data_bytes || (slot & 7)) {
        atomicOr(err, ERR_BOUNDS);
        continue;
      }
      uint64_t* sp = reinterpret_cast<uint64_t*>(a.arena + slot);
      if (a.verify && *sp != a.hostp[b]) atomicOr(err, ERR_VERIFY);
      *sp = reinterpret_cast<uint64_t>(a.arena) + off[k];
    }
    __syncthreads();  // s_tile / s_off / s_prefix are reused by the next tile
  }

  // the last CTA out resets the tile counter for the next launch
  if (tid == 0) {
    __threadfence();
    uint32_t d = atomicAdd(&a.ctrl[CTRL_DONE], 1u);
    if (d == gridDim.x - 1) {
      atomicExch(&a.ctrl[CTRL_TILE], 0u);
      atomicExch(&a.ctrl[CTRL_DONE], 0u);
    }
  }
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

template <typename T, int KIND>
__global__ void __launch_bounds__(LEAF_THREADS) leaf_kernel(LeafArgs a) {
  using VT = typename V16<T>::type;
  constexpr int EPU = V16<T>::N;
  const T sc = (T)a.scale;
  const Segment* seg = a.seg;
  auto ub = [&](uint32_t s) { return __ldg(&seg[s].ubeg); };
  for (uint64_t t = blockIdx.x; t * LEAF_TILE < a.units; t += gridDim.x) {
    const uint64_t u0 = t * LEAF_TILE;
    // the tile's segments are [lo, hi]; most tiles lie inside one segment
    const uint32_t lo = __ldg(&a.tile_seg[t]), hi = __ldg(&a.tile_seg[t + 1]);
    VT xv[LEAF_UNROLL], yv[LEAF_UNROLL];
    VT* xp[LEAF_UNROLL];
    const VT* yp[LEAF_UNROLL];
    uint32_t tail[LEAF_UNROLL];  // elements of this unit; EPU = a full vector
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {
      const uint64_t u = u0 + threadIdx.x + k * LEAF_THREADS;
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
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {
      if (tail[k] == EPU) {
        xv[k] = ldcs(xp[k]);
        if (KIND == DC_OP_AXPY_HALF) yv[k] = ldcs(yp[k]);
      }
    }
#pragma unroll
    for (uint32_t k = 0; k < LEAF_UNROLL; k++) {
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
  static int occ = occupancy(relocate_kernel, RELOC_THREADS, 0);
  uint32_t grid = (uint32_t)std::min<uint64_t>(a.ntiles, (uint64_t)sm_count * occ);
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

cudaError_t launch_move(const MoveArgs& a, cudaStream_t s, int sm_count) {
  if (a.units == 0 || a.nd == 0) return cudaSuccess;
  static int occ = occupancy(move_kernel, LEAF_THREADS, 0);
  uint64_t tiles = (a.units + LEAF_TILE - 1) / LEAF_TILE;
  uint32_t grid = (uint32_t)std::min<uint64_t>(tiles, (uint64_t)sm_count * occ);
  move_kernel<<<grid, LEAF_THREADS, 0, s>>>(a);
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
