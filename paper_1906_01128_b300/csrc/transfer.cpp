// transfer.cpp — moving a plan's blocks between host memory and the arena.
//
// The data region travels in one of two ways:
//   staged (default)  every block is marshalled into the plan's pinned arena
//                     (Algorithm 1: one contiguous buffer) by host threads and
//                     sent by DMA in chunks, each chunk as soon as it is
//                     marshalled.
//   mapped (DC_PLAN_MAP_HOST)  the whole pages strictly inside each large
//                     array are page-locked in place, and one move-kernel launch
//                     reads them straight from the caller's memory (one
//                     transfer per effective-address array, as in the paper's
//                     pointerchain scheme, Sec. 4.1.1 item 3, but all arrays in
//                     one launch); array heads/tails, small arrays and structs
//                     are marshalled meanwhile and moved by a second launch.
//                     The copy back writes array interiors straight back.
// Only pages wholly inside an array are registered, so no other object's bytes
// are ever page-locked.  A staged plan of many small blocks copies whole host
// spans instead of single blocks (span staging, spans.cpp); the staged copy back
// is a DMA into the pinned arena in chunks and a host scatter per chunk.
#include <immintrin.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <memory>

#include "internal.hpp"

namespace dc {

namespace {

// The host side's granularity (overridable when building, for measurements).
#ifndef DC_PIECE_BYTES
#define DC_PIECE_BYTES (512ull << 10)
#endif
#ifndef DC_UNIT_BYTES
#define DC_UNIT_BYTES (256ull << 10)
#endif
#ifndef DC_CHUNK_BYTES
#define DC_CHUNK_BYTES (16ull << 20)
#endif
#ifndef DC_BACK_CHUNK_BYTES
#define DC_BACK_CHUNK_BYTES (8ull << 20)
#endif
constexpr uint64_t PIECE_BYTES = DC_PIECE_BYTES;  // largest memcpy one host thread does at once
constexpr uint64_t UNIT_BYTES = DC_UNIT_BYTES;    // host work handed out at once
constexpr uint64_t UNIT_PIECES = 4096;
constexpr uint64_t CHUNK_BYTES = DC_CHUNK_BYTES;  // staged bytes per DMA chunk
constexpr uint64_t BACK_CHUNK_BYTES = DC_BACK_CHUNK_BYTES;  // copied-back bytes per DMA chunk
constexpr uint64_t PAGE = 4096;

uint64_t page_up(uint64_t x) { return (x + PAGE - 1) / PAGE * PAGE; }
uint64_t page_down(uint64_t x) { return x / PAGE * PAGE; }

}  // namespace

uint64_t interior_bytes(const HostBlock& b) {
  if (in_host_arena(b.host, b.bytes, nullptr)) return b.bytes;  // the whole block
  if (b.lane == 0) return 0;  // struct blocks always go through the pinned arena
  const uint64_t h = (uint64_t)(uintptr_t)b.host;
  const uint64_t lo = page_up(h), hi = page_down(h + b.bytes);
  return hi > lo && hi - lo >= DC_MAP_MIN_BYTES ? hi - lo : 0;
}

void plan_moves(const dc_plan_s* p, const std::vector<uint32_t>& list, dc_plan_s::Moves* m, bool host_order,
                uint64_t chunk_bytes, bool stage_all) {
  *m = dc_plan_s::Moves();
  if (!chunk_bytes) chunk_bytes = CHUNK_BYTES;
  for (uint32_t b : list) {
    const HostBlock& B = p->blocks[b];
    uint8_t* host = const_cast<uint8_t*>(B.host);
    if (!stage_all && p->ihi[b] > p->ilo[b]) {
      m->interiors.push_back(b);
      const uint64_t head = p->ilo[b] - (uint64_t)(uintptr_t)host;
      const uint64_t tail = p->ihi[b] - (uint64_t)(uintptr_t)host;
      if (head) m->frags.push_back({B.off, head, host});
      if (tail < B.bytes) m->frags.push_back({B.off + tail, B.bytes - tail, host + tail});
    } else {
      m->frags.push_back({B.off, B.bytes, host});
    }
  }
  split_moves(m, host_order, chunk_bytes);
}

// The second half of planning a transfer: m->frags split into pieces and work
// units, the runs of the destination range, and (arena order) DMA chunks.
void split_moves(dc_plan_s::Moves* m, bool host_order, uint64_t chunk_bytes) {
  if (!chunk_bytes) chunk_bytes = CHUNK_BYTES;
  for (const auto& f : m->frags)
    for (uint64_t o = 0; o < f.len; o += PIECE_BYTES)
      m->pieces.push_back({f.off + o, std::min(PIECE_BYTES, f.len - o), f.host + o});
  if (host_order)
    std::sort(m->pieces.begin(), m->pieces.end(), [](const dc_plan_s::Frag& a, const dc_plan_s::Frag& b) {
      return a.host < b.host;
    });
  for (uint64_t i = 0; i < m->pieces.size();) {
    uint64_t j = i, bytes = 0;
    while (j < m->pieces.size() && bytes < UNIT_BYTES && j - i < UNIT_PIECES) bytes += m->pieces[j++].len;
    m->units.push_back({i, j});
    i = j;
  }
  // runs: fragments separated only by block padding travel together
  for (const auto& f : m->frags) {
    if (!m->runs.empty() && f.off - m->runs.back().hi < 16)
      m->runs.back().hi = f.off + f.len;
    else
      m->runs.push_back({f.off, f.off + f.len});
  }
  if (host_order) return;
  // chunks of ~CHUNK_BYTES of staged bytes, with the runs clipped to them
  size_t r = 0;
  for (uint64_t u = 0; u < m->units.size();) {
    uint64_t v = u, bytes = 0;
    while (v < m->units.size() && bytes < chunk_bytes) {
      for (uint64_t k = m->units[v].first; k < m->units[v].last; k++) bytes += m->pieces[k].len;
      v++;
    }
    const uint64_t lo = m->pieces[m->units[u].first].off;
    const uint64_t hi = v < m->units.size() ? m->pieces[m->units[v].first].off : ~0ull;
    const uint64_t cfirst = m->copies.size();
    while (r < m->runs.size() && m->runs[r].lo < hi) {
      const uint64_t a = std::max(m->runs[r].lo, lo), b = std::min(m->runs[r].hi, hi);
      if (b > a) m->copies.push_back({a, b});
      if (m->runs[r].hi <= hi)
        r++;
      else
        break;
    }
    m->chunks.push_back({u, v, cfirst, m->copies.size()});
    u = v;
  }
}

void plan_transfers(dc_plan_s* p) {
  const uint64_t nb = p->blocks.size();
  p->ilo.assign(nb, 0);
  p->ihi.assign(nb, 0);
  p->idev.assign(nb, 0);
  {  // blocks in a host arena: the GPU reads and writes them in place (struct
     // blocks with NULL-slot fix-ups excepted: those go through the pinned arena)
    const std::vector<uint8_t> fixup = null_fixups(p);
    for (uint32_t b = 0; b < nb; b++) {
      uint64_t dev;
      const HostBlock& B = p->blocks[b];
      if (fixup[b] || !in_host_arena(B.host, B.bytes, &dev)) continue;
      p->ilo[b] = (uint64_t)(uintptr_t)B.host;
      p->ihi[b] = p->ilo[b] + B.bytes;
      p->idev[b] = dev;
      p->has_arena_blocks = true;
    }
  }
  if (p->flags & DC_PLAN_MAP_HOST) {
    for (uint32_t b = 0; b < nb; b++) {
      const HostBlock& B = p->blocks[b];
      if (p->ihi[b] > p->ilo[b] || !interior_bytes(B)) continue;
      const uint64_t lo = page_up((uint64_t)(uintptr_t)B.host), hi = page_down((uint64_t)(uintptr_t)B.host + B.bytes);
      void* dptr = nullptr;
      if (cudaHostRegister((void*)lo, hi - lo, cudaHostRegisterMapped) != cudaSuccess) {
        cudaGetLastError();  // not a sticky error: this array is staged instead
        continue;
      }
      p->registered.push_back({(void*)lo, hi - lo});
      if (cudaHostGetDevicePointer(&dptr, (void*)lo, 0) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      p->ilo[b] = lo;
      p->ihi[b] = hi;
      p->idev[b] = (uint64_t)(uintptr_t)dptr;
    }
  }
  std::vector<uint32_t> all(nb);
  for (uint32_t b = 0; b < nb; b++) all[b] = b;
  plan_moves(p, all, &p->h2d, (p->flags & DC_PLAN_MAP_HOST) != 0);  // staged copies go chunk by chunk
  p->h2d_span = dc_plan_s::Moves();
  p->span_nulls.clear();
  if (p->span_mode) {  // the spans move instead, in staging order, chunk by chunk
    for (const HostSpan& S : p->spans) p->h2d_span.frags.push_back({S.stage, S.bytes, const_cast<uint8_t*>(S.host)});
    split_moves(&p->h2d_span, false, 0);
    p->span_nulls = span_null_offsets(p);
  }
  p->transfers_ready = true;
}

void release_transfers(dc_plan_s* p) {
  for (auto& r : p->registered) cudaHostUnregister(r.first);
  p->registered.clear();
}

// Upload a move table (descriptors + per-tile first descriptor) on `s`.  The
// sources are pageable vectors: cudaMemcpyAsync returns once it has staged
// them, so they may go away afterwards.
dc_status upload(dc_plan_s* p, const std::vector<MoveDesc>& d, uint64_t desc_off, uint64_t tile_off, uint64_t cap,
                 uint64_t* nd, uint64_t* units, cudaStream_t s) {
  *nd = d.size();
  *units = d.empty() ? 0 : d.back().ubeg + (d.back().bytes + 15) / 16;
  if (d.empty()) return DC_OK;
  if (d.size() > cap) return fail(DC_EINVAL, "move table larger than planned");
  std::vector<uint32_t> tiles;
  const uint64_t ntiles = (*units + LEAF_TILE - 1) / LEAF_TILE;
  if (ntiles + 1 > p->L.tseg_cap) return fail(DC_EINVAL, "move tile table larger than planned");
  for (uint64_t t = 0, k = 0; t < ntiles; t++) {
    while (k + 1 < d.size() && d[k + 1].ubeg <= t * LEAF_TILE) k++;
    tiles.push_back((uint32_t)k);
  }
  tiles.push_back((uint32_t)(d.size() - 1));
  DC_CUDA(cudaMemcpyAsync(p->dev + desc_off, d.data(), d.size() * sizeof(MoveDesc), cudaMemcpyHostToDevice, s));
  DC_CUDA(cudaMemcpyAsync(p->dev + tile_off, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, s));
  return DC_OK;
}

void push_desc(std::vector<MoveDesc>* d, uint64_t src, uint64_t dst, uint64_t bytes) {
  uint64_t u = d->empty() ? 0 : d->back().ubeg + (d->back().bytes + 15) / 16;
  d->push_back({src, dst, bytes, u});
}

dc_status launch_table(dc_plan_s* p, uint64_t desc_off, uint64_t tile_off, uint64_t nd, uint64_t units,
                       cudaStream_t s) {
  if (!nd) return DC_OK;
  MoveArgs a;
  a.d = reinterpret_cast<const MoveDesc*>(p->dev + desc_off);
  a.tile_desc = reinterpret_cast<const uint32_t*>(p->dev + tile_off);
  a.nd = (uint32_t)nd;
  a.units = units;
  DC_CUDA(launch_move(a, s, p->sm_count));
  return DC_OK;
}

namespace {

// Copies of at least NT_MIN bytes use streaming stores: the destination lines are written without
// being read first (a plain copy reads every destination line before writing it), and they do
// not displace the cache.  The store fence at the end makes them visible before the copy returns.
#ifndef DC_NT_MIN
#define DC_NT_MIN 4096
#endif
constexpr size_t NT_MIN = DC_NT_MIN;

__attribute__((target("avx2"))) void copy_stream(uint8_t* dst, const uint8_t* src, size_t n) {
  const size_t head = (32 - ((uintptr_t)dst & 31)) & 31;
  memcpy(dst, src, head);
  dst += head;
  src += head;
  n -= head;
  size_t i = 0;
  for (; i + 128 <= n; i += 128) {
    const __m256i a = _mm256_loadu_si256(reinterpret_cast<const __m256i*>(src + i));
    const __m256i b = _mm256_loadu_si256(reinterpret_cast<const __m256i*>(src + i + 32));
    const __m256i c = _mm256_loadu_si256(reinterpret_cast<const __m256i*>(src + i + 64));
    const __m256i d = _mm256_loadu_si256(reinterpret_cast<const __m256i*>(src + i + 96));
    _mm256_stream_si256(reinterpret_cast<__m256i*>(dst + i), a);
    _mm256_stream_si256(reinterpret_cast<__m256i*>(dst + i + 32), b);
    _mm256_stream_si256(reinterpret_cast<__m256i*>(dst + i + 64), c);
    _mm256_stream_si256(reinterpret_cast<__m256i*>(dst + i + 96), d);
  }
  memcpy(dst + i, src + i, n - i);
  _mm_sfence();
}

void copy_block(uint8_t* dst, const uint8_t* src, size_t n) {
  static const bool avx2 = __builtin_cpu_supports("avx2");
  if (avx2 && n >= NT_MIN)
    copy_stream(dst, src, n);
  else
    memcpy(dst, src, n);
}

}  // namespace

void host_copy(dc_plan_s* p, const dc_plan_s::Moves& m, uint64_t ufirst, uint64_t ulast, bool to_arena) {
  auto unit = [&](uint64_t u) {
    for (uint64_t k = m.units[u].first; k < m.units[u].last; k++) {
      const auto& pc = m.pieces[k];
      if (to_arena)
        copy_block(p->pinned + pc.off, pc.host, pc.len);
      else
        copy_block(pc.host, p->pinned + pc.off, pc.len);
    }
  };
  Pool& pool = *p->pool;
  if (ulast - ufirst <= 1 || pool.size() == 1) {
    for (uint64_t u = ufirst; u < ulast; u++) unit(u);
  } else {
    pool.parallel_for(ulast - ufirst, [&](uint64_t i) { unit(ufirst + i); });
  }
}

void null_slots_upto(dc_plan_s* p, size_t* ns, uint64_t hi) {
  while (*ns < p->null_slots.size() && p->null_slots[*ns] < hi) {
    memset(p->pinned + p->null_slots[*ns], 0, 8);
    (*ns)++;
  }
}

dc_status upload_h2d_tables(dc_plan_s* p, cudaStream_t s) {
  const uint64_t base = (uint64_t)(uintptr_t)p->dev;
  std::vector<MoveDesc> d;
  for (uint32_t b : p->h2d.interiors)
    push_desc(&d, p->idev[b], base + p->blocks[b].off + (p->ilo[b] - (uint64_t)(uintptr_t)p->blocks[b].host),
              p->ihi[b] - p->ilo[b]);
  dc_status st = upload(p, d, p->L.mva, p->L.mvat, p->L.tab_cap, &p->h2d_int_nd, &p->h2d_int_units, s);
  if (st) return st;
  d.clear();
  if (p->flags & DC_PLAN_MAP_HOST)  // the staged bytes also move by kernel, from the mapped pinned arena
    for (const auto& r : p->h2d.runs) push_desc(&d, (uint64_t)(uintptr_t)p->pinned_dev + r.lo, base + r.lo, r.hi - r.lo);
  st = upload(p, d, p->L.mvb, p->L.mvbt, p->L.tab_cap, &p->h2d_frag_nd, &p->h2d_frag_units, s);
  if (st || !p->span_mode) return st;
  std::vector<PlaceDesc> pd;
  build_place_table(p, &pd);
  if (pd.size() > p->L.spd_cap) return fail(DC_EINVAL, "placement table larger than planned");
  p->span_nd = pd.size();
  if (!pd.empty())
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.spd, pd.data(), pd.size() * sizeof(PlaceDesc), cudaMemcpyHostToDevice, s));
  return DC_OK;
}

dc_status transfer_to_device(dc_plan_s* p, cudaStream_t s) {
  const dc_plan_s::Moves& m = p->h2d;
  // array interiors: one launch reads them all from the caller's pages
  dc_status st = launch_table(p, p->L.mva, p->L.mvat, p->h2d_int_nd, p->h2d_int_units, s);
  if (st) return st;
  size_t ns = 0;
  if (p->flags & DC_PLAN_MAP_HOST) {
    {
      Trace tr("dc_deep_copy", "marshal");
      host_copy(p, m, 0, m.units.size(), true);
      null_slots_upto(p, &ns, ~0ull);
    }
    return launch_table(p, p->L.mvb, p->L.mvbt, p->h2d_frag_nd, p->h2d_frag_units, s);
  }
  if (p->span_mode) {  // the spans into the staging region, then every block to its place
    st = send_staged(p, p->h2d_span, p->span_nulls, p->dev + p->L.spn, s);
    if (st) return st;
    PlaceArgs a;
    a.d = reinterpret_cast<const PlaceDesc*>(p->dev + p->L.spd);
    a.nd = p->span_nd;
    a.stage = p->dev + p->L.spn;
    a.arena = p->dev;
    a.stage_bytes = p->L.spd - p->L.spn;  // the region, rounded up: 16-byte reads of a piece's last vector stay inside
    a.data_bytes = p->data_bytes;
    a.err = reinterpret_cast<uint32_t*>(p->dev + p->L.ctrl) + CTRL_ERR;
    DC_CUDA(launch_place(a, s, p->sm_count));
    return DC_OK;
  }
  return send_staged(p, m, p->null_slots, p->dev, s);
}

// Algorithm 1's contiguous buffer.  The pool's threads take the work units in
// destination order (the arena's, or the span staging area's) without stopping
// at chunk ends; each unit zeroes the NULL slots in its range after its copies,
// and the thread that finishes a chunk's last unit queues the chunk's DMA to
// `dev`, so the link starts on a chunk as soon as its bytes are in the pinned
// arena.
dc_status send_staged(dc_plan_s* p, const dc_plan_s::Moves& m, const std::vector<uint64_t>& nulls, uint8_t* dev,
                      cudaStream_t s) {
  Trace tr("dc_deep_copy", "marshal+copies");
  const size_t nc = m.chunks.size();
  if (!nc) return DC_OK;
  std::vector<uint32_t> unit_chunk(m.units.size());
  std::unique_ptr<std::atomic<uint64_t>[]> left(new std::atomic<uint64_t>[nc]);
  for (size_t c = 0; c < nc; c++) {
    const auto& ch = m.chunks[c];
    for (uint64_t u = ch.ufirst; u < ch.ulast; u++) unit_chunk[u] = (uint32_t)c;
    left[c].store(ch.ulast - ch.ufirst);
  }
  std::atomic<int> failed{0};
  cudaError_t first = cudaSuccess;
  auto finish_chunk = [&](size_t c) {
    const auto& ch = m.chunks[c];
    for (uint64_t k = ch.cfirst; k < ch.clast; k++) {
      const cudaError_t e = cudaMemcpyAsync(dev + m.copies[k].lo, p->pinned + m.copies[k].lo,
                                            m.copies[k].hi - m.copies[k].lo, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess && failed.exchange(1) == 0) first = e;
    }
  };
  auto unit = [&](uint64_t u) {
    const uint64_t k0 = m.units[u].first, k1 = m.units[u].last;
    for (uint64_t k = k0; k < k1; k++) {
      const auto& pc = m.pieces[k];
      copy_block(p->pinned + pc.off, pc.host, pc.len);
    }
    // the NULL-slot fix-ups of the unit's range, clipped to it: a slot that
    // straddles two units is zeroed by each for its own bytes, after its copy
    const uint64_t lo = m.pieces[k0].off, hi = m.pieces[k1 - 1].off + m.pieces[k1 - 1].len;
    for (auto it = std::lower_bound(nulls.begin(), nulls.end(), lo >= 7 ? lo - 7 : 0); it != nulls.end() && *it < hi;
         ++it) {
      const uint64_t a = std::max(*it, lo), b = std::min(*it + 8, hi);
      if (b > a) memset(p->pinned + a, 0, b - a);
    }
    const uint32_t c = unit_chunk[u];
    if (left[c].fetch_sub(1, std::memory_order_acq_rel) == 1) finish_chunk(c);
  };
  pool_of(p).parallel_for(m.units.size(), unit);
  if (failed.load()) return cuda_fail(first, "cudaMemcpyAsync (deep copy chunk)");
  return DC_OK;
}

// The copy back: array interiors in mapped caller pages go by one move-kernel
// launch straight into those pages; every other written byte goes by DMA into
// the pinned arena in chunks of about BACK_CHUNK_BYTES, each with an event, and
// the pool scatters chunk c into the caller's arrays while the chunks after it
// are still on the link.  The device's error word is read first (after
// every kernel queued before the copy back): if a kernel recorded an error,
// nothing is scattered and the error is returned.
dc_status transfer_back(dc_plan_s* p, const std::vector<uint32_t>& list, uint64_t key, cudaStream_t s) {
  if (key != p->back_key) {
    std::vector<uint32_t> sorted(list);  // chunks follow arena order
    std::sort(sorted.begin(), sorted.end());
    plan_moves(p, sorted, &p->back, false, BACK_CHUNK_BYTES);
    const uint64_t base = (uint64_t)(uintptr_t)p->dev;
    std::vector<MoveDesc> d;
    for (uint32_t b : p->back.interiors)  // interiors straight into the caller's pages
      push_desc(&d, base + p->blocks[b].off + (p->ilo[b] - (uint64_t)(uintptr_t)p->blocks[b].host), p->idev[b],
                p->ihi[b] - p->ilo[b]);
    dc_status st = upload(p, d, p->L.bk, p->L.bkt, p->L.tab_cap, &p->bk_nd, &p->bk_units, s);
    if (st) return st;
    p->back_key = key;
  }
  const dc_plan_s::Moves& m = p->back;
  if (!p->back_err) DC_CUDA(cudaEventCreateWithFlags(&p->back_err, cudaEventDisableTiming));
  while (p->back_ev.size() < m.chunks.size()) {
    cudaEvent_t e;
    DC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p->back_ev.push_back(e);
  }
  uint32_t* word = pinned_error_word(p);
  {
    Trace tr("dc_copy_back", "enqueue");
    DC_CUDA(cudaMemcpyAsync(word, p->dev + p->L.ctrl + CTRL_ERR * 4, 4, cudaMemcpyDeviceToHost, s));
    DC_CUDA(cudaEventRecord(p->back_err, s));
    dc_status st = launch_table(p, p->L.bk, p->L.bkt, p->bk_nd, p->bk_units, s);
    if (st) return st;
    for (size_t c = 0; c < m.chunks.size(); c++) {
      for (uint64_t k = m.chunks[c].cfirst; k < m.chunks[c].clast; k++)
        DC_CUDA(cudaMemcpyAsync(p->pinned + m.copies[k].lo, p->dev + m.copies[k].lo, m.copies[k].hi - m.copies[k].lo,
                                cudaMemcpyDeviceToHost, s));
      DC_CUDA(cudaEventRecord(p->back_ev[c], s));
    }
  }
  {
    Trace tr("dc_copy_back", "error word");
    dc_status st = wait_event(p->back_err);
    if (st) return st;
  }
  if (*word) return device_error(p, s);  // waits for the stream, clears the word and reports it
  Trace tr("dc_copy_back", "scatter");
  // One pass of the pool over every unit in arena order, with no stop between
  // chunks: the first thread to take a unit of chunk c waits for c's event
  // (polling and yielding its core) and marks c ready for the others.
  const size_t nc = m.chunks.size();
  std::vector<uint32_t> unit_chunk(m.units.size());
  for (size_t c = 0; c < nc; c++)
    for (uint64_t u = m.chunks[c].ufirst; u < m.chunks[c].ulast; u++) unit_chunk[u] = (uint32_t)c;
  std::unique_ptr<std::atomic<uint8_t>[]> ready(new std::atomic<uint8_t>[nc]);
  for (size_t c = 0; c < nc; c++) ready[c].store(0);
  std::atomic<int> failed{0};
  pool_of(p).parallel_for(m.units.size(), [&](uint64_t u) {
    const uint32_t c = unit_chunk[u];
    if (!ready[c].load(std::memory_order_acquire)) {
      if (wait_event(p->back_ev[c]) != DC_OK) {
        failed.store(1);
        return;
      }
      ready[c].store(1, std::memory_order_release);
    }
    for (uint64_t k = m.units[u].first; k < m.units[u].last; k++) {
      const auto& pc = m.pieces[k];
      copy_block(pc.host, p->pinned + pc.off, pc.len);
    }
  });
  if (failed.load()) return fail(DC_ECUDA, "copy back: a chunk's transfer failed");
  return sync_stream(p, s);  // the interiors' launch, when no chunk follows it
}

}  // namespace dc
