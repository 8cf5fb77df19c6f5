// runtime.cpp — the C ABI (include/dc.h): plan lifetime, device binding, the
// marshal + transfer + relocation of a deep copy (Fig 2; Algorithm 1), chain
// resolution (Sec. 3), the leaf kernels, copy back (Algorithm 2 step 5) and the
// managed-memory comparison path.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "internal.hpp"

using namespace dc;

static std::atomic<uint64_t> g_launches{0};
void dc::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

constexpr uint64_t WORD_AREA = 256;            // pinned words for small device -> host reads

uint64_t align256(uint64_t x) { return round_up(x, 256); }

DevLayout make_layout(const dc_plan_s* p) {
  DevLayout L;
  const uint64_t nb = p->blocks.size();
  uint64_t o = align256(p->data_bytes);
  const uint64_t nrec = std::max<uint64_t>(1, p->rrec.size());
  L.rec = o;  // relocation records, and two spare ones (copies of a tile's records start and end on 16 bytes)
  o = align256(o + (nrec + 2) * sizeof(RelocRec));
  L.hostp = o;  // per record: the target's host address
  o = align256(o + nrec * 8);
  L.soff = o;  // per record: the target's arena offset
  o = align256(o + nrec * 8);
  L.ntiles = p->rtiles.size();
  L.status = o;  // (tile, lane) groups
  o = align256(o + p->rseg.size() * sizeof(RelocSeg));
  L.rtile = o;  // per tile: its records and groups
  o = align256(o + std::max<uint64_t>(1, p->rtiles.size()) * sizeof(RelocTile));
  L.seltile = o;  // the tiles a selective deep copy relocates (a subset of the above)
  o = align256(o + std::max<uint64_t>(1, p->rtiles.size()) * sizeof(RelocTile));
  L.ctrl = o;
  o = align256(o + CTRL_WORDS * 4);
  // one leaf segment per selected struct, or with DC_PLAN_PACK_SMALL up to 8 for an
  // array off a 16-byte boundary (a head shorter than a vector, or pieces of one)
  L.seg_cap = std::max<uint64_t>(1, p->nstructs) * ((p->flags & DC_PLAN_PACK_SMALL) ? 8 : 1);
  L.seg = o;
  o = align256(o + L.seg_cap * sizeof(Segment));
  // every segment has at least one 16-byte unit and lives in the data region
  L.tseg_cap = (p->data_bytes / 16 + L.seg_cap) / LEAF_TILE + 2;
  L.tseg = o;
  o = align256(o + L.tseg_cap * 4);
  L.cseg = o;
  o = align256(o + L.seg_cap * sizeof(ChaseSeg));
  L.step_cap = std::max<uint64_t>(1, p->sum_depth);
  L.steps = o;
  o = align256(o + L.step_cap * sizeof(ChaseStep));
  // move tables: at most one descriptor per block plus two per array interior
  uint64_t interiors = 0;
  for (const auto& b : p->blocks) interiors += interior_bytes(b) ? 1 : 0;
  L.tab_cap = nb + 2 * interiors;
  for (uint64_t* t : {&L.mva, &L.mvat, &L.mvb, &L.mvbt, &L.bk, &L.bkt, &L.sta, &L.stat, &L.stb, &L.stbt}) {
    *t = o;
    bool tiles = (t == &L.mvat || t == &L.mvbt || t == &L.bkt || t == &L.stat || t == &L.stbt);
    o = align256(o + (tiles ? L.tseg_cap * 4 : L.tab_cap * sizeof(MoveDesc)));
  }
  L.sts = o;  // fused-step segments and their tile table
  o = align256(o + L.seg_cap * sizeof(StreamSeg));
  L.stst = o;
  o = align256(o + L.tseg_cap * 4);
  L.walk_cap = (uint64_t)p->max_depth + 2;
  L.walk = o;
  o = align256(o + L.walk_cap * sizeof(ChaseStep) + 16);
  if (p->span_mode) {  // the staged spans, and the placement table (a piece per PLACE_PIECE bytes of a block)
    L.spn = o;
    o = align256(o + p->span_bytes);
    L.spd_cap = nb + p->data_bytes / PLACE_PIECE + 1;
    L.spd = o;
    o = align256(o + L.spd_cap * sizeof(PlaceDesc));
  }
  L.total = o;
  return L;
}

// pinned table staging: [segments][tile table][chase segments][chase steps][walk steps][words]
uint64_t tab_seg(const DevLayout& L) { (void)L; return 0; }
uint64_t tab_tseg(const DevLayout& L) { return align256(L.seg_cap * sizeof(Segment)); }
uint64_t tab_cseg(const DevLayout& L) { return tab_tseg(L) + align256(L.tseg_cap * 4); }
uint64_t tab_steps(const DevLayout& L) { return tab_cseg(L) + align256(L.seg_cap * sizeof(ChaseSeg)); }
uint64_t tab_walk(const DevLayout& L) { return tab_steps(L) + align256(L.step_cap * sizeof(ChaseStep)); }
uint64_t tab_words(const DevLayout& L) { return tab_walk(L) + align256(L.walk_cap * sizeof(ChaseStep)); }
uint64_t tab_total(const DevLayout& L) { return tab_words(L) + WORD_AREA; }

unsigned default_threads() {
  unsigned hc = std::thread::hardware_concurrency();
  if (hc == 0) hc = 1;
  return std::min(hc, 32u);
}

}  // namespace

Pool& dc::pool_of(dc_plan_s* p) {
  if (!p->pool) {
    if (p->nthreads) {
      p->own_pool.reset(new Pool(p->nthreads));
      p->pool = p->own_pool.get();
    } else {  // plans share one pool: thousands of plans must not mean thousands of threads
      static Pool shared(default_threads());
      p->pool = &shared;
    }
  }
  return *p->pool;
}

uint32_t* dc::pinned_error_word(dc_plan_s* p) { return reinterpret_cast<uint32_t*>(p->pin_tab + tab_words(p->L)); }

dc_status dc::device_error(dc_plan_s* p, cudaStream_t s) {
  uint32_t* word = pinned_error_word(p);
  DC_CUDA(cudaMemcpyAsync(word, p->dev + p->L.ctrl + CTRL_ERR * 4, 4, cudaMemcpyDeviceToHost, s));
  dc_status st = sync_stream(p, s);
  if (st) return st;
  uint32_t e = *word;
  if (!e) return DC_OK;
  DC_CUDA(cudaMemsetAsync(p->dev + p->L.ctrl + CTRL_ERR * 4, 0, 4, s));
  if ((st = sync_stream(p, s))) return st;
  if (e & ERR_BOUNDS) return fail(DC_EDEVICE_BOUNDS, "a kernel found an offset outside its buffers (0x%x)", e);
  if (e & ERR_TIMEOUT) return fail(DC_ETIMEOUT, "a device-side wait gave up (0x%x)", e);
  return fail(DC_EVERIFY, "relocation check: a pointer slot did not hold the recorded host address");
}

OpKey dc::key_of(const dc_op* op) {
  OpKey k;
  k.kind = op->kind;
  k.sel = op->sel;
  k.type = op->type;
  k.x = op->x_field;
  k.y = op->kind == DC_OP_AXPY_HALF ? op->y_field : 0;
  if (op->sel == DC_SEL_CHAIN) k.path.assign(op->path, op->path + op->path_len);
  return k;
}

dc_status dc::pick(const dc_plan_s* p, const dc_op* op, std::vector<Pick>* out) {
  std::vector<std::pair<uint32_t, uint64_t>> sel;
  dc_status st = select_structs(p, op, &sel);
  if (st) return st;
  const SchemaCopy& S = p->schema;
  const uint32_t np = S.nptr[op->type];
  const int32_t ix = S.ptr_index[op->type][op->x_field];
  const int32_t iy = op->kind == DC_OP_AXPY_HALF ? S.ptr_index[op->type][op->y_field] : -1;
  out->clear();
  out->reserve(sel.size());
  for (auto& se : sel) {
    const uint64_t base = p->blocks[se.first].ptr_first + se.second * np;
    uint32_t bx = p->ptr_target[base + ix];
    uint32_t by = iy >= 0 ? p->ptr_target[base + iy] : NONE;
    if (iy >= 0) {
      uint64_t nx = bx == NONE ? 0 : p->blocks[bx].count, ny = by == NONE ? 0 : p->blocks[by].count;
      if (nx != ny) return fail(DC_EINVAL, "op: x has %llu elements but y has %llu", (unsigned long long)nx,
                                (unsigned long long)ny);
    }
    if (bx == NONE) continue;
    out->push_back({se.first, se.second, bx, by});
  }
  std::sort(out->begin(), out->end(), [&](const Pick& a, const Pick& b) { return a.bx < b.bx; });
  return DC_OK;
}

namespace {

// chase steps from its tree's root to struct (sblk, elem), appended to
// `steps`; returns the root block
uint32_t chain_steps(const dc_plan_s* p, uint32_t sblk, uint64_t elem, std::vector<ChaseStep>* steps) {
  size_t start = steps->size();
  const SchemaCopy& S = p->schema;
  while (p->blocks[sblk].parent != NONE) {
    const HostBlock& B = p->blocks[sblk];
    const HostBlock& P = p->blocks[B.parent];
    uint32_t psize = S.types[P.type].size;
    steps->push_back({B.slot_off % psize, S.types[B.type].size, elem});
    elem = B.slot_off / psize;
    sblk = B.parent;
  }
  std::reverse(steps->begin() + start, steps->end());
  return sblk;
}

}  // namespace

// Host waits for the GPU.  cudaEventSynchronize spins a core while it waits;
// the library's host threads (a server's slots, the pool) then keep cores from
// the threads that marshal and scatter.  With DC_YIELD_WAITS (the default) a
// waiting thread polls the event and yields the core between polls.
#ifndef DC_YIELD_WAITS
#define DC_YIELD_WAITS 1
#endif
dc_status dc::wait_event(cudaEvent_t e) {
  if (!e) return DC_OK;
#if DC_YIELD_WAITS
  for (;;) {
    const cudaError_t r = cudaEventQuery(e);
    if (r == cudaSuccess) return DC_OK;
    if (r != cudaErrorNotReady) return cuda_fail(r, "cudaEventQuery");
    std::this_thread::yield();
  }
#else
  DC_CUDA(cudaEventSynchronize(e));
  return DC_OK;
#endif
}

dc_status dc::sync_stream(dc_plan_s* p, cudaStream_t s) {
  if (!p->sync_ev) DC_CUDA(cudaEventCreateWithFlags(&p->sync_ev, cudaEventDisableTiming));
  DC_CUDA(cudaEventRecord(p->sync_ev, s));
  return wait_event(p->sync_ev);
}

namespace {

dc_status path_steps(const dc_plan_s* p, const dc_step* path, uint32_t len, std::vector<ChaseStep>* out) {
  uint32_t blk, ty;
  uint64_t within, elem;
  dc_status st = resolve(p, 0, path, len, &blk, &within, &ty, &elem);  // validates the chain
  if (st) return st;
  const SchemaCopy& S = p->schema;
  uint32_t ti = S.root_type;
  out->clear();
  for (uint32_t k = 0; k < len; k++) {
    const dc_field& F = S.fields[ti][path[k].field];
    uint32_t sz = F.kind == DC_F_ARRAY ? F.elem_size : S.types[F.child_type].size;
    out->push_back({F.offset, sz, path[k].index});
    if (F.kind == DC_F_CHILD) ti = (uint32_t)F.child_type;
  }
  return DC_OK;
}

}  // namespace

extern "C" {

const char* dc_last_error(void) { return last_error(); }

const char* dc_status_name(dc_status s) {
  switch (s) {
    case DC_OK: return "DC_OK";
    case DC_EINVAL: return "DC_EINVAL";
    case DC_ENOMEM: return "DC_ENOMEM";
    case DC_ECUDA: return "DC_ECUDA";
    case DC_EALIAS: return "DC_EALIAS";
    case DC_ECYCLE: return "DC_ECYCLE";
    case DC_EBUDGET: return "DC_EBUDGET";
    case DC_ETIMEOUT: return "DC_ETIMEOUT";
    case DC_EDEVICE_BOUNDS: return "DC_EDEVICE_BOUNDS";
    case DC_ESTATE: return "DC_ESTATE";
    case DC_EVERIFY: return "DC_EVERIFY";
  }
  return "unknown";
}

uint64_t dc_kernel_launches(void) { return g_launches.load(); }

dc_status dc_plan(const dc_schema* schema, const void* host_root, dc_plan_t* out) {
  if (!host_root) {
    if (out) *out = nullptr;
    return fail(DC_EINVAL, "host_root is NULL");
  }
  return dc_plan_forest(schema, &host_root, 1, out);
}

dc_status dc_plan_forest(const dc_schema* schema, const void* const* roots, uint64_t nroots, dc_plan_t* out) {
  if (!out) return fail(DC_EINVAL, "out is NULL");
  *out = nullptr;
  dc_plan_s* p = new (std::nothrow) dc_plan_s;
  if (!p) return fail(DC_ENOMEM, "out of host memory");
  dc_status st;
  try {
    st = build_plan(schema, roots, nroots, p);
  } catch (const std::bad_alloc&) {
    st = fail(DC_ENOMEM, "out of host memory while planning");
  }
  if (st) {
    delete p;
    return st;
  }
  plan_spans(p);
  choose_spans(p);
  p->L = make_layout(p);
  if (debug_on()) p->flags |= DC_PLAN_VERIFY;
  *out = p;
  return DC_OK;
}

dc_status dc_plan_set_flags(dc_plan_t p, uint32_t flags) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  const uint32_t before = p->flags;
  flags |= debug_on() ? DC_PLAN_VERIFY : 0u;
  if ((before ^ flags) & DC_PLAN_PACK_SMALL) {  // another layout: offsets and tables again
    if (p->dev) return fail(DC_ESTATE, "DC_PLAN_PACK_SMALL changes the layout: set it before dc_bind_device");
    p->flags = flags;
    dc_status st = layout(p);
    if (st) {
      p->flags = before;
      layout(p);
    }
    choose_spans(p);
    p->L = make_layout(p);  // the device regions follow the data bytes and the segment capacity
    return st;
  }
  if ((before ^ flags) & (DC_PLAN_MAP_HOST | DC_PLAN_SPANS)) {  // span staging on or off
    if (p->dev) return fail(DC_ESTATE, "DC_PLAN_MAP_HOST and DC_PLAN_SPANS are set before dc_bind_device");
    p->flags = flags;
    choose_spans(p);
    p->L = make_layout(p);
    return DC_OK;
  }
  p->flags = flags;
  return DC_OK;
}

dc_status dc_plan_set_threads(dc_plan_t p, uint32_t n) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  p->nthreads = n;
  p->pool = nullptr;
  p->own_pool.reset();
  return DC_OK;
}

dc_status dc_plan_info_get(dc_plan_t p, dc_plan_info* out) {
  if (!p || !out) return fail(DC_EINVAL, "NULL argument");
  out->data_bytes = p->data_bytes;
  out->device_bytes = p->L.total;
  out->payload_bytes = p->payload;
  out->nblocks = p->blocks.size();
  out->nrelocs = p->blocks.size() - p->roots.size();
  out->nstructs = p->nstructs;
  out->nstruct_blocks = p->nstruct_blocks;
  out->root_offset = 0;
  out->ntrees = p->roots.size();
  out->struct_bytes = p->struct_bytes;
  out->reloc_table_bytes =
      p->rrec.size() * sizeof(RelocRec) + p->rseg.size() * sizeof(RelocSeg) + p->rtiles.size() * sizeof(RelocTile);
  out->staging_bytes = p->span_mode ? p->span_bytes : 0;
  return DC_OK;
}

dc_status dc_plan_arena_bytes(dc_plan_t p, uint64_t* bytes, uint64_t* nblocks, uint64_t* nrelocs) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (bytes) *bytes = p->L.total;
  if (nblocks) *nblocks = p->blocks.size();
  if (nrelocs) *nrelocs = p->blocks.size() - p->roots.size();
  return DC_OK;
}

dc_status dc_plan_root(dc_plan_t p, uint64_t tree, uint64_t* offset) {
  if (!p || !offset) return fail(DC_EINVAL, "NULL argument");
  if (tree >= p->roots.size()) return fail(DC_EINVAL, "tree %llu out of range", (unsigned long long)tree);
  *offset = p->blocks[p->roots[tree]].off;
  return DC_OK;
}

dc_status dc_plan_block(dc_plan_t p, uint64_t i, uint64_t* host, uint64_t* off, uint64_t* bytes, uint32_t* lane,
                        uint32_t* parent, uint32_t* slot_off) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (i >= p->blocks.size()) return fail(DC_EINVAL, "block %llu out of range", (unsigned long long)i);
  const HostBlock& b = p->blocks[i];
  if (host) *host = (uint64_t)(uintptr_t)b.host;
  if (off) *off = b.off;
  if (bytes) *bytes = b.bytes;
  if (lane) *lane = b.lane;
  if (parent) *parent = b.parent;
  if (slot_off) *slot_off = b.slot_off;
  return DC_OK;
}

dc_status dc_plan_destroy(dc_plan_t p) {
  if (!p) return DC_OK;
  if (p->h2d_done) cudaEventSynchronize(p->h2d_done);
  if (p->tab_done) cudaEventSynchronize(p->tab_done);
  if (p->pinned && !p->borrowed_pinned) cudaFreeHost(p->pinned);
  if (p->pin_tab && !p->borrowed_pinned) cudaFreeHost(p->pin_tab);
  release_transfers(p);
  if (p->h2d_done) cudaEventDestroy(p->h2d_done);
  if (p->tab_done) cudaEventDestroy(p->tab_done);
  for (cudaEvent_t e : p->step_ev) {
    cudaEventSynchronize(e);
    cudaEventDestroy(e);
  }
  if (p->back_err) cudaEventDestroy(p->back_err);
  if (p->sync_ev) cudaEventDestroy(p->sync_ev);
  for (cudaEvent_t e : p->back_ev) cudaEventDestroy(e);
  delete p;
  return DC_OK;
}

dc_status dc_bind_device(dc_plan_t p, void* dev, uint64_t bytes, dc_stream_t stream) {
  if (!p || !dev) return fail(DC_EINVAL, "NULL argument");
  if ((uintptr_t)dev % 256) return fail(DC_EINVAL, "device buffer must be 256-byte aligned");
  if (bytes < p->L.total)
    return fail(DC_EBUDGET, "device buffer holds %llu bytes, the plan needs %llu", (unsigned long long)bytes,
                (unsigned long long)p->L.total);
  cudaStream_t s = stream;
  DC_CUDA(cudaGetDevice(&p->device));
  DC_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
  if (p->h2d_done) DC_CUDA(cudaEventSynchronize(p->h2d_done));
  if (!p->pinned) {
    const uint64_t pin = pin_arena_bytes(p);
    cudaError_t e = host_alloc((void**)&p->pinned, std::max<uint64_t>(pin, 16), cudaHostAllocMapped);
    if (e != cudaSuccess) {
      p->pinned = nullptr;
      return fail(DC_ENOMEM, "pinned arena of %llu bytes: %s", (unsigned long long)pin, cudaGetErrorString(e));
    }
    DC_CUDA(cudaHostGetDevicePointer((void**)&p->pinned_dev, p->pinned, 0));
    // padding between blocks stays zero: the marshal writes blocks only
    Pool& pool = pool_of(p);
    const uint64_t n = (pin + (64ull << 20) - 1) / (64ull << 20);
    pool.parallel_for(n, [&](uint64_t i) {
      uint64_t lo = i * (64ull << 20), hi = std::min<uint64_t>(pin, lo + (64ull << 20));
      memset(p->pinned + lo, 0, hi - lo);
    });
  }
  if (!p->transfers_ready) plan_transfers(p);
  if (!p->pin_tab || p->pin_tab_bytes < tab_total(p->L)) {
    if (p->pin_tab && !p->borrowed_pinned) cudaFreeHost(p->pin_tab);
    p->pin_tab_bytes = tab_total(p->L);
    cudaError_t e = host_alloc((void**)&p->pin_tab, p->pin_tab_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      p->pin_tab = nullptr;
      return fail(DC_ENOMEM, "pinned table staging: %s", cudaGetErrorString(e));
    }
  }
  if (!p->h2d_done) DC_CUDA(cudaEventCreateWithFlags(&p->h2d_done, cudaEventDisableTiming));
  if (!p->tab_done) DC_CUDA(cudaEventCreateWithFlags(&p->tab_done, cudaEventDisableTiming));
  p->dev = (uint8_t*)dev;
  p->dev_bytes = bytes;
  const uint64_t nrec = p->rrec.size();
  p->rec_scan = (p->flags & DC_PLAN_DEVICE_SCAN) != 0;
  std::vector<RelocRec> size_rec;  // DC_PLAN_DEVICE_SCAN: slice heads' offsets and sizes
  if (nrec && p->rec_scan) {
    size_rec.resize(nrec);
    scan_records(p, size_rec.data());
  }
  if (nrec) {
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.rec, p->rec_scan ? size_rec.data() : p->rrec.data(), nrec * sizeof(RelocRec),
                            cudaMemcpyHostToDevice, s));
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.hostp, p->rec_host.data(), nrec * 8, cudaMemcpyHostToDevice, s));
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.soff, p->rec_off.data(), nrec * 8, cudaMemcpyHostToDevice, s));
  }
  DC_CUDA(cudaMemsetAsync(p->dev + p->L.ctrl, 0, CTRL_WORDS * 4, s));
  DC_CUDA(cudaMemcpyAsync(p->dev + p->L.status, p->rseg.data(), p->rseg.size() * sizeof(RelocSeg),
                          cudaMemcpyHostToDevice, s));
  if (!p->rtiles.empty())
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.rtile, p->rtiles.data(), p->rtiles.size() * sizeof(RelocTile),
                            cudaMemcpyHostToDevice, s));
  {
    dc_status st = upload_h2d_tables(p, s);
    if (st) return st;
  }
  DC_CUDA(cudaStreamSynchronize(s));
  p->back_key = ~0ull;
  p->bk_nd = 0;
  p->step_key = OpKey();
  p->leaf_key = OpKey();
  p->chase_key = OpKey();
  p->written = nullptr;
  p->op_run = false;
  return DC_OK;
}

}  // extern "C"

uint64_t dc::pinned_need(const dc_plan_s* p) { return round_up(pin_arena_bytes(p), 256) + tab_total(p->L); }

dc_status dc::bind_borrowed(dc_plan_s* p, void* dev, uint64_t bytes, uint8_t* pinned, uint8_t* pinned_dev,
                            cudaStream_t s) {
  if (p->pinned && !p->borrowed_pinned) return fail(DC_ESTATE, "plan already owns a pinned arena");
  p->borrowed_pinned = true;
  p->pinned = pinned;
  p->pinned_dev = pinned_dev;
  p->pin_tab = pinned + round_up(pin_arena_bytes(p), 256);
  p->pin_tab_bytes = tab_total(p->L);
  return dc_bind_device(p, dev, bytes, s);
}

dc_status dc::lend_pinned(dc_plan_s* p, uint8_t* pinned, uint8_t* pinned_dev) {
  if (!p->borrowed_pinned) return fail(DC_ESTATE, "the plan owns its pinned arena");
  if (p->flags & DC_PLAN_MAP_HOST) return fail(DC_ESTATE, "mapped plans keep the pinned range they were bound with");
  p->pinned = pinned;
  p->pinned_dev = pinned_dev;
  p->pin_tab = pinned + round_up(pin_arena_bytes(p), 256);
  p->step_key = OpKey();  // the round trip's device tables hold pinned addresses: rebuild them
  return DC_OK;
}

extern "C" {

dc_status dc_device_base(dc_plan_t p, uint64_t* base) {
  if (!p || !base) return fail(DC_EINVAL, "NULL argument");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  *base = (uint64_t)(uintptr_t)p->dev;
  return DC_OK;
}

dc_status dc_relocate(dc_plan_t p, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  // Fig 2 step d: rebuild every pointer on the device
  const RelocArgs a = reloc_args(p);
  DC_CUDA(launch_relocate(a, s, p->sm_count));
  return DC_OK;
}

dc_status dc_deep_copy(dc_plan_t p, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  // the previous deep copy's transfers read the same pinned arena
  dc_status st = wait_event(p->h2d_done);
  if (st) return st;
  pool_of(p);
  if ((st = transfer_to_device(p, s))) return st;
  DC_CUDA(cudaEventRecord(p->h2d_done, s));
  return dc_relocate(p, stream);
}

// A selective deep copy (Sec. 2): the struct blocks on the way to every struct
// the op selects (for SEL_CHAIN: the blocks its chain passes through) and the
// op's x and y arrays of those structs go through the pinned arena to the
// device; then only the relocation tiles that hold those struct blocks' slots
// run.  Nothing else of the data region is written.
dc_status dc_deep_copy_selected(dc_plan_t p, const dc_op* op, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  dc_status st = check_op(p, op);
  if (st) return st;
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  OpKey key = key_of(op);
  if (!(key == p->sel_key)) {
    std::vector<std::pair<uint32_t, uint64_t>> structs;
    if ((st = select_structs(p, op, &structs))) return st;
    std::vector<Pick> picks;
    if ((st = pick(p, op, &picks))) return st;
    const uint64_t nb = p->blocks.size();
    std::vector<uint8_t> mark(nb, 0);
    for (const auto& se : structs)  // the struct block and every struct block above it
      for (uint32_t b = se.first; b != NONE && !mark[b]; b = p->blocks[b].parent) mark[b] = 1;
    for (const auto& k : picks) {
      mark[k.bx] = 1;
      if (k.by != NONE) mark[k.by] = 1;
    }
    std::vector<uint32_t> list;
    for (uint32_t b = 0; b < nb; b++)
      if (mark[b]) list.push_back(b);
    plan_moves(p, list, &p->sel, false, 0, true);  // every selected byte through the pinned arena
    // the listed relocation tiles (ascending t) that overlap a selected struct block
    p->sel_tiles.clear();
    for (uint32_t b : list) {
      const HostBlock& B = p->blocks[b];
      if (B.lane != 0 || !B.bytes) continue;
      const uint64_t t0 = B.off / RELOC_SPAN, t1 = (B.off + B.bytes - 1) / RELOC_SPAN;
      auto it = std::lower_bound(p->rtiles.begin(), p->rtiles.end(), t0,
                                 [](const RelocTile& a, uint64_t t) { return a.t < t; });
      for (; it != p->rtiles.end() && it->t <= t1; ++it)
        if (p->sel_tiles.empty() || p->sel_tiles.back().t < it->t) p->sel_tiles.push_back(*it);
    }
    if (!p->sel_tiles.empty())
      DC_CUDA(cudaMemcpyAsync(p->dev + p->L.seltile, p->sel_tiles.data(), p->sel_tiles.size() * sizeof(RelocTile),
                              cudaMemcpyHostToDevice, s));
    p->sel_key = key;
  }
  if ((st = wait_event(p->h2d_done))) return st;  // an earlier transfer may still read the pinned arena
  if ((st = send_staged(p, p->sel, p->null_slots, p->dev, s))) return st;
  DC_CUDA(cudaEventRecord(p->h2d_done, s));
  RelocArgs a = reloc_args(p);
  a.tiles = reinterpret_cast<const RelocTile*>(p->dev + p->L.seltile);
  a.ntiles = (uint32_t)p->sel_tiles.size();
  a.verify = 0;  // the tiles' other structs were not copied: their slots hold no host address
  DC_CUDA(launch_relocate(a, s, p->sm_count));
  return DC_OK;
}

dc_status dc_resolve_offset(dc_plan_t p, const dc_step* path, uint32_t len, uint64_t* offset) {
  return dc_resolve_offset_in(p, 0, path, len, offset);
}

dc_status dc_resolve_offset_in(dc_plan_t p, uint64_t tree, const dc_step* path, uint32_t len, uint64_t* offset) {
  if (!p || !offset) return fail(DC_EINVAL, "NULL argument");
  uint32_t blk, ty;
  uint64_t within;
  dc_status st = resolve(p, tree, path, len, &blk, &within, &ty, nullptr);
  if (st) return st;
  *offset = p->blocks[blk].off + within;
  return DC_OK;
}

dc_status dc_resolve_chain(dc_plan_t p, const dc_step* path, uint32_t len, uint64_t* dev_addr) {
  return dc_resolve_chain_in(p, 0, path, len, dev_addr);
}

dc_status dc_resolve_chain_in(dc_plan_t p, uint64_t tree, const dc_step* path, uint32_t len, uint64_t* dev_addr) {
  if (!p || !dev_addr) return fail(DC_EINVAL, "NULL argument");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  uint64_t off;
  dc_status st = dc_resolve_offset_in(p, tree, path, len, &off);
  if (st) return st;
  *dev_addr = (uint64_t)(uintptr_t)p->dev + off;
  return DC_OK;
}

}  // extern "C"

dc_status dc::build_leaf_table(dc_plan_s* p, const dc_op* op, cudaStream_t s) {
  const dc_field& X = p->schema.fields[op->type][op->x_field];
  OpKey key = key_of(op);
  if (key == p->leaf_key) return DC_OK;
  std::vector<Pick> picks;
  dc_status st;
  if ((st = pick(p, op, &picks))) return st;
  if ((st = wait_event(p->tab_done))) return st;
  Segment* seg = reinterpret_cast<Segment*>(p->pin_tab + tab_seg(p->L));
  const uint64_t base = (uint64_t)(uintptr_t)p->dev;
  const uint64_t esz = X.elem_size;
  const bool axpy = op->kind == DC_OP_AXPY_HALF;
  uint64_t units = 0, nseg = 0;
  p->leaf_written.clear();
  p->leaf_gen = ++p->gen;
  p->leaf_hist.assign(40, 0);
  for (size_t i = 0; i < picks.size(); i++) {
    const HostBlock& bx = p->blocks[picks[i].bx];
    const uint64_t x = base + bx.off, y = picks[i].by == NONE ? 0 : base + p->blocks[picks[i].by].off;
    p->leaf_written.push_back(picks[i].bx);
    uint32_t lg = 0;
    while (lg < 39 && (1ull << lg) < bx.count) lg++;
    p->leaf_hist[lg]++;
    if (nseg) {  // x (and y) continue the previous segment after at most its padding: one stream
      Segment& g = seg[nseg - 1];
      const uint64_t end = g.x + g.n * esz;
      if (x >= end && x - end < 16 && (x - g.x) % esz == 0 && (!axpy || y - g.y == x - g.x) && g.x % 16 == 0 &&
          (!axpy || g.y % 16 == 0)) {
        g.n = (x - g.x) / esz + bx.count;
        continue;
      }
    }
    // A segment streams in 16-byte vectors from its start, which must lie on 16
    // bytes (a DC_PLAN_PACK_SMALL arena has arrays that do not): the elements
    // before the next boundary become a segment of their own, shorter than a
    // vector, which the kernels update element by element; if x and y are not
    // on the same side of a boundary, the whole (small) array goes that way.
    uint64_t n = bx.count, xx = x, yy = y;
    const uint64_t epu = 16 / esz;
    if (xx % 16 || (axpy && yy % 16)) {
      if (!axpy || xx % 16 == yy % 16) {
        const uint64_t head = std::min<uint64_t>(n, (16 - xx % 16) / esz);
        if (nseg >= p->L.seg_cap) return fail(DC_EINVAL, "segment table larger than planned");
        seg[nseg++] = Segment{xx, yy, head, 0};
        xx += head * esz;
        yy += axpy ? head * esz : 0;
        n -= head;
      } else {
        for (; n; n -= std::min<uint64_t>(n, epu - 1)) {
          const uint64_t c = std::min<uint64_t>(n, epu - 1);
          if (nseg >= p->L.seg_cap) return fail(DC_EINVAL, "segment table larger than planned");
          seg[nseg++] = Segment{xx, yy, c, 0};
          xx += c * esz;
          yy += c * esz;
        }
      }
    }
    if (n) {
      if (nseg >= p->L.seg_cap) return fail(DC_EINVAL, "segment table larger than planned");
      seg[nseg++] = Segment{xx, yy, n, 0};
    }
  }
  for (uint64_t i = 0; i < nseg; i++) {
    seg[i].ubeg = units;
    units += (seg[i].n * esz + 15) / 16;
  }
  // tile -> segment holding the tile's first unit (two-pointer walk)
  uint32_t* tseg = reinterpret_cast<uint32_t*>(p->pin_tab + tab_tseg(p->L));
  const uint64_t ntiles = (units + LEAF_TILE - 1) / LEAF_TILE;
  if (ntiles + 1 > p->L.tseg_cap) return fail(DC_EINVAL, "tile table larger than planned");
  for (uint64_t t = 0, sg = 0; t < ntiles; t++) {
    const uint64_t u = t * LEAF_TILE;
    while (sg + 1 < nseg && seg[sg + 1].ubeg <= u) sg++;
    tseg[t] = (uint32_t)sg;
  }
  tseg[ntiles] = nseg ? (uint32_t)(nseg - 1) : 0;
  if (nseg) {
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.seg, seg, nseg * sizeof(Segment), cudaMemcpyHostToDevice, s));
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.tseg, tseg, (ntiles + 1) * 4, cudaMemcpyHostToDevice, s));
  }
  DC_CUDA(cudaEventRecord(p->tab_done, s));
  p->leaf_nseg = nseg;
  p->leaf_units = units;
  p->leaf_key = key;
  return DC_OK;
}

LeafArgs dc::leaf_args(const dc_plan_s* p, const dc_op* op) {
  const dc_field& X = p->schema.fields[op->type][op->x_field];
  LeafArgs a;
  a.seg = reinterpret_cast<const Segment*>(p->dev + p->L.seg);
  a.tile_seg = reinterpret_cast<const uint32_t*>(p->dev + p->L.tseg);
  a.nseg = (uint32_t)p->leaf_nseg;
  a.units = p->leaf_units;
  a.kind = op->kind;
  a.f64 = X.elem_kind == DC_E_F64;
  a.scale = op->scale;
  a.ctrl = reinterpret_cast<uint32_t*>(p->dev + p->L.ctrl);
  return a;
}

RelocArgs dc::reloc_args(const dc_plan_s* p) {
  RelocArgs a;
  a.arena = p->dev;
  a.data_bytes = p->data_bytes;
  a.struct_bytes = p->struct_bytes;
  a.rec = reinterpret_cast<const RelocRec*>(p->dev + p->L.rec);
  a.seg = reinterpret_cast<const RelocSeg*>(p->dev + p->L.status);
  a.tiles = reinterpret_cast<const RelocTile*>(p->dev + p->L.rtile);
  a.rec_host = reinterpret_cast<const uint64_t*>(p->dev + p->L.hostp);
  a.rec_off = reinterpret_cast<const uint64_t*>(p->dev + p->L.soff);
  a.ctrl = reinterpret_cast<uint32_t*>(p->dev + p->L.ctrl);
  a.nrec = (uint32_t)p->rrec.size();
  a.nseg = (uint32_t)(p->rseg.size() - 1);
  a.ntiles = (uint32_t)p->L.ntiles;
  a.verify = (p->flags & DC_PLAN_VERIFY) ? 1u : 0u;
  a.scan = p->rec_scan ? 1u : 0u;
  a.unit_shift = p->unit_shift;
  return a;
}

extern "C" {

dc_status dc_update_leaves(dc_plan_t p, const dc_op* op, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  dc_status st = check_op(p, op);
  if (st) return st;
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  {
    Trace tr("dc_update_leaves", "tables");
    if ((st = build_leaf_table(p, op, s))) return st;
  }
  p->written = &p->leaf_written;
  p->written_gen = p->leaf_gen;
  p->op_run = true;
  DC_CUDA(launch_leaf(leaf_args(p, op), s, p->sm_count));
  return DC_OK;
}

dc_status dc_update_chase(dc_plan_t p, const dc_op* op, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  dc_status st = check_op(p, op);
  if (st) return st;
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  const SchemaCopy& S = p->schema;
  const dc_field& X = S.fields[op->type][op->x_field];
  OpKey key = key_of(op);
  if (!(key == p->chase_key)) {
    std::vector<Pick> picks;
    if ((st = pick(p, op, &picks))) return st;
    if ((st = wait_event(p->tab_done))) return st;
    ChaseSeg* seg = reinterpret_cast<ChaseSeg*>(p->pin_tab + tab_cseg(p->L));
    ChaseStep* stp = reinterpret_cast<ChaseStep*>(p->pin_tab + tab_steps(p->L));
    std::vector<ChaseStep> steps;
    uint64_t elems = 0;
    p->chase_written.clear();
    p->chase_gen = ++p->gen;
    for (size_t i = 0; i < picks.size(); i++) {
      uint32_t first = (uint32_t)steps.size();
      const uint32_t root = chain_steps(p, picks[i].sblk, picks[i].elem, &steps);
      seg[i].root = (uint64_t)(uintptr_t)p->dev + p->blocks[root].off;
      seg[i].step_first = first;
      seg[i].nsteps = (uint32_t)(steps.size() - first);
      seg[i].n = p->blocks[picks[i].bx].count;
      seg[i].ebeg = elems;
      elems += seg[i].n;
      p->chase_written.push_back(picks[i].bx);
    }
    if (steps.size() > p->L.step_cap) return fail(DC_EINVAL, "chase table larger than planned");
    if (!steps.empty()) memcpy(stp, steps.data(), steps.size() * sizeof(ChaseStep));
    if (!picks.empty())
      DC_CUDA(cudaMemcpyAsync(p->dev + p->L.cseg, seg, picks.size() * sizeof(ChaseSeg), cudaMemcpyHostToDevice, s));
    if (!steps.empty())
      DC_CUDA(cudaMemcpyAsync(p->dev + p->L.steps, stp, steps.size() * sizeof(ChaseStep), cudaMemcpyHostToDevice,
                              s));
    DC_CUDA(cudaEventRecord(p->tab_done, s));
    p->chase_nseg = picks.size();
    p->chase_elems = elems;
    p->chase_key = key;
  }
  p->written = &p->chase_written;
  p->written_gen = p->chase_gen;
  p->op_run = true;
  ChaseArgs a;
  a.seg = reinterpret_cast<const ChaseSeg*>(p->dev + p->L.cseg);
  a.steps = reinterpret_cast<const ChaseStep*>(p->dev + p->L.steps);
  a.nseg = (uint32_t)p->chase_nseg;
  a.elems = p->chase_elems;
  a.x_off = X.offset;
  a.y_off = op->kind == DC_OP_AXPY_HALF ? S.fields[op->type][op->y_field].offset : 0;
  a.kind = op->kind;
  a.f64 = X.elem_kind == DC_E_F64;
  a.scale = op->scale;
  DC_CUDA(launch_chase(a, s, p->sm_count));
  return DC_OK;
}

dc_status dc_verify_chain(dc_plan_t p, const dc_step* path, uint32_t len, dc_stream_t stream, uint64_t* dev_addr) {
  if (!p || !dev_addr) return fail(DC_EINVAL, "NULL argument");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  std::vector<ChaseStep> steps;
  dc_status st = path_steps(p, path, len, &steps);
  if (st) return st;
  if (steps.size() > p->L.walk_cap) return fail(DC_EINVAL, "path longer than the tree");
  cudaStream_t s = stream;
  if ((st = wait_event(p->tab_done))) return st;
  ChaseStep* stp = reinterpret_cast<ChaseStep*>(p->pin_tab + tab_walk(p->L));
  if (!steps.empty()) memcpy(stp, steps.data(), steps.size() * sizeof(ChaseStep));
  uint8_t* dsteps = p->dev + p->L.walk;
  uint64_t* dout = reinterpret_cast<uint64_t*>(dsteps + p->L.walk_cap * sizeof(ChaseStep));
  if (!steps.empty())
    DC_CUDA(cudaMemcpyAsync(dsteps, stp, steps.size() * sizeof(ChaseStep), cudaMemcpyHostToDevice, s));
  DC_CUDA(launch_walk((uint64_t)(uintptr_t)p->dev, reinterpret_cast<const ChaseStep*>(dsteps),
                      (uint32_t)steps.size(), 0, dout, s));
  uint64_t* word = reinterpret_cast<uint64_t*>(p->pin_tab + tab_words(p->L) + 8);
  DC_CUDA(cudaMemcpyAsync(word, dout, 8, cudaMemcpyDeviceToHost, s));
  DC_CUDA(cudaStreamSynchronize(s));
  *dev_addr = *word;
  return DC_OK;
}

dc_status dc_copy_back(dc_plan_t p, uint32_t flags, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  static const std::vector<uint32_t> none;
  std::vector<uint32_t> all;
  uint64_t key;
  if (flags & DC_COPY_ALL_ARRAYS) {
    key = 0;
    if (p->back_key != 0)
      for (uint32_t b = (uint32_t)p->nstruct_blocks; b < p->blocks.size(); b++) all.push_back(b);
  } else {
    if (!p->op_run) return fail(DC_ESTATE, "no update has run: nothing to copy back");
    key = p->written_gen;
  }
  pool_of(p);
  const std::vector<uint32_t>& list = (flags & DC_COPY_ALL_ARRAYS) ? all : (key == p->back_key ? none : *p->written);
  return transfer_back(p, list, key, stream);
}

dc_status dc_sync(dc_plan_t p, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  Trace tr("dc_sync", "wait");
  return device_error(p, stream);
}

// ---- UVM comparison path ----------------------------------------------------------

dc_status dc_uvm_build(const dc_schema* schema, const void* host_root, dc_uvm_t* out) {
  if (!out) return fail(DC_EINVAL, "out is NULL");
  *out = nullptr;
  dc_plan_t plan = nullptr;
  dc_status st = dc_plan(schema, host_root, &plan);
  if (st) return st;
  dc_uvm_s* u = new (std::nothrow) dc_uvm_s;
  if (!u) {
    dc_plan_destroy(plan);
    return fail(DC_ENOMEM, "out of host memory");
  }
  u->plan = plan;
  auto cleanup = [&](dc_status s2) {
    dc_uvm_destroy(u);
    return s2;
  };
  cudaError_t e = cudaGetDevice(&u->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaGetDevice"));
  e = cudaDeviceGetAttribute(&u->sm_count, cudaDevAttrMultiProcessorCount, u->device);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaDeviceGetAttribute"));
  const uint64_t nb = plan->blocks.size();
  u->managed.assign(nb, nullptr);
  for (uint64_t b = 0; b < nb; b++) {  // one managed allocation per block, like a managed malloc
    e = cudaMallocManaged(&u->managed[b], std::max<uint64_t>(plan->blocks[b].bytes, 1));
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMallocManaged"));
    memcpy(u->managed[b], plan->blocks[b].host, plan->blocks[b].bytes);
  }
  for (uint64_t b = 1; b < nb; b++) {  // host pointers -> managed pointers
    const HostBlock& B = plan->blocks[b];
    uint64_t v = (uint64_t)(uintptr_t)u->managed[b];
    memcpy((uint8_t*)u->managed[B.parent] + B.slot_off, &v, 8);
  }
  for (uint64_t off : plan->null_slots) {  // count-0 slots hold NULL
    auto it = std::upper_bound(plan->blocks.begin(), plan->blocks.begin() + plan->nstruct_blocks, off,
                               [](uint64_t o, const HostBlock& hb) { return o < hb.off; });
    uint32_t b = (uint32_t)(it - plan->blocks.begin()) - 1;
    memset((uint8_t*)u->managed[b] + (off - plan->blocks[b].off), 0, 8);
  }
  u->root = (uint64_t)(uintptr_t)u->managed[0];
  u->seg_cap = std::max<uint64_t>(1, plan->nstructs);
  u->step_cap = std::max<uint64_t>(1, plan->sum_depth);
  e = cudaMalloc((void**)&u->dseg, u->seg_cap * sizeof(ChaseSeg));
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc"));
  e = cudaMalloc((void**)&u->dsteps, u->step_cap * sizeof(ChaseStep));
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc"));
  *out = u;
  return DC_OK;
}

dc_status dc_uvm_root(dc_uvm_t u, uint64_t* root) {
  if (!u || !root) return fail(DC_EINVAL, "NULL argument");
  *root = u->root;
  return DC_OK;
}

dc_status dc_uvm_prefetch(dc_uvm_t u, int to_device, dc_stream_t stream) {
  if (!u) return fail(DC_EINVAL, "uvm is NULL");
  cudaMemLocation loc;
  loc.type = to_device ? cudaMemLocationTypeDevice : cudaMemLocationTypeHost;
  loc.id = to_device ? u->device : 0;
  for (uint64_t b = 0; b < u->managed.size(); b++)
    DC_CUDA(cudaMemPrefetchAsync(u->managed[b], std::max<uint64_t>(u->plan->blocks[b].bytes, 1), loc, 0, stream));
  return DC_OK;
}

dc_status dc_uvm_update(dc_uvm_t u, const dc_op* op, dc_stream_t stream) {
  if (!u) return fail(DC_EINVAL, "uvm is NULL");
  dc_plan_s* p = u->plan;
  dc_status st = check_op(p, op);
  if (st) return st;
  const SchemaCopy& S = p->schema;
  const dc_field& X = S.fields[op->type][op->x_field];
  cudaStream_t s = stream;
  OpKey key = key_of(op);
  if (!(key == u->key)) {
    std::vector<Pick> picks;
    if ((st = pick(p, op, &picks))) return st;
    std::vector<ChaseSeg> seg(picks.size());
    std::vector<ChaseStep> steps;
    uint64_t elems = 0;
    u->written.clear();
    for (size_t i = 0; i < picks.size(); i++) {
      uint32_t first = (uint32_t)steps.size();
      const uint32_t root = chain_steps(p, picks[i].sblk, picks[i].elem, &steps);
      seg[i] = ChaseSeg{(uint64_t)(uintptr_t)u->managed[root], first, (uint32_t)(steps.size() - first), p->blocks[picks[i].bx].count, elems};
      elems += seg[i].n;
      u->written.push_back(picks[i].bx);
    }
    if (steps.size() > u->step_cap) return fail(DC_EINVAL, "chase table larger than planned");
    if (!seg.empty()) DC_CUDA(cudaMemcpy(u->dseg, seg.data(), seg.size() * sizeof(ChaseSeg), cudaMemcpyHostToDevice));
    if (!steps.empty())
      DC_CUDA(cudaMemcpy(u->dsteps, steps.data(), steps.size() * sizeof(ChaseStep), cudaMemcpyHostToDevice));
    u->nseg = seg.size();
    u->elems = elems;
    u->key = key;
  }
  ChaseArgs a;
  a.seg = u->dseg;
  a.steps = u->dsteps;
  a.nseg = (uint32_t)u->nseg;
  a.elems = u->elems;
  a.x_off = X.offset;
  a.y_off = op->kind == DC_OP_AXPY_HALF ? S.fields[op->type][op->y_field].offset : 0;
  a.kind = op->kind;
  a.f64 = X.elem_kind == DC_E_F64;
  a.scale = op->scale;
  DC_CUDA(launch_chase(a, s, u->sm_count));
  return DC_OK;
}

dc_status dc_uvm_sync(dc_uvm_t u, dc_stream_t stream) {
  if (!u) return fail(DC_EINVAL, "uvm is NULL");
  DC_CUDA(cudaStreamSynchronize(stream));
  return DC_OK;
}

dc_status dc_uvm_copy_back(dc_uvm_t u, const void* host_root, uint32_t flags) {
  if (!u) return fail(DC_EINVAL, "uvm is NULL");
  dc_plan_s* p = u->plan;
  if (host_root != p->blocks[0].host) return fail(DC_EINVAL, "host_root is not the tree this UVM copy was built from");
  DC_CUDA(cudaDeviceSynchronize());
  if (flags & DC_COPY_ALL_ARRAYS) {
    for (uint64_t b = p->nstruct_blocks; b < p->blocks.size(); b++)
      memcpy(const_cast<uint8_t*>(p->blocks[b].host), u->managed[b], p->blocks[b].bytes);
  } else {
    for (uint32_t b : u->written) memcpy(const_cast<uint8_t*>(p->blocks[b].host), u->managed[b], p->blocks[b].bytes);
  }
  return DC_OK;
}

dc_status dc_uvm_destroy(dc_uvm_t u) {
  if (!u) return DC_OK;
  if (!u->managed.empty() || u->dseg || u->dsteps) cudaDeviceSynchronize();
  for (void* m : u->managed)
    if (m) cudaFree(m);
  if (u->dseg) cudaFree(u->dseg);
  if (u->dsteps) cudaFree(u->dsteps);
  dc_plan_destroy(u->plan);
  delete u;
  return DC_OK;
}

}  // extern "C"
