// plan.cpp — the host walk of a pointer-linked structure (dc_plan).
//
// Algorithm 1's first step (determineTotalBytes) and its allocation requests:
// one iterative depth-first walk over the field-offset schema records every
// block (the root struct, each non-empty array, each non-empty child-struct
// array) with the pointer slot that refers to it.  The blocks are then laid out
// in lanes (all struct blocks first, then one lane per ARRAY field), each block
// on a 16-byte boundary (small arrays closer with DC_PLAN_PACK_SMALL), which
// fixes the arena and the relocation table.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <optional>

#include "internal.hpp"

namespace dc {

static thread_local char g_err[1024];

dc_status fail(dc_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

dc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(DC_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

const char* last_error() { return g_err; }

bool OpKey::operator==(const OpKey& o) const {
  if (kind != o.kind || sel != o.sel || type != o.type || x != o.x || y != o.y ||
      path.size() != o.path.size())
    return false;
  for (size_t i = 0; i < path.size(); i++)
    if (path[i].field != o.path[i].field || path[i].index != o.path[i].index) return false;
  return true;
}

dc_status copy_schema(const dc_schema* s, SchemaCopy* out) {
  if (!s || !s->types || s->ntypes == 0 || s->root_type >= s->ntypes)
    return fail(DC_EINVAL, "schema: missing types or bad root type");
  out->types.assign(s->types, s->types + s->ntypes);
  out->fields.resize(s->ntypes);
  out->ptr_index.resize(s->ntypes);
  out->nptr.assign(s->ntypes, 0);
  out->lane_of.resize(s->ntypes);
  out->root_type = s->root_type;
  uint32_t lane = 1;
  for (uint32_t t = 0; t < s->ntypes; t++) {
    const dc_type& T = s->types[t];
    if (T.size == 0 || (T.nfields && !T.fields)) return fail(DC_EINVAL, "type %u: empty", t);
    if (T.align == 0 || T.align > 16 || (T.align & (T.align - 1)))
      return fail(DC_EINVAL, "type %u: alignment %u is not a power of two <= 16", t, T.align);
    out->fields[t].assign(T.fields, T.fields + T.nfields);
    out->types[t].fields = out->fields[t].data();
    out->ptr_index[t].assign(T.nfields, -1);
    out->lane_of[t].assign(T.nfields, 0);
    bool has_ptr = false;
    for (uint32_t f = 0; f < T.nfields; f++) {
      const dc_field& F = T.fields[f];
      if (F.kind == DC_F_SCALAR) {
        if (F.elem_size != 4 && F.elem_size != 8)
          return fail(DC_EINVAL, "type %u field %u: scalar size must be 4 or 8", t, f);
        if ((uint64_t)F.offset + F.elem_size > T.size)
          return fail(DC_EINVAL, "type %u field %u: outside the struct", t, f);
        continue;
      }
      if (F.kind != DC_F_ARRAY && F.kind != DC_F_CHILD)
        return fail(DC_EINVAL, "type %u field %u: unknown kind %d", t, f, F.kind);
      // the relocation writes 8-byte pointer slots: they must be naturally aligned
      if (F.offset % 8 || (uint64_t)F.offset + 8 > T.size)
        return fail(DC_EINVAL, "type %u field %u: pointer slot not 8-byte aligned inside the struct",
                    t, f);
      if (F.count_field >= 0) {
        if ((uint32_t)F.count_field >= T.nfields || T.fields[F.count_field].kind != DC_F_SCALAR)
          return fail(DC_EINVAL, "type %u field %u: count field is not a scalar", t, f);
      }
      if (F.kind == DC_F_ARRAY) {
        if (F.elem_size == 0) return fail(DC_EINVAL, "type %u field %u: zero element size", t, f);
        out->lane_of[t][f] = lane++;
      } else if (F.child_type < 0 || (uint32_t)F.child_type >= s->ntypes) {
        return fail(DC_EINVAL, "type %u field %u: bad child type", t, f);
      }
      out->ptr_index[t][f] = (int32_t)out->nptr[t]++;
      has_ptr = true;
    }
    if (has_ptr && T.size % 8)
      return fail(DC_EINVAL, "type %u: size %u must be a multiple of 8 (it holds pointers)", t, T.size);
  }
  out->nlanes = lane;
  return DC_OK;
}

static bool read_count(const dc_type& T, const uint8_t* s, const dc_field& F, uint64_t* n) {
  if (F.count_field < 0) {
    *n = F.count_const;
    return true;
  }
  const dc_field& C = T.fields[F.count_field];
  int64_t v;
  if (C.elem_size == 8) {
    memcpy(&v, s + C.offset, 8);
  } else {
    int32_t w;
    memcpy(&w, s + C.offset, 4);
    v = w;
  }
  if (v < 0) return false;
  *n = (uint64_t)v;
  return true;
}

namespace {

// A block's host byte range and its emission index.
struct Span {
  uint64_t start, end;
  uint32_t id;
};

struct Frame {
  uint32_t blk;    // emission index of the struct block
  uint64_t elem;   // element of that block
  uint32_t type;
  uint32_t field;  // next field to descend into
  uint64_t k;      // next element of that field's child array
};

struct Walker {
  dc_plan_s* p;
  const SchemaCopy& S;
  std::vector<HostBlock> emitted;
  // struct ranges: start -> (end, id).  A struct block that overlaps one already
  // emitted stops the walk at once, so a cycle of child pointers cannot make it
  // loop; arrays are leaves, and the overlap pass after the walk checks them.
  std::map<uint64_t, std::pair<uint64_t, uint32_t>> structs;
  std::vector<std::pair<uint32_t, uint64_t>> null_slots;      // (emission index, slot offset)

  explicit Walker(dc_plan_s* pl) : p(pl), S(pl->schema) {}

  bool is_ancestor(uint32_t maybe, uint32_t blk) const {
    for (uint32_t b = blk; b != NONE; b = emitted[b].parent)
      if (b == maybe) return true;
    return false;
  }

  dc_status emit(const uint8_t* host, uint64_t bytes, uint64_t count, uint32_t lane, uint32_t type,
                 uint32_t field, uint32_t parent, uint64_t slot_off, uint32_t depth, uint32_t* id) {
    if (emitted.size() >= (size_t)NONE - 1) return fail(DC_EINVAL, "too many blocks");
    if (slot_off > 0xFFFFFFFFull) return fail(DC_EINVAL, "child array too large for a 32-bit slot offset");
    if (round_up(bytes, 16) / 16 > 0xFFFFFFFFull) return fail(DC_EINVAL, "block larger than 64 GiB");
    uint64_t a = (uint64_t)(uintptr_t)host;
    if (field == NONE) {  // a struct block: it must not overlap another struct block
      auto it = structs.upper_bound(a);
      uint32_t other = NONE;
      if (it != structs.end() && it->first < a + bytes) other = it->second.second;
      if (it != structs.begin()) {
        auto pv = std::prev(it);
        if (pv->second.first > a) other = pv->second.second;
      }
      if (other != NONE) {
        if (parent != NONE && is_ancestor(other, parent))
          return fail(DC_ECYCLE, "a pointer leads back into an ancestor struct block (host 0x%llx)",
                      (unsigned long long)a);
        return fail(DC_EALIAS, "struct block at 0x%llx overlaps another", (unsigned long long)a);
      }
      structs.emplace(a, std::make_pair(a + bytes, (uint32_t)emitted.size()));
    }
    HostBlock b{};
    b.host = host;
    b.bytes = bytes;
    b.count = count;
    b.lane = lane;
    b.type = type;
    b.field = field;
    b.parent = parent;
    b.slot_off = (uint32_t)slot_off;
    b.depth = depth;
    b.ptr_first = 0;
    if (field == NONE) {
      b.ptr_first = p->ptr_target.size();
      p->ptr_target.resize(p->ptr_target.size() + count * S.nptr[type], NONE);
      p->nstructs += count;
      p->nstruct_blocks++;
      p->sum_depth += count * depth;
      if (depth > p->max_depth) p->max_depth = depth;
    }
    p->payload += bytes;
    *id = (uint32_t)emitted.size();
    emitted.push_back(b);
    return DC_OK;
  }

  // Emit the blocks one struct points to (field order).
  dc_status visit(uint32_t blk, uint64_t elem, uint32_t type) {
    const dc_type& T = S.types[type];
    const uint8_t* s = emitted[blk].host + elem * T.size;
    for (uint32_t f = 0; f < T.nfields; f++) {
      const dc_field& F = T.fields[f];
      if (F.kind == DC_F_SCALAR) continue;
      uint64_t n;
      if (!read_count(T, s, F, &n)) return fail(DC_EINVAL, "negative count (type %u field %u)", type, f);
      const uint8_t* ptr;
      memcpy(&ptr, s + F.offset, sizeof ptr);
      if (n == 0) {  // nothing to point at: the copy holds NULL in this slot
        if (ptr) null_slots.push_back({blk, elem * T.size + F.offset});
        continue;
      }
      if (!ptr)
        return fail(DC_EINVAL, "NULL pointer with count %llu (type %u field %u)", (unsigned long long)n,
                    type, f);
      uint64_t esz = F.kind == DC_F_ARRAY ? F.elem_size : S.types[F.child_type].size;
      if (n > UINT64_MAX / esz) return fail(DC_EINVAL, "block size overflows (type %u field %u)", type, f);
      uint32_t id;
      uint32_t depth = emitted[blk].depth;
      dc_status st = F.kind == DC_F_ARRAY
                         ? emit(ptr, n * esz, n, S.lane_of[type][f], type, f, blk,
                                elem * T.size + F.offset, depth, &id)
                         : emit(ptr, n * esz, n, 0, (uint32_t)F.child_type, NONE, blk,
                                elem * T.size + F.offset, depth + 1, &id);
      if (st) return st;
      p->ptr_target[emitted[blk].ptr_first + elem * S.nptr[type] + S.ptr_index[type][f]] = id;
    }
    return DC_OK;
  }

  dc_status run(const uint8_t* root) {
    uint32_t rt = S.root_type;
    uint32_t rid;
    dc_status st = emit(root, S.types[rt].size, 1, 0, rt, NONE, NONE, 0, 0, &rid);
    if (st) return st;
    std::vector<Frame> stack;
    if ((st = visit(rid, 0, rt))) return st;
    stack.push_back({rid, 0, rt, 0, 0});
    while (!stack.empty()) {
      Frame& fr = stack.back();
      const dc_type& T = S.types[fr.type];
      bool pushed = false;
      while (fr.field < T.nfields) {
        const dc_field& F = T.fields[fr.field];
        if (F.kind != DC_F_CHILD) {
          fr.field++;
          continue;
        }
        uint32_t tgt = p->ptr_target[emitted[fr.blk].ptr_first + fr.elem * S.nptr[fr.type] +
                                     S.ptr_index[fr.type][fr.field]];
        if (tgt == NONE || fr.k >= emitted[tgt].count) {
          fr.field++;
          fr.k = 0;
          continue;
        }
        uint64_t k = fr.k++;
        uint32_t ct = (uint32_t)F.child_type;
        if ((st = visit(tgt, k, ct))) return st;
        stack.push_back({tgt, k, ct, 0, 0});
        pushed = true;
        break;
      }
      if (!pushed) stack.pop_back();
    }
    return DC_OK;
  }
};

}  // namespace

// Block offsets and the relocation tables (the second half of dc_plan; run
// again by dc_plan_set_flags when DC_PLAN_PACK_SMALL changes).  Lanes follow
// each other in the arena, each starting on 16 bytes; every block starts on 16
// bytes, except that with DC_PLAN_PACK_SMALL an array block of fewer than
// DC_PACK_BYTES bytes starts at the next multiple of its element alignment (8
// bytes for f64, else 4): arrays of a few elements then lie back to back.  The
// relocation records hold offsets in units of the smallest block alignment: 16
// bytes, or 4 with packing.
dc_status layout(dc_plan_s* p) {
  const bool pack = (p->flags & DC_PLAN_PACK_SMALL) != 0;
  const uint32_t shift = pack ? 2 : 4, unit = 1u << shift;
  p->unit_shift = shift;
  const uint64_t nb = p->blocks.size();
  const uint32_t nl = p->schema.nlanes;
  const std::vector<uint64_t>& lane_start = p->lane_start;
  uint64_t off = 0;
  for (uint32_t l = 0; l < nl; l++) {
    off = round_up(off, 16);
    for (uint64_t i = lane_start[l]; i < lane_start[l + 1]; i++) {
      HostBlock& b = p->blocks[i];
      uint64_t al = 16;
      if (pack && l > 0 && b.bytes < DC_PACK_BYTES)
        al = p->schema.fields[b.type][b.field].elem_kind == DC_E_F64 ? 8 : 4;
      off = round_up(off, al);
      b.off = off;
      off += b.bytes;
      if (round_up(b.bytes, unit) >> shift > 0xFFFFFFFFull)
        return fail(DC_EINVAL, "block of %llu bytes: larger than 2^32 record units", (unsigned long long)b.bytes);
    }
  }
  p->data_bytes = round_up(off, 16);
  p->struct_bytes = p->nstruct_blocks ? p->blocks[p->nstruct_blocks - 1].off +
                                            round_up(p->blocks[p->nstruct_blocks - 1].bytes, 16)
                                      : 0;
  if (p->struct_bytes / 8 > 0xFFFFFFFFull) return fail(DC_EINVAL, "struct lane larger than 32 GiB");

  Trace phase("dc_plan", "reloc_tables");
  // Relocation tables: tile t covers the struct-lane bytes [t, t+1) * RELOC_SPAN;
  // its records are, lane by lane, the consecutive blocks whose slots lie there.
  const uint64_t ntiles = (p->struct_bytes + RELOC_SPAN - 1) / RELOC_SPAN;
  const uint64_t nr = p->roots.size();
  std::vector<uint64_t> cur(lane_start.begin(), lane_start.end() - 1), last(nl, 0);
  cur[0] += nr;  // the roots are pointed at by no slot
  auto slot = [&](uint64_t b) { return p->blocks[p->blocks[b].parent].off + p->blocks[b].slot_off; };
  p->rrec.clear();
  p->rseg.clear();
  p->rtiles.clear();
  p->rec_host.clear();
  p->rec_off.clear();
  p->rec_size.clear();
  p->rec_size.reserve(nb - nr);
  p->rrec.reserve(nb - nr);
  p->rec_host.reserve(nb - nr);
  p->rec_off.reserve(nb - nr);
  for (uint64_t t = 0; t < ntiles; t++) {
    const uint32_t tr0 = (uint32_t)p->rrec.size(), tg0 = (uint32_t)p->rseg.size();
    const uint64_t hi = (t + 1) * RELOC_SPAN;
    for (uint32_t l = 0; l < nl; l++) {
      // a record holds its target's offset from the group base in 32 bits of
      // units: a target 2^32 units or more past the base starts a new group
      uint64_t base = 0;
      bool open = false;
      for (; cur[l] < lane_start[l + 1] && slot(cur[l]) < hi; cur[l]++) {
        const HostBlock& b = p->blocks[cur[l]];
        const uint64_t sl = slot(cur[l]);
        if (b.parent == NONE || sl < last[l] || sl % 8)
          return fail(DC_EINVAL, "internal: lane %u is not in slot order at block %llu", l,
                      (unsigned long long)cur[l]);
        last[l] = sl + 8;
        const uint64_t u = b.off >> shift;
        if (!open || u - base > 0xFFFFFFFFull) {
          base = u;
          open = true;
          p->rseg.push_back(RelocSeg{base, (uint32_t)p->rrec.size(), 0});
        }
        const uint64_t g = p->rseg.size() - 1 - tg0;  // checked against RELOC_MAXGROUPS below
        const uint64_t w = (sl - t * RELOC_SPAN) / 8;  // < RELOC_MAXREC
        p->rrec.push_back(RelocRec{(uint32_t)(u - base), (uint32_t)(w | std::min<uint64_t>(g, 0xFFFF) << 16)});
        p->rec_host.push_back((uint64_t)(uintptr_t)b.host);
        p->rec_off.push_back(b.off);
        // the scan form's size: the distance to the next block of the lane (the
        // block's bytes and the padding after it), < 2^32 units (checked above)
        const uint64_t next = cur[l] + 1 < lane_start[l + 1] ? p->blocks[cur[l] + 1].off : round_up(b.off + b.bytes, unit);
        p->rec_size.push_back((uint32_t)((next - b.off) >> shift));
      }
    }
    if (p->rseg.size() - tg0 > RELOC_MAXGROUPS)
      return fail(DC_EINVAL, "relocation tile %llu needs more than %u lane groups", (unsigned long long)t,
                  RELOC_MAXGROUPS);
    const uint32_t nrt = (uint32_t)p->rrec.size() - tr0, ngt = (uint32_t)p->rseg.size() - tg0;
    if (nrt) p->rtiles.push_back(RelocTile{(uint32_t)t, tr0, tg0, nrt | ngt << 16});
  }
  p->rseg.push_back(RelocSeg{0, (uint32_t)p->rrec.size(), 0});
  for (uint32_t l = 0; l < nl; l++)
    if (cur[l] != lane_start[l + 1]) return fail(DC_EINVAL, "internal: lane %u has slots outside the struct lane", l);
  return DC_OK;
}

void scan_records(const dc_plan_s* p, RelocRec* out) {
  for (const RelocTile& T : p->rtiles) {
    const uint32_t ng = T.counts >> 16;
    for (uint32_t g = T.g0; g < T.g0 + ng; g++)
      for (uint32_t i = p->rseg[g].rec_begin; i < p->rseg[g + 1].rec_begin; i++) {
        const bool head = (i - T.r0) % SCAN_SLICE == 0 || i == p->rseg[g].rec_begin;
        out[i] = head ? RelocRec{p->rrec[i].off, p->rrec[i].where | SCAN_HEAD} : RelocRec{p->rec_size[i - 1], p->rrec[i].where};
      }
  }
}

dc_status build_plan(const dc_schema* schema, const void* const* roots, uint64_t nroots, dc_plan_s* p) {
  if (!roots || nroots == 0) return fail(DC_EINVAL, "no root");
  dc_status st = copy_schema(schema, &p->schema);
  if (st) return st;
  std::optional<Trace> phase;  // one traced phase at a time
  phase.emplace("dc_plan", "walk");
  Walker w(p);
  std::vector<uint32_t> root_ids;
  for (uint64_t i = 0; i < nroots; i++) {  // trees one after another; they must not share blocks
    if (!roots[i]) return fail(DC_EINVAL, "root %llu is NULL", (unsigned long long)i);
    root_ids.push_back((uint32_t)w.emitted.size());
    if ((st = w.run((const uint8_t*)roots[i]))) return st;
  }
  std::vector<HostBlock>& E = w.emitted;
  const uint64_t nb = E.size();

  // every block must be disjoint from every other (arrays included): sort the
  // blocks' host ranges by start and compare neighbours
  phase.emplace("dc_plan", "overlap");
  {
    std::vector<Span> by(nb);
    for (uint64_t i = 0; i < nb; i++) {
      const uint64_t a = (uint64_t)(uintptr_t)E[i].host;
      by[i] = Span{a, a + E[i].bytes, (uint32_t)i};
    }
    std::sort(by.begin(), by.end(), [](const Span& x, const Span& y) { return x.start < y.start; });
    for (uint64_t i = 1; i < nb; i++) {
      if (by[i - 1].end > by[i].start) {
        const uint32_t ia = by[i - 1].id, ib = by[i].id;
        const HostBlock& a = E[ia];
        const HostBlock& b = E[ib];
        // only child pointers can close a cycle: two struct blocks, one inside the other's ancestry
        const bool cyc = a.field == NONE && b.field == NONE &&
                         (w.is_ancestor(ia, b.parent) || w.is_ancestor(ib, a.parent));
        return fail(cyc ? DC_ECYCLE : DC_EALIAS, "host blocks at 0x%llx and 0x%llx overlap",
                    (unsigned long long)by[i - 1].start, (unsigned long long)by[i].start);
      }
    }
  }

  phase.emplace("dc_plan", "lanes");
  // Lanes in slot order: lane 0 holds the roots, then the child arrays breadth
  // first (each struct block's children by slot offset); every array lane holds
  // its blocks in the order of their parents, then of their slot offsets.  So
  // within every lane the slots that point at consecutive blocks ascend.
  const uint32_t nl = p->schema.nlanes;
  if (nl > RELOC_MAXGROUPS)
    return fail(DC_EINVAL, "the schema has %u ARRAY fields; at most %u are supported", nl - 1, RELOC_MAXGROUPS - 1);
  std::vector<uint32_t> kbeg(nb + 1, 0), kid(nb);
  for (uint64_t i = 0; i < nb; i++)
    if (E[i].parent != NONE) kbeg[E[i].parent + 1]++;
  for (uint64_t i = 0; i < nb; i++) kbeg[i + 1] += kbeg[i];
  {
    std::vector<uint32_t> fill(kbeg.begin(), kbeg.end() - 1);
    for (uint64_t i = 0; i < nb; i++)
      if (E[i].parent != NONE) kid[fill[E[i].parent]++] = (uint32_t)i;
  }
  // the walk emits a struct block's children element by element, each element's
  // in field order, so they are in slot order unless the schema lists its pointer
  // fields out of offset order
  auto by_slot = [&](uint32_t a, uint32_t b) { return E[a].slot_off < E[b].slot_off; };
  for (uint64_t i = 0; i < nb; i++)
    if (!std::is_sorted(kid.begin() + kbeg[i], kid.begin() + kbeg[i + 1], by_slot))
      std::sort(kid.begin() + kbeg[i], kid.begin() + kbeg[i + 1], by_slot);
  std::vector<std::vector<uint32_t>> lanes(nl);
  for (uint32_t r : root_ids) lanes[0].push_back(r);
  for (size_t q = 0; q < lanes[0].size(); q++)
    for (uint32_t k = kbeg[lanes[0][q]]; k < kbeg[lanes[0][q] + 1]; k++) lanes[E[kid[k]].lane].push_back(kid[k]);
  std::vector<uint64_t> lane_start(nl + 1, 0);
  for (uint32_t l = 0; l < nl; l++) lane_start[l + 1] = lane_start[l] + lanes[l].size();
  if (lane_start[nl] != nb) return fail(DC_EINVAL, "internal: %llu of %llu blocks reached in the lane order",
                                        (unsigned long long)lane_start[nl], (unsigned long long)nb);
  phase.emplace("dc_plan", "remap");
  std::vector<uint32_t> new_id(nb);
  for (uint32_t l = 0; l < nl; l++)
    for (size_t j = 0; j < lanes[l].size(); j++) new_id[lanes[l][j]] = (uint32_t)(lane_start[l] + j);
  // gather the blocks in arena order
  p->blocks.clear();
  p->blocks.reserve(nb);
  for (uint32_t l = 0; l < nl; l++)
    for (uint32_t old : lanes[l]) {
      HostBlock b = E[old];
      if (b.parent != NONE) b.parent = new_id[b.parent];
      p->blocks.push_back(b);
    }
  lanes.clear();
  for (auto& t : p->ptr_target)
    if (t != NONE) t = new_id[t];
  p->roots.clear();
  for (uint32_t r : root_ids) p->roots.push_back(new_id[r]);
  p->lane_start = lane_start;
  {
    dc_status st = layout(p);
    if (st) return st;
  }
  p->null_slots.clear();
  for (auto& ns : w.null_slots) p->null_slots.push_back(p->blocks[new_id[ns.first]].off + ns.second);
  std::sort(p->null_slots.begin(), p->null_slots.end());
  return DC_OK;
}

dc_status resolve(const dc_plan_s* p, uint64_t tree, const dc_step* path, uint32_t len, uint32_t* block,
                  uint64_t* within, uint32_t* type, uint64_t* elem_out) {
  if (len && !path) return fail(DC_EINVAL, "path is NULL");
  if (tree >= p->roots.size()) return fail(DC_EINVAL, "tree %llu out of range", (unsigned long long)tree);
  const SchemaCopy& S = p->schema;
  uint32_t blk = p->roots[tree];  // the tree's root struct block
  uint64_t elem = 0;
  uint32_t ti = S.root_type;
  for (uint32_t k = 0; k < len; k++) {
    const dc_type& T = S.types[ti];
    if (path[k].field >= T.nfields) return fail(DC_EINVAL, "step %u: no field %u", k, path[k].field);
    const dc_field& F = T.fields[path[k].field];
    if (F.kind == DC_F_SCALAR) return fail(DC_EINVAL, "step %u: field %u is a scalar", k, path[k].field);
    uint32_t tgt =
        p->ptr_target[p->blocks[blk].ptr_first + elem * S.nptr[ti] + S.ptr_index[ti][path[k].field]];
    if (tgt == NONE) return fail(DC_EINVAL, "step %u: pointer is empty", k);
    if (path[k].index >= p->blocks[tgt].count)
      return fail(DC_EINVAL, "step %u: index %llu out of range (%llu)", k,
                  (unsigned long long)path[k].index, (unsigned long long)p->blocks[tgt].count);
    if (F.kind == DC_F_ARRAY) {
      if (k + 1 != len) return fail(DC_EINVAL, "step %u: an array step must be the last", k);
      *block = tgt;
      *within = path[k].index * F.elem_size;
      *type = NONE;
      if (elem_out) *elem_out = 0;
      return DC_OK;
    }
    blk = tgt;
    elem = path[k].index;
    ti = (uint32_t)F.child_type;
  }
  *block = blk;
  *within = elem * S.types[ti].size;
  *type = ti;
  if (elem_out) *elem_out = elem;
  return DC_OK;
}

dc_status check_op(const dc_plan_s* p, const dc_op* op) {
  if (!op) return fail(DC_EINVAL, "op is NULL");
  const SchemaCopy& S = p->schema;
  if (op->kind != DC_OP_AXPY_HALF && op->kind != DC_OP_SCALE) return fail(DC_EINVAL, "op: unknown kind");
  if (op->sel != DC_SEL_ALL && op->sel != DC_SEL_CHAIN) return fail(DC_EINVAL, "op: unknown selection");
  if (op->sel == DC_SEL_CHAIN && op->path_len && !op->path) return fail(DC_EINVAL, "op: path is NULL");
  if (op->type >= S.types.size()) return fail(DC_EINVAL, "op: bad type");
  const dc_type& T = S.types[op->type];
  if (op->x_field >= T.nfields || T.fields[op->x_field].kind != DC_F_ARRAY)
    return fail(DC_EINVAL, "op: x_field is not an ARRAY field");
  const dc_field& X = T.fields[op->x_field];
  if (!((X.elem_kind == DC_E_F32 && X.elem_size == 4) || (X.elem_kind == DC_E_F64 && X.elem_size == 8)))
    return fail(DC_EINVAL, "op: x must be an f32 or f64 array");
  if (op->kind == DC_OP_AXPY_HALF) {
    if (op->y_field >= T.nfields || T.fields[op->y_field].kind != DC_F_ARRAY)
      return fail(DC_EINVAL, "op: y_field is not an ARRAY field");
    const dc_field& Y = T.fields[op->y_field];
    if (Y.elem_kind != X.elem_kind || Y.elem_size != X.elem_size)
      return fail(DC_EINVAL, "op: x and y differ in element type");
    if (op->y_field == op->x_field) return fail(DC_EINVAL, "op: x and y are the same field");
  }
  return DC_OK;
}

dc_status select_structs(const dc_plan_s* p, const dc_op* op,
                         std::vector<std::pair<uint32_t, uint64_t>>* out) {
  out->clear();
  if (op->sel == DC_SEL_CHAIN) {
    uint32_t blk, ty;
    uint64_t within, elem;
    dc_status st = resolve(p, 0, op->path, op->path_len, &blk, &within, &ty, &elem);
    if (st) return st;
    if (ty == NONE) return fail(DC_EINVAL, "op: the chain must end on a struct, not an array element");
    if (ty != op->type)
      return fail(DC_EINVAL, "op: the chain reaches a struct of type %u, not %u", ty, op->type);
    out->push_back({blk, elem});
    return DC_OK;
  }
  for (uint64_t b = 0; b < p->nstruct_blocks; b++) {
    const HostBlock& B = p->blocks[b];
    if (B.type != op->type) continue;
    for (uint64_t e = 0; e < B.count; e++) out->push_back({(uint32_t)b, e});
  }
  return DC_OK;
}

void path_to(const dc_plan_s* p, uint32_t block, uint64_t elem, std::vector<dc_step>* out) {
  out->clear();
  const SchemaCopy& S = p->schema;
  while (p->blocks[block].parent != NONE) {
    const HostBlock& B = p->blocks[block];
    const HostBlock& P = p->blocks[B.parent];
    uint32_t psize = S.types[P.type].size;
    uint32_t foff = B.slot_off % psize;
    uint32_t field = 0;
    for (uint32_t f = 0; f < S.types[P.type].nfields; f++)
      if (S.fields[P.type][f].kind == DC_F_CHILD && S.fields[P.type][f].offset == foff) field = f;
    out->push_back({field, elem});
    elem = B.slot_off / psize;
    block = B.parent;
  }
  std::reverse(out->begin(), out->end());
}

}  // namespace dc
