// plan_shim.cpp — test infrastructure: the host walk and layout (build_plan)
// behind a C entry point, built with AddressSanitizer and UBSan by
// tests/test_host_sanitizers.py and run on the CPU.  Besides planning, it
// checks the relocation tables the way the relocation kernel reads them:
// every slot inside its tile, each record in the lane group it names, each
// group's base plus the record's offset equal to the plan's own offset of the
// target block, the slot the record names being the one that points at that
// block, the running sum of the records' sizes within each group equal to the
// record's offset, and the device-scan records (slice heads with offsets, the
// rest with their predecessors' sizes), summed per slice from each head as the
// device-scan relocation does, equal to the same offsets.  With `pack`
// the plan is laid out again with DC_PLAN_PACK_SMALL (as dc_plan_set_flags does)
// and every block's alignment is checked against the packing rule.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "internal.hpp"

namespace {
char g_msg[256];
int bad(const char* what, unsigned long long a, unsigned long long b) {
  std::snprintf(g_msg, sizeof g_msg, "%s (%llu, %llu)", what, a, b);
  return 1000;
}
}  // namespace

extern "C" const char* shim_message() { return g_msg; }

// Returns the dc_status of planning, 1000 when a table check fails (message in
// shim_message()), else 0; out[0..5] = blocks, records, groups, listed tiles, data bytes, struct bytes.
extern "C" int shim_plan(const dc_schema* schema, const void* const* roots, uint64_t nroots, int pack,
                         uint64_t* out) {
  dc_plan_s* p = new dc_plan_s;
  int st = dc::build_plan(schema, roots, nroots, p);
  if (!st && pack) {
    p->flags |= DC_PLAN_PACK_SMALL;
    st = dc::layout(p);
  }
  if (st) {
    delete p;
    return st;
  }
  const uint32_t shift = p->unit_shift;
  if (shift != (pack ? 2u : 4u)) {
    delete p;
    return bad("record unit", shift, pack);
  }
  for (size_t i = 0; i < p->blocks.size(); i++) {  // the layout rule, block by block
    const dc::HostBlock& b = p->blocks[i];
    const bool small = pack && b.lane > 0 && b.bytes < DC_PACK_BYTES;
    const uint64_t al = !small ? 16 : p->schema.fields[b.type][b.field].elem_kind == DC_E_F64 ? 8 : 4;
    const bool lane_first = i == 0 || p->blocks[i - 1].lane != b.lane;
    uint64_t want = i ? p->blocks[i - 1].off + p->blocks[i - 1].bytes : 0;  // the previous block's end
    if (lane_first) want = (want + 15) / 16 * 16;                             // a lane starts on 16 bytes
    want = (want + al - 1) / al * al;
    if (b.off != want) {
      delete p;
      return bad("block offset breaks the layout rule", i, b.off);
    }
  }
  out[0] = p->blocks.size();
  out[1] = p->rrec.size();
  out[2] = p->rseg.size() - 1;
  out[3] = p->rtiles.size();
  out[4] = p->data_bytes;
  out[5] = p->struct_bytes;
  int rc = 0;
  uint64_t seen = 0;
  std::unordered_map<uint64_t, size_t> by_off;  // arena offset -> block
  for (size_t i = 0; i < p->blocks.size(); i++) by_off.emplace(p->blocks[i].off, i);
  for (const dc::RelocTile& T : p->rtiles) {
    const uint32_t nr = T.counts & 0xFFFFu, ng = T.counts >> 16;
    const uint64_t lo = (uint64_t)T.t * dc::RELOC_SPAN, hi = std::min<uint64_t>(p->struct_bytes, lo + dc::RELOC_SPAN);
    if (!nr || !ng || ng > dc::RELOC_MAXGROUPS || T.r0 != seen || T.g0 + ng > p->rseg.size() - 1) {
      rc = bad("tile header", T.t, T.counts);
      break;
    }
    seen = T.r0 + nr;
    if (p->rseg[T.g0].rec_begin != T.r0 || p->rseg[T.g0 + ng].rec_begin != T.r0 + nr) {
      rc = bad("tile groups do not cover its records", T.t, ng);
      break;
    }
    for (uint32_t g = T.g0; g < T.g0 + ng && !rc; g++) {
      const dc::RelocSeg& G = p->rseg[g];
      uint64_t prefix = 0;  // the device-scan form: sizes summed from the group's first record
      for (uint32_t i = G.rec_begin; i < p->rseg[g + 1].rec_begin; i++) {
        const dc::RelocRec& R = p->rrec[i];
        if (prefix != R.off) {
          rc = bad("prefix of the group's sizes differs from the record's offset", prefix, R.off);
          break;
        }
        prefix += p->rec_size[i];
        const uint64_t slot = lo + (uint64_t)(R.where & 0xFFFFu) * 8;
        if (slot + 8 > hi) {
          rc = bad("slot outside its tile", slot, T.t);
          break;
        }
        if ((R.where >> 16) != g - T.g0) {
          rc = bad("record names another lane group", R.where >> 16, g - T.g0);
          break;
        }
        if ((G.base + R.off) << shift != p->rec_off[i]) {
          rc = bad("base + offset differs from the plan's offset", (G.base + R.off) << shift, p->rec_off[i]);
          break;
        }
        // the slot is the one that points at the block at that offset
        const auto b = by_off.find(p->rec_off[i]);
        if (b == by_off.end() || p->blocks[b->second].parent == dc::NONE ||
            p->blocks[p->blocks[b->second].parent].off + p->blocks[b->second].slot_off != slot) {
          rc = bad("the slot does not point at the record's target", slot, p->rec_off[i]);
          break;
        }
      }
    }
    if (rc) break;
  }
  if (!rc && seen != p->rrec.size()) rc = bad("records outside every tile", seen, p->rrec.size());
  // The device-scan records, summed the way the kernel does (per tile, slices of
  // 32 records, each sum restarting at a head), give back every record's offset.
  std::vector<dc::RelocRec> sr(p->rrec.size());
  if (!rc) dc::scan_records(p, sr.data());
  for (const dc::RelocTile& T : p->rtiles) {
    if (rc) break;
    const uint32_t nr = T.counts & 0xFFFFu;
    uint32_t sum = 0;
    for (uint32_t j = 0; j < nr; j++) {
      const dc::RelocRec& R = sr[T.r0 + j];
      const bool head = (R.where & dc::SCAN_HEAD) != 0;
      if ((j % dc::SCAN_SLICE == 0) != (head && j % dc::SCAN_SLICE == 0) ||
          (R.where & ~dc::SCAN_HEAD) != p->rrec[T.r0 + j].where) {
        rc = bad("scan record's head flag or slot word", T.r0 + j, R.where);
        break;
      }
      sum = head ? R.off : sum + R.off;
      if (sum != p->rrec[T.r0 + j].off) {
        rc = bad("the scan records' segmented sum differs from the record's offset", sum, p->rrec[T.r0 + j].off);
        break;
      }
    }
  }
  delete p;
  return rc;
}

// Span staging on the CPU: plan with `flags` (DC_PLAN_PACK_SMALL lays the plan
// out again), then check the spans (host order, gaps of SPAN_GAP or more between
// them, staging offsets in order with their host address's phase modulo 16)
// and the placement table (pieces in staging order that, taken in arena order,
// cover every staged block exactly, read inside the staging area, and pad only up to the block's 16-byte
// slot end or the next block).  With `emulate`, copy the spans into a staging
// buffer as the deep copy does (reading the gaps: only for trees whose blocks
// share one allocation), zero the NULL-slot fix-ups, apply the table to an
// arena image filled with 0xAB, and check every block's bytes and that every
// other byte of the data region is zero.  out[0..3] = span staging on, staging
// bytes, spans, pieces.  Returns 1000 on a failed check (message in
// shim_message()), else the planning status.
extern "C" int shim_spans(const dc_schema* schema, const void* const* roots, uint64_t nroots, uint32_t flags,
                          int emulate, uint64_t* out) {
  dc_plan_s* p = new dc_plan_s;
  int st = dc::build_plan(schema, roots, nroots, p);
  if (!st && (flags & DC_PLAN_PACK_SMALL)) {
    p->flags |= DC_PLAN_PACK_SMALL;
    st = dc::layout(p);
  }
  if (st) {
    delete p;
    return st;
  }
  dc::plan_spans(p);
  p->flags |= flags;
  dc::choose_spans(p);
  out[0] = p->span_mode;
  out[1] = p->span_bytes;
  out[2] = p->spans.size();
  out[3] = 0;
  if (!p->span_mode) {
    delete p;
    return 0;
  }
  int rc = 0;
  for (size_t i = 0; i < p->spans.size() && !rc; i++) {
    const dc::HostSpan& S = p->spans[i];
    if (S.stage % 16 != (uint64_t)(uintptr_t)S.host % 16 || S.stage + S.bytes > p->span_bytes)
      rc = bad("span's staging offset", i, S.stage);
    else if (i && (S.host < p->spans[i - 1].host + p->spans[i - 1].bytes ||
                   (uint64_t)(S.host - (p->spans[i - 1].host + p->spans[i - 1].bytes)) < dc::SPAN_GAP ||
                   S.stage < p->spans[i - 1].stage + p->spans[i - 1].bytes))
      rc = bad("spans out of order or closer than the merge gap", i, S.stage);
  }
  std::vector<dc::PlaceDesc> pd;
  dc::build_place_table(p, &pd);
  out[3] = pd.size();
  for (size_t i = 1; i < pd.size() && !rc; i++)  // staging order
    if ((pd[i].src & ((1ull << 60) - 1)) < (pd[i - 1].src & ((1ull << 60) - 1))) rc = bad("pieces not in staging order", i, 0);
  std::sort(pd.begin(), pd.end(), [](const dc::PlaceDesc& a, const dc::PlaceDesc& b) { return a.dst < b.dst; });
  size_t k = 0;
  const uint64_t nb = p->blocks.size();
  for (uint64_t b = 0; b < nb && !rc; b++) {  // the pieces of each block, in arena order
    const dc::HostBlock& B = p->blocks[b];
    const dc::HostSpan& S = dc::span_at(p, B.host);
    if (B.host < S.host || B.host + B.bytes > S.host + S.bytes) {
      rc = bad("block outside its span", b, B.off);
      break;
    }
    const uint64_t end = B.off + B.bytes, next = b + 1 < nb ? p->blocks[b + 1].off : p->data_bytes;
    for (uint64_t o = 0; o < B.bytes && !rc; k++) {
      if (k >= pd.size()) {
        rc = bad("placement table ends early", b, o);
        break;
      }
      const uint64_t src = pd[k].src & ((1ull << 60) - 1), pad = pd[k].src >> 60, dst = pd[k].dst >> 16;
      const uint64_t w = (pd[k].dst & 0xFFFFu) + 1, n = w - pad;
      const bool last = o + n == B.bytes;
      if (dst != B.off + o || src != S.stage + (uint64_t)(B.host - S.host) + o || n > dc::PLACE_PIECE ||
          src + n > p->span_bytes)
        rc = bad("piece's source or destination", b, o);
      else if (pad >= 16 || (!last && pad) || (last && dst + w != std::min(dc::round_up(end, 16), next)))
        rc = bad("piece's padding", b, pad);
      o += n;
    }
  }
  if (!rc && k != pd.size()) rc = bad("placement table has extra pieces", k, pd.size());
  if (!rc && emulate) {
    std::vector<uint8_t> stage(p->span_bytes, 0), img(p->data_bytes, 0xAB);
    for (const dc::HostSpan& S : p->spans) memcpy(stage.data() + S.stage, S.host, S.bytes);
    for (uint64_t o : dc::span_null_offsets(p)) memset(stage.data() + o, 0, 8);
    for (const dc::PlaceDesc& d : pd) {
      const uint64_t src = d.src & ((1ull << 60) - 1), pad = d.src >> 60, dst = d.dst >> 16;
      const uint64_t w = (d.dst & 0xFFFFu) + 1;
      memcpy(img.data() + dst, stage.data() + src, w - pad);
      memset(img.data() + dst + (w - pad), 0, pad);
    }
    std::vector<uint8_t> want(p->data_bytes, 0);  // the blocks' bytes, NULL slots zeroed; zero elsewhere
    for (const dc::HostBlock& B : p->blocks) memcpy(want.data() + B.off, B.host, B.bytes);
    for (uint64_t o : p->null_slots) memset(want.data() + o, 0, 8);
    for (uint64_t i = 0; i < p->data_bytes && !rc; i++)
      if (img[i] != want[i]) rc = bad("emulated arena byte", i, img[i]);
  }
  delete p;
  return rc;
}
