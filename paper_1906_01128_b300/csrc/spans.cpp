// spans.cpp — span staging's host side: which blocks a deep copy stages, the
// host spans they lie in (blocks less than SPAN_GAP bytes apart, merged), the
// rule that picks span staging, and the placement table that puts every staged
// block at its arena offset once the spans are on the device (place_kernel).
// Host only: no CUDA call, so the host sanitizer tests build it on the CPU.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "internal.hpp"

namespace dc {

// The struct block that holds arena offset `off` (a slot of a struct block).
uint64_t struct_block_at(const dc_plan_s* p, uint64_t off) {
  auto it = std::upper_bound(p->blocks.begin(), p->blocks.begin() + p->nstruct_blocks, off,
                             [](uint64_t o, const HostBlock& hb) { return o < hb.off; });
  return (uint64_t)(it - p->blocks.begin()) - 1;
}

// Per block: 1 if it is a struct block with a NULL-slot fix-up (such blocks go
// through the pinned arena even when they live in a host arena).
std::vector<uint8_t> null_fixups(const dc_plan_s* p) {
  std::vector<uint8_t> fixup(p->blocks.size(), 0);
  for (uint64_t off : p->null_slots) fixup[struct_block_at(p, off)] = 1;
  return fixup;
}

// The span holding host address h (spans are in host order, h inside one).
const HostSpan& span_at(const dc_plan_s* p, const uint8_t* h) {
  auto it = std::upper_bound(p->spans.begin(), p->spans.end(), h,
                             [](const uint8_t* a, const HostSpan& sp) { return a < sp.host; });
  return *(it - 1);
}

void plan_spans(dc_plan_s* p) {
  p->spans.clear();
  p->span_bytes = 0;
  p->span_worth = false;
  p->spans_built = false;
  p->span_nstaged = p->span_staged = 0;
  const std::vector<uint8_t> fixup = null_fixups(p);
  for (uint64_t b = 0; b < p->blocks.size(); b++) {  // the blocks a full deep copy stages
    const HostBlock& B = p->blocks[b];
    if ((!fixup[b] && in_host_arena(B.host, B.bytes, nullptr)) || !B.bytes) continue;
    p->span_nstaged++;
    p->span_staged += B.bytes;
  }
  const char* v = getenv("DC_SPANS");
  p->span_rule = !(v && v[0] == '0') && p->span_nstaged >= DC_SPAN_MIN_BLOCKS &&
                 p->span_staged < (uint64_t)DC_SPAN_MAX_MEAN * p->span_nstaged;
}

namespace {

// The spans themselves (a sort of the staged blocks by host address), built
// the first time span staging is asked for or the rule's counts allow it.
void build_spans(dc_plan_s* p) {
  p->spans_built = true;
  const std::vector<uint8_t> fixup = null_fixups(p);
  std::vector<std::pair<const uint8_t*, uint64_t>> hb;
  hb.reserve(p->span_nstaged);
  for (uint64_t b = 0; b < p->blocks.size(); b++) {
    const HostBlock& B = p->blocks[b];
    if ((!fixup[b] && in_host_arena(B.host, B.bytes, nullptr)) || !B.bytes) continue;
    hb.push_back({B.host, B.bytes});
  }
  std::sort(hb.begin(), hb.end());
  for (const auto& x : hb) {
    if (!p->spans.empty()) {
      HostSpan& S = p->spans.back();
      const uint8_t* end = S.host + S.bytes;
      if (x.first >= end && (uint64_t)(x.first - end) < SPAN_GAP) {  // blocks never overlap
        S.bytes = (uint64_t)(x.first + x.second - S.host);
        continue;
      }
    }
    p->spans.push_back({x.first, x.second, 0});
  }
  uint64_t o = 0;
  for (HostSpan& S : p->spans) {  // each span keeps its host address's phase modulo 16
    o = round_up(o, 16) + ((uintptr_t)S.host & 15);
    S.stage = o;
    o += S.bytes;
  }
  p->span_bytes = round_up(o, 16);
  p->span_worth = p->span_rule && p->span_bytes * 4 <= p->span_staged * 5;
}

}  // namespace

void choose_spans(dc_plan_s* p) {
  p->span_mode = false;
  if ((p->flags & DC_PLAN_MAP_HOST) || !p->span_nstaged) return;
  if (!(p->flags & DC_PLAN_SPANS) && !p->span_rule) return;  // no sort where the rule cannot fire
  if (!p->spans_built) build_spans(p);
  p->span_mode = !p->spans.empty() && ((p->flags & DC_PLAN_SPANS) || p->span_worth);
}

uint64_t pin_arena_bytes(const dc_plan_s* p) {
  return std::max(p->data_bytes, p->span_mode ? p->span_bytes : 0);
}

std::vector<uint64_t> span_null_offsets(const dc_plan_s* p) {
  std::vector<uint64_t> out;
  for (uint64_t off : p->null_slots) {  // where each NULL-slot fix-up lies in the staging area
    const HostBlock& B = p->blocks[struct_block_at(p, off)];
    const uint8_t* h = B.host + (off - B.off);
    const HostSpan& S = span_at(p, h);
    out.push_back(S.stage + (uint64_t)(h - S.host));
  }
  std::sort(out.begin(), out.end());
  return out;
}

void build_place_table(const dc_plan_s* p, std::vector<PlaceDesc>* out) {
  // every staged block from its place in the staging area to the arena, in
  // pieces of at most PLACE_PIECE bytes; the last piece also zeroes the block's
  // slot up to 16 bytes where the next block does not start before that
  out->clear();
  const uint64_t nb = p->blocks.size();
  for (uint64_t b = 0; b < nb; b++) {
    const HostBlock& B = p->blocks[b];
    if ((b < p->ihi.size() && p->ihi[b] > p->ilo[b]) || !B.bytes) continue;  // moved in place (a host arena)
    const HostSpan& S = span_at(p, B.host);
    const uint64_t src = S.stage + (uint64_t)(B.host - S.host), end = B.off + B.bytes;
    const uint64_t next = b + 1 < nb ? p->blocks[b + 1].off : p->data_bytes;
    const uint64_t pad = std::min(round_up(end, 16), std::max(next, end)) - end;
    for (uint64_t o = 0; o < B.bytes; o += PLACE_PIECE) {
      const uint64_t n = std::min(PLACE_PIECE, B.bytes - o), z = o + n == B.bytes ? pad : 0;
      out->push_back({(src + o) | (z << 60), (B.off + o) << 16 | (n + z - 1)});
    }
  }
  // in staging order: a warp then reads consecutive bytes, and its writes go to a
  // few runs of consecutive slots, one per lane (no two pieces write the same byte)
  std::sort(out->begin(), out->end(), [](const PlaceDesc& a, const PlaceDesc& b) {
    return (a.src & ((1ull << 60) - 1)) < (b.src & ((1ull << 60) - 1));
  });
}

}  // namespace dc
