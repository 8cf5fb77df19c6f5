// step.cpp — dc_roundtrip: Algorithm 2's transfer, kernel and transfer back as one
// pipelined call.
//
// Blocks the op does not touch (structs, other arrays) move as in
// dc_deep_copy; the relocation runs; then one stream_kernel launch reads the
// selected x and y arrays from host memory, applies the leaf update, writes x
// and y into the arena and the updated x straight back to the host.  The host
// -> device and device -> host traffic of the leaf arrays thus overlap on the
// link instead of following each other.  Needs a DC_PLAN_MAP_HOST plan whose
// selected arrays start on 16-byte host addresses and on 16 bytes in the arena;
// otherwise the call runs dc_deep_copy, dc_update_leaves and dc_copy_back in
// turn (same results).
//
// The pass runs in tile groups (up to STEP_GROUPS launches): the host
// marshals the array pieces that group g+1 reads from the pinned arena and
// scatters the pieces group g-1 wrote there while the device streams group g.
#include <algorithm>

#include "internal.hpp"

using namespace dc;

namespace {

constexpr uint64_t STEP_GROUPS = 8;
constexpr uint64_t STEP_GROUP_MIN = 4ull << 20;  // x bytes per group at least

// The op's blocks and the rest, their moves, and (when the fused kernel can
// run: `direct` and 16-byte aligned host arrays) its device tables.
dc_status build_step(dc_plan_s* p, const dc_op* op, bool direct, cudaStream_t s) {
  std::vector<Pick> picks;
  dc_status st = pick(p, op, &picks);
  if (st) return st;
  const uint64_t nb = p->blocks.size();
  const bool axpy = op->kind == DC_OP_AXPY_HALF;
  p->step_fused = direct;
  std::vector<uint8_t> mark(nb, 0);
  for (const auto& k : picks) {
    mark[k.bx] = 1;
    if (axpy && k.by != NONE) mark[k.by] = 1;
    if ((uintptr_t)p->blocks[k.bx].host % 16 || (axpy && (uintptr_t)p->blocks[k.by].host % 16)) p->step_fused = false;
    if (p->blocks[k.bx].off % 16 || (axpy && p->blocks[k.by].off % 16)) p->step_fused = false;  // packed arenas
  }
  std::vector<uint32_t> rest, xy, x;
  for (uint32_t b = 0; b < nb; b++) (mark[b] ? xy : rest).push_back(b);
  for (const auto& k : picks) x.push_back(k.bx);
  std::sort(x.begin(), x.end());
  plan_moves(p, rest, &p->step_rest);
  plan_moves(p, xy, &p->step_xy);      // the parts of x and y outside mapped interiors
  plan_moves(p, x, &p->step_xback);    // the parts of x the host scatters afterwards
  p->step_written = x;
  p->step_gen = ++p->gen;
  if (!p->step_fused) return DC_OK;
  const uint64_t base = (uint64_t)(uintptr_t)p->dev, pin = (uint64_t)(uintptr_t)p->pinned_dev;
  std::vector<MoveDesc> d;
  for (uint32_t b : p->step_rest.interiors)
    push_desc(&d, p->idev[b], base + p->blocks[b].off + (p->ilo[b] - (uint64_t)(uintptr_t)p->blocks[b].host),
              p->ihi[b] - p->ilo[b]);
  if ((st = upload(p, d, p->L.sta, p->L.stat, p->L.tab_cap, &p->st_int_nd, &p->st_int_units, s))) return st;
  d.clear();
  for (const auto& r : p->step_rest.runs) push_desc(&d, pin + r.lo, base + r.lo, r.hi - r.lo);
  if ((st = upload(p, d, p->L.stb, p->L.stbt, p->L.tab_cap, &p->st_run_nd, &p->st_run_units, s))) return st;
  // the fused segments
  const uint64_t esz = p->schema.fields[op->type][op->x_field].elem_size;
  std::vector<StreamSeg> seg(picks.size());
  uint64_t u = 0;
  for (size_t i = 0; i < picks.size(); i++) {
    const HostBlock& X = p->blocks[picks[i].bx];
    StreamSeg g{};
    g.xd = base + X.off;
    g.n = X.count;
    g.ubeg = u;
    g.xh = (uint64_t)(uintptr_t)X.host;
    g.xlo = p->ilo[picks[i].bx];
    g.xhi = p->ihi[picks[i].bx];
    g.xi = p->idev[picks[i].bx];
    g.xp = pin + X.off;
    if (axpy) {
      const HostBlock& Y = p->blocks[picks[i].by];
      g.yd = base + Y.off;
      g.yh = (uint64_t)(uintptr_t)Y.host;
      g.ylo = p->ilo[picks[i].by];
      g.yhi = p->ihi[picks[i].by];
      g.yi = p->idev[picks[i].by];
      g.yp = pin + Y.off;
    }
    seg[i] = g;
    u += (X.count * esz + 15) / 16;
  }
  p->st_nseg = seg.size();
  p->st_units = u;
  const uint64_t ntiles = (u + LEAF_TILE - 1) / LEAF_TILE;
  // tile groups: a piece in the pinned arena is marshalled for the group of its array's first
  // tile and scattered after the group of its last tile
  // groups only pay when there are host copies to overlap: the bytes of x and y that go through
  // the pinned arena (the rest is read and written in place by the kernel)
  uint64_t staged = 0;
  for (const auto& f : p->step_xy.frags) staged += f.len;
  const uint64_t ng = staged < STEP_GROUP_MIN
                          ? 1
                          : std::max<uint64_t>(1, std::min<uint64_t>({STEP_GROUPS, ntiles, u * 16 / STEP_GROUP_MIN}));
  p->step_cut.assign(ng + 1, 0);
  for (uint64_t g = 0; g <= ng; g++) p->step_cut[g] = ntiles * g / ng;
  auto group_of = [&](uint64_t t) {
    return (uint64_t)(std::upper_bound(p->step_cut.begin(), p->step_cut.end(), t) - p->step_cut.begin()) - 1;
  };
  std::vector<std::vector<uint32_t>> in(ng), out(ng);
  for (size_t i = 0; i < picks.size(); i++) {
    const uint64_t nu = (p->blocks[picks[i].bx].count * esz + 15) / 16;
    const uint64_t t0 = seg[i].ubeg / LEAF_TILE, t1 = (seg[i].ubeg + std::max<uint64_t>(nu, 1) - 1) / LEAF_TILE;
    in[std::min(group_of(t0), ng - 1)].push_back(picks[i].bx);
    if (axpy) in[std::min(group_of(t0), ng - 1)].push_back(picks[i].by);
    out[std::min(group_of(t1), ng - 1)].push_back(picks[i].bx);
  }
  p->step_in.assign(ng, dc_plan_s::Moves());
  p->step_out.assign(ng, dc_plan_s::Moves());
  for (uint64_t g = 0; g < ng; g++) {
    std::sort(in[g].begin(), in[g].end());
    std::sort(out[g].begin(), out[g].end());
    plan_moves(p, in[g], &p->step_in[g]);
    plan_moves(p, out[g], &p->step_out[g]);
  }
  while (p->step_ev.size() < ng) {
    cudaEvent_t e;
    DC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    p->step_ev.push_back(e);
  }
  if (!seg.empty()) {
    if (ntiles + 1 > p->L.tseg_cap || seg.size() > p->L.seg_cap) return fail(DC_EINVAL, "step table larger than planned");
    std::vector<uint32_t> tiles;
    for (uint64_t t = 0, k = 0; t < ntiles; t++) {
      while (k + 1 < seg.size() && seg[k + 1].ubeg <= t * LEAF_TILE) k++;
      tiles.push_back((uint32_t)k);
    }
    tiles.push_back((uint32_t)(seg.size() - 1));
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.sts, seg.data(), seg.size() * sizeof(StreamSeg), cudaMemcpyHostToDevice, s));
    DC_CUDA(cudaMemcpyAsync(p->dev + p->L.stst, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, s));
  }
  return DC_OK;
}

dc_status prepare_step(dc_plan_s* p, const dc_op* op, cudaStream_t s) {
  const bool direct = (p->flags & DC_PLAN_MAP_HOST) || p->has_arena_blocks;
  OpKey key = key_of(op);
  if (key == p->step_key) return DC_OK;
  dc_status st = wait_event(p->h2d_done);
  if (st) return st;
  if ((st = build_step(p, op, direct, s))) return st;
  p->step_key = key;
  return DC_OK;
}

// The fused pass, group by group: marshal group g's pieces, launch its tiles, and while the
// device streams it, scatter the pieces of group g-1.  Ends with the stream synchronized and the
// device error word read.  On an error the caller's x arrays may hold part of the results.
dc_status run_step_groups(dc_plan_s* p, const dc_op* op, cudaStream_t s) {
  StreamArgs a;
  a.seg = reinterpret_cast<const StreamSeg*>(p->dev + p->L.sts);
  a.tile_seg = reinterpret_cast<const uint32_t*>(p->dev + p->L.stst);
  a.nseg = (uint32_t)p->st_nseg;
  a.units = p->st_units;
  a.kind = op->kind;
  a.f64 = p->schema.fields[op->type][op->x_field].elem_kind == DC_E_F64;
  a.scale = op->scale;
  const uint64_t ng = p->step_in.size();
  dc_status st0;
  for (uint64_t g = 0; g < ng; g++) {
    {
      Trace tr("dc_roundtrip", "marshal");
      host_copy(p, p->step_in[g], 0, p->step_in[g].units.size(), true);
    }
    a.t_begin = p->step_cut[g];
    a.t_end = p->step_cut[g + 1];
    DC_CUDA(launch_stream(a, s, p->sm_count));
    DC_CUDA(cudaEventRecord(p->step_ev[g], s));
    if (g) {
      Trace tr("dc_roundtrip", "scatter");
      if ((st0 = wait_event(p->step_ev[g - 1]))) return st0;
      host_copy(p, p->step_out[g - 1], 0, p->step_out[g - 1].units.size(), false);
    }
  }
  DC_CUDA(cudaEventRecord(p->h2d_done, s));  // the pinned arena is free once the pass has read it
  p->written = &p->step_written;
  p->written_gen = p->step_gen;
  p->op_run = true;
  dc_status st;
  {
    Trace tr("dc_roundtrip", "device+wait");
    if ((st = device_error(p, s))) return st;  // synchronizes the stream
  }
  Trace tr("dc_roundtrip", "scatter");
  if (ng) host_copy(p, p->step_out[ng - 1], 0, p->step_out[ng - 1].units.size(), false);
  return DC_OK;
}

}  // namespace

extern "C" dc_status dc_roundtrip(dc_plan_t p, const dc_op* op, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  dc_status st = check_op(p, op);
  if (st) return st;
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  pool_of(p);
  {
    Trace tr("dc_roundtrip", "tables");
    if ((st = prepare_step(p, op, s))) return st;
  }
  if (!p->step_fused) {
    if ((st = dc_deep_copy(p, stream))) return st;
    if ((st = dc_update_leaves(p, op, stream))) return st;
    return dc_copy_back(p, 0, stream);
  }
  if ((st = wait_event(p->h2d_done))) return st;  // the pinned arena is rewritten below
  // blocks outside the op: as in dc_deep_copy
  if ((st = launch_table(p, p->L.sta, p->L.stat, p->st_int_nd, p->st_int_units, s))) return st;
  {
    Trace tr("dc_roundtrip", "marshal");
    host_copy(p, p->step_rest, 0, p->step_rest.units.size(), true);
    size_t ns = 0;
    null_slots_upto(p, &ns, ~0ull);
  }
  if ((st = launch_table(p, p->L.stb, p->L.stbt, p->st_run_nd, p->st_run_units, s))) return st;
  if ((st = dc_relocate(p, stream))) return st;
  // the selected arrays: host -> update -> arena and host, in one pass per tile group
  return run_step_groups(p, op, s);
}

extern "C" dc_status dc_roundtrip_selected(dc_plan_t p, const dc_op* op, dc_stream_t stream) {
  if (!p) return fail(DC_EINVAL, "plan is NULL");
  dc_status st = check_op(p, op);
  if (st) return st;
  if (!p->dev) return fail(DC_ESTATE, "no device buffer bound");
  cudaStream_t s = stream;
  pool_of(p);
  if ((st = prepare_step(p, op, s))) return st;
  if ((st = wait_event(p->h2d_done))) return st;
  // only the op's arrays move, by their effective addresses (Sec. 3)
  if (p->step_fused) return run_step_groups(p, op, s);
  host_copy(p, p->step_xy, 0, p->step_xy.units.size(), true);
  for (const auto& r : p->step_xy.runs)
    DC_CUDA(cudaMemcpyAsync(p->dev + r.lo, p->pinned + r.lo, r.hi - r.lo, cudaMemcpyHostToDevice, s));
  DC_CUDA(cudaEventRecord(p->h2d_done, s));
  if ((st = dc_update_leaves(p, op, stream))) return st;
  return dc_copy_back(p, 0, stream);
}
