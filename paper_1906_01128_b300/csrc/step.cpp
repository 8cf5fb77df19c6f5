// step.cpp — dc_roundtrip: Algorithm 2's transfer, kernel and transfer back as one
// pipelined call.
//
// Blocks the op does not touch (structs, other arrays) move as in
// dc_deep_copy; the relocation runs; then one stream_kernel launch reads the
// selected x and y arrays from host memory, applies the leaf update, writes x
// and y into the arena and the updated x straight back to the host.  The host
// -> device and device -> host traffic of the leaf arrays thus overlap on the
// link instead of following each other.  Needs a DC_PLAN_MAP_HOST plan whose
// selected arrays start on 16-byte host addresses; otherwise the call runs
// dc_deep_copy, dc_update_leaves and dc_copy_back in turn (same results).
#include <algorithm>

#include "internal.hpp"

using namespace dc;

namespace {

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
  if (!seg.empty()) {
    const uint64_t ntiles = (u + LEAF_TILE - 1) / LEAF_TILE;
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

dc_status launch_step_kernel(dc_plan_s* p, const dc_op* op, cudaStream_t s) {
  StreamArgs a;
  a.seg = reinterpret_cast<const StreamSeg*>(p->dev + p->L.sts);
  a.tile_seg = reinterpret_cast<const uint32_t*>(p->dev + p->L.stst);
  a.nseg = (uint32_t)p->st_nseg;
  a.units = p->st_units;
  a.kind = op->kind;
  a.f64 = p->schema.fields[op->type][op->x_field].elem_kind == DC_E_F64;
  a.scale = op->scale;
  DC_CUDA(launch_stream(a, s, p->sm_count));
  p->written = &p->step_written;
  p->written_gen = p->step_gen;
  p->op_run = true;
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
  if ((st = prepare_step(p, op, s))) return st;
  if (!p->step_fused) {
    if ((st = dc_deep_copy(p, stream))) return st;
    if ((st = dc_update_leaves(p, op, stream))) return st;
    return dc_copy_back(p, 0, stream);
  }
  if ((st = wait_event(p->h2d_done))) return st;  // the pinned arena is rewritten below
  // blocks outside the op: as in dc_deep_copy
  if ((st = launch_table(p, p->L.sta, p->L.stat, p->st_int_nd, p->st_int_units, s))) return st;
  host_copy(p, p->step_rest, 0, p->step_rest.units.size(), true);
  host_copy(p, p->step_xy, 0, p->step_xy.units.size(), true);
  size_t ns = 0;
  null_slots_upto(p, &ns, ~0ull);
  if ((st = launch_table(p, p->L.stb, p->L.stbt, p->st_run_nd, p->st_run_units, s))) return st;
  DC_CUDA(cudaEventRecord(p->h2d_done, s));
  if ((st = dc_relocate(p, stream))) return st;
  // the selected arrays: host -> update -> arena and host, in one pass
  if ((st = launch_step_kernel(p, op, s))) return st;
  if ((st = device_error(p, s))) return st;  // synchronizes the stream
  // x bytes that went through the pinned arena (outside mapped interiors)
  host_copy(p, p->step_xback, 0, p->step_xback.units.size(), false);
  return DC_OK;
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
  host_copy(p, p->step_xy, 0, p->step_xy.units.size(), true);
  if (p->step_fused) {
    if ((st = launch_step_kernel(p, op, s))) return st;
    DC_CUDA(cudaEventRecord(p->h2d_done, s));
    if ((st = device_error(p, s))) return st;
    host_copy(p, p->step_xback, 0, p->step_xback.units.size(), false);
    return DC_OK;
  }
  for (const auto& r : p->step_xy.runs)
    DC_CUDA(cudaMemcpyAsync(p->dev + r.lo, p->pinned + r.lo, r.hi - r.lo, cudaMemcpyHostToDevice, s));
  DC_CUDA(cudaEventRecord(p->h2d_done, s));
  if ((st = dc_update_leaves(p, op, stream))) return st;
  return dc_copy_back(p, 0, stream);
}
