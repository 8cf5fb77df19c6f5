// internal.hpp — plan tables, device-buffer layout and kernel entry points
// shared by the host runtime (runtime.cpp, plan.cpp) and the kernels
// (kernels.cu).  Not part of the public ABI (include/dc.h is).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../include/dc.h"
#include "pool.hpp"
#include "trace.hpp"

namespace dc {

constexpr uint32_t NONE = 0xFFFFFFFFu;

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// ---- error reporting ---------------------------------------------------------
dc_status fail(dc_status s, const char* fmt, ...);
// debug.cpp: DC_DEBUG=1 (every plan verifies) and DC_FAULT_HOST_ALLOC=1 (pinned allocations fail)
bool debug_on();
cudaError_t host_alloc(void** ptr, size_t bytes, unsigned int flags);

// try_wait rounds before an mbarrier wait gives up (well over a second)
constexpr uint32_t WAIT_LIMIT = 1u << 22;
// The limit of the first wait of every pipeline step of the bulk-copy kernels:
// WAIT_LIMIT unless DC_WAIT_LIMIT (decimal, read at every launch) lowers it.
uint32_t first_wait_limit();
dc_status cuda_fail(cudaError_t e, const char* what);
const char* last_error();
#define DC_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return dc::cuda_fail(e_, #call);  \
  } while (0)

// ---- device-side records -----------------------------------------------------

// The relocation's tables.  Every lane of the arena holds its blocks in the
// order of the slots that point at them (lane 0: the roots, then child arrays
// breadth first), so the blocks whose slots lie in one RELOC_SPAN-byte range
// of the struct lane are, in every lane, a run of consecutive blocks.  A
// relocation tile is such a range; its records are grouped by lane, each
// group holding consecutive target blocks.
//
// Offsets in the relocation tables are in record units: 16 bytes, or 4 bytes
// for DC_PLAN_PACK_SMALL plans (the plan's unit_shift: 4 or 2).
// One pointer slot: the target block's arena offset in units relative to its
// lane group's base (DC_PLAN_DEVICE_SCAN records, below, hold sizes instead),
// and where the slot is: its 8-byte word within the tile (low 16 bits) and its
// lane group's index within the tile (high 16 bits).
struct RelocRec {
  uint32_t off;
  uint32_t where;
};
static_assert(sizeof(RelocRec) == 8, "RelocRec is 8 bytes");
// DC_PLAN_DEVICE_SCAN records.  A tile's records are cut into slices of 32
// (tile-relative indexes 32k .. 32k + 31), one warp scan each.  A record that
// starts a slice or a lane group is a head: `off` holds its own offset from
// the group's base (0 at a group's first record) and `where` has SCAN_HEAD
// set; any other record holds the size in units of the record before it (the
// units from that target to the next block of the lane).  A target's offset is
// then the sum of `off` from its segment's head to itself.
constexpr uint32_t SCAN_HEAD = 0x8000u;  // above the slot word (< 1024, one per 8 bytes of a tile)
constexpr uint32_t SCAN_SLICE = 32;
// One (tile, lane) group: the arena offset in units of its first target block
// and the index of its first record; the plan starts a new group where a target
// lies 2^32 units or more past the base.  The table ends with a group whose
// rec_begin is the record count.
struct RelocSeg {
  uint64_t base;
  uint32_t rec_begin, pad;
};
static_assert(sizeof(RelocSeg) == 16, "RelocSeg is 16 bytes");
// One relocation tile with at least one slot: the tile (its struct bytes are
// [t, t+1) * RELOC_SPAN), its first record and lane group, and the counts
// (records in the low 16 bits, lane groups in the high 16 bits).  Only such
// tiles are listed.
struct RelocTile {
  uint32_t t, r0, g0, counts;
};
static_assert(sizeof(RelocTile) == 16, "RelocTile is one 16-byte vector");
constexpr uint32_t RELOC_SPAN = 8192;             // struct-lane bytes per relocation tile
constexpr uint32_t RELOC_MAXREC = RELOC_SPAN / 8;  // at most one slot per 8 bytes
constexpr uint32_t RELOC_MAXGROUPS = 64;           // lanes per plan (struct lane + array fields)

// A resolved leaf segment for the streaming kernel: effective addresses of
// x and y, the element count, and the exclusive prefix of 16-byte units
// (ceil(n * elem_size / 16)) over the table.
struct Segment {
  uint64_t x, y, n, ubeg;
};
static_assert(sizeof(Segment) == 32, "Segment is 32 bytes");

// An unresolved chain for the pointer-chasing kernel: start at `root` and
// follow steps[step_first .. step_first + nsteps); ebeg is the exclusive
// prefix of elements over the table.
struct ChaseSeg {
  uint64_t root;
  uint32_t step_first, nsteps;
  uint64_t n, ebeg;
};
static_assert(sizeof(ChaseSeg) == 32, "ChaseSeg is 32 bytes");

struct ChaseStep {
  uint32_t field_off;   // byte offset of the CHILD pointer in the current struct
  uint32_t child_size;  // sizeof the child struct
  uint64_t index;       // element of the child array
};
static_assert(sizeof(ChaseStep) == 16, "ChaseStep is 16 bytes");

// Control words in device scratch.
// CTRL_NEXT / CTRL_DONE: the fused launch's leaf-tile counter and finished-CTA
// count; both are zero between launches (the last CTA of a launch resets them).
enum CtrlWord : uint32_t { CTRL_ERR = 2, CTRL_NEXT = 4 /* words 4-5: 64-bit */, CTRL_DONE = 6, CTRL_WORDS = 16 };
enum DeviceErr : uint32_t { ERR_BOUNDS = 1u, ERR_TIMEOUT = 2u, ERR_VERIFY = 4u };

constexpr uint32_t RELOC_THREADS = 256;

// ---- kernels (kernels.cu) ------------------------------------------------------

struct RelocArgs {
  uint8_t* arena;
  uint64_t data_bytes;
  uint64_t struct_bytes;       // the struct lane is [0, struct_bytes) of the arena
  const RelocRec* rec;         // nrec records, tile by tile
  const RelocSeg* seg;         // nseg groups + the closing one
  const RelocTile* tiles;      // ntiles entries: the tiles that hold a slot
  const uint64_t* rec_host;    // DC_PLAN_VERIFY: host address of each record's target
  const uint64_t* rec_off;     // DC_PLAN_VERIFY: arena offset of each record's target
  uint32_t* ctrl;
  uint32_t nrec, nseg, ntiles, verify;
  uint32_t scan;  // records hold sizes (DC_PLAN_DEVICE_SCAN), not offsets
  uint32_t wait_limit = WAIT_LIMIT;  // try_wait rounds of a tile's first wait (0: give up at once)
  uint32_t unit_shift = 4;           // offsets in the tables are in units of 1 << unit_shift bytes
};

constexpr uint32_t LEAF_THREADS = 256;
constexpr uint32_t LEAF_UNROLL = 4;
constexpr uint32_t LEAF_TILE = LEAF_THREADS * LEAF_UNROLL;  // 16-byte units per tile

struct LeafArgs {
  const Segment* seg;
  const uint32_t* tile_seg;  // per tile: the segment holding its first unit; one extra entry = nseg - 1
  uint32_t nseg;
  uint64_t units;  // total 16-byte units
  int kind;        // dc_op_kind
  int f64;         // element type: 0 f32, 1 f64
  double scale;
  uint32_t* ctrl;  // the plan's control words (error bits)
  uint32_t wait_limit = WAIT_LIMIT;  // try_wait rounds of a sub-tile's first wait (0: give up at once)
};

// One block to move between host and device memory: src and dst are device-
// visible addresses (a mapped host page or the arena); ubeg is the exclusive
// prefix of 16-byte units over the table.
struct MoveDesc {
  uint64_t src, dst, bytes, ubeg;
};
static_assert(sizeof(MoveDesc) == 32, "MoveDesc is 32 bytes");

struct MoveArgs {
  const MoveDesc* d;
  const uint32_t* tile_desc;  // per tile of LEAF_TILE units: its first descriptor; one extra entry
  uint32_t nd;
  uint64_t units;
};

// One piece of a staged block for the span placement (place_kernel): `src`
// holds the piece's offset in the staging region (low 60 bits) and the zero
// bytes written after it (high 4 bits, < 16); `dst` holds its arena offset
// (high 48 bits) and the bytes written there minus one (low 16 bits).  A piece
// writes its bytes and then zeros up to its 16-byte slot end where the arena
// leaves room, so that writes fill whole sectors.  Pieces are in staging order.
struct PlaceDesc {
  uint64_t src, dst;
};
static_assert(sizeof(PlaceDesc) == 16, "PlaceDesc is 16 bytes");
constexpr uint64_t PLACE_PIECE = 32768;  // bytes of a piece at most (the rest of a block is further pieces)

struct PlaceArgs {
  const PlaceDesc* d;
  uint64_t nd;
  const uint8_t* stage;     // the staging region
  uint8_t* arena;
  uint64_t stage_bytes, data_bytes;
  uint32_t* err;            // ERR_BOUNDS for a piece outside either region
};

// One selected struct of a fused round trip (dc_roundtrip): its x and y blocks in the
// arena (xd, yd), their element count, the unit prefix, and for each of x and
// y where its bytes live on the host side: the host address, the mapped
// interior [lo, hi) of caller pages with its device address, and the block's
// place in the mapped pinned arena (for the bytes outside the interior).
struct StreamSeg {
  uint64_t xd, yd, n, ubeg;
  uint64_t xh, xlo, xhi, xi, xp;
  uint64_t yh, ylo, yhi, yi, yp;
  uint64_t pad[2];
};
static_assert(sizeof(StreamSeg) == 128, "StreamSeg is 128 bytes");

struct StreamArgs {
  const StreamSeg* seg;
  const uint32_t* tile_seg;
  uint32_t nseg;
  uint64_t units;
  uint64_t t_begin, t_end;  // the launch's tiles (of LEAF_TILE units)
  int kind, f64;
  double scale;
};

struct ChaseArgs {
  const ChaseSeg* seg;
  const ChaseStep* steps;
  uint32_t nseg;
  uint64_t elems;
  uint32_t x_off, y_off;
  int kind, f64;
  double scale;
};

cudaError_t launch_relocate(const RelocArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_leaf(const LeafArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_chase(const ChaseArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_move(const MoveArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_place(const PlaceArgs& a, cudaStream_t s, int sm_count);
// threads: 128, 256 or 512 per CTA; ctas_per_sm: 0 = as many as fit.  With
// max_per_sm set, launches nothing and reports how many CTAs fit on an SM.
cudaError_t launch_fused(const RelocArgs& r, const LeafArgs& l, uint32_t threads, uint32_t ctas_per_sm, int sm_count,
                         cudaStream_t s, int* max_per_sm);
cudaError_t launch_stream(const StreamArgs& a, cudaStream_t s, int sm_count);
cudaError_t launch_walk(uint64_t root, const ChaseStep* steps, uint32_t nsteps, uint64_t final_add,
                        uint64_t* out, cudaStream_t s);
void count_launch();

// ---- host plan -----------------------------------------------------------------

struct HostBlock {
  const uint8_t* host;
  uint64_t bytes;
  uint64_t count;     // elements (structs or array elements)
  uint64_t off;       // arena offset
  uint64_t ptr_first; // struct blocks: first index into Plan::ptr_target
  uint32_t lane;
  uint32_t type;      // struct blocks: struct type; arrays: owning struct type
  uint32_t field;     // arrays: field index in `type`; struct blocks: NONE
  uint32_t parent;    // arena index of the struct block with the slot; NONE = root
  uint32_t slot_off;  // byte offset of the slot in the parent block
  uint32_t depth;     // struct blocks: tree level of their structs
};

struct SchemaCopy {
  std::vector<dc_type> types;
  std::vector<std::vector<dc_field>> fields;
  std::vector<std::vector<int32_t>> ptr_index;  // [type][field] -> pointer-field index or -1
  std::vector<uint32_t> nptr;                   // [type] -> number of pointer fields
  std::vector<std::vector<uint32_t>> lane_of;   // [type][field] -> lane (ARRAY fields)
  uint32_t nlanes = 1;
  uint32_t root_type = 0;
};

dc_status copy_schema(const dc_schema* s, SchemaCopy* out);

// Layout of the caller's device buffer (byte offsets).
struct DevLayout {
  uint64_t data = 0, rec = 0, hostp = 0, soff = 0, status = 0, rtile = 0, seltile = 0, ctrl = 0;
  uint64_t seg = 0, tseg = 0, cseg = 0, steps = 0, walk = 0, total = 0;
  uint64_t mva = 0, mvat = 0, mvb = 0, mvbt = 0, bk = 0, bkt = 0;  // move tables + their tile tables
  uint64_t sta = 0, stat = 0, stb = 0, stbt = 0, sts = 0, stst = 0;  // fused-step tables
  uint64_t seg_cap = 0, tseg_cap = 0, step_cap = 0, walk_cap = 0, ntiles = 0, tab_cap = 0;
  // span staging (dc_plan_s::span_mode): the staged host spans and the placement
  // table that puts their blocks in the arena (0 bytes without span staging)
  uint64_t spn = 0, spd = 0, spd_cap = 0;
};

// One host span: staged blocks close together in host memory (gaps under
// SPAN_GAP bytes), copied as one range; `stage` is its offset in the staging
// area, with the host address's phase modulo 16.
struct HostSpan {
  const uint8_t* host;
  uint64_t bytes, stage;
};
constexpr uint64_t SPAN_GAP = 1024;  // a gap of less than a page: every page a span touches holds a block byte

struct OpKey {
  int32_t kind = -1, sel = -1;
  uint32_t type = 0, x = 0, y = 0;
  std::vector<dc_step> path;
  bool operator==(const OpKey& o) const;
};

}  // namespace dc

struct dc_plan_s {
  dc::SchemaCopy schema;
  std::vector<dc::HostBlock> blocks;     // arena order
  std::vector<uint32_t> ptr_target;      // per struct element, per pointer field: block or NONE
  std::vector<dc::RelocRec> rrec;        // relocation records, tile by tile
  std::vector<dc::RelocSeg> rseg;        // (tile, lane) groups + the closing one
  std::vector<dc::RelocTile> rtiles;     // per relocation tile: its records and lane groups
  std::vector<uint64_t> rec_host;        // per record: the target's host address (DC_PLAN_VERIFY)
  std::vector<uint64_t> rec_off;         // per record: the target's arena offset (DC_PLAN_VERIFY)
  std::vector<uint32_t> rec_size;        // per record: units to the next block of the lane (DC_PLAN_DEVICE_SCAN)
  std::vector<uint64_t> lane_start;      // lane l's blocks are [lane_start[l], lane_start[l+1])
  uint32_t unit_shift = 4;               // the tables' units: 16 bytes, or 4 with DC_PLAN_PACK_SMALL
  bool rec_scan = false;                 // the bound buffer holds scan records (DC_PLAN_DEVICE_SCAN)
  uint64_t struct_bytes = 0;             // bytes of the struct lane (lane 0)
  std::vector<uint64_t> null_slots;      // arena offsets of slots with count 0 but a non-NULL host value
  std::vector<uint32_t> roots;           // arena index of each tree's root struct block
  uint64_t nstructs = 0, nstruct_blocks = 0, payload = 0, data_bytes = 0, sum_depth = 0;
  uint32_t max_depth = 0;
  uint32_t flags = 0;
  uint32_t nthreads = 0;

  // runtime state
  uint8_t* dev = nullptr;
  uint64_t dev_bytes = 0;
  dc::DevLayout L;
  uint8_t* pinned = nullptr;      // data-region staging arena (cudaHostAlloc)
  uint8_t* pin_tab = nullptr;     // segment / chase table staging (cudaHostAlloc)
  bool borrowed_pinned = false;   // pinned memory lent by a server (not freed by the plan)
  uint64_t pin_tab_bytes = 0;
  cudaEvent_t h2d_done = nullptr; // last deep copy's transfers
  cudaEvent_t tab_done = nullptr; // last table upload
  int sm_count = 0;
  int device = -1;
  dc::OpKey leaf_key, chase_key;  // ops whose tables are on the device
  uint64_t leaf_nseg = 0, leaf_units = 0, chase_nseg = 0, chase_elems = 0;
  const std::vector<uint32_t>* written = nullptr;  // arrays the last update wrote (leaf_written or chase_written)
  std::vector<uint32_t> leaf_written, chase_written;  // ascending arena indices
  std::vector<uint64_t> leaf_hist;  // log2 histogram of the selected arrays' lengths (the autotuner's key)
  uint32_t tuned_threads = 0, tuned_ctas = 0;  // split chosen by dc_autotune (0 = default)
  dc::OpKey tuned_key;
  uint64_t gen = 0;                // bumped whenever a written list is rebuilt
  uint64_t leaf_gen = 0, chase_gen = 0, written_gen = 0;
  bool op_run = false;
  std::unique_ptr<dc::Pool> own_pool;  // only when dc_plan_set_threads asked for one
  dc::Pool* pool = nullptr;
  // transfers (transfer.cpp), planned at the first bind
  struct Frag { uint64_t off, len; uint8_t* host; };  // staged bytes: arena offset, length, host address
  struct Unit { uint64_t first, last; };              // pieces [first, last), one host thread at a time
  struct Copy { uint64_t lo, hi; };                   // a range of the data region
  struct Chunk { uint64_t ufirst, ulast, cfirst, clast; };
  struct Moves {
    std::vector<Frag> frags;          // staged bytes, arena order
    std::vector<Frag> pieces;         // frags split for host threads
    std::vector<Unit> units;
    std::vector<Copy> runs;           // frags separated only by padding, merged
    std::vector<Copy> copies;         // runs clipped to chunks (DMA)
    std::vector<Chunk> chunks;
    std::vector<uint32_t> interiors;  // blocks whose interior moves through mapped caller pages
  };
  bool transfers_ready = false;
  uint8_t* pinned_dev = nullptr;      // device view of the (mapped) pinned arena
  std::vector<uint64_t> ilo, ihi, idev;  // per block: mapped interior host range, its device address
  std::vector<std::pair<void*, uint64_t>> registered;  // caller pages this plan page-locked
  bool has_arena_blocks = false;       // some blocks live in a host arena (moved directly)
  Moves h2d;
  uint64_t h2d_int_nd = 0, h2d_int_units = 0, h2d_frag_nd = 0, h2d_frag_units = 0;
  // Span staging: a deep copy of many small blocks copies whole host spans (the
  // blocks and the gaps between them) into the pinned staging area, moves them
  // to the device staging region by DMA, and places every block in the arena
  // with one move-kernel launch (the host copies stream instead of handling
  // each block).
  std::vector<dc::HostSpan> spans;    // host order (built on first need)
  uint64_t span_bytes = 0;            // staging area bytes
  uint64_t span_nstaged = 0, span_staged = 0;  // the blocks a full deep copy stages, and their bytes
  bool span_rule = false;             // their count and mean size allow span staging
  bool spans_built = false;
  bool span_worth = false;            // ... and their spans hold at most 5/4 of their bytes
  bool span_mode = false;             // dc_deep_copy stages by spans
  Moves h2d_span;                     // frags: the spans, at their staging offsets
  std::vector<uint64_t> span_nulls;   // NULL-slot fix-ups, as staging offsets (sorted)
  uint64_t span_nd = 0;                // pieces in the placement table
  uint64_t back_key = ~0ull;          // generation of the block list `back` was built for (0 = all arrays)
  Moves back;
  uint64_t bk_nd = 0, bk_units = 0;
  Moves sel;                          // the last selective deep copy's blocks
  dc::OpKey sel_key;
  std::vector<dc::RelocTile> sel_tiles;  // relocation tiles holding its struct blocks' slots
  // the copy back's events: the error word's read, then one per DMA chunk of `back`
  cudaEvent_t back_err = nullptr;
  std::vector<cudaEvent_t> back_ev;
  cudaEvent_t sync_ev = nullptr;      // sync_stream's marker
  // the fused round trip (step.cpp), cached per op
  dc::OpKey step_key;
  bool step_fused = false;
  Moves step_rest, step_xy, step_xback;
  // the fused pass in tile groups: group g's tiles [step_cut[g], step_cut[g+1]) launch once its
  // pieces in step_in[g] are marshalled; step_out[g] are scattered once they complete
  std::vector<uint64_t> step_cut;
  std::vector<Moves> step_in, step_out;
  std::vector<cudaEvent_t> step_ev;
  uint64_t st_int_nd = 0, st_int_units = 0, st_run_nd = 0, st_run_units = 0, st_nseg = 0, st_units = 0;
  std::vector<uint32_t> step_written;
  uint64_t step_gen = 0;
};

struct dc_uvm_s {
  dc_plan_s* plan = nullptr;         // host tables of the tree (no device buffer)
  std::vector<void*> managed;        // per block (arena order)
  uint64_t root = 0;
  dc::ChaseSeg* dseg = nullptr;      // device tables for the chase kernel
  dc::ChaseStep* dsteps = nullptr;
  uint64_t seg_cap = 0, step_cap = 0;
  std::vector<uint32_t> written;
  dc::OpKey key;
  uint64_t nseg = 0, elems = 0;
  int sm_count = 0;
  int device = -1;
};

namespace dc {
// Block offsets and relocation tables from the blocks in lane order (plan.cpp).
dc_status layout(dc_plan_s* p);
// The DC_PLAN_DEVICE_SCAN form of the plan's records (plan.cpp), one per record into `out`.
void scan_records(const dc_plan_s* p, RelocRec* out);
dc_status build_plan(const dc_schema* schema, const void* const* roots, uint64_t nroots, dc_plan_s* p);
// Resolve a chain over the plan tables to (block, byte offset in block, type
// of the struct reached or NONE when the last step was an ARRAY step, element).
dc_status resolve(const dc_plan_s* p, uint64_t tree, const dc_step* path, uint32_t len, uint32_t* block,
                  uint64_t* within, uint32_t* type, uint64_t* elem);
// The structs an op selects: (struct block, element) pairs.
dc_status select_structs(const dc_plan_s* p, const dc_op* op,
                         std::vector<std::pair<uint32_t, uint64_t>>* out);
dc_status check_op(const dc_plan_s* p, const dc_op* op);
// arena.cpp: is [host, host + bytes) inside a host arena?  Its device view.
bool in_host_arena(const void* host, uint64_t bytes, uint64_t* dev);
// transfer.cpp
uint64_t interior_bytes(const HostBlock& b);
// host_order: hand out the host copies in host-address order (sequential on the
// caller's side); such Moves have no DMA chunks.  Otherwise they follow the
// arena, chunk by chunk.
// Split a block list's staged bytes into pieces, host work units and (unless
// host_order) DMA chunks of about chunk_bytes (0: the deep copy's chunk size).
void plan_moves(const dc_plan_s* p, const std::vector<uint32_t>& list, dc_plan_s::Moves* m, bool host_order = true,
                uint64_t chunk_bytes = 0, bool stage_all = false);
// Marshal a chunked move list (plan_moves with host_order false) into the
// pinned arena, zero the NULL slots `nulls` (offsets in the list's destination
// range, sorted) and queue each chunk's DMA to `dev` + offset as it completes.
dc_status send_staged(dc_plan_s* p, const dc_plan_s::Moves& m, const std::vector<uint64_t>& nulls, uint8_t* dev,
                      cudaStream_t s);
void plan_transfers(dc_plan_s* p);
// Pieces, units, runs and (unless host_order) chunks of m->frags.
void split_moves(dc_plan_s::Moves* m, bool host_order, uint64_t chunk_bytes);
// The staged blocks' count and bytes, and whether the span rule may fire (at planning).
void plan_spans(dc_plan_s* p);
// span_mode from the plan's flags and span_worth (at planning and flag changes).
void choose_spans(dc_plan_s* p);
// Bytes of the pinned arena: the data region, or the span staging area if larger.
uint64_t pin_arena_bytes(const dc_plan_s* p);
// The placement table of a span-staged plan (spans.cpp): one PlaceDesc per piece, staging order.
void build_place_table(const dc_plan_s* p, std::vector<PlaceDesc>* out);
// The plan's NULL-slot fix-ups as offsets in the span staging area, sorted (spans.cpp).
std::vector<uint64_t> span_null_offsets(const dc_plan_s* p);
// The struct block holding arena offset `off`; per block, 1 for a struct block with a
// NULL-slot fix-up; the span holding host address h (spans.cpp).
uint64_t struct_block_at(const dc_plan_s* p, uint64_t off);
std::vector<uint8_t> null_fixups(const dc_plan_s* p);
const HostSpan& span_at(const dc_plan_s* p, const uint8_t* h);
void release_transfers(dc_plan_s* p);
dc_status upload_h2d_tables(dc_plan_s* p, cudaStream_t s);
dc_status transfer_to_device(dc_plan_s* p, cudaStream_t s);
dc_status transfer_back(dc_plan_s* p, const std::vector<uint32_t>& list, uint64_t key, cudaStream_t s);
dc_status upload(dc_plan_s* p, const std::vector<MoveDesc>& d, uint64_t desc_off, uint64_t tile_off, uint64_t cap,
                 uint64_t* nd, uint64_t* units, cudaStream_t s);
void push_desc(std::vector<MoveDesc>* d, uint64_t src, uint64_t dst, uint64_t bytes);
dc_status launch_table(dc_plan_s* p, uint64_t desc_off, uint64_t tile_off, uint64_t nd, uint64_t units,
                       cudaStream_t s);
void host_copy(dc_plan_s* p, const dc_plan_s::Moves& m, uint64_t ufirst, uint64_t ulast, bool to_arena);
void null_slots_upto(dc_plan_s* p, size_t* ns, uint64_t hi);
// runtime.cpp
dc_status device_error(dc_plan_s* p, cudaStream_t s);
// The pinned host word that device_error reads the device's error word into.
uint32_t* pinned_error_word(dc_plan_s* p);
Pool& pool_of(dc_plan_s* p);
OpKey key_of(const dc_op* op);
dc_status wait_event(cudaEvent_t e);
// Wait until the plan's work queued on `s` so far has completed (an event
// recorded on `s`, waited for as wait_event does).
dc_status sync_stream(dc_plan_s* p, cudaStream_t s);
// x (and y) target blocks of the structs an op selects; structs whose x is empty are skipped
struct Pick {
  uint32_t sblk;
  uint64_t elem;
  uint32_t bx, by;
};
dc_status pick(const dc_plan_s* p, const dc_op* op, std::vector<Pick>* out);
dc_status build_leaf_table(dc_plan_s* p, const dc_op* op, cudaStream_t s);
LeafArgs leaf_args(const dc_plan_s* p, const dc_op* op);
RelocArgs reloc_args(const dc_plan_s* p);
// Pinned bytes a plan needs (arena + table staging), and binding with pinned
// memory lent by the caller (the request server's pool; mapped).
uint64_t pinned_need(const dc_plan_s* p);
dc_status bind_borrowed(dc_plan_s* p, void* dev, uint64_t bytes, uint8_t* pinned, uint8_t* pinned_dev, cudaStream_t s);
// Give a plan bound with borrowed pinned memory another pinned range of the
// same size (pinned_need) for its next calls; the caller makes sure nothing
// of the plan's earlier calls is in flight.  Not for DC_PLAN_MAP_HOST plans.
dc_status lend_pinned(dc_plan_s* p, uint8_t* pinned, uint8_t* pinned_dev);
// The chain of (field, index) steps from the root to struct (block, elem).
void path_to(const dc_plan_s* p, uint32_t block, uint64_t elem, std::vector<dc_step>* out);
}  // namespace dc
