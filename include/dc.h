/*
 * dc.h — C ABI of the B300 deep-copy library (libdc.so).
 *
 * Moves a nested, pointer-linked host structure into one device arena,
 * rebuilds every pointer so it is valid on the device, resolves pointer
 * chains to effective device addresses, runs the leaf-array kernel through
 * those addresses and copies the results back.  The operations follow the
 * paper's statement of the problem: the four deep-copy steps of Fig 2 (Sec. 2),
 * the marshalling of Algorithm 1 (Sec. 4.1.1 item 2), effective-address
 * extraction of a pointer chain (Sec. 3), the scaling kernels of Sec. 4.1.2 and
 * Listing 2, and the main-program flow of Algorithm 2.
 *
 * Conventions for every call
 *   - Returns a dc_status and never aborts; dc_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).
 *   - Pointers are plain host or device addresses; sizes are bytes unless the
 *     name says otherwise.  A dc_stream_t is a cudaStream_t (NULL = the legacy
 *     default stream).  Calls on one plan must be ordered on one stream (or
 *     the caller must order the streams); a plan is not thread-safe.
 *   - Device work is asynchronous and stream-ordered.  Errors a kernel finds
 *     (an index outside its buffers, a device-side wait that gave up, a
 *     failed relocation check) are recorded in a device word and reported by
 *     the next dc_sync() (or dc_copy_back()) on that plan.  The only device-
 *     side waits are a kernel's waits for its own bulk copies; each gives up
 *     after about a second, records DC_ETIMEOUT, waits (bounded) for the
 *     copies still in flight and returns.  For tests, DC_WAIT_LIMIT=N in the
 *     environment (read at every launch) lowers the first wait of every
 *     pipeline step to N try-wait rounds (0: give up at once).
 *   - Ownership: the caller owns the host tree and must not change its shape
 *     (pointers, counts) or free it before dc_plan_destroy, nor write its
 *     arrays while a dc_deep_copy is in flight (until dc_sync, or any later
 *     blocking call on the same stream).  The caller owns the device
 *     buffer given to dc_bind_device (e.g. a torch uint8 tensor).  The library
 *     owns the plan's tables, its pinned staging arena and managed trees;
 *     dc_plan_destroy / dc_uvm_destroy free them.
 */
#ifndef DC_H
#define DC_H

#include <stddef.h>
#include <stdint.h>

/* Every entry point below is exported from the library; nothing else is. */
#if defined(__GNUC__)
#define DC_API __attribute__((visibility("default")))
#else
#define DC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dc_stream_t;

typedef enum {
  DC_OK = 0,
  DC_EINVAL = 1,         /* bad argument, schema, path or structure */
  DC_ENOMEM = 2,         /* host or pinned allocation failed */
  DC_ECUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
  DC_EALIAS = 4,         /* two blocks overlap (one reached twice, an array pointing into a
                            struct, ...): not a tree */
  DC_ECYCLE = 5,         /* a child pointer leads into an ancestor struct block */
  DC_EBUDGET = 6,        /* the bound device buffer is smaller than the plan needs */
  DC_ETIMEOUT = 7,       /* a device-side wait gave up after its iteration limit */
  DC_EDEVICE_BOUNDS = 8, /* a kernel found an index or offset outside its buffers */
  DC_ESTATE = 9,         /* call out of order (no device buffer bound, no op run, ...) */
  DC_EVERIFY = 10        /* relocation check: a slot did not hold the expected host address */
} dc_status;

/* ---- schema: C struct types described by field offsets -------------------- */

typedef enum { DC_F_SCALAR = 0, DC_F_ARRAY = 1, DC_F_CHILD = 2 } dc_field_kind;
typedef enum { DC_E_F32 = 0, DC_E_F64 = 1, DC_E_BYTES = 2 } dc_elem_kind;

typedef struct {
  int32_t kind;         /* dc_field_kind */
  uint32_t offset;      /* byte offset of the member in its struct */
  uint32_t elem_size;   /* SCALAR: 4 or 8 (signed integer); ARRAY: bytes per element */
  int32_t count_field;  /* ARRAY/CHILD: index of the SCALAR field holding the
                           element count, or -1 to use count_const */
  uint64_t count_const; /* ARRAY/CHILD: element count when count_field == -1 */
  int32_t child_type;   /* CHILD: index into dc_schema.types of the pointee type */
  int32_t elem_kind;    /* ARRAY: dc_elem_kind; leaf ops need F32 or F64 */
} dc_field;

/* A struct type: `size` bytes (sizeof), alignment `align` (<= 16).  An ARRAY
 * member is a pointer to `count` primitive elements; a CHILD member is a
 * pointer to a contiguous array of `count` structs of child_type (count 1 for
 * a plain struct pointer, as in Listing 1's simulation->atoms).  A pointer
 * whose count is 0 may be anything; the copy holds NULL there.  Pointer
 * members must sit at 8-byte aligned offsets. */
typedef struct {
  uint32_t size, align, nfields;
  const dc_field* fields;
} dc_type;

typedef struct {
  uint32_t ntypes, root_type;
  const dc_type* types;
} dc_schema;

/* One arrow of a pointer chain: follow member `field` of the current struct
 * and take element `index` of what it points to.  A CHILD step moves to that
 * child struct; an ARRAY step selects an element and must be the last step. */
typedef struct {
  uint32_t field;
  uint64_t index;
} dc_step;

typedef enum { DC_OP_AXPY_HALF = 0, DC_OP_SCALE = 1 } dc_op_kind;
typedef enum { DC_SEL_ALL = 0, DC_SEL_CHAIN = 1 } dc_sel;

/* A leaf-kernel request.
 *   AXPY_HALF: x[i] = x[i] + 0.5*y[i], computed as __fadd_rn(x, __fmul_rn(0.5f, y))
 *              for F32 arrays (one IEEE rounding per operation), likewise in F64.
 *   SCALE:     x[i] = x[i] * scale (the paper's scaling kernel, Sec. 4.1.2 item 1
 *              and Listing 2); scale is rounded to float for F32 arrays.
 *   SEL_ALL:   every struct of `type` in the tree (the allinit-allused layout).
 *   SEL_CHAIN: the one struct of `type` that `path` (CHILD steps only) reaches
 *              from the root (the LLused layouts; Listing 2's chain).
 * x_field / y_field are ARRAY fields of `type` with the same count and kind. */
typedef struct {
  int32_t kind;  /* dc_op_kind */
  double scale;
  int32_t sel;   /* dc_sel */
  const dc_step* path;
  uint32_t path_len;
  uint32_t type;
  uint32_t x_field, y_field;
} dc_op;

typedef struct dc_plan_s* dc_plan_t;
typedef struct dc_uvm_s* dc_uvm_t;

typedef struct {
  uint64_t data_bytes;     /* arena data region: every block at a 16-byte aligned offset;
                              the size of the H2D of dc_deep_copy */
  uint64_t device_bytes;   /* bytes the buffer passed to dc_bind_device must hold:
                              data region + block table + scratch */
  uint64_t payload_bytes;  /* sum of block sizes without padding */
  uint64_t nblocks;        /* root struct + non-empty arrays + non-empty child arrays */
  uint64_t nrelocs;        /* pointer slots rewritten by the relocation (nblocks - ntrees) */
  uint64_t nstructs;       /* struct instances in the tree */
  uint64_t nstruct_blocks; /* blocks that hold structs (root + child arrays) */
  uint64_t root_offset;    /* offset of the (first) root struct in the data region (0) */
  uint64_t ntrees;         /* trees in the plan (1, or the count given to dc_plan_forest) */
  uint64_t struct_bytes;   /* bytes of lane 0 (every struct block, padded), at the start of
                              the data region: the relocation reads and writes this range */
  uint64_t reloc_table_bytes; /* the relocation's tables (8 B per slot, 16 B per lane group
                                 of a tile, 16 B per tile that holds a slot) */
  uint64_t staging_bytes;  /* the span staging area when dc_deep_copy stages by host spans
                              (DC_PLAN_SPANS), else 0 */
} dc_plan_info;

/* Plan flags (dc_plan_set_flags, before dc_bind_device). */
#define DC_PLAN_VERIFY 1u /* relocation also checks that every slot still holds the
                             host address the plan recorded (DC_EVERIFY otherwise) */
#define DC_PLAN_MAP_HOST 2u /* move the whole pages inside each array of at least
                             DC_MAP_MIN_BYTES straight between the caller's memory and
                             the arena (one kernel launch for all of them) instead of
                             through the pinned arena.  dc_bind_device page-locks and
                             maps those pages in place (cudaHostRegister) until
                             dc_plan_destroy; only pages wholly inside an array are
                             touched.  While they are registered, a cudaMemcpy by the
                             caller that starts inside such a page range and runs past
                             its end fails. */
#define DC_MAP_MIN_BYTES (64u << 10)
#define DC_PLAN_DEVICE_SCAN 4u /* the relocation computes the targets' arena offsets on
                             the device from their padded sizes: a tile's records are
                             cut into slices of 32, each slice's first record carries
                             its own offset, the others the size of the record before
                             them, and one segmented warp-shuffle prefix sum per slice,
                             added to each lane group's base, gives the offsets.
                             Without it (the default) every record carries the offset
                             the plan's layout assigned; the device image is the same.
                             Read at dc_bind_device; dc_relocate_static ignores it. */
#define DC_PLAN_PACK_SMALL 8u /* lay array blocks of fewer than DC_PACK_BYTES bytes out
                             at their element alignment (8 bytes for f64, else 4)
                             instead of on 16 bytes, so that many small arrays lie
                             back to back and the leaf update streams over them
                             without padding (the relocation tables then count in
                             4-byte units: a lane group spans at most 16 GiB and a
                             block less than 16 GiB).  Struct blocks and larger
                             arrays stay on 16 bytes; every lane starts on 16 bytes.
                             Changing it reruns the plan's layout, so it is set before
                             dc_bind_device (DC_ESTATE after).  dc_plan_arena_bytes
                             and dc_plan_block give the packed offsets.  dc_roundtrip
                             takes its three-call path when a selected array is not
                             on 16 bytes in the arena. */
#define DC_PACK_BYTES 64u
#define DC_PLAN_SPANS 16u /* stage the deep copy by host spans even where the plan's own
                             rule would not (that rule: at least DC_SPAN_MIN_BLOCKS
                             staged blocks averaging under DC_SPAN_MAX_MEAN bytes, whose
                             spans hold at most 5/4 of their bytes).  A span is a run of
                             staged blocks in host memory with gaps of under 1 KiB
                             between them; dc_deep_copy copies each span whole into the
                             pinned arena (the gap bytes included: they lie on pages
                             that also hold the tree's blocks, are read, moved to the
                             device and never used), moves the spans by DMA to a
                             staging region of the device buffer, and one kernel launch
                             places every block at its arena offset.  The device buffer
                             then holds the staging region too (dc_plan_info's
                             staging_bytes); the pinned arena is the larger of the data
                             region and the staging area.  Ignored with DC_PLAN_MAP_HOST;
                             set it before dc_bind_device.  The environment variable
                             DC_SPANS=0, read at dc_plan, turns the plan's own rule
                             off: a program run under a memory checker (AddressSanitizer
                             and the like) would report the reads between allocations. */
#define DC_SPAN_MIN_BLOCKS 1024u
#define DC_SPAN_MAX_MEAN 4096u

/* dc_plan — walk the host structure from `host_root` (one struct of
 * schema->root_type) and lay out its device arena (Algorithm 1's first step,
 * determineTotalBytes, and its allocation requests; Fig 2 step a).  Host only:
 * touches no GPU.
 * Layout: blocks are grouped in lanes — lane 0 holds every struct block (the
 * root, then the child arrays breadth first, each struct block's children in
 * the order of their slots), then one lane per ARRAY field (in type, field
 * order) holding its blocks in the order of their parents in lane 0, then of
 * their slots.  So in every lane, consecutive blocks are pointed at by
 * ascending slots.  Every block starts on a 16-byte boundary.
 * Errors: DC_EINVAL (NULL pointer with a non-zero count, negative count, bad
 * schema), DC_ECYCLE (a child pointer leads into an ancestor struct block),
 * DC_EALIAS (any other two blocks overlap: the structure is not a tree),
 * DC_ENOMEM.  With DC_TRACE=1 the walk, the overlap check, the lane order, the
 * remap and the relocation tables are timed. */
DC_API dc_status dc_plan(const dc_schema* schema, const void* host_root, dc_plan_t* out);
/* dc_plan_forest — one plan (one arena, one relocation, one leaf stream) for
 * `nroots` independent trees of the same schema (the batched form of the deep
 * copy): lane 0 starts with the roots in the order given, and the lanes hold
 * every tree's blocks in the slot order above.  SEL_ALL ops cover
 * every tree; SEL_CHAIN paths and dc_resolve_chain / dc_verify_chain start at
 * tree 0 (dc_resolve_chain_in takes a tree index).  The trees must not share
 * blocks (DC_EALIAS). */
DC_API dc_status dc_plan_forest(const dc_schema* schema, const void* const* roots, uint64_t nroots, dc_plan_t* out);
/* Offset of tree `tree`'s root struct in the data region. */
DC_API dc_status dc_plan_root(dc_plan_t plan, uint64_t tree, uint64_t* offset);
DC_API dc_status dc_plan_set_flags(dc_plan_t plan, uint32_t flags);
DC_API dc_status dc_plan_info_get(dc_plan_t plan, dc_plan_info* out);
/* dc_plan_arena_bytes — the three sizes a caller needs before dc_bind_device:
 * the bytes the device buffer must hold (info.device_bytes: the data region of
 * Algorithm 1's determineTotalBytes plus the plan's tables and scratch), the
 * block count and the pointer slots the relocation rewrites.  Host only.  Any
 * output pointer may be NULL.  Errors: DC_EINVAL (NULL plan). */
DC_API dc_status dc_plan_arena_bytes(dc_plan_t plan, uint64_t* bytes, uint64_t* nblocks, uint64_t* nrelocs);
/* Block `i` in arena order: its host address, arena offset, byte size, lane,
 * and its relocation entry — the struct block holding the pointer slot that
 * refers to it (UINT32_MAX for the root) and that slot's byte offset inside
 * it.  Any output pointer may be NULL. */
DC_API dc_status dc_plan_block(dc_plan_t plan, uint64_t i, uint64_t* host_addr, uint64_t* offset,
                        uint64_t* bytes, uint32_t* lane, uint32_t* parent, uint32_t* slot_off);
/* Host threads used by marshal and copy-back scatter (0 = all online cores). */
DC_API dc_status dc_plan_set_threads(dc_plan_t plan, uint32_t nthreads);
DC_API dc_status dc_plan_destroy(dc_plan_t plan);

/* dc_bind_device — give the plan a caller-owned device buffer of at least
 * info.device_bytes bytes, 256-byte aligned (a torch CUDA uint8 tensor
 * qualifies).  Uploads the block table and clears the scratch on `stream`
 * (blocking).  The plan's first bind also allocates its pinned staging arena:
 * info.data_bytes of page-locked host memory (or info.staging_bytes, if larger,
 * for a plan staged by host spans).
 * Errors: DC_EBUDGET, DC_EINVAL (misaligned), DC_ENOMEM, DC_ECUDA. */
DC_API dc_status dc_bind_device(dc_plan_t plan, void* dev_buffer, uint64_t bytes, dc_stream_t stream);

/* dc_deep_copy — move the tree into the arena (Fig 2 steps b-c), then run
 * the relocation kernel, which rebuilds every pointer slot to the device
 * address of its target (Fig 2 step d; Algorithm 1's attach loop).  By
 * default every block is marshalled into the pinned arena (Algorithm 1: one
 * contiguous buffer) by the plan's host threads, which take work units of
 * about 256 KiB in arena order; each 16 MiB chunk of the arena goes by DMA as
 * soon as its last unit is marshalled, while the threads go on with the next
 * chunks (the call returns once every chunk is queued).  A plan staged by host
 * spans (DC_PLAN_SPANS, or the plan's own rule for many small blocks) copies
 * whole spans the same way into the staging area, sends them to the device
 * buffer's staging region, and one kernel launch puts every block at its arena
 * offset before the relocation.  With DC_PLAN_MAP_HOST
 * the interiors of large arrays are
 * read straight from the caller's pages by one kernel launch (one transfer
 * per effective-address array, as in the paper's pointerchain scheme,
 * Sec. 4.1.1 item 3) while the rest is marshalled.  Returns once the copies
 * and the kernel are queued; with DC_PLAN_MAP_HOST the caller's arrays are
 * read until the stream gets there.  Errors: DC_ESTATE (nothing bound),
 * DC_ECUDA. */
DC_API dc_status dc_deep_copy(dc_plan_t plan, dc_stream_t stream);

/* dc_deep_copy_selected — a selective deep copy (Sec. 2: only what the
 * computation reaches is replicated; the allinit-LLused and LLinit-LLused
 * layouts of Sec. 4.1.2 and Listing 2's chain): for `op`, the struct blocks
 * on the way from the root to every struct the op selects (with DC_SEL_CHAIN,
 * the blocks its chain passes through: the root struct and each child array
 * it indexes into) and those structs' x (and y) arrays are marshalled into the
 * pinned arena and sent to the device; then the relocation runs only over the
 * 8 KiB ranges of the struct lane that hold those blocks' pointer slots.  No
 * other byte of the data region is written, so the device holds a walkable
 * copy of the chain (dc_verify_chain, dc_update_chase) and the op's arrays
 * (dc_update_leaves, dc_copy_back); other arrays and structs are not current,
 * and pointer slots of unselected structs in the same 8 KiB ranges are set to
 * their targets' device addresses whatever those hold.  Every block goes
 * through the pinned arena (DC_PLAN_MAP_HOST's mapped pages are not used);
 * no DC_PLAN_VERIFY check.  Returns once the copies and the kernel are
 * queued.  Errors: DC_EINVAL (op), DC_ESTATE (nothing bound), DC_ECUDA. */
DC_API dc_status dc_deep_copy_selected(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_relocate — the relocation kernel of dc_deep_copy alone (Fig 2 step d):
 * rewrite every pointer slot of the data region already in device memory to
 * the device address of its target (the buffer's base + the target's arena
 * offset, which the plan's relocation records hold).  For a data region that
 * is already resident (filled by an earlier dc_deep_copy or by the caller);
 * the result is the same whatever the slots held.  Errors: DC_ESTATE, DC_ECUDA. */
DC_API dc_status dc_relocate(dc_plan_t plan, dc_stream_t stream);

/* dc_resolve_chain — the effective device address of a pointer chain
 * (Sec. 3: extract it once, before the compute region): the struct the CHILD
 * steps reach, or &array[index] for a final ARRAY step.  Host only, O(path
 * length), reads no device memory.  Errors: DC_EINVAL (bad field, index out
 * of range, NULL link), DC_ESTATE (nothing bound).
 * dc_resolve_offset gives the same place as an offset in the data region
 * and needs no device buffer. */
DC_API dc_status dc_resolve_chain(dc_plan_t plan, const dc_step* path, uint32_t len, uint64_t* dev_addr);
DC_API dc_status dc_resolve_offset(dc_plan_t plan, const dc_step* path, uint32_t len, uint64_t* offset);
DC_API dc_status dc_resolve_chain_in(dc_plan_t plan, uint64_t tree, const dc_step* path, uint32_t len, uint64_t* dev_addr);
DC_API dc_status dc_resolve_offset_in(dc_plan_t plan, uint64_t tree, const dc_step* path, uint32_t len, uint64_t* offset);

/* dc_update_leaves — run the leaf kernel on the device copy through resolved
 * addresses: the selected structs' chains are resolved on the host and the
 * kernel streams over (x, y, n) segments with no pointer loads, bringing x
 * and y into shared memory by 1-D bulk copies (with DC_LEAF_TMA=0 in the
 * environment, read at every call, by direct 16-byte loads instead; the
 * results are the same).  Arrays that follow each other in the arena with
 * only block padding between them (and whose y arrays do the same) are one
 * segment: the update then also rewrites the padding bytes between them (up
 * to 15 per block), which belong to no block.  Errors: DC_EINVAL (op fields /
 * path / counts), DC_ESTATE, DC_ECUDA. */
DC_API dc_status dc_update_leaves(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_relocate_update — dc_relocate and dc_update_leaves(op) in one persistent
 * kernel launch: work items are the relocation's tiles, then the leaf
 * update's tiles.  The two are independent (the update goes through
 * addresses resolved on the host), so for a forest (dc_plan_forest) one launch
 * relocates and updates every tree.  Uses the split dc_autotune chose for this
 * plan and op, else one cached for the same kind of op and length histogram in
 * this process, else 256 threads per CTA and as many CTAs as fit.  Once the op's
 * tables are on the device (after a first call) the call only launches a
 * kernel, so it can be captured in a CUDA graph.  Errors: as
 * dc_update_leaves. */
DC_API dc_status dc_relocate_update(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_autotune — time dc_relocate_update's launch on the bound arena under each
 * work split (128, 256 or 512 threads per CTA, i.e. 8, 4 or 2 blocks or
 * 16-byte units per thread per tile; 1, 2, 4 or 8 CTAs per SM, as far as they
 * fit; each timed over three back-to-back launches), keep the fastest for the
 * plan and cache it for the process under a key made of the op's kind and
 * element size, the plan's block count and the log2 histogram of the selected
 * arrays' lengths.  Blocking.  Each timing run applies
 * the update, so the arena's x arrays change: tune before the deep copy of
 * the data that matters, or deep copy again afterwards.  Outputs may be NULL. */
DC_API dc_status dc_autotune(dc_plan_t plan, const dc_op* op, dc_stream_t stream, uint32_t* threads,
                      uint32_t* ctas_per_sm);
/* dc_set_split — use this split for dc_relocate_update(op) on this plan
 * instead of timing the candidates: `threads` per CTA (128, 256 or 512) and
 * `ctas_per_sm` CTAs per SM (0 = as many as fit; more than fit are clamped at
 * launch).  For a split tuned earlier, or to repeat a run with the same launch
 * shape.  Host only.  Errors: DC_EINVAL (NULL plan, bad op, other thread
 * counts). */
DC_API dc_status dc_set_split(dc_plan_t plan, const dc_op* op, uint32_t threads, uint32_t ctas_per_sm);

/* dc_update_chase — the same update, computed the way an unresolved chain
 * is: every element walks root -> ... -> struct -> x/y with device loads the
 * compiler may not hoist (Listing 2's loop body; Sec. 3).  Comparison path. */
DC_API dc_status dc_update_chase(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_verify_chain — walk `path` on the device with one thread, reading the
 * relocated pointers, and return the address it reaches (blocking).  Lets a
 * caller check dc_resolve_chain against the device image. */
DC_API dc_status dc_verify_chain(dc_plan_t plan, const dc_step* path, uint32_t len, dc_stream_t stream,
                          uint64_t* dev_addr);

/* dc_copy_back — transfer back (Algorithm 2 step 5): the arrays the last
 * dc_update_* wrote (the x arrays of the selected structs), or every ARRAY
 * block with DC_COPY_ALL_ARRAYS, are copied device -> pinned arena -> the
 * original host arrays: by DMA in chunks of about 8 MiB, each scattered into
 * the host arrays by the plan's host threads while the later chunks are still
 * in transfer (array interiors in pages DC_PLAN_MAP_HOST mapped go straight
 * into those pages by one kernel launch).  Pointers, scalars and struct bytes
 * on the host are never written.  Blocking: returns when the host arrays hold
 * the results.  The device's error word is read before any host byte is
 * written: if an earlier kernel recorded an error, nothing is scattered and
 * that error is returned.  Errors: DC_ESTATE (no op run and no flag),
 * DC_ECUDA, plus any device error recorded by earlier kernels. */
#define DC_COPY_ALL_ARRAYS 1u
DC_API dc_status dc_copy_back(dc_plan_t plan, uint32_t flags, dc_stream_t stream);

/* dc_roundtrip — dc_deep_copy, dc_update_leaves(op) and dc_copy_back(0) as one
 * call (Algorithm 2 steps 3-5: transfer, run the kernel once, transfer back),
 * with the same results.  With a DC_PLAN_MAP_HOST plan, or a tree built in
 * dc_host_arena memory, whose selected arrays start on 16-byte host addresses,
 * the blocks the op does not touch move as in dc_deep_copy, and one kernel
 * then reads each selected x and y element from host memory, applies the
 * update, writes x and y into the arena and the new x straight back to the
 * host: the two directions of the link overlap instead of following each
 * other.  The kernel runs in up to eight tile groups while host threads stage
 * the next group's array heads and tails and return the previous group's.
 * Otherwise it runs the three calls in turn.
 * Blocking: returns when the host arrays hold the results.  Errors: as the
 * three calls. */
DC_API dc_status dc_roundtrip(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_roundtrip_selected — the paper's pointerchain transfer scheme (Sec. 3;
 * Sec. 4.1.1 item 3): only the arrays the op reads and writes move, each to its
 * effective device address; the update runs and x comes back.  Structs and
 * other arrays are neither copied nor relocated (their device copies are
 * whatever an earlier deep copy left), so it suits kernels that work through
 * resolved addresses only.  The host result equals dc_roundtrip's.
 * Blocking.  Errors: as dc_roundtrip. */
DC_API dc_status dc_roundtrip_selected(dc_plan_t plan, const dc_op* op, dc_stream_t stream);

/* dc_sync — wait for the plan's work on `stream` and report (then clear) the
 * device error word: DC_EDEVICE_BOUNDS, DC_ETIMEOUT or DC_EVERIFY. */
DC_API dc_status dc_sync(dc_plan_t plan, dc_stream_t stream);

/* Device address of the bound buffer's data region (for callers that want
 * to read the device image, e.g. to check it). */
DC_API dc_status dc_device_base(dc_plan_t plan, uint64_t* dev_base);

/* ---- comparison path: Unified Virtual Memory (Sec. 2; Sec. 4.1.1 item 1) ----
 * dc_uvm_build replicates the host tree into managed memory, one
 * cudaMallocManaged allocation per block (as if every malloc of the
 * application were managed); its pointers are valid on host and device with
 * no relocation.  dc_uvm_update runs the pointer-chasing leaf kernel on it, so
 * pages migrate on demand; dc_uvm_prefetch moves every block to the device
 * (to_device = 1) or back to the host (0) first.  dc_uvm_copy_back copies
 * the written arrays (all arrays with DC_COPY_ALL_ARRAYS) into the original
 * host tree: the host reads managed memory.  dc_uvm_root gives the managed
 * root's address. */
DC_API dc_status dc_uvm_build(const dc_schema* schema, const void* host_root, dc_uvm_t* out);
DC_API dc_status dc_uvm_root(dc_uvm_t uvm, uint64_t* managed_root);
DC_API dc_status dc_uvm_prefetch(dc_uvm_t uvm, int to_device, dc_stream_t stream);
DC_API dc_status dc_uvm_update(dc_uvm_t uvm, const dc_op* op, dc_stream_t stream);
DC_API dc_status dc_uvm_copy_back(dc_uvm_t uvm, const void* host_root, uint32_t flags);
DC_API dc_status dc_uvm_sync(dc_uvm_t uvm, dc_stream_t stream);
DC_API dc_status dc_uvm_destroy(dc_uvm_t uvm);

/* ---- several GPUs -------------------------------------------------------------
 * dc_partition_by_bytes — assign n independent trees (payload sizes
 * bytes[0..n)) to nparts GPUs with no exchange between them: greedy LPT,
 * trees in decreasing size (stable), each to the part with the fewest bytes
 * so far (the lower part index on ties).  part_of[i] receives tree i's part;
 * part_bytes (nparts entries, may be NULL) each part's total.  No part
 * exceeds the mean by more than the largest tree, and the result depends on
 * the inputs alone, so every rank can compute it independently.  Host only.
 * Errors: DC_EINVAL (nparts = 0, NULL arrays with n > 0, total overflow). */
DC_API dc_status dc_partition_by_bytes(const uint64_t* bytes, uint64_t n, uint32_t nparts, uint32_t* part_of,
                                       uint64_t* part_bytes);

/* ---- relocation that allocates nothing ---------------------------------------
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate memory at the point where they relocate.  Examples: code
 * embedded in an application whose device memory is handed out only by that
 * application's own pool (a cudaMalloc there would bypass its accounting or
 * fail under its cap), or a hot path that must not allocate because
 * cudaMalloc/cudaFree can synchronize the whole device.  Such a caller owns
 * only the device copy of the data region (info.data_bytes, holding the
 * marshalled image, e.g. from its own copy of dc_deep_copy's transfer).
 *
 * dc_relocate_static does dc_relocate's work on `dev_data` (16-byte aligned,
 * at least data_bytes long; pointers become dev_data + block offset) with all
 * of its scratch in one fixed device array of DC_STATIC_SCRATCH_BYTES bytes
 * inside the library, which every GPU that loads the library keeps until the
 * process exits.  Limits: plans of at most DC_STATIC_MAX_BLOCKS blocks whose
 * pointer slots lie in at most DC_STATIC_MAX_TILES of the 8 KiB ranges the
 * struct blocks are relocated in (DC_EBUDGET otherwise); no DC_PLAN_VERIFY
 * check.  It calls no cudaMalloc,
 * cudaHostAlloc, cudaFree or other allocating routine.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and the array
 * keeps the previous call's contents (the call clears what must start at
 * zero), so calls whose work overlaps on the GPU race: order them on one
 * stream.  If `dev_status` is not NULL, the device word it points to receives
 * the kernel's error bits once the work completes: 0 = success; bit 0 (1) = an
 * offset outside the buffers (what dc_sync reports as DC_EDEVICE_BOUNDS); bit 1
 * (2) = a wait for the kernel's own bulk copies gave up (DC_ETIMEOUT).  Test
 * the bits, not equality: both can be set. */
#define DC_STATIC_MAX_BLOCKS 65536u
#define DC_STATIC_MAX_TILES 16384u /* 8 KiB ranges of struct bytes that hold a pointer slot */
#define DC_STATIC_SCRATCH_BYTES 1835776u /* 512 KiB records + 1 MiB lane groups + 256 KiB tile table + control words */
DC_API dc_status dc_relocate_static(dc_plan_t plan, void* dev_data, uint64_t data_bytes, uint32_t* dev_status,
                             dc_stream_t stream);

/* ---- host arenas (Algorithm 1's allocation requests served from one buffer) ----
 * A host arena is pinned, mapped host memory of the library's own; blocks
 * handed out by dc_host_arena_alloc (16-byte aligned at least) are blocks a
 * tree can be built from.  A plan recognises blocks inside an arena and
 * moves them between the arena and the device without any marshal or
 * scatter: the deep copy reads them and the copy back writes them in place,
 * one kernel launch each way, whatever their sizes (no DC_PLAN_MAP_HOST
 * needed; nothing outside the arena is touched).  dc_roundtrip then also
 * takes its fused path.  dc_host_arena_alloc returns NULL when the arena is
 * full; dc_host_arena_reset forgets every allocation (no plan may still use
 * them); an arena must outlive the plans that use it. */
typedef struct dc_host_arena_s* dc_host_arena_t;
DC_API dc_status dc_host_arena_create(uint64_t bytes, dc_host_arena_t* out);
DC_API void* dc_host_arena_alloc(dc_host_arena_t arena, uint64_t bytes, uint64_t align);
DC_API dc_status dc_host_arena_used(dc_host_arena_t arena, uint64_t* used);
DC_API dc_status dc_host_arena_reset(dc_host_arena_t arena);
DC_API dc_status dc_host_arena_destroy(dc_host_arena_t arena);

/* ---- served requests (a request loop with continuous batching) ----------------
 * A server deep-copies and updates trees on request.  It owns `dev_pool`
 * (a caller-owned device buffer, the HBM budget) and a mapped pinned host
 * pool of `pinned_bytes`, both sub-allocated first-fit, and `nslots` worker
 * slots, each a host thread with its own CUDA stream.  Requests are admitted
 * as they arrive and as slots and memory free up, so the work of requests on
 * different slots overlaps on the device; requests on one key keep their
 * order.  A served tree stays resident (plan, arena, pinned staging) until
 * its memory is needed; then the least recently used idle tree is evicted.
 * A request's result is the same as dc_roundtrip's on a fresh plan: the host
 * tree's x arrays hold the update.  A request with `retouch` set on a resident
 * key skips the deep copy (its device copy already equals the host tree,
 * which the caller asserts it has not changed since).  With
 * DC_SERVER_SEQUENTIAL the requests are handled one at a time in arrival
 * order and nothing stays resident (the plain per-structure path).
 * All requests of a server share one schema; trees must not change shape
 * while resident. */
typedef struct dc_server_s* dc_server_t;
typedef struct {
  uint64_t key;          /* identifies the tree (equal keys = the same tree) */
  const void* host_root; /* its root */
  double arrival_s;      /* arrival time, seconds after dc_server_run starts */
  int32_t retouch;       /* 1: the host tree is unchanged since this key's last request */
} dc_request;
typedef struct {
  uint64_t served, failed, resident_hits, evictions;
  uint64_t h2d_bytes, d2h_bytes;       /* payload deep-copied / copied back */
  uint64_t peak_resident_bytes, resident_bytes;
  double wall_s;                       /* time spent in dc_server_run */
} dc_server_stats;
#define DC_SERVER_SEQUENTIAL 1u
DC_API dc_status dc_server_create(const dc_schema* schema, void* dev_pool, uint64_t dev_bytes, uint64_t pinned_bytes,
                           uint32_t nslots, uint32_t flags, dc_server_t* out);
/* Run a request stream: each request is injected at its arrival time and
 * served with `op`; returns when all are done.  latency_ms[i] (may be NULL)
 * receives the time from request i's arrival to its results being in host
 * memory, or -1 if it failed (the first failure's status is returned). */
DC_API dc_status dc_server_run(dc_server_t server, const dc_request* requests, uint64_t n, const dc_op* op,
                        double* latency_ms);
DC_API dc_status dc_server_stats_get(dc_server_t server, dc_server_stats* out);
DC_API dc_status dc_server_destroy(dc_server_t server);

/* ---- misc ------------------------------------------------------------------ */
DC_API const char* dc_last_error(void);
DC_API const char* dc_status_name(dc_status s);
/* Number of kernels this library has launched in this process (all paths). */
DC_API uint64_t dc_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DC_H */
