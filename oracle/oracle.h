/*
 * oracle.h — CPU oracle for the deep-copy hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct C written from the
 * paper.  Only the test suite, the package's smoke entry point and the CPU
 * baseline leg of the benchmark may load it.  It shares no code with the CUDA
 * path: it declares its own mirror of the field-offset schema.
 *
 * Functions and the passage each follows:
 *   or_deep_copy      full deep copy (Sec. 2, Fig 2 steps a-d): every struct,
 *                     array and child array is replicated into a fresh arena
 *                     and every copied pointer is made to point at the replica.
 *   or_count          structure counters; for the paper's Linear and Dense
 *                     shapes the payload equals Eq 1 / Eq 2 / Eq 3 (+ padding
 *                     of the 12-byte last-level struct, see tests).
 *   or_update         the leaf kernel: x[i] = x[i] + 0.5f*y[i] (fp32) or the
 *                     paper's scaling kernel x[i] *= scale (Sec. 4.1.2 item 1,
 *                     Listing 2), on every struct (allused) or on the struct a
 *                     pointer chain reaches (LLused / Listing 2's chain).
 *   or_update_parallel  the same on every host core (OpenMP): the benchmark's
 *                     multi-core CPU baseline, pinned to or_update.
 *   or_copy_back      transfer back of the arrays the kernel wrote (Alg 2 step 5).
 *   or_trees_equal    the results check (Alg 2 step 6): two trees have the same
 *                     shape, the same scalar/padding bytes and the same arrays.
 *   or_check_image    checks a device image of a deep copy against its source:
 *                     same shape, byte-equal data, every pointer inside the
 *                     arena, 16-byte aligned, and no two blocks overlapping.
 *                     or_check_image_packed allows arrays of fewer than
 *                     pack_below bytes to start on their element alignment (8
 *                     bytes for f64, else 4), the packed layout's promise.
 *   or_check_chain_image  checks a device image of a selective deep copy of
 *                     one pointer chain (Sec. 2: only what the chain reaches is
 *                     replicated) along that chain: each struct block the chain
 *                     passes through holds its source's non-pointer bytes,
 *                     every pointer the chain follows and the x / y array
 *                     pointers of the struct it reaches lie inside the arena
 *                     (16-byte aligned, not the source address), and those
 *                     arrays hold the source's bytes.  Off the chain nothing
 *                     is read.
 *   or_image_resolve  follows a pointer chain through a device image (the
 *                     effective address of Sec. 3) by reading its pointers.
 *   or_host_resolve   the same chain in a host tree.
 * Parity is pinned for every function by the non-GPU tests (tables, closed
 * forms, hand-built trees, planted mistakes); none is "parity unpinned".
 */
#ifndef DC_ORACLE_H
#define DC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SCALAR = 0, OR_ARRAY = 1, OR_CHILD = 2 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_MISMATCH = 3 };
enum { OR_OP_AXPY_HALF = 0, OR_OP_SCALE = 1 };
enum { OR_SEL_ALL = 0, OR_SEL_CHAIN = 1 };

typedef struct {
  int32_t kind;
  uint32_t offset;
  uint32_t elem_size;
  int32_t count_field;
  uint64_t count_const;
  int32_t child_type;
  int32_t elem_kind; /* 0 f32, 1 f64, 2 raw bytes */
} or_field;

typedef struct {
  uint32_t size, align, nfields;
  const or_field* fields;
} or_type;

typedef struct {
  uint32_t ntypes, root_type;
  const or_type* types;
} or_schema;

/* Bump arena.  Copied pointers are written as ptr_base + (block - base);
 * ptr_base == 0 means base itself (a usable host copy). */
typedef struct {
  uint8_t* base;
  uint64_t cap, used;
  uint64_t ptr_base;
} or_arena;

typedef struct {
  uint64_t nstructs;      /* struct instances */
  uint64_t nblocks;       /* root + non-empty arrays + non-empty child arrays */
  uint64_t payload_bytes; /* sum of block bytes */
  uint64_t padded_bytes;  /* sum of block bytes rounded up to 16 */
  uint64_t nptr;          /* non-null pointers (= nblocks - 1) */
  uint32_t levels;
  uint64_t per_level[64]; /* struct instances per level (root = 0) */
} or_counts;

typedef struct {
  uint32_t field;
  uint64_t index;
} or_step;

typedef struct {
  int32_t kind;   /* OR_OP_* */
  double scale;   /* OR_OP_SCALE; rounded to float for f32 arrays */
  int32_t sel;    /* OR_SEL_* */
  const or_step* path;
  uint32_t path_len;
  uint32_t type;  /* struct type owning x_field / y_field */
  uint32_t x_field, y_field;
} or_op;

int or_count(const or_schema* s, const void* root, or_counts* out);
int or_deep_copy(const or_schema* s, const void* src_root, or_arena* a, void** dst_root);
int or_update(const or_schema* s, void* root, const or_op* op);
/* The same update with the selected arrays split into 2^16-element chunks
 * that `nthreads` OpenMP threads (0 = all) apply in parallel: the CPU
 * baseline on every host core.  Not a parity reference; its results equal
 * or_update's bit for bit.  or_threads() = the threads it uses by default. */
int or_update_parallel(const or_schema* s, void* root, const or_op* op, int nthreads);
int or_threads(void);
int or_copy_back(const or_schema* s, const void* copy_root, void* src_root, const or_op* op,
                 int all_arrays);
int or_trees_equal(const or_schema* s, const void* a, const void* b, char* msg, size_t msglen);
int or_check_image(const or_schema* s, const void* src_root, const void* image,
                   uint64_t image_bytes, uint64_t dev_base, uint64_t root_off, or_counts* seen,
                   char* msg, size_t msglen);
int or_check_image_packed(const or_schema* s, const void* src_root, const void* image,
                          uint64_t image_bytes, uint64_t dev_base, uint64_t root_off, uint64_t pack_below,
                          or_counts* seen, char* msg, size_t msglen);
/* y_field < 0: the op has no y array.  The path's steps are CHILD fields. */
int or_check_chain_image(const or_schema* s, const void* src_root, const void* image, uint64_t image_bytes,
                         uint64_t dev_base, uint64_t root_off, const or_step* path, uint32_t len, int32_t x_field,
                         int32_t y_field, char* msg, size_t msglen);
int or_image_resolve(const or_schema* s, const void* image, uint64_t image_bytes,
                     uint64_t dev_base, uint64_t root_off, const or_step* path, uint32_t len,
                     uint64_t* dev_addr);
int or_host_resolve(const or_schema* s, const void* root, const or_step* path, uint32_t len,
                    uint64_t* host_addr);

#ifdef __cplusplus
}
#endif
#endif
