/*
 * treegen — seeded synthetic inputs for the deep-copy benchmarks.
 *
 * Builds nested, pointer-linked host structures (structs whose members point
 * to arrays and to child-struct arrays) in ordinary malloc'd host memory, the
 * way an application would before a deep copy (Fig 2 step a; Alg 2 steps 1-2).
 * Every block is a separate heap allocation, so the host tree is scattered.
 *
 * This module is shared test/bench infrastructure: it generates inputs for the
 * CPU oracle and for the CUDA path alike and contains none of the deep-copy
 * arithmetic (no arena layout, no relocation, no leaf update).
 *
 * Randomness
 *   - shape stream: xoshiro256** seeded by SplitMix64(seed); it draws counts
 *     (lognormal via Box-Muller, uniform ints), scalar values, struct filler
 *     bytes and one 64-bit key per array;
 *   - array values are counter-based: element i of an array with key K takes
 *     h = mix64(K + (i+1) * 0x9E3779B97F4A7C15) (SplitMix64 finaliser), so the
 *     fill is identical for any thread count.
 *   - f32 value: (float)((int64_t)h >> 40) * 2^-23, a multiple of 2^-23 in
 *     [-1, 1); f64 value: (double)((int64_t)h >> 11) * 2^-52 in [-1, 1).
 */
#ifndef TREEGEN_H
#define TREEGEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { TG_SCALAR = 0, TG_ARRAY = 1, TG_CHILD = 2 };
enum { TG_F32 = 0, TG_F64 = 1, TG_BYTES = 2 };
enum { TG_DIST_CONST = 0, TG_DIST_UNIFORM = 1, TG_DIST_LOGNORMAL = 2 };

/* Field descriptor. SCALAR: elem_size 4 or 8 (signed integer). ARRAY: a pointer
 * to count_field/count_const elements of elem_size bytes, filled per elem_kind.
 * CHILD: a pointer to a contiguous array of `count` structs of child_type. */
typedef struct {
  int32_t kind;
  uint32_t offset;
  uint32_t elem_size;
  int32_t count_field; /* index of the SCALAR field holding the count, or -1 */
  uint64_t count_const;
  int32_t child_type;
  int32_t elem_kind;
} tg_field;

typedef struct {
  uint32_t size, align, nfields;
  const tg_field* fields;
} tg_type;

typedef struct {
  uint32_t ntypes, root_type;
  const tg_type* types;
} tg_schema;

/* A distribution for a count: CONST a; UNIFORM integer in [a, b];
 * LOGNORMAL with median a, sigma b, clamped to [1, c]. */
typedef struct {
  int32_t dist;
  double a, b, c;
} tg_dist;

/* The value of SCALAR field `field` of every struct of `type`: `interior` on
 * levels 0..levels-2, `leaf` on level levels-1 (root = level 0). */
typedef struct {
  uint32_t type, field;
  tg_dist interior, leaf;
} tg_rule;

typedef struct {
  uint32_t levels;   /* CHILD pointers on level levels-1 are NULL, count 0 */
  uint32_t nrules;
  const tg_rule* rules;
  uint32_t nthreads; /* value-fill threads, 0 = all online cores */
} tg_shape;

typedef struct tg_tree_s tg_tree;

/* Build one tree. Count fields without a rule are 0; other scalars and all
 * struct bytes not covered by a field take random values. NULL on error. */
tg_tree* tg_build(const tg_schema* s, const tg_shape* shape, uint64_t seed);
/* The same, with every block taken from `alloc(ctx, bytes, 16)` instead of
 * malloc (e.g. an arena); tg_free then frees none of the blocks. */
typedef void* (*tg_alloc_fn)(void* ctx, uint64_t bytes, uint64_t align);
tg_tree* tg_build_ex(const tg_schema* s, const tg_shape* shape, uint64_t seed, tg_alloc_fn alloc, void* ctx);
/* Same draws as tg_build, nothing allocated: the tree's payload bytes. */
int tg_dry_bytes(const tg_schema* s, const tg_shape* shape, uint64_t seed, uint64_t* bytes);
void* tg_root(const tg_tree* t);
uint64_t tg_payload_bytes(const tg_tree* t); /* sum of block bytes */
uint64_t tg_nstructs(const tg_tree* t);
uint64_t tg_nblocks(const tg_tree* t);       /* root + non-empty arrays + non-empty child arrays */
uint64_t tg_nelems(const tg_tree* t, uint32_t type, uint32_t field); /* elements in that ARRAY field */
void tg_free(tg_tree* t);
const char* tg_error(void);

#ifdef __cplusplus
}
#endif
#endif
