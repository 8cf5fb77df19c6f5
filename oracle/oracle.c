/*
 * oracle.c — CPU oracle for the deep-copy hot path.  TEST INFRASTRUCTURE ONLY
 * (see oracle.h).  Recursive, single-threaded, no blocking or reordering
 * beyond what the paper's steps state.  Compiled with -ffp-contract=off so the
 * leaf update rounds once per operation, as IEEE-754 single precision does.
 */
#include "oracle.h"

#include <omp.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ---- small helpers ------------------------------------------------------ */

static void say(char* msg, size_t len, const char* fmt, ...) {
  if (!msg || !len) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, len, fmt, ap);
  va_end(ap);
}

static int64_t scalar_at(const uint8_t* s, const or_field* f) {
  if (f->elem_size == 8) {
    int64_t v;
    memcpy(&v, s + f->offset, 8);
    return v;
  }
  int32_t v;
  memcpy(&v, s + f->offset, 4);
  return v;
}

static void* ptr_at(const uint8_t* s, const or_field* f) {
  void* p;
  memcpy(&p, s + f->offset, sizeof p);
  return p;
}

static uint64_t u64_at(const uint8_t* s, uint64_t off) {
  uint64_t v;
  memcpy(&v, s + off, 8);
  return v;
}

static void set_ptr(uint8_t* s, const or_field* f, uint64_t v) { memcpy(s + f->offset, &v, 8); }

/* The element count of an ARRAY or CHILD field: the value of its count
 * scalar, or its constant.  A negative count is an invalid structure. */
static int count_of(const or_type* T, const uint8_t* s, const or_field* f, uint64_t* n) {
  if (f->count_field < 0) {
    *n = f->count_const;
    return OR_OK;
  }
  int64_t v = scalar_at(s, &T->fields[f->count_field]);
  if (v < 0) return OR_EINVAL;
  *n = (uint64_t)v;
  return OR_OK;
}

static uint64_t block_bytes(const or_schema* sc, const or_field* f, uint64_t n) {
  if (f->kind == OR_ARRAY) return n * f->elem_size;
  return n * sc->types[f->child_type].size;
}

static uint64_t round16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

/* ---- counters ------------------------------------------------------------ */

static int count_struct(const or_schema* sc, uint32_t ti, const uint8_t* s, uint32_t level,
                        or_counts* c) {
  const or_type* T = &sc->types[ti];
  c->nstructs++;
  if (level < 64) c->per_level[level]++;
  if (level + 1 > c->levels) c->levels = level + 1;
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind == OR_SCALAR) continue;
    uint64_t n;
    if (count_of(T, s, f, &n)) return OR_EINVAL;
    if (n == 0) continue;
    const uint8_t* p = (const uint8_t*)ptr_at(s, f);
    if (!p) return OR_EINVAL;
    uint64_t b = block_bytes(sc, f, n);
    c->nblocks++;
    c->nptr++;
    c->payload_bytes += b;
    c->padded_bytes += round16(b);
    if (f->kind == OR_CHILD) {
      uint32_t cs = sc->types[f->child_type].size;
      for (uint64_t j = 0; j < n; j++) {
        int rc = count_struct(sc, (uint32_t)f->child_type, p + j * cs, level + 1, c);
        if (rc) return rc;
      }
    }
  }
  return OR_OK;
}

int or_count(const or_schema* s, const void* root, or_counts* out) {
  memset(out, 0, sizeof *out);
  if (!s || !root) return OR_EINVAL;
  uint32_t rs = s->types[s->root_type].size;
  out->nblocks = 1;
  out->payload_bytes = rs;
  out->padded_bytes = round16(rs);
  return count_struct(s, s->root_type, (const uint8_t*)root, 0, out);
}

/* ---- deep copy (Fig 2) ----------------------------------------------------- */

static uint8_t* bump(or_arena* a, uint64_t bytes) {
  uint64_t at = round16(a->used);
  if (at + bytes > a->cap) return NULL;
  a->used = at + bytes;
  return a->base + at;
}

static uint64_t as_pointer(const or_arena* a, const uint8_t* block) {
  uint64_t base = a->ptr_base ? a->ptr_base : (uint64_t)(uintptr_t)a->base;
  return base + (uint64_t)(block - a->base);
}

/* dst already holds a byte copy of the struct at src (step b/c); replicate
 * what each pointer field points to and re-point the field (step d). */
static int copy_struct(const or_schema* sc, uint32_t ti, const uint8_t* src, uint8_t* dst,
                       or_arena* a) {
  const or_type* T = &sc->types[ti];
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind == OR_SCALAR) continue;
    uint64_t n;
    if (count_of(T, src, f, &n)) return OR_EINVAL;
    if (n == 0) {
      set_ptr(dst, f, 0);
      continue;
    }
    const uint8_t* from = (const uint8_t*)ptr_at(src, f);
    if (!from) return OR_EINVAL;
    uint64_t bytes = block_bytes(sc, f, n);
    uint8_t* to = bump(a, bytes);
    if (!to) return OR_ENOMEM;
    memcpy(to, from, bytes);
    set_ptr(dst, f, as_pointer(a, to));
    if (f->kind == OR_CHILD) {
      uint32_t cs = sc->types[f->child_type].size;
      for (uint64_t j = 0; j < n; j++) {
        int rc = copy_struct(sc, (uint32_t)f->child_type, from + j * cs, to + j * cs, a);
        if (rc) return rc;
      }
    }
  }
  return OR_OK;
}

int or_deep_copy(const or_schema* s, const void* src_root, or_arena* a, void** dst_root) {
  if (!s || !src_root || !a || !a->base) return OR_EINVAL;
  uint32_t rs = s->types[s->root_type].size;
  uint8_t* root = bump(a, rs);
  if (!root) return OR_ENOMEM;
  memcpy(root, src_root, rs);
  if (dst_root) *dst_root = root;
  return copy_struct(s, s->root_type, (const uint8_t*)src_root, root, a);
}

/* ---- leaf update ----------------------------------------------------------- */

static int apply(const or_schema* sc, const or_op* op, uint8_t* node) {
  const or_type* T = &sc->types[op->type];
  const or_field* fx = &T->fields[op->x_field];
  uint64_t n;
  if (fx->kind != OR_ARRAY || count_of(T, node, fx, &n)) return OR_EINVAL;
  if (n == 0) return OR_OK;
  uint8_t* x = (uint8_t*)ptr_at(node, fx);
  if (op->kind == OR_OP_SCALE) {
    if (fx->elem_kind == 0) {
      float a = (float)op->scale;
      float* xf = (float*)x;
      for (uint64_t i = 0; i < n; i++) xf[i] = xf[i] * a;
    } else if (fx->elem_kind == 1) {
      double* xd = (double*)x;
      for (uint64_t i = 0; i < n; i++) xd[i] = xd[i] * op->scale;
    } else {
      return OR_EINVAL;
    }
    return OR_OK;
  }
  const or_field* fy = &T->fields[op->y_field];
  uint64_t ny;
  if (fy->kind != OR_ARRAY || count_of(T, node, fy, &ny) || ny != n ||
      fy->elem_kind != fx->elem_kind)
    return OR_EINVAL;
  const uint8_t* y = (const uint8_t*)ptr_at(node, fy);
  if (fx->elem_kind == 0) {
    float* xf = (float*)x;
    const float* yf = (const float*)y;
    for (uint64_t i = 0; i < n; i++) {
      float half = 0.5f * yf[i];
      xf[i] = xf[i] + half;
    }
  } else if (fx->elem_kind == 1) {
    double* xd = (double*)x;
    const double* yd = (const double*)y;
    for (uint64_t i = 0; i < n; i++) {
      double half = 0.5 * yd[i];
      xd[i] = xd[i] + half;
    }
  } else {
    return OR_EINVAL;
  }
  return OR_OK;
}

static int update_all(const or_schema* sc, uint32_t ti, uint8_t* s, const or_op* op) {
  const or_type* T = &sc->types[ti];
  if (ti == op->type) {
    int rc = apply(sc, op, s);
    if (rc) return rc;
  }
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind != OR_CHILD) continue;
    uint64_t n;
    if (count_of(T, s, f, &n)) return OR_EINVAL;
    uint8_t* c = (uint8_t*)ptr_at(s, f);
    uint32_t cs = sc->types[f->child_type].size;
    for (uint64_t j = 0; j < n; j++) {
      int rc = update_all(sc, (uint32_t)f->child_type, c + j * cs, op);
      if (rc) return rc;
    }
  }
  return OR_OK;
}

/* Follow (field, index) steps through CHILD fields from the root; returns the
 * struct reached and its type. */
static int walk_chain(const or_schema* sc, uint8_t* root, const or_step* path, uint32_t len,
                      uint8_t** node, uint32_t* type) {
  uint8_t* s = root;
  uint32_t ti = sc->root_type;
  for (uint32_t k = 0; k < len; k++) {
    const or_type* T = &sc->types[ti];
    if (path[k].field >= T->nfields) return OR_EINVAL;
    const or_field* f = &T->fields[path[k].field];
    uint64_t n;
    if (f->kind != OR_CHILD || count_of(T, s, f, &n) || path[k].index >= n) return OR_EINVAL;
    s = (uint8_t*)ptr_at(s, f) + path[k].index * sc->types[f->child_type].size;
    ti = (uint32_t)f->child_type;
  }
  *node = s;
  *type = ti;
  return OR_OK;
}

int or_update(const or_schema* s, void* root, const or_op* op) {
  if (!s || !root || !op || op->type >= s->ntypes) return OR_EINVAL;
  if (op->x_field >= s->types[op->type].nfields) return OR_EINVAL;
  if (op->kind == OR_OP_AXPY_HALF && op->y_field >= s->types[op->type].nfields) return OR_EINVAL;
  if (op->sel == OR_SEL_ALL) return update_all(s, s->root_type, (uint8_t*)root, op);
  uint8_t* node;
  uint32_t ti;
  int rc = walk_chain(s, (uint8_t*)root, op->path, op->path_len, &node, &ti);
  if (rc) return rc;
  if (ti != op->type) return OR_EINVAL;
  return apply(s, op, node);
}

/* ---- the same update on every host core (the CPU baseline on N cores) ------
 * Not a parity reference.  It collects the structs the op selects, as
 * or_update visits them, then splits each one's arrays into chunks of
 * 2^16 elements and applies the same per-element arithmetic as apply() to the
 * chunks in parallel (OpenMP).  Elements are independent, so the result is
 * bit-identical to or_update's. */

typedef struct {
  uint8_t** v;
  uint64_t n, cap;
} node_list;

static int push_node(node_list* l, uint8_t* node) {
  if (l->n == l->cap) {
    uint64_t cap = l->cap ? 2 * l->cap : 1024;
    uint8_t** v = (uint8_t**)realloc(l->v, cap * sizeof *v);
    if (!v) return OR_ENOMEM;
    l->v = v;
    l->cap = cap;
  }
  l->v[l->n++] = node;
  return OR_OK;
}

static int collect_all(const or_schema* sc, uint32_t ti, uint8_t* s, const or_op* op, node_list* out) {
  const or_type* T = &sc->types[ti];
  if (ti == op->type) {
    int rc = push_node(out, s);
    if (rc) return rc;
  }
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind != OR_CHILD) continue;
    uint64_t n;
    if (count_of(T, s, f, &n)) return OR_EINVAL;
    uint8_t* c = (uint8_t*)ptr_at(s, f);
    uint32_t cs = sc->types[f->child_type].size;
    for (uint64_t j = 0; j < n; j++) {
      int rc = collect_all(sc, (uint32_t)f->child_type, c + j * cs, op, out);
      if (rc) return rc;
    }
  }
  return OR_OK;
}

/* elements [lo, hi) of one selected struct's x (and y), as apply() does them */
static void apply_range(const or_op* op, int kind, uint8_t* x, const uint8_t* y, uint64_t lo, uint64_t hi) {
  if (op->kind == OR_OP_SCALE) {
    if (kind == 0) {
      float a = (float)op->scale;
      float* xf = (float*)x;
      for (uint64_t i = lo; i < hi; i++) xf[i] = xf[i] * a;
    } else {
      double* xd = (double*)x;
      for (uint64_t i = lo; i < hi; i++) xd[i] = xd[i] * op->scale;
    }
  } else if (kind == 0) {
    float* xf = (float*)x;
    const float* yf = (const float*)y;
    for (uint64_t i = lo; i < hi; i++) {
      float half = 0.5f * yf[i];
      xf[i] = xf[i] + half;
    }
  } else {
    double* xd = (double*)x;
    const double* yd = (const double*)y;
    for (uint64_t i = lo; i < hi; i++) {
      double half = 0.5 * yd[i];
      xd[i] = xd[i] + half;
    }
  }
}

int or_update_parallel(const or_schema* s, void* root, const or_op* op, int nthreads) {
  if (!s || !root || !op || op->type >= s->ntypes) return OR_EINVAL;
  const or_type* T = &s->types[op->type];
  if (op->x_field >= T->nfields) return OR_EINVAL;
  if (op->kind == OR_OP_AXPY_HALF && op->y_field >= T->nfields) return OR_EINVAL;
  node_list nodes = {0};
  int rc;
  if (op->sel == OR_SEL_ALL) {
    rc = collect_all(s, s->root_type, (uint8_t*)root, op, &nodes);
  } else {
    uint8_t* node;
    uint32_t ti;
    rc = walk_chain(s, (uint8_t*)root, op->path, op->path_len, &node, &ti);
    if (!rc) rc = ti != op->type ? OR_EINVAL : push_node(&nodes, node);
  }
  /* the chunks: (node, first element) pairs, checked as apply() checks them */
  const uint64_t CH = 1u << 16;
  uint64_t nchunks = 0;
  const or_field* fx = &T->fields[op->x_field];
  const or_field* fy = op->kind == OR_OP_AXPY_HALF ? &T->fields[op->y_field] : NULL;
  for (uint64_t k = 0; !rc && k < nodes.n; k++) {
    uint64_t n, ny;
    if (fx->kind != OR_ARRAY || count_of(T, nodes.v[k], fx, &n) || fx->elem_kind > 1) rc = OR_EINVAL;
    else if (fy && (fy->kind != OR_ARRAY || count_of(T, nodes.v[k], fy, &ny) || ny != n ||
                    fy->elem_kind != fx->elem_kind)) rc = OR_EINVAL;
    else nchunks += (n + CH - 1) / CH;
  }
  uint64_t* chunk = NULL;  /* per chunk: node index, first element, end */
  if (!rc && nchunks) {
    chunk = (uint64_t*)malloc(3 * nchunks * sizeof *chunk);
    if (!chunk) rc = OR_ENOMEM;
  }
  if (!rc) {
    uint64_t c = 0;
    for (uint64_t k = 0; k < nodes.n; k++) {
      uint64_t n = 0;
      count_of(T, nodes.v[k], fx, &n);
      for (uint64_t lo = 0; lo < n; lo += CH, c++) {
        chunk[3 * c] = k;
        chunk[3 * c + 1] = lo;
        chunk[3 * c + 2] = lo + CH < n ? lo + CH : n;
      }
    }
    const int nt = nthreads > 0 ? nthreads : omp_get_num_procs();  /* this call only */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
    for (int64_t c2 = 0; c2 < (int64_t)nchunks; c2++) {
      uint8_t* node = nodes.v[chunk[3 * c2]];
      apply_range(op, fx->elem_kind, (uint8_t*)ptr_at(node, fx), fy ? (const uint8_t*)ptr_at(node, fy) : NULL,
                  chunk[3 * c2 + 1], chunk[3 * c2 + 2]);
    }
  }
  free(chunk);
  free(nodes.v);
  return rc;
}

int or_threads(void) { return omp_get_num_procs(); }

/* ---- copy back (Alg 2 step 5) ---------------------------------------------- */

static int back_struct(const or_schema* sc, uint32_t ti, const uint8_t* from, uint8_t* to,
                       const or_op* op, int all) {
  const or_type* T = &sc->types[ti];
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind == OR_SCALAR) continue;
    uint64_t n;
    if (count_of(T, to, f, &n)) return OR_EINVAL;
    if (n == 0) continue;
    const uint8_t* pf = (const uint8_t*)ptr_at(from, f);
    uint8_t* pt = (uint8_t*)ptr_at(to, f);
    if (f->kind == OR_ARRAY) {
      int wanted = all || (op && ti == op->type && fi == op->x_field);
      if (wanted) memcpy(pt, pf, block_bytes(sc, f, n));
    } else if (all || (op && op->sel == OR_SEL_ALL)) {
      uint32_t cs = sc->types[f->child_type].size;
      for (uint64_t j = 0; j < n; j++) {
        int rc = back_struct(sc, (uint32_t)f->child_type, pf + j * cs, pt + j * cs, op, all);
        if (rc) return rc;
      }
    }
  }
  return OR_OK;
}

int or_copy_back(const or_schema* s, const void* copy_root, void* src_root, const or_op* op,
                 int all_arrays) {
  if (!s || !copy_root || !src_root) return OR_EINVAL;
  if (all_arrays || !op || op->sel == OR_SEL_ALL)
    return back_struct(s, s->root_type, (const uint8_t*)copy_root, (uint8_t*)src_root, op,
                       all_arrays || !op);
  uint8_t *from, *to;
  uint32_t tf, tt;
  int rc = walk_chain(s, (uint8_t*)copy_root, op->path, op->path_len, &from, &tf);
  if (rc) return rc;
  rc = walk_chain(s, (uint8_t*)src_root, op->path, op->path_len, &to, &tt);
  if (rc) return rc;
  if (tf != op->type || tt != op->type) return OR_EINVAL;
  const or_type* T = &s->types[op->type];
  const or_field* fx = &T->fields[op->x_field];
  uint64_t n;
  if (count_of(T, to, fx, &n)) return OR_EINVAL;
  if (n) memcpy(ptr_at(to, fx), ptr_at(from, fx), block_bytes(s, fx, n));
  return OR_OK;
}

/* ---- results check (Alg 2 step 6) ------------------------------------------ */

/* Is byte `b` of a struct of type T inside one of its pointer slots? */
static int in_pointer_slot(const or_type* T, uint32_t b) {
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind != OR_SCALAR && b >= f->offset && b < f->offset + 8) return 1;
  }
  return 0;
}

static int eq_struct(const or_schema* sc, uint32_t ti, const uint8_t* a, const uint8_t* b,
                     char* msg, size_t len, const char* where) {
  const or_type* T = &sc->types[ti];
  for (uint32_t k = 0; k < T->size; k++)
    if (!in_pointer_slot(T, k) && a[k] != b[k]) {
      say(msg, len, "%s: struct byte %u differs", where, k);
      return OR_MISMATCH;
    }
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind == OR_SCALAR) continue;
    uint64_t n;
    if (count_of(T, a, f, &n)) return OR_EINVAL;
    const uint8_t* pa = (const uint8_t*)ptr_at(a, f);
    const uint8_t* pb = (const uint8_t*)ptr_at(b, f);
    if (n == 0) continue;
    if (!pa || !pb) {
      say(msg, len, "%s.field%u: null pointer with count %llu", where, fi, (unsigned long long)n);
      return OR_MISMATCH;
    }
    if (f->kind == OR_ARRAY) {
      if (memcmp(pa, pb, block_bytes(sc, f, n))) {
        uint64_t e = 0;
        while (e < n * f->elem_size && pa[e] == pb[e]) e++;
        say(msg, len, "%s.field%u: array differs at byte %llu", where, fi, (unsigned long long)e);
        return OR_MISMATCH;
      }
    } else {
      uint32_t cs = sc->types[f->child_type].size;
      for (uint64_t j = 0; j < n; j++) {
        char w[512];
        snprintf(w, sizeof w, "%s.field%u[%llu]", where, fi, (unsigned long long)j);
        int rc = eq_struct(sc, (uint32_t)f->child_type, pa + j * cs, pb + j * cs, msg, len, w);
        if (rc) return rc;
      }
    }
  }
  return OR_OK;
}

int or_trees_equal(const or_schema* s, const void* a, const void* b, char* msg, size_t msglen) {
  if (!s || !a || !b) return OR_EINVAL;
  say(msg, msglen, "equal");
  return eq_struct(s, s->root_type, (const uint8_t*)a, (const uint8_t*)b, msg, msglen, "root");
}

/* ---- device image check ---------------------------------------------------- */

typedef struct {
  uint64_t lo, hi;
} span;

typedef struct {
  const or_schema* sc;
  const uint8_t* img;
  uint64_t bytes, base;
  span* spans;
  uint64_t nspans, cap;
  or_counts* seen;
  char* msg;
  size_t len;
  uint64_t pack_below; /* arrays of fewer bytes may start on their element alignment */
} img_ctx;

static int add_span(img_ctx* c, uint64_t lo, uint64_t hi) {
  if (c->nspans == c->cap) {
    uint64_t nc = c->cap ? 2 * c->cap : 256;
    span* ns = (span*)realloc(c->spans, nc * sizeof(span));
    if (!ns) return OR_ENOMEM;
    c->spans = ns;
    c->cap = nc;
  }
  c->spans[c->nspans].lo = lo;
  c->spans[c->nspans].hi = hi;
  c->nspans++;
  return OR_OK;
}

static int img_struct(img_ctx* c, uint32_t ti, const uint8_t* src, uint64_t off, uint32_t level,
                      const char* where) {
  const or_type* T = &c->sc->types[ti];
  const uint8_t* im = c->img + off;
  c->seen->nstructs++;
  if (level < 64) c->seen->per_level[level]++;
  if (level + 1 > c->seen->levels) c->seen->levels = level + 1;
  for (uint32_t k = 0; k < T->size; k++)
    if (!in_pointer_slot(T, k) && im[k] != src[k]) {
      say(c->msg, c->len, "%s: struct byte %u differs from the source", where, k);
      return OR_MISMATCH;
    }
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const or_field* f = &T->fields[fi];
    if (f->kind == OR_SCALAR) continue;
    uint64_t n;
    if (count_of(T, src, f, &n)) return OR_EINVAL;
    uint64_t p = u64_at(im, f->offset);
    const uint8_t* sp = (const uint8_t*)ptr_at(src, f);
    if (n == 0) {
      if (p != 0) {
        say(c->msg, c->len, "%s.field%u: count 0 but pointer 0x%llx", where, fi,
            (unsigned long long)p);
        return OR_MISMATCH;
      }
      continue;
    }
    if (!sp) return OR_EINVAL;
    uint64_t b = block_bytes(c->sc, f, n);
    if (p == (uint64_t)(uintptr_t)sp) {
      say(c->msg, c->len, "%s.field%u: still the source address", where, fi);
      return OR_MISMATCH;
    }
    if (p < c->base || p - c->base > c->bytes || b > c->bytes - (p - c->base)) {
      say(c->msg, c->len, "%s.field%u: pointer 0x%llx outside the arena", where, fi,
          (unsigned long long)p);
      return OR_MISMATCH;
    }
    uint64_t o = p - c->base;
    /* every block starts on 16 bytes; in a packed layout an array of fewer than
     * pack_below bytes may start on 8 bytes (f64) or 4 (other elements) */
    const uint64_t al = (f->kind == OR_ARRAY && b < c->pack_below) ? (f->elem_kind == 1 ? 8 : 4) : 16;
    if (o % al) {
      say(c->msg, c->len, "%s.field%u: block offset %llu not %llu-byte aligned", where, fi, (unsigned long long)o,
          (unsigned long long)al);
      return OR_MISMATCH;
    }
    int rc = add_span(c, o, o + b);
    if (rc) return rc;
    c->seen->nblocks++;
    c->seen->nptr++;
    c->seen->payload_bytes += b;
    c->seen->padded_bytes += round16(b);
    if (f->kind == OR_ARRAY) {
      if (memcmp(c->img + o, sp, b)) {
        say(c->msg, c->len, "%s.field%u: array bytes differ from the source", where, fi);
        return OR_MISMATCH;
      }
    } else {
      uint32_t cs = c->sc->types[f->child_type].size;
      for (uint64_t j = 0; j < n; j++) {
        char w[512];
        snprintf(w, sizeof w, "%s.field%u[%llu]", where, fi, (unsigned long long)j);
        rc = img_struct(c, (uint32_t)f->child_type, sp + j * cs, o + j * cs, level + 1, w);
        if (rc) return rc;
      }
    }
  }
  return OR_OK;
}

static int span_cmp(const void* a, const void* b) {
  const span* x = (const span*)a;
  const span* y = (const span*)b;
  return x->lo < y->lo ? -1 : x->lo > y->lo ? 1 : 0;
}

int or_check_image(const or_schema* s, const void* src_root, const void* image,
                   uint64_t image_bytes, uint64_t dev_base, uint64_t root_off, or_counts* seen,
                   char* msg, size_t msglen) {
  return or_check_image_packed(s, src_root, image, image_bytes, dev_base, root_off, 0, seen, msg, msglen);
}

int or_check_image_packed(const or_schema* s, const void* src_root, const void* image,
                          uint64_t image_bytes, uint64_t dev_base, uint64_t root_off, uint64_t pack_below,
                          or_counts* seen, char* msg, size_t msglen) {
  or_counts local;
  if (!seen) seen = &local;
  memset(seen, 0, sizeof *seen);
  if (!s || !src_root || !image) return OR_EINVAL;
  uint32_t rs = s->types[s->root_type].size;
  if (root_off % 16 || root_off > image_bytes || rs > image_bytes - root_off) {
    say(msg, msglen, "root block outside the arena");
    return OR_MISMATCH;
  }
  img_ctx c = {s, (const uint8_t*)image, image_bytes, dev_base, NULL, 0, 0, seen, msg, msglen, pack_below};
  int rc = add_span(&c, root_off, root_off + rs);
  seen->nblocks = 1;
  seen->payload_bytes = rs;
  seen->padded_bytes = round16(rs);
  if (!rc) rc = img_struct(&c, s->root_type, (const uint8_t*)src_root, root_off, 0, "root");
  if (!rc) {
    qsort(c.spans, c.nspans, sizeof(span), span_cmp);
    for (uint64_t i = 1; i < c.nspans; i++)
      if (c.spans[i].lo < c.spans[i - 1].hi) {
        say(msg, msglen, "blocks at offsets %llu and %llu overlap",
            (unsigned long long)c.spans[i - 1].lo, (unsigned long long)c.spans[i].lo);
        rc = OR_MISMATCH;
        break;
      }
  }
  free(c.spans);
  if (!rc) say(msg, msglen, "ok");
  return rc;
}

/* ---- selective deep copy of one chain (Sec. 2) ---------------------------- */

/* One pointer of the chain in the image: `p` must be a device address inside
 * the arena with the whole `b`-byte block after it, 16-byte aligned (the
 * layout's block alignment), and not the source's own address. */
static int chain_ptr(uint64_t p, uint64_t b, const void* src_ptr, uint64_t image_bytes, uint64_t dev_base,
                     const char* what, char* msg, size_t msglen) {
  if (p == (uint64_t)(uintptr_t)src_ptr) {
    say(msg, msglen, "%s: still the source address", what);
    return OR_MISMATCH;
  }
  if (p < dev_base || p - dev_base > image_bytes || b > image_bytes - (p - dev_base)) {
    say(msg, msglen, "%s: pointer 0x%llx outside the arena", what, (unsigned long long)p);
    return OR_MISMATCH;
  }
  if ((p - dev_base) % 16) {
    say(msg, msglen, "%s: block offset %llu not 16-byte aligned", what, (unsigned long long)(p - dev_base));
    return OR_MISMATCH;
  }
  return OR_OK;
}

/* Every struct of a struct block on the chain carries its source's bytes
 * outside its pointer slots. */
static int chain_block(const or_schema* sc, uint32_t ti, const uint8_t* src, const uint8_t* im, uint64_t n,
                       uint32_t step, char* msg, size_t msglen) {
  const or_type* T = &sc->types[ti];
  for (uint64_t j = 0; j < n; j++)
    for (uint32_t k = 0; k < T->size; k++)
      if (!in_pointer_slot(T, k) && im[j * T->size + k] != src[j * T->size + k]) {
        say(msg, msglen, "chain block %u, struct %llu: byte %u differs from the source", step,
            (unsigned long long)j, k);
        return OR_MISMATCH;
      }
  return OR_OK;
}

int or_check_chain_image(const or_schema* s, const void* src_root, const void* image, uint64_t image_bytes,
                         uint64_t dev_base, uint64_t root_off, const or_step* path, uint32_t len, int32_t x_field,
                         int32_t y_field, char* msg, size_t msglen) {
  if (!s || !src_root || !image) return OR_EINVAL;
  const uint8_t* img = (const uint8_t*)image;
  uint32_t ti = s->root_type;
  if (root_off % 16 || root_off > image_bytes || s->types[ti].size > image_bytes - root_off) {
    say(msg, msglen, "root block outside the arena");
    return OR_MISMATCH;
  }
  /* the struct block the walk is in: its source, its image offset, its length
   * in structs, and the struct of it the chain takes */
  const uint8_t* blk_src = (const uint8_t*)src_root;
  uint64_t blk_off = root_off, blk_n = 1, at = 0;
  for (uint32_t k = 0;; k++) {
    const or_type* T = &s->types[ti];
    int rc = chain_block(s, ti, blk_src, img + blk_off, blk_n, k, msg, msglen);
    if (rc) return rc;
    const uint8_t* cur_src = blk_src + at * T->size;
    const uint8_t* cur_img = img + blk_off + at * T->size;
    if (k == len) { /* the struct the chain reaches: its x and y arrays */
      int32_t fields[2] = {x_field, y_field};
      for (int a = 0; a < 2; a++) {
        if (fields[a] < 0) continue;
        if ((uint32_t)fields[a] >= T->nfields) return OR_EINVAL;
        const or_field* f = &T->fields[fields[a]];
        uint64_t n;
        if (f->kind != OR_ARRAY || count_of(T, cur_src, f, &n)) return OR_EINVAL;
        uint64_t p = u64_at(cur_img, f->offset);
        if (n == 0) {
          if (p != 0) {
            say(msg, msglen, "field%d: count 0 but pointer 0x%llx", fields[a], (unsigned long long)p);
            return OR_MISMATCH;
          }
          continue;
        }
        const uint8_t* sp = (const uint8_t*)ptr_at(cur_src, f);
        if (!sp) return OR_EINVAL;
        uint64_t b = block_bytes(s, f, n);
        char what[64];
        snprintf(what, sizeof what, "field%d of the chain's last struct", fields[a]);
        if ((rc = chain_ptr(p, b, sp, image_bytes, dev_base, what, msg, msglen))) return rc;
        if (memcmp(img + (p - dev_base), sp, b)) {
          say(msg, msglen, "%s: array bytes differ from the source", what);
          return OR_MISMATCH;
        }
      }
      say(msg, msglen, "ok");
      return OR_OK;
    }
    if (path[k].field >= T->nfields) return OR_EINVAL;
    const or_field* f = &T->fields[path[k].field];
    uint64_t n;
    if (f->kind != OR_CHILD || count_of(T, cur_src, f, &n) || path[k].index >= n) return OR_EINVAL;
    const uint8_t* sp = (const uint8_t*)ptr_at(cur_src, f);
    if (!sp) return OR_EINVAL;
    const uint32_t cs = s->types[f->child_type].size;
    uint64_t p = u64_at(cur_img, f->offset);
    char what[64];
    snprintf(what, sizeof what, "chain step %u (field %u)", k, path[k].field);
    if ((rc = chain_ptr(p, n * cs, sp, image_bytes, dev_base, what, msg, msglen))) return rc;
    blk_src = sp;
    blk_off = p - dev_base;
    blk_n = n;
    at = path[k].index;
    ti = (uint32_t)f->child_type;
  }
}

/* ---- effective addresses of pointer chains (Sec. 3) ------------------------ */

int or_image_resolve(const or_schema* s, const void* image, uint64_t image_bytes,
                     uint64_t dev_base, uint64_t root_off, const or_step* path, uint32_t len,
                     uint64_t* dev_addr) {
  if (!s || !image || !dev_addr) return OR_EINVAL;
  const uint8_t* img = (const uint8_t*)image;
  uint64_t off = root_off;
  uint32_t ti = s->root_type;
  for (uint32_t k = 0; k < len; k++) {
    const or_type* T = &s->types[ti];
    if (off > image_bytes || T->size > image_bytes - off) return OR_EINVAL;
    if (path[k].field >= T->nfields) return OR_EINVAL;
    const or_field* f = &T->fields[path[k].field];
    uint64_t n;
    if (f->kind == OR_SCALAR || count_of(T, img + off, f, &n) || path[k].index >= n)
      return OR_EINVAL;
    uint64_t p = u64_at(img + off, f->offset);
    if (p < dev_base) return OR_EINVAL;
    if (f->kind == OR_ARRAY) {
      if (k + 1 != len) return OR_EINVAL;
      *dev_addr = p + path[k].index * f->elem_size;
      return OR_OK;
    }
    off = p - dev_base + path[k].index * s->types[f->child_type].size;
    ti = (uint32_t)f->child_type;
  }
  *dev_addr = dev_base + off;
  return OR_OK;
}

int or_host_resolve(const or_schema* s, const void* root, const or_step* path, uint32_t len,
                    uint64_t* host_addr) {
  if (!s || !root || !host_addr) return OR_EINVAL;
  const uint8_t* p = (const uint8_t*)root;
  uint32_t ti = s->root_type;
  for (uint32_t k = 0; k < len; k++) {
    const or_type* T = &s->types[ti];
    if (path[k].field >= T->nfields) return OR_EINVAL;
    const or_field* f = &T->fields[path[k].field];
    uint64_t n;
    if (f->kind == OR_SCALAR || count_of(T, p, f, &n) || path[k].index >= n) return OR_EINVAL;
    const uint8_t* q = (const uint8_t*)ptr_at(p, f);
    if (f->kind == OR_ARRAY) {
      if (k + 1 != len) return OR_EINVAL;
      *host_addr = (uint64_t)(uintptr_t)(q + path[k].index * f->elem_size);
      return OR_OK;
    }
    p = q + path[k].index * s->types[f->child_type].size;
    ti = (uint32_t)f->child_type;
  }
  *host_addr = (uint64_t)(uintptr_t)p;
  return OR_OK;
}
