/*
 * treegen — seeded synthetic host structures (see treegen.h for the recipe).
 * Shared input generator: no deep-copy arithmetic lives here.
 */
#define _GNU_SOURCE
#include "treegen.h"

#include <math.h>
#include <pthread.h>
#include <stdarg.h>
#include <stdatomic.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define TG_MAX_STRUCT 1024u
#define TG_MAX_FIELDS 64u
#define TG_MAX_LEVELS 1024u

static __thread char g_err[512];

static void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

const char* tg_error(void) { return g_err; }

/* ---- random streams ---------------------------------------------------- */

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t s[4];
} rng_t;

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(rng_t* r) { /* xoshiro256** */
  uint64_t* s = r->s;
  uint64_t result = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return result;
}

static void rng_seed(rng_t* r, uint64_t seed) {
  uint64_t x = seed;
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static double rng_unit(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1p-53; }

static double rng_normal(rng_t* r) { /* Box-Muller, cosine branch */
  double u1 = 1.0 - rng_unit(r); /* (0, 1] */
  double u2 = rng_unit(r);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

static int64_t draw(rng_t* r, const tg_dist* d) {
  switch (d->dist) {
    case TG_DIST_CONST:
      return (int64_t)d->a;
    case TG_DIST_UNIFORM: {
      int64_t lo = (int64_t)d->a, hi = (int64_t)d->b;
      if (hi < lo) return lo;
      return lo + (int64_t)(rng_next(r) % (uint64_t)(hi - lo + 1));
    }
    case TG_DIST_LOGNORMAL: {
      double z = rng_normal(r);
      double v = exp(log(d->a) + d->b * z);
      long long n = llround(v);
      if (n < 1) n = 1;
      if (d->c >= 1 && n > (long long)d->c) n = (long long)d->c;
      return n;
    }
  }
  return 0;
}

/* ---- tree bookkeeping -------------------------------------------------- */

typedef struct {
  void* ptr;
  uint64_t n;
  int32_t kind;
  uint32_t elem_size;
  uint64_t key;
} fill_job;

struct tg_tree_s {
  void* root;
  void** allocs;
  uint64_t nallocs, cap_allocs;
  fill_job* jobs;
  uint64_t njobs, cap_jobs;
  uint64_t payload, nstructs, nblocks;
  uint32_t ntypes;
  uint64_t* elems; /* ntypes * TG_MAX_FIELDS */
};

typedef struct {
  const tg_schema* s;
  const tg_shape* sh;
  rng_t rng;
  tg_tree* t;
  int dry;
  tg_alloc_fn alloc;
  void* actx;
  uint64_t payload, nstructs, nblocks;
  uint8_t is_count[64][TG_MAX_FIELDS];
} ctx_t;

static int push_alloc(tg_tree* t, void* p) {
  if (t->nallocs == t->cap_allocs) {
    uint64_t nc = t->cap_allocs ? 2 * t->cap_allocs : 1024;
    void** na = realloc(t->allocs, nc * sizeof(void*));
    if (!na) return -1;
    t->allocs = na;
    t->cap_allocs = nc;
  }
  t->allocs[t->nallocs++] = p;
  return 0;
}

static int push_job(tg_tree* t, fill_job j) {
  if (t->njobs == t->cap_jobs) {
    uint64_t nc = t->cap_jobs ? 2 * t->cap_jobs : 1024;
    fill_job* nj = realloc(t->jobs, nc * sizeof(fill_job));
    if (!nj) return -1;
    t->jobs = nj;
    t->cap_jobs = nc;
  }
  t->jobs[t->njobs++] = j;
  return 0;
}

static int64_t read_scalar(const uint8_t* p, const tg_field* f) {
  if (f->elem_size == 8) {
    int64_t v;
    memcpy(&v, p + f->offset, 8);
    return v;
  }
  int32_t v;
  memcpy(&v, p + f->offset, 4);
  return v;
}

static void write_scalar(uint8_t* p, const tg_field* f, int64_t v) {
  if (f->elem_size == 8) {
    memcpy(p + f->offset, &v, 8);
  } else {
    int32_t w = (int32_t)v;
    memcpy(p + f->offset, &w, 4);
  }
}

static uint64_t field_count(const uint8_t* p, const tg_type* T, const tg_field* f) {
  if (f->count_field < 0) return f->count_const;
  int64_t v = read_scalar(p, &T->fields[f->count_field]);
  return v < 0 ? 0 : (uint64_t)v;
}

static const tg_rule* find_rule(const tg_shape* sh, uint32_t type, uint32_t field) {
  for (uint32_t i = 0; i < sh->nrules; i++)
    if (sh->rules[i].type == type && sh->rules[i].field == field) return &sh->rules[i];
  return NULL;
}

static void* tg_alloc(ctx_t* c, uint64_t bytes) {
  if (c->alloc) return c->alloc(c->actx, bytes ? bytes : 1, 16);
  void* p = malloc(bytes ? bytes : 1);
  if (!p) return NULL;
  if (push_alloc(c->t, p)) {
    free(p);
    return NULL;
  }
  return p;
}

/* Fill the struct of type `ti` at `dst` (level `level`); recurse into children. */
static int build_struct(ctx_t* c, uint32_t ti, uint8_t* dst, uint32_t level) {
  const tg_type* T = &c->s->types[ti];
  uint8_t buf[TG_MAX_STRUCT];
  c->nstructs++;
  /* struct bytes (padding and non-count scalars included) start random */
  for (uint32_t o = 0; o < T->size; o += 8) {
    uint64_t r = rng_next(&c->rng);
    uint32_t k = T->size - o < 8 ? T->size - o : 8;
    memcpy(buf + o, &r, k);
  }
  int leaf = (level + 1 >= c->sh->levels);
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const tg_field* f = &T->fields[fi];
    if (f->kind != TG_SCALAR || !c->is_count[ti][fi]) continue;
    const tg_rule* r = find_rule(c->sh, ti, fi);
    int64_t v = r ? draw(&c->rng, leaf ? &r->leaf : &r->interior) : 0;
    write_scalar(buf, f, v);
  }
  if (leaf) { /* the last level has no children */
    for (uint32_t fi = 0; fi < T->nfields; fi++) {
      const tg_field* f = &T->fields[fi];
      if (f->kind == TG_CHILD && f->count_field >= 0) write_scalar(buf, &T->fields[f->count_field], 0);
    }
  }
  /* arrays and child blocks, in field order */
  uint8_t* child_ptr[TG_MAX_FIELDS];
  uint64_t child_n[TG_MAX_FIELDS];
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const tg_field* f = &T->fields[fi];
    child_ptr[fi] = NULL;
    child_n[fi] = 0;
    if (f->kind == TG_ARRAY) {
      uint64_t n = field_count(buf, T, f);
      void* p = NULL;
      uint64_t key = rng_next(&c->rng);
      if (n) {
        uint64_t bytes = n * f->elem_size;
        c->payload += bytes;
        c->nblocks++;
        if (!c->dry) {
          p = tg_alloc(c, bytes);
          if (!p) {
            set_err("out of host memory (%llu bytes)", (unsigned long long)bytes);
            return -1;
          }
          fill_job j = {p, n, f->elem_kind, f->elem_size, key};
          if (push_job(c->t, j)) return -1;
          c->t->elems[ti * TG_MAX_FIELDS + fi] += n;
        }
      }
      memcpy(buf + f->offset, &p, sizeof p);
    } else if (f->kind == TG_CHILD) {
      uint64_t n = leaf ? 0 : field_count(buf, T, f);
      const tg_type* C = &c->s->types[f->child_type];
      void* p = NULL;
      if (n) {
        uint64_t bytes = n * C->size;
        c->payload += bytes;
        c->nblocks++;
        if (!c->dry) {
          p = tg_alloc(c, bytes);
          if (!p) {
            set_err("out of host memory (%llu bytes)", (unsigned long long)bytes);
            return -1;
          }
        }
      }
      memcpy(buf + f->offset, &p, sizeof p);
      child_ptr[fi] = p;
      child_n[fi] = n;
    }
  }
  if (!c->dry) memcpy(dst, buf, T->size);
  for (uint32_t fi = 0; fi < T->nfields; fi++) {
    const tg_field* f = &T->fields[fi];
    if (f->kind != TG_CHILD || child_n[fi] == 0) continue;
    const tg_type* C = &c->s->types[f->child_type];
    for (uint64_t j = 0; j < child_n[fi]; j++) {
      uint8_t* d = c->dry ? NULL : child_ptr[fi] + j * C->size;
      if (build_struct(c, (uint32_t)f->child_type, d, level + 1)) return -1;
    }
  }
  return 0;
}

static int check_schema(const tg_schema* s, const tg_shape* sh) {
  if (!s || !s->types || s->ntypes == 0 || s->ntypes > 64 || s->root_type >= s->ntypes) {
    set_err("bad schema header");
    return -1;
  }
  if (!sh || sh->levels == 0 || sh->levels > TG_MAX_LEVELS) {
    set_err("shape.levels must be in [1, %u]", TG_MAX_LEVELS);
    return -1;
  }
  for (uint32_t ti = 0; ti < s->ntypes; ti++) {
    const tg_type* T = &s->types[ti];
    if (T->size == 0 || T->size > TG_MAX_STRUCT || T->nfields > TG_MAX_FIELDS || (T->nfields && !T->fields)) {
      set_err("type %u: bad size or field count", ti);
      return -1;
    }
    for (uint32_t fi = 0; fi < T->nfields; fi++) {
      const tg_field* f = &T->fields[fi];
      uint32_t w = f->kind == TG_SCALAR ? f->elem_size : 8;
      if (f->offset + w > T->size) {
        set_err("type %u field %u: outside the struct", ti, fi);
        return -1;
      }
      if (f->kind == TG_SCALAR && f->elem_size != 4 && f->elem_size != 8) {
        set_err("type %u field %u: scalar size must be 4 or 8", ti, fi);
        return -1;
      }
      if (f->kind == TG_CHILD && (f->child_type < 0 || (uint32_t)f->child_type >= s->ntypes)) {
        set_err("type %u field %u: bad child type", ti, fi);
        return -1;
      }
      if (f->kind != TG_SCALAR && f->count_field >= 0 &&
          ((uint32_t)f->count_field >= T->nfields || T->fields[f->count_field].kind != TG_SCALAR)) {
        set_err("type %u field %u: count field is not a scalar", ti, fi);
        return -1;
      }
    }
  }
  return 0;
}

static void init_ctx(ctx_t* c, const tg_schema* s, const tg_shape* sh, uint64_t seed) {
  memset(c, 0, sizeof *c);
  c->s = s;
  c->sh = sh;
  rng_seed(&c->rng, seed);
  for (uint32_t ti = 0; ti < s->ntypes; ti++) {
    const tg_type* T = &s->types[ti];
    for (uint32_t fi = 0; fi < T->nfields; fi++) {
      const tg_field* f = &T->fields[fi];
      if (f->kind != TG_SCALAR && f->count_field >= 0) c->is_count[ti][f->count_field] = 1;
    }
  }
}

/* ---- parallel value fill ------------------------------------------------ */

typedef struct {
  const fill_job* job;
  uint64_t lo, hi;
} fill_piece;

typedef struct {
  const fill_piece* pieces;
  uint64_t npieces;
  atomic_uint_fast64_t next;
} fill_ctx;

static void fill_range(const fill_job* j, uint64_t lo, uint64_t hi) {
  const uint64_t phi = 0x9E3779B97F4A7C15ull;
  if (j->kind == TG_F32) {
    float* p = (float*)j->ptr;
    for (uint64_t i = lo; i < hi; i++) {
      uint64_t h = mix64(j->key + (i + 1) * phi);
      p[i] = (float)((int64_t)h >> 40) * 0x1p-23f;
    }
  } else if (j->kind == TG_F64) {
    double* p = (double*)j->ptr;
    for (uint64_t i = lo; i < hi; i++) {
      uint64_t h = mix64(j->key + (i + 1) * phi);
      p[i] = (double)((int64_t)h >> 11) * 0x1p-52;
    }
  } else {
    uint8_t* p = (uint8_t*)j->ptr;
    uint64_t total = hi * j->elem_size;
    for (uint64_t b = lo * j->elem_size; b < total; b++) {
      uint64_t h = mix64(j->key + (b + 1) * phi);
      p[b] = (uint8_t)(h >> 56);
    }
  }
}

static void* fill_worker(void* arg) {
  fill_ctx* fc = (fill_ctx*)arg;
  for (;;) {
    uint64_t k = atomic_fetch_add(&fc->next, 1);
    if (k >= fc->npieces) break;
    const fill_piece* p = &fc->pieces[k];
    fill_range(p->job, p->lo, p->hi);
  }
  return NULL;
}

static int fill_all(tg_tree* t, uint32_t nthreads) {
  const uint64_t piece = 1u << 20;
  uint64_t np = 0;
  for (uint64_t i = 0; i < t->njobs; i++) np += (t->jobs[i].n + piece - 1) / piece;
  fill_piece* pcs = malloc((np ? np : 1) * sizeof *pcs);
  if (!pcs) return -1;
  uint64_t k = 0;
  for (uint64_t i = 0; i < t->njobs; i++)
    for (uint64_t lo = 0; lo < t->jobs[i].n; lo += piece) {
      pcs[k].job = &t->jobs[i];
      pcs[k].lo = lo;
      pcs[k].hi = lo + piece < t->jobs[i].n ? lo + piece : t->jobs[i].n;
      k++;
    }
  fill_ctx fc;
  fc.pieces = pcs;
  fc.npieces = np;
  atomic_init(&fc.next, 0);
  long ncpu = sysconf(_SC_NPROCESSORS_ONLN);
  uint32_t nt = nthreads ? nthreads : (uint32_t)(ncpu > 0 ? ncpu : 1);
  if (nt > 64) nt = 64;
  if (np < 4 * (uint64_t)nt && t->payload < (64ull << 20)) nt = 1;
  pthread_t th[64];
  uint32_t started = 0;
  for (uint32_t i = 1; i < nt; i++)
    if (pthread_create(&th[started], NULL, fill_worker, &fc) == 0) started++;
  fill_worker(&fc);
  for (uint32_t i = 0; i < started; i++) pthread_join(th[i], NULL);
  free(pcs);
  return 0;
}

/* ---- public API --------------------------------------------------------- */

tg_tree* tg_build(const tg_schema* s, const tg_shape* sh, uint64_t seed) {
  return tg_build_ex(s, sh, seed, NULL, NULL);
}

tg_tree* tg_build_ex(const tg_schema* s, const tg_shape* sh, uint64_t seed, tg_alloc_fn alloc, void* actx) {
  if (check_schema(s, sh)) return NULL;
  tg_tree* t = calloc(1, sizeof *t);
  if (!t) return NULL;
  t->ntypes = s->ntypes;
  t->elems = calloc((size_t)s->ntypes * TG_MAX_FIELDS, sizeof(uint64_t));
  ctx_t* c = malloc(sizeof *c);
  if (!t->elems || !c) {
    free(c);
    tg_free(t);
    set_err("out of host memory");
    return NULL;
  }
  init_ctx(c, s, sh, seed);
  c->t = t;
  c->alloc = alloc;
  c->actx = actx;
  const tg_type* R = &s->types[s->root_type];
  t->root = tg_alloc(c, R->size);
  if (!t->root) {
    free(c);
    tg_free(t);
    set_err("out of host memory");
    return NULL;
  }
  c->payload = R->size;
  c->nblocks = 1;
  if (build_struct(c, s->root_type, (uint8_t*)t->root, 0)) {
    free(c);
    tg_free(t);
    return NULL;
  }
  t->payload = c->payload;
  t->nstructs = c->nstructs;
  t->nblocks = c->nblocks;
  free(c);
  if (fill_all(t, sh->nthreads)) {
    tg_free(t);
    set_err("out of host memory (fill)");
    return NULL;
  }
  free(t->jobs);
  t->jobs = NULL;
  t->njobs = t->cap_jobs = 0;
  return t;
}

int tg_dry_bytes(const tg_schema* s, const tg_shape* sh, uint64_t seed, uint64_t* bytes) {
  if (check_schema(s, sh)) return -1;
  ctx_t* c = malloc(sizeof *c);
  if (!c) return -1;
  init_ctx(c, s, sh, seed);
  c->dry = 1;
  c->payload = s->types[s->root_type].size;
  int rc = build_struct(c, s->root_type, NULL, 0);
  *bytes = c->payload;
  free(c);
  return rc;
}

void* tg_root(const tg_tree* t) { return t ? t->root : NULL; }
uint64_t tg_payload_bytes(const tg_tree* t) { return t ? t->payload : 0; }
uint64_t tg_nstructs(const tg_tree* t) { return t ? t->nstructs : 0; }
uint64_t tg_nblocks(const tg_tree* t) { return t ? t->nblocks : 0; }

uint64_t tg_nelems(const tg_tree* t, uint32_t type, uint32_t field) {
  if (!t || type >= t->ntypes || field >= TG_MAX_FIELDS) return 0;
  return t->elems[type * TG_MAX_FIELDS + field];
}

void tg_free(tg_tree* t) {
  if (!t) return;
  for (uint64_t i = 0; i < t->nallocs; i++) free(t->allocs[i]);
  free(t->allocs);
  free(t->jobs);
  free(t->elems);
  free(t);
}
