/*
 * graphgen.c -- seeded synthetic graph generators.
 *
 * This module produces INPUTS only: edge lists (src[i], dst[i]) of int32
 * vertex ids.  It holds none of the triangle-counting method's arithmetic
 * (no degree ordering, no orientation, no adjacency sort, no intersection);
 * the GPU path and the CPU oracle both consume what it writes and neither
 * shares any other code with it.
 *
 * Randomness: every random number is a pure function of (seed, stream,
 * counter) built from the SplitMix64 output function of Steele, Lea and
 * Flood ("Fast splittable pseudorandom number generators", OOPSLA 2014):
 * value = mix(key(seed, stream) + (counter + 1) * 0x9e3779b97f4a7c15).
 * Because draws are addressed by counter, the multi-threaded loops below
 * produce the same bytes for any thread count and on any host.  Floating
 * point appears only in the random geometric graph, where it is confined to
 * exact operations plus IEEE-rounded products/sums; the build passes
 * -ffp-contract=off so that no fused multiply-add changes a comparison
 * between x86_64 and aarch64.
 *
 * Graph families (workloads of the paper's evaluation, stand-ins for its
 * datasets):
 *   gg_er            Erdos-Renyi G(n, m): uniform pairs, loops skipped,
 *                    redrawn until m distinct undirected edges.
 *   gg_rmat          R-MAT (Chakrabarti, Zhan & Faloutsos 2004) raw draws
 *                    with a random vertex permutation; loops and duplicates
 *                    are kept (the library under test removes them).
 *   gg_rmat_distinct R-MAT draws until m distinct non-loop undirected edges;
 *                    the output lists each of those edges once, in the order
 *                    of its first draw, in the direction it was first drawn.
 *   gg_rgg           random geometric graph in the unit square: an edge iff
 *                    the Euclidean distance is < r; ids shuffled; each edge
 *                    once, random direction, random order.
 *   gg_ba            Barabasi-Albert preferential attachment; ids shuffled.
 *   gg_ws            Watts-Strogatz ring lattice with rewired edges; ids
 *                    shuffled.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define GG_GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Key of an independent stream: one SplitMix64 step from a seed/stream mix. */
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix(seed * GG_GOLDEN + (stream + 1) * 0xd1b54a32d192ed03ULL);
}

/* counter-th 64-bit output of the stream with this key. */
static inline uint64_t gg_rand(uint64_t key, uint64_t ctr) {
  return gg_mix(key + (ctr + 1) * GG_GOLDEN);
}

/* Uniform integer in [0, bound) from 32 random bits (multiply-shift). */
static inline uint32_t gg_below(uint32_t bits, uint32_t bound) {
  return (uint32_t)(((uint64_t)bits * (uint64_t)bound) >> 32);
}

/* Stream ids.  Fixed forever: changing one changes every stored input hash. */
enum {
  GG_S_ER = 1,
  GG_S_RMAT = 2,
  GG_S_RMAT_PERM = 3,
  GG_S_RGG_POINTS = 4,
  GG_S_RGG_PERM = 5,
  GG_S_RGG_DIR = 6,
  GG_S_RGG_SHUFFLE = 7,
  GG_S_BA = 8,
  GG_S_BA_PERM = 9,
  GG_S_WS = 10,
  GG_S_WS_PERM = 11,
};

/* ------------------------------------------------------------------ */
/* tiny parallel-for over [0, n) in contiguous chunks                   */
/* ------------------------------------------------------------------ */
typedef void (*gg_body_fn)(void *ctx, int64_t lo, int64_t hi, int tid);

typedef struct {
  gg_body_fn fn;
  void *ctx;
  int64_t lo, hi;
  int tid;
} gg_task;

static void *gg_task_run(void *p) {
  gg_task *t = (gg_task *)p;
  t->fn(t->ctx, t->lo, t->hi, t->tid);
  return NULL;
}

static int gg_nthreads(void) {
  const char *e = getenv("GG_THREADS");
  long t = e ? atol(e) : sysconf(_SC_NPROCESSORS_ONLN);
  if (t < 1) t = 1;
  if (t > 64) t = 64;
  return (int)t;
}

static void gg_parallel_min(int64_t n, int nt, gg_body_fn fn, void *ctx, int64_t serial_below) {
  if (nt < 1) nt = 1;
  if (nt > n) nt = (int)(n > 0 ? n : 1);
  if (n < serial_below || nt == 1) {
    fn(ctx, 0, n, 0);
    return;
  }
  pthread_t th[64];
  gg_task tk[64];
  int started[64];
  for (int i = 0; i < nt; ++i) {
    tk[i].fn = fn;
    tk[i].ctx = ctx;
    tk[i].lo = n * i / nt;
    tk[i].hi = n * (i + 1) / nt;
    tk[i].tid = i;
    started[i] = pthread_create(&th[i], NULL, gg_task_run, &tk[i]) == 0;
    if (!started[i]) gg_task_run(&tk[i]);
  }
  for (int i = 0; i < nt; ++i)
    if (started[i]) pthread_join(th[i], NULL);
}

static void gg_parallel(int64_t n, int nt, gg_body_fn fn, void *ctx) {
  gg_parallel_min(n, nt, fn, ctx, 4096);
}

/* ------------------------------------------------------------------ */
/* open-addressing set of undirected edges (generator bookkeeping only) */
/* ------------------------------------------------------------------ */
static inline uint64_t gg_pair_key(uint32_t u, uint32_t v) {
  uint32_t a = u < v ? u : v, b = u < v ? v : u;
  return ((uint64_t)a << 32) | (uint64_t)b;
}

static uint64_t gg_pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

/* ------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m)                                                  */
/* ------------------------------------------------------------------ */
/* Writes m distinct non-loop undirected edges; returns the number of draws
 * used, or -1 on invalid arguments, -2 on allocation failure. */
int64_t gg_er(int32_t n, int64_t m, uint64_t seed, int32_t *src, int32_t *dst) {
  if (n < 0 || m < 0) return -1;
  if (m == 0) return 0;
  if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
  uint64_t cap = gg_pow2_at_least((uint64_t)m * 2 + 16);
  uint64_t *tab = (uint64_t *)calloc(cap, sizeof(uint64_t));
  if (!tab) return -2;
  const uint64_t key = gg_key(seed, GG_S_ER);
  int64_t got = 0, draws = 0;
  while (got < m) {
    uint64_t r = gg_rand(key, (uint64_t)draws++);
    uint32_t u = gg_below((uint32_t)r, (uint32_t)n);
    uint32_t v = gg_below((uint32_t)(r >> 32), (uint32_t)n);
    if (u == v) continue;
    uint64_t k = gg_pair_key(u, v) + 1; /* 0 marks an empty slot */
    uint64_t h = gg_mix(k) & (cap - 1);
    int fresh = 1;
    while (tab[h]) {
      if (tab[h] == k) { fresh = 0; break; }
      h = (h + 1) & (cap - 1);
    }
    if (!fresh) continue;
    tab[h] = k;
    src[got] = (int32_t)u;
    dst[got] = (int32_t)v;
    ++got;
  }
  free(tab);
  return draws;
}

/* ------------------------------------------------------------------ */
/* R-MAT                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  int scale;
  uint64_t key;
  uint64_t ta, tab, tabc; /* cumulative quadrant thresholds over 2^32 */
  const int32_t *perm;    /* NULL: identity */
  int32_t *src, *dst;
} gg_rmat_ctx;

static void gg_rmat_body(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const gg_rmat_ctx *c = (const gg_rmat_ctx *)p;
  const int words = (c->scale + 1) / 2; /* two 32-bit level draws per word */
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int lvl = 0; lvl < c->scale; ++lvl) {
      if ((lvl & 1) == 0) w = gg_rand(c->key, (uint64_t)i * (uint64_t)words + (uint64_t)(lvl >> 1));
      uint64_t r = (lvl & 1) ? (w >> 32) : (w & 0xffffffffULL);
      uint32_t bu, bv;
      if (r < c->ta) { bu = 0; bv = 0; }
      else if (r < c->tab) { bu = 0; bv = 1; }
      else if (r < c->tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    if (c->perm) {
      u = (uint32_t)c->perm[u];
      v = (uint32_t)c->perm[v];
    }
    c->src[i] = (int32_t)u;
    c->dst[i] = (int32_t)v;
  }
}

/* Fisher-Yates permutation of [0, n) driven by one stream. */
static void gg_permutation(int32_t *perm, int64_t n, uint64_t key) {
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = gg_rand(key, (uint64_t)i);
    int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}

static int gg_rmat_setup(gg_rmat_ctx *c, int scale, double a, double b, double cc,
                         uint64_t seed) {
  if (scale < 1 || scale > 30) return -1;
  if (!(a >= 0 && b >= 0 && cc >= 0 && a + b + cc <= 1.0)) return -1;
  c->scale = scale;
  c->key = gg_key(seed, GG_S_RMAT);
  c->ta = (uint64_t)(a * 4294967296.0);
  c->tab = (uint64_t)((a + b) * 4294967296.0);
  c->tabc = (uint64_t)((a + b + cc) * 4294967296.0);
  return 0;
}

/* `draws` raw R-MAT pairs over 2^scale vertices; with permute != 0 the ids
 * go through one seeded random permutation.  Returns 0, or -1 / -2. */
int gg_rmat(int scale, int64_t draws, double a, double b, double c, uint64_t seed,
            int permute, int32_t *src, int32_t *dst) {
  gg_rmat_ctx ctx;
  if (draws < 0 || gg_rmat_setup(&ctx, scale, a, b, c, seed)) return -1;
  int32_t *perm = NULL;
  if (permute) {
    int64_t nv = (int64_t)1 << scale;
    perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!perm) return -2;
    gg_permutation(perm, nv, gg_key(seed, GG_S_RMAT_PERM));
  }
  ctx.perm = perm;
  ctx.src = src;
  ctx.dst = dst;
  gg_parallel(draws, gg_nthreads(), gg_rmat_body, &ctx);
  free(perm);
  return 0;
}

typedef struct {
  const int32_t *src, *dst;
  uint64_t *tkey;   /* pair key + 1, 0 = empty */
  uint32_t *tidx;   /* first draw index of the key */
  uint64_t mask;
  uint8_t *mark;
  int64_t distinct_per_thread[64];
} gg_dedup_ctx;

static void gg_dedup_insert(void *p, int64_t lo, int64_t hi, int tid) {
  gg_dedup_ctx *c = (gg_dedup_ctx *)p;
  int64_t fresh = 0;
  for (int64_t i = lo; i < hi; ++i) {
    uint32_t u = (uint32_t)c->src[i], v = (uint32_t)c->dst[i];
    if (u == v) continue;
    uint64_t k = gg_pair_key(u, v) + 1;
    uint64_t h = gg_mix(k) & c->mask;
    for (;;) {
      uint64_t cur = __atomic_load_n(&c->tkey[h], __ATOMIC_ACQUIRE);
      if (cur == 0) {
        uint64_t expect = 0;
        if (__atomic_compare_exchange_n(&c->tkey[h], &expect, k, 0, __ATOMIC_ACQ_REL,
                                        __ATOMIC_ACQUIRE)) {
          ++fresh;
          break;
        }
        cur = expect;
      }
      if (cur == k) break;
      h = (h + 1) & c->mask;
    }
    /* keep the smallest draw index that produced this key */
    uint32_t old = __atomic_load_n(&c->tidx[h], __ATOMIC_RELAXED);
    while ((uint32_t)i < old &&
           !__atomic_compare_exchange_n(&c->tidx[h], &old, (uint32_t)i, 1, __ATOMIC_RELAXED,
                                        __ATOMIC_RELAXED)) {
    }
  }
  c->distinct_per_thread[tid] = fresh;
}

static void gg_dedup_mark(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  gg_dedup_ctx *c = (gg_dedup_ctx *)p;
  for (int64_t h = lo; h < hi; ++h)
    if (c->tkey[h]) c->mark[c->tidx[h]] = 1;
}

/* R-MAT draws (permuted ids) until m_target distinct non-loop undirected
 * edges have appeared.  src/dst receive those m_target edges, each once, in
 * the order and direction of its first draw.  Returns the number of draws
 * consumed, or -1 (bad arguments) / -2 (allocation failure). */
int64_t gg_rmat_distinct(int scale, int64_t m_target, double a, double b, double c,
                         uint64_t seed, int32_t *src, int32_t *dst) {
  if (m_target < 0) return -1;
  if (m_target == 0) return 0;
  double nv = (double)((int64_t)1 << scale);
  if ((double)m_target > 0.5 * nv * (nv - 1.0)) return -1;
  int64_t cap = m_target + m_target / 8 + 4096;
  for (;;) {
    if (cap >= (int64_t)0xffffffffLL) return -1;
    int32_t *ds = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *dd = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!ds || !dd) { free(ds); free(dd); return -2; }
    int rc = gg_rmat(scale, cap, a, b, c, seed, 1, ds, dd);
    if (rc) { free(ds); free(dd); return rc; }
    gg_dedup_ctx x;
    memset(&x, 0, sizeof(x));
    uint64_t slots = gg_pow2_at_least((uint64_t)cap * 2);
    x.src = ds;
    x.dst = dd;
    x.mask = slots - 1;
    x.tkey = (uint64_t *)calloc(slots, sizeof(uint64_t));
    x.tidx = (uint32_t *)malloc(sizeof(uint32_t) * slots);
    x.mark = (uint8_t *)calloc((size_t)cap, 1);
    if (!x.tkey || !x.tidx || !x.mark) {
      free(ds); free(dd); free(x.tkey); free(x.tidx); free(x.mark);
      return -2;
    }
    memset(x.tidx, 0xff, sizeof(uint32_t) * slots);
    int nt = gg_nthreads();
    gg_parallel(cap, nt, gg_dedup_insert, &x);
    int64_t distinct = 0;
    for (int i = 0; i < 64; ++i) distinct += x.distinct_per_thread[i];
    int64_t used = -1;
    if (distinct >= m_target) {
      gg_parallel((int64_t)slots, nt, gg_dedup_mark, &x);
      int64_t got = 0;
      for (int64_t i = 0; i < cap; ++i) {
        if (!x.mark[i]) continue;
        src[got] = ds[i];
        dst[got] = dd[i];
        if (++got == m_target) { used = i + 1; break; }
      }
    }
    free(ds); free(dd); free(x.tkey); free(x.tidx); free(x.mark);
    if (used >= 0) return used;
    cap += cap / 4;
  }
}

/* One R-MAT graph on n vertices (n need not be a power of two): draws at
 * scale ceil(log2 n), pairs with an id >= n rejected, ids permuted within
 * [0, n), until m distinct non-loop undirected edges, each written once in
 * its first direction.  Single-threaded (batches run many in parallel).
 * Returns the draws used, or -1 (bad arguments), -2 (allocation failure),
 * -4 (no m distinct edges within 256 m + 2^20 draws). */
int64_t gg_rmat_graph(int32_t n, int64_t m, double a, double b, double c, uint64_t seed,
                      int32_t *src, int32_t *dst) {
  if (n < 2 || m < 0) return -1;
  if (m == 0) return 0;
  if ((double)m > 0.5 * (double)n * (double)(n - 1)) return -1;
  int scale = 1;
  while (((int64_t)1 << scale) < n) ++scale;
  gg_rmat_ctx ctx;
  if (gg_rmat_setup(&ctx, scale, a, b, c, seed)) return -1;
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint64_t cap = gg_pow2_at_least((uint64_t)m * 2 + 16);
  uint64_t *tab = (uint64_t *)calloc(cap, sizeof(uint64_t));
  if (!perm || !tab) { free(perm); free(tab); return -2; }
  gg_permutation(perm, n, gg_key(seed, GG_S_RMAT_PERM));
  const int words = (scale + 1) / 2;
  const int64_t limit = 256 * m + (1 << 20);
  int64_t got = 0, draws = 0;
  while (got < m) {
    if (draws >= limit) { free(perm); free(tab); return -4; }
    const int64_t i = draws++;
    uint32_t u = 0, v = 0;
    uint64_t w = 0;
    for (int lvl = 0; lvl < scale; ++lvl) {
      if ((lvl & 1) == 0) w = gg_rand(ctx.key, (uint64_t)i * (uint64_t)words + (uint64_t)(lvl >> 1));
      uint64_t r = (lvl & 1) ? (w >> 32) : (w & 0xffffffffULL);
      uint32_t bu, bv;
      if (r < ctx.ta) { bu = 0; bv = 0; }
      else if (r < ctx.tab) { bu = 0; bv = 1; }
      else if (r < ctx.tabc) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    if (u >= (uint32_t)n || v >= (uint32_t)n || u == v) continue;
    uint64_t k = gg_pair_key(u, v) + 1;
    uint64_t h = gg_mix(k) & (cap - 1);
    int fresh = 1;
    while (tab[h]) {
      if (tab[h] == k) { fresh = 0; break; }
      h = (h + 1) & (cap - 1);
    }
    if (!fresh) continue;
    tab[h] = k;
    src[got] = perm[u];
    dst[got] = perm[v];
    ++got;
  }
  free(perm);
  free(tab);
  return draws;
}

/* ------------------------------------------------------------------ */
/* random geometric graph                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  int32_t g;          /* cells per side; cell side 1/g >= r */
  double r2;
  const double *x, *y;
  const int32_t *cstart; /* g*g+1 offsets into order[] */
  const int32_t *order;  /* point indices grouped by cell */
  int64_t *row_count;    /* edges found per cell row */
  const int64_t *row_base;
  int32_t *pa, *pb;      /* point-index pairs (emit pass) */
  uint64_t key_pts;
} gg_rgg_ctx;

static void gg_rgg_points(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  gg_rgg_ctx *c = (gg_rgg_ctx *)p;
  double *x = (double *)c->x, *y = (double *)c->y;
  for (int64_t i = lo; i < hi; ++i) {
    x[i] = (double)(gg_rand(c->key_pts, 2 * (uint64_t)i) >> 11) * 0x1.0p-53;
    y[i] = (double)(gg_rand(c->key_pts, 2 * (uint64_t)i + 1) >> 11) * 0x1.0p-53;
  }
}

/* Visits every unordered close pair once: a point against later points of
 * its own cell and all points of the cells right, down-left, down and
 * down-right of it.  emit == 0 counts, emit == 1 writes. */
static void gg_rgg_rows(gg_rgg_ctx *c, int64_t lo, int64_t hi, int emit) {
  static const int dxs[4] = {1, -1, 0, 1}, dys[4] = {0, 1, 1, 1};
  const int g = c->g;
  for (int64_t cy = lo; cy < hi; ++cy) {
    int64_t cnt = 0, out = emit ? c->row_base[cy] : 0;
    for (int cx = 0; cx < g; ++cx) {
      int64_t cell = cy * g + cx;
      for (int32_t s = c->cstart[cell]; s < c->cstart[cell + 1]; ++s) {
        int32_t p = c->order[s];
        double px = c->x[p], py = c->y[p];
        for (int32_t t = s + 1; t < c->cstart[cell + 1]; ++t) {
          int32_t q = c->order[t];
          double dx = px - c->x[q], dy = py - c->y[q];
          if (dx * dx + dy * dy < c->r2) {
            if (emit) { c->pa[out] = p; c->pb[out] = q; ++out; }
            ++cnt;
          }
        }
        for (int k = 0; k < 4; ++k) {
          int nx = cx + dxs[k], ny = (int)cy + dys[k];
          if (nx < 0 || nx >= g || ny >= g) continue;
          int64_t nc = (int64_t)ny * g + nx;
          for (int32_t t = c->cstart[nc]; t < c->cstart[nc + 1]; ++t) {
            int32_t q = c->order[t];
            double dx = px - c->x[q], dy = py - c->y[q];
            if (dx * dx + dy * dy < c->r2) {
              if (emit) { c->pa[out] = p; c->pb[out] = q; ++out; }
              ++cnt;
            }
          }
        }
      }
    }
    if (!emit) c->row_count[cy] = cnt;
  }
}

static void gg_rgg_count_body(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  gg_rgg_rows((gg_rgg_ctx *)p, lo, hi, 0);
}

static void gg_rgg_emit_body(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  gg_rgg_rows((gg_rgg_ctx *)p, lo, hi, 1);
}

/* Random geometric graph on n seeded uniform points of [0,1)^2, edge iff
 * distance < r.  Writes at most `cap` edges.  Returns the edge count m, or
 * -1 (bad arguments), -2 (allocation failure), -(3 + m) if cap < m. */
int64_t gg_rgg(int32_t n, double r, uint64_t seed, int32_t *src, int32_t *dst, int64_t cap) {
  if (n < 0 || !(r > 0.0) || r > 1.0) return -1;
  gg_rgg_ctx c;
  memset(&c, 0, sizeof(c));
  c.n = n;
  c.r2 = r * r;
  c.g = (int32_t)(1.0 / r);
  if (c.g < 1) c.g = 1;
  if ((int64_t)c.g * c.g > 1LL << 28) return -1;
  const int64_t cells = (int64_t)c.g * c.g;
  double *x = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  double *y = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  int32_t *cstart = (int32_t *)calloc((size_t)cells + 1, sizeof(int32_t));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  int32_t *cellof = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  int64_t *row_count = (int64_t *)calloc((size_t)c.g, sizeof(int64_t));
  int64_t *row_base = (int64_t *)calloc((size_t)c.g + 1, sizeof(int64_t));
  int64_t ret = 0;
  if (!x || !y || !cstart || !order || !cellof || !row_count || !row_base) { ret = -2; goto done; }
  c.x = x;
  c.y = y;
  c.key_pts = gg_key(seed, GG_S_RGG_POINTS);
  int nt = gg_nthreads();
  gg_parallel(n, nt, gg_rgg_points, &c);
  for (int32_t i = 0; i < n; ++i) {
    int32_t cx = (int32_t)(x[i] * c.g), cy = (int32_t)(y[i] * c.g);
    if (cx >= c.g) cx = c.g - 1;
    if (cy >= c.g) cy = c.g - 1;
    cellof[i] = cy * c.g + cx;
    ++cstart[cellof[i] + 1];
  }
  for (int64_t k = 0; k < cells; ++k) cstart[k + 1] += cstart[k];
  {
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)cells);
    if (!fill) { ret = -2; goto done; }
    memcpy(fill, cstart, sizeof(int32_t) * (size_t)cells);
    for (int32_t i = 0; i < n; ++i) order[fill[cellof[i]]++] = i;
    free(fill);
  }
  c.cstart = cstart;
  c.order = order;
  c.row_count = row_count;
  gg_parallel_min(c.g, nt, gg_rgg_count_body, &c, 64);
  for (int32_t k = 0; k < c.g; ++k) row_base[k + 1] = row_base[k] + row_count[k];
  const int64_t m = row_base[c.g];
  if (m > cap) { ret = -(3 + m); goto done; }
  c.row_base = row_base;
  c.pa = src;
  c.pb = dst;
  gg_parallel_min(c.g, nt, gg_rgg_emit_body, &c, 64);
  {
    /* shuffle ids, pick a random direction per edge, shuffle edge order */
    int32_t *perm = order; /* reuse: point order no longer needed */
    gg_permutation(perm, n, gg_key(seed, GG_S_RGG_PERM));
    const uint64_t kdir = gg_key(seed, GG_S_RGG_DIR);
    for (int64_t e = 0; e < m; ++e) {
      int32_t a = perm[src[e]], b = perm[dst[e]];
      if (gg_rand(kdir, (uint64_t)e) & 1) { int32_t t = a; a = b; b = t; }
      src[e] = a;
      dst[e] = b;
    }
    const uint64_t ksh = gg_key(seed, GG_S_RGG_SHUFFLE);
    for (int64_t i = m - 1; i > 0; --i) {
      uint64_t r = gg_rand(ksh, (uint64_t)i);
      int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(i + 1)) >> 64);
      int32_t ts = src[i], td = dst[i];
      src[i] = src[j]; dst[i] = dst[j];
      src[j] = ts; dst[j] = td;
    }
  }
  ret = m;
done:
  free(x); free(y); free(cstart); free(order); free(cellof); free(row_count); free(row_base);
  return ret;
}

/* The n points gg_rgg(n, ., seed, ...) places, before id shuffling: point i
 * is (x[i], y[i]).  Exposed so a test can check the distance rule. */
void gg_rgg_point_coords(int32_t n, uint64_t seed, double *x, double *y) {
  gg_rgg_ctx c;
  memset(&c, 0, sizeof(c));
  c.x = x;
  c.y = y;
  c.key_pts = gg_key(seed, GG_S_RGG_POINTS);
  gg_parallel(n, gg_nthreads(), gg_rgg_points, &c);
}

/* The id permutation gg_rgg applies: point i gets vertex id perm[i]. */
void gg_rgg_permutation(int32_t n, uint64_t seed, int32_t *perm) {
  gg_permutation(perm, n, gg_key(seed, GG_S_RGG_PERM));
}

/* ------------------------------------------------------------------ */
/* Barabasi-Albert                                                      */
/* ------------------------------------------------------------------ */
/* Preferential attachment (Barabasi & Albert, Science 286, 1999): a clique
 * on k + 1 vertices, then each further vertex v = k+1 .. n-1 joins k
 * distinct earlier vertices, each drawn with probability proportional to its
 * degree at that moment: a uniform draw from the list of all edge endpoints
 * so far, drawn again if it repeats one of v's earlier picks.  The draws are
 * one stream, consumed in order (the process is sequential).  Ids go through
 * one seeded permutation; the pairs are listed in creation order as (new
 * vertex, its pick).  Writes k(k+1)/2 + (n-k-1)k pairs and returns that
 * count, or -1 (bad arguments) / -2 (allocation failure). */
int64_t gg_ba(int32_t n, int32_t k, uint64_t seed, int32_t *src, int32_t *dst) {
  if (k < 1 || n < k + 1) return -1;
  const int64_t m = (int64_t)k * (k + 1) / 2 + (int64_t)(n - k - 1) * k;
  if (2 * m >= ((int64_t)1 << 32)) return -1;
  int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m));
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
  if (!ends || !perm || !pick) {
    free(ends); free(perm); free(pick);
    return -2;
  }
  int64_t e = 0, nends = 0;
  for (int32_t u = 0; u <= k; ++u)
    for (int32_t v = u + 1; v <= k; ++v) {
      src[e] = v;
      dst[e] = u;
      ++e;
      ends[nends++] = u;
      ends[nends++] = v;
    }
  const uint64_t key = gg_key(seed, GG_S_BA);
  uint64_t ctr = 0;
  for (int32_t v = k + 1; v < n; ++v) {
    const uint32_t bound = (uint32_t)nends;  /* endpoints before v's edges */
    int got = 0;
    while (got < k) {
      const uint64_t r = gg_rand(key, ctr++);
      int32_t w = ends[gg_below((uint32_t)r, bound)];
      int fresh = 1;
      for (int i = 0; i < got; ++i)
        if (pick[i] == w) { fresh = 0; break; }
      if (fresh) pick[got++] = w;
      if (got < k) {  /* the high half of the word is a second draw */
        w = ends[gg_below((uint32_t)(r >> 32), bound)];
        fresh = 1;
        for (int i = 0; i < got; ++i)
          if (pick[i] == w) { fresh = 0; break; }
        if (fresh) pick[got++] = w;
      }
    }
    for (int i = 0; i < k; ++i) {
      src[e] = v;
      dst[e] = pick[i];
      ++e;
      ends[nends++] = pick[i];
      ends[nends++] = v;
    }
  }
  gg_permutation(perm, n, gg_key(seed, GG_S_BA_PERM));
  for (int64_t i = 0; i < m; ++i) {
    src[i] = perm[src[i]];
    dst[i] = perm[dst[i]];
  }
  free(ends); free(perm); free(pick);
  return m;
}

/* ------------------------------------------------------------------ */
/* Watts-Strogatz                                                       */
/* ------------------------------------------------------------------ */
/* Small world (Watts & Strogatz, Nature 393, 1998): vertices 0 .. n-1 on a
 * ring, each joined to its k nearest neighbours on either side (n k edges,
 * edge (u, u+j mod n) for j = 1..k has index u k + j - 1).  With probability
 * p (a 32-bit word below p_threshold = p 2^32) an edge's far end moves to a
 * uniform vertex w whose ring distance to u exceeds k (so w is neither u nor
 * one of u's lattice neighbours); up to seven candidates are drawn, and the
 * edge stays if all seven fail.  Every decision and candidate depends only on
 * (seed, edge index), so the loop runs in parallel.  Two moved edges may
 * coincide (about (n k p)^2 / n^2 of them): such repeats stay in the output,
 * as in raw R-MAT draws.  Ids go through one seeded permutation.  Writes
 * n k pairs and returns that count, or -1 / -2. */
typedef struct {
  int32_t n, k;
  uint64_t thr, key;
  const int32_t *perm;
  int32_t *src, *dst;
} gg_ws_ctx;

static void gg_ws_body(void *p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  const gg_ws_ctx *c = (const gg_ws_ctx *)p;
  const uint32_t n = (uint32_t)c->n;
  for (int64_t e = lo; e < hi; ++e) {
    const uint32_t u = (uint32_t)(e / c->k);
    const uint32_t j = (uint32_t)(e % c->k) + 1;
    uint32_t v = (u + j) % n;
    const uint64_t base = (uint64_t)e * 8;
    if ((gg_rand(c->key, base) & 0xffffffffULL) < c->thr) {
      for (uint64_t a = 1; a < 8; ++a) {
        const uint32_t w = gg_below((uint32_t)(gg_rand(c->key, base + a) >> 32), n);
        const uint32_t d = w >= u ? w - u : w + n - u;
        const uint32_t ring = d < n - d ? d : n - d;
        if (ring > (uint32_t)c->k) {
          v = w;
          break;
        }
      }
    }
    c->src[e] = c->perm[u];
    c->dst[e] = c->perm[v];
  }
}

int64_t gg_ws(int32_t n, int32_t k, double p, uint64_t seed, int32_t *src, int32_t *dst) {
  if (k < 1 || n < 2 * k + 2 || !(p >= 0.0 && p <= 1.0)) return -1;
  const int64_t m = (int64_t)n * k;
  if (m > (int64_t)0x7fffffff) return -1;
  int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!perm) return -2;
  gg_permutation(perm, n, gg_key(seed, GG_S_WS_PERM));
  gg_ws_ctx c;
  c.n = n;
  c.k = k;
  c.thr = (uint64_t)(p * 4294967296.0);
  c.key = gg_key(seed, GG_S_WS);
  c.perm = perm;
  c.src = src;
  c.dst = dst;
  gg_parallel(m, gg_nthreads(), gg_ws_body, &c);
  free(perm);
  return m;
}
