/*
 * forward.c -- CPU oracle for exact triangle counting.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check in __graft_entry__ and the CPU-baseline / reference legs of bench.py
 * may load or call this file.  The GPU library never calls it and shares no
 * code with it (no headers, helpers or tables in common).
 *
 * Plain, slow, single-threaded and written to be checked by eye against
 * Polak, "Counting Triangles in Large Graphs on GPU" (arXiv 1503.00576):
 *
 *   oracle_forward          the sequential forward algorithm of Sec. II-B
 *                           (Schank & Wagner; Latapy), step by step:
 *                             1. an order on vertices consistent with degree,
 *                             2. keep, for each vertex, only neighbours that
 *                                come after it in that order,
 *                             3. sort every kept list by vertex id,
 *                             4. for every kept (directed) edge (u, v) add the
 *                                size of N+(u) intersect N+(v), computed by a
 *                                two-pointer merge.
 *                           Each triangle is found exactly once, from its
 *                           order-smallest vertex u and middle vertex v.
 *   oracle_vertex_triangles t(v) straight from the definition: the number of
 *                           edges of the graph whose both ends are neighbours
 *                           of v (no ordering, no orientation).  Used for
 *                           sampled checks on graphs too large for a full run.
 *
 * Input conventions (the readings taken where the paper is silent):
 *   - Sec. III-A assumes a clean edge array (no self-loops, no multi-edges,
 *     each edge twice).  This oracle accepts any list of pairs, treats every
 *     pair as undirected, drops self-loops and collapses repeats, so a clean
 *     input gives exactly the paper's result.
 *   - Degrees are those of the cleaned simple graph.
 *   - Ties in degree are broken by vertex id, lower id first (the
 *     preprocessing of Sec. III-B that marks backward edges only says to
 *     compare identifiers on a tie); tie_high_first = 1 flips the tie-break,
 *     which must not change any count.
 *   - Every id must satisfy 0 <= id < n (n is an argument, not max id + 1).
 *
 * Status codes: 0 ok, 1 invalid argument, 2 id out of range, 3 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_INVALID = 1, OR_RANGE = 2, OR_NOMEM = 3 };

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return (x > y) - (x < y);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* The cleaned simple graph: sorted, distinct pairs (a, b) with a < b,
 * packed as a * 2^32 + b.  Returns the status; *edges is malloc'ed. */
static int clean_edges(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                       uint64_t **edges, int64_t *m_out) {
  *edges = NULL;
  *m_out = 0;
  for (int64_t i = 0; i < m_in; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return OR_RANGE;
  uint64_t *e = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m_in > 0 ? m_in : 1));
  if (!e) return OR_NOMEM;
  int64_t k = 0;
  for (int64_t i = 0; i < m_in; ++i) {
    int32_t a = src[i], b = dst[i];
    if (a == b) continue; /* self-loop */
    if (a > b) { int32_t t = a; a = b; b = t; }
    e[k++] = ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
  }
  qsort(e, (size_t)k, sizeof(uint64_t), cmp_u64);
  int64_t m = 0;
  for (int64_t i = 0; i < k; ++i)
    if (m == 0 || e[i] != e[m - 1]) e[m++] = e[i];
  *edges = e;
  *m_out = m;
  return OR_OK;
}

/* u comes before v in the degree order of Sec. II-B. */
static int precedes(int32_t u, int32_t v, const int32_t *deg, int tie_high_first) {
  if (deg[u] != deg[v]) return deg[u] < deg[v];
  return tie_high_first ? (u > v) : (u < v);
}

/*
 * Forward algorithm.  Outputs (each optional except total):
 *   total            number of triangles T
 *   t[n]             triangles containing each vertex
 *   deg[n]           degree in the cleaned graph
 *   m_out            number of distinct undirected edges m
 *   max_out_deg      the longest forward list, max_v |N+(v)|
 */
int oracle_forward(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                   int tie_high_first, uint64_t *total, int64_t *t, int32_t *deg,
                   int64_t *m_out, int64_t *max_out_deg) {
  if (m_in < 0 || n < 0 || !total) return OR_INVALID;
  uint64_t *e = NULL;
  int64_t m = 0;
  int rc = clean_edges(src, dst, m_in, n, &e, &m);
  if (rc) return rc;

  /* degrees of the simple graph */
  int32_t *d = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!d || !off || !nbr) { free(e); free(d); free(off); free(nbr); return OR_NOMEM; }
  for (int64_t i = 0; i < m; ++i) {
    ++d[(int32_t)(e[i] >> 32)];
    ++d[(int32_t)(e[i] & 0xffffffffu)];
  }

  /* orient each edge from its order-smaller end: N+(u) keeps v iff u < v in
   * the order; lay the lists out one after another */
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = (int32_t)(e[i] >> 32), b = (int32_t)(e[i] & 0xffffffffu);
    int32_t u = precedes(a, b, d, tie_high_first) ? a : b;
    ++off[u + 1];
  }
  for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) { free(e); free(d); free(off); free(nbr); return OR_NOMEM; }
  for (int32_t v = 0; v < n; ++v) fill[v] = off[v];
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = (int32_t)(e[i] >> 32), b = (int32_t)(e[i] & 0xffffffffu);
    if (precedes(a, b, d, tie_high_first)) nbr[fill[a]++] = b;
    else nbr[fill[b]++] = a;
  }
  free(fill);
  free(e);

  /* sort every forward list by vertex id */
  int64_t longest = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t len = off[v + 1] - off[v];
    if (len > longest) longest = len;
    qsort(nbr + off[v], (size_t)len, sizeof(int32_t), cmp_i32);
  }

  if (t) memset(t, 0, sizeof(int64_t) * (size_t)n);

  /* every forward edge (u, v) adds |N+(u) & N+(v)|, by a two-pointer merge */
  uint64_t T = 0;
  for (int32_t u = 0; u < n; ++u) {
    for (int64_t k = off[u]; k < off[u + 1]; ++k) {
      int32_t v = nbr[k];
      int64_t i = off[u], iend = off[u + 1];
      int64_t j = off[v], jend = off[v + 1];
      while (i < iend && j < jend) {
        if (nbr[i] < nbr[j]) {
          ++i;
        } else if (nbr[i] > nbr[j]) {
          ++j;
        } else {
          int32_t w = nbr[i];
          ++T;
          if (t) { ++t[u]; ++t[v]; ++t[w]; }
          ++i;
          ++j;
        }
      }
    }
  }

  *total = T;
  if (deg) memcpy(deg, d, sizeof(int32_t) * (size_t)n);
  if (m_out) *m_out = m;
  if (max_out_deg) *max_out_deg = longest;
  free(d);
  free(off);
  free(nbr);
  return OR_OK;
}

/* Forward lists only (steps 1-3 of the algorithm), for invariant checks:
 * out_deg[v] = |N+(v)|.  Same conventions as oracle_forward. */
int oracle_out_degrees(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                       int tie_high_first, int32_t *out_deg) {
  if (m_in < 0 || n < 0 || !out_deg) return OR_INVALID;
  uint64_t *e = NULL;
  int64_t m = 0;
  int rc = clean_edges(src, dst, m_in, n, &e, &m);
  if (rc) return rc;
  int32_t *d = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
  if (!d) { free(e); return OR_NOMEM; }
  for (int64_t i = 0; i < m; ++i) {
    ++d[(int32_t)(e[i] >> 32)];
    ++d[(int32_t)(e[i] & 0xffffffffu)];
  }
  memset(out_deg, 0, sizeof(int32_t) * (size_t)n);
  for (int64_t i = 0; i < m; ++i) {
    int32_t a = (int32_t)(e[i] >> 32), b = (int32_t)(e[i] & 0xffffffffu);
    ++out_deg[precedes(a, b, d, tie_high_first) ? a : b];
  }
  free(d);
  free(e);
  return OR_OK;
}

/*
 * t(v) for the k vertices vs[0..k) by the definition: the number of distinct
 * edges {a, b} (a != b) with both a and b adjacent to v.  Two passes over the
 * raw pair list; repeated pairs and self-loops are handled by working on the
 * set of distinct canonical pairs found.
 */
int oracle_vertex_triangles(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                            const int32_t *vs, int64_t k, int64_t *out) {
  if (m_in < 0 || n < 0 || k < 0 || (k > 0 && (!vs || !out))) return OR_INVALID;
  for (int64_t i = 0; i < m_in; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return OR_RANGE;
  for (int64_t s = 0; s < k; ++s)
    if (vs[s] < 0 || vs[s] >= n) return OR_RANGE;
  if (k == 0) return OR_OK;

  /* which sampled vertices each vertex is a neighbour of: a linked list of
   * (sample index) entries per vertex, built from the distinct neighbour
   * sets N(vs[s]) */
  int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!head) return OR_NOMEM;
  for (int32_t v = 0; v < n; ++v) head[v] = -1;
  int64_t cap = 1024, used = 0;
  int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  int64_t *who = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
  int32_t *nb = NULL;
  uint64_t *rec = NULL;
  int rc = OR_OK;
  if (!next || !who) { rc = OR_NOMEM; goto out; }
  for (int64_t s = 0; s < k; ++s) {
    int32_t v = vs[s];
    int64_t cnt = 0;
    for (int64_t i = 0; i < m_in; ++i)
      if ((src[i] == v) != (dst[i] == v)) ++cnt;
    free(nb);
    nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!nb) { rc = OR_NOMEM; goto out; }
    cnt = 0;
    for (int64_t i = 0; i < m_in; ++i) {
      if (src[i] == v && dst[i] != v) nb[cnt++] = dst[i];
      else if (dst[i] == v && src[i] != v) nb[cnt++] = src[i];
    }
    qsort(nb, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < cnt; ++i) {
      if (i > 0 && nb[i] == nb[i - 1]) continue;
      if (used == cap) {
        cap *= 2;
        int64_t *n2 = (int64_t *)realloc(next, sizeof(int64_t) * (size_t)cap);
        if (!n2) { rc = OR_NOMEM; goto out; }
        next = n2;
        int64_t *w2 = (int64_t *)realloc(who, sizeof(int64_t) * (size_t)cap);
        if (!w2) { rc = OR_NOMEM; goto out; }
        who = w2;
      }
      who[used] = s;
      next[used] = head[nb[i]];
      head[nb[i]] = used;
      ++used;
    }
  }

  /* every pair whose two ends are both neighbours of sample s is a
   * candidate edge of s's neighbourhood; record (s, canonical pair) */
  int64_t rcap = 1024, nrec = 0;
  rec = (uint64_t *)malloc(sizeof(uint64_t) * 2 * (size_t)rcap);
  if (!rec) { rc = OR_NOMEM; goto out; }
  for (int64_t i = 0; i < m_in; ++i) {
    int32_t a = src[i], b = dst[i];
    if (a == b || head[a] < 0 || head[b] < 0) continue;
    if (a > b) { int32_t t = a; a = b; b = t; }
    for (int64_t p = head[a]; p >= 0; p = next[p]) {
      for (int64_t q = head[b]; q >= 0; q = next[q]) {
        if (who[p] != who[q]) continue;
        if (nrec == rcap) {
          rcap *= 2;
          uint64_t *r2 = (uint64_t *)realloc(rec, sizeof(uint64_t) * 2 * (size_t)rcap);
          if (!r2) { rc = OR_NOMEM; goto out; }
          rec = r2;
        }
        rec[2 * nrec] = (uint64_t)who[p];
        rec[2 * nrec + 1] = ((uint64_t)(uint32_t)a << 32) | (uint64_t)(uint32_t)b;
        ++nrec;
      }
    }
  }
  /* count the distinct pairs recorded for each sample */
  for (int64_t s = 0; s < k; ++s) out[s] = 0;
  if (nrec > 0) {
    /* sort the pair keys of each sample separately: gather, sort, count */
    uint64_t *buf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nrec);
    if (!buf) { rc = OR_NOMEM; goto out; }
    for (int64_t s = 0; s < k; ++s) {
      int64_t c = 0;
      for (int64_t r = 0; r < nrec; ++r)
        if ((int64_t)rec[2 * r] == s) buf[c++] = rec[2 * r + 1];
      qsort(buf, (size_t)c, sizeof(uint64_t), cmp_u64);
      int64_t distinct = 0;
      for (int64_t r = 0; r < c; ++r)
        if (r == 0 || buf[r] != buf[r - 1]) ++distinct;
      out[s] = distinct;
    }
    free(buf);
  }
out:
  free(head);
  free(next);
  free(who);
  free(nb);
  free(rec);
  return rc;
}
