// group.cu -- partner groups for the counting phase.
//
// The counting phase adds |N+(u) & N+(v)| over every forward edge (u, v)
// (Sec. II-B).  The intersection is symmetric in u and v, and the counting
// kernel computes it by hashing one list and streaming the other through
// the hash set, which costs one probe per element of the streamed list.
// Streaming the shorter list is cheapest, so every forward edge is assigned
// to the endpoint whose forward list is longer:
//
//   h = v if |N+(v)| > |N+(u)| else u,     l = the other endpoint,
//
// and the edges are grouped by h: k_group_keys writes the key h << b | l of
// every edge, and a stable LSD radix sort over the h bits (the passes of
// preprocess.cu) leaves the partners l of each group together, its last
// pass counting the group sizes.  A group then hashes N+(h) once and
// streams N+(l) for each of its partners l.  On the R-MAT graphs of the
// benchmarks this cuts the probes by a factor of 2.7 against always
// streaming N+(v).
//
// The lists themselves are sorted here (Sec. II-B sorts every forward list;
// the paper merges them, this path hashes, and uses the order only to skip
// the leading blocks of a streamed list that lie below the hashed list's
// smallest id -- a third of all blocks on R-MAT scale 24).
#include <climits>

#include "tc_common.cuh"

namespace tc {
namespace {

constexpr int kGroupThreads = 256;
constexpr int kGroupUnroll = 4;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// sorted forward lists
// ---------------------------------------------------------------------------
constexpr int kListThreads = 256;
constexpr int kListWarps = kListThreads / 32;
constexpr int kLongListThreads = 512;
constexpr int kLongListBlocks = 4;  // CTAs per SM: a CTA mostly waits at its barriers

__device__ __forceinline__ void cswap(int32_t &a, int32_t &b) {
  const int32_t x = min(a, b);
  b = max(a, b);
  a = x;
}

// Batcher's odd-even merge sort network for 8 keys (19 comparators).
__device__ __forceinline__ void sort8(int32_t (&x)[8]) {
  cswap(x[0], x[1]); cswap(x[2], x[3]); cswap(x[4], x[5]); cswap(x[6], x[7]);
  cswap(x[0], x[2]); cswap(x[1], x[3]); cswap(x[4], x[6]); cswap(x[5], x[7]);
  cswap(x[1], x[2]); cswap(x[5], x[6]);
  cswap(x[0], x[4]); cswap(x[1], x[5]); cswap(x[2], x[6]); cswap(x[3], x[7]);
  cswap(x[2], x[4]); cswap(x[3], x[5]);
  cswap(x[1], x[2]); cswap(x[3], x[4]); cswap(x[5], x[6]);
}

// Bitonic sort of 32 E keys held E per lane, key e*32 + lane in x[e] of
// lane `lane` (a warp-striped layout: loads and stores stay coalesced),
// ascending.  Exchanges between keys 32 or more apart stay in a lane;
// closer ones are shuffles.
template <int E>
__device__ __forceinline__ void warp_sort_regs(int32_t (&x)[E]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int je = j >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if ((e & je) == 0) {
            const bool up = ((e * 32) & k) == 0;
            const int32_t a = x[e], b = x[e | je];
            x[e] = up ? min(a, b) : max(a, b);
            x[e | je] = up ? max(a, b) : min(a, b);
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int32_t y = __shfl_xor_sync(kFull, x[e], j);
          const bool up = ((e * 32 + lane) & k) == 0, low = (lane & j) == 0;
          x[e] = low == up ? min(x[e], y) : max(x[e], y);
        }
      }
    }
  }
}

// Where the list sort leaves its results (see launch_sort_lists).
struct ListOut {
  int32_t *col4;   // sorted lists, padded with -1 to whole 32-byte blocks
  int32_t *dlen;   // length of a list that held repeats, after dropping them
  int32_t *dcorr;  // per rank: repeated edges dropped at that vertex
  Ctrl *ctrl;
};

// A repeat of edge (u, x) in the sorted list of u is dropped: it had added
// one to the degree of both ends.
__device__ __forceinline__ void drop_repeat(int32_t u, int32_t x, const ListOut &o) {
  atomicAdd(&o.dcorr[u], 1);
  atomicAdd(&o.dcorr[x], 1);
  *(volatile uint32_t *)&o.ctrl->dups = 1u;
}

// Key e*32 + lane of a warp-striped sorted list repeats the key before it.
template <int E>
__device__ __forceinline__ bool warp_repeat(const int32_t (&x)[E], int e, int32_t d) {
  const int lane = threadIdx.x & 31;
  int32_t p = __shfl_up_sync(kFull, x[e], 1);
  const int32_t q = __shfl_sync(kFull, x[e > 0 ? e - 1 : 0], 31);
  if (lane == 0) p = q;
  const int i = e * 32 + lane;
  return i > 0 && i < d && x[e] == p;
}

// The warp sorts list v (d entries from col + b) into col4 from entry w4,
// with E keys per lane (32 E >= d), dropping repeated entries.
template <int E>
__device__ __forceinline__ void warp_sort_list(const int32_t *__restrict__ col, int32_t b,
                                               int32_t d, long long w4, int32_t v,
                                               const ListOut &o) {
  const int lane = threadIdx.x & 31;
  int32_t x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    x[e] = i < d ? __ldg(col + b + i) : INT32_MAX;
  }
  warp_sort_regs<E>(x);
  const int r8 = (d + 7) & ~7;
  uint32_t reps = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) reps |= __ballot_sync(kFull, warp_repeat<E>(x, e, d));
  if (reps == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = e * 32 + lane;
      if (i < r8) o.col4[w4 + i] = i < d ? x[e] : -1;
    }
    return;
  }
  // some entry repeats (an edge given more than once): compact the rest
  const uint32_t lt = (1u << lane) - 1u;
  int len = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    const bool rep = warp_repeat<E>(x, e, d);
    const bool keep = i < d && !rep;
    const uint32_t bk = __ballot_sync(kFull, keep);
    if (keep) o.col4[w4 + len + __popc(bk & lt)] = x[e];
    if (rep) drop_repeat(v, x[e], o);
    len += __popc(bk);
  }
  for (int i = len + lane; i < r8; i += 32) o.col4[w4 + i] = -1;
  if (lane == 0) o.dlen[v] = len;
}

// Bitonic sort of buf[0..P) (P a power of two) by a whole block of G
// threads, ascending.
template <int G>
__device__ __forceinline__ void bitonic_smem(int32_t *buf, int P, int rank) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = rank; i < P / 2; i += G) {
        const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1)), hi = lo + j;
        const int32_t a = buf[lo], b = buf[hi];
        if ((a > b) == ((lo & k) == 0)) {
          buf[lo] = b;
          buf[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Exclusive scan of one value per thread over a block of G threads; *total
// gets the sum.  All threads must call it; s_warp holds G / 32 words.
template <int G>
__device__ __forceinline__ uint32_t block_scan(uint32_t x, uint32_t *s_warp, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < G / 32; ++w) {
    const uint32_t t = s_warp[w];
    if (w < warp) before += t;
    all += t;
  }
  __syncthreads();  // s_warp is reused by the next call
  *total = all;
  return before + incl - x;
}

// Copies the sorted list buf[0..d) of vertex v to dst without its repeated
// entries, padded with -1 up to r8 entries, by a block of G threads (buf in
// shared or global memory, written before the last barrier).
template <int G>
__device__ void cta_unique_copy(const int32_t *buf, int32_t d, int32_t *__restrict__ dst,
                                int32_t r8, int32_t v, const ListOut &o, uint32_t *s_warp,
                                int32_t *s_len) {
  constexpr int PER = 16;  // consecutive entries per thread
  const int tid = threadIdx.x;
  int32_t len = 0;  // uniform: entries written so far
  for (int32_t t0 = 0; t0 < d; t0 += G * PER) {
    const int32_t j0 = t0 + tid * PER;
    uint32_t keep = 0, cnt = 0;
    int32_t prev = (j0 > 0 && j0 < d) ? buf[j0 - 1] : 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int32_t j = j0 + q;
      if (j < d) {
        const int32_t x = buf[j];
        const bool k = j == 0 || x != prev;
        if (!k) drop_repeat(v, x, o);
        prev = x;
        keep |= (uint32_t)k << q;
        cnt += k;
      }
    }
    uint32_t total;
    uint32_t pos = (uint32_t)len + block_scan<G>(cnt, s_warp, &total);
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if ((keep >> q) & 1u) dst[pos++] = buf[j0 + q];
    len += (int32_t)total;
  }
  for (int32_t j = len + tid; j < r8; j += G) dst[j] = -1;
  if (tid == 0) {
    if (len < d) o.dlen[v] = len;
    *s_len = len;
  }
}

// Every forward list into col4, sorted ascending, without repeated entries
// and padded with -1 to whole 32-byte blocks.  Warps take 32 consecutive
// vertices at a time: a list of up to 8 entries is sorted by its own lane in
// registers (a sorting network), one of up to kWarpSortMax entries by the
// warp in registers (bitonic, up to 16 keys per lane); longer lists go to
// k_sort_long_lists_warp and k_sort_long_lists.
__global__ void __launch_bounds__(kListThreads)
k_sort_lists(const int32_t *__restrict__ col, const int32_t *__restrict__ off,
             const int32_t *__restrict__ voff, int32_t n, ListOut o,
             int32_t *__restrict__ long_lists) {
  Ctrl *ctrl = o.ctrl;
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t warps = gridDim.x * kListWarps;
  for (uint32_t c = blockIdx.x * kListWarps + warp; c * 32u < (uint32_t)n; c += warps) {
    const uint32_t v = c * 32u + lane;
    int32_t b = 0, d = 0;
    long long w4 = 0;  // first col4 entry of the list
    if (v < (uint32_t)n) {
      b = __ldg(off + v);
      d = __ldg(off + v + 1) - b;
      w4 = 4ll * __ldg(voff + v);
    }
    if (d > 0 && d <= 8) {
      int32_t x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = i < d ? __ldg(col + b + i) : INT32_MAX;
      sort8(x);
      uint32_t reps = 0;  // bit i: entry i repeats entry i - 1
#pragma unroll
      for (int i = 1; i < 8; ++i) reps |= (uint32_t)(i < d && x[i] == x[i - 1]) << i;
      if (reps == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (i >= d) x[i] = -1;
        int4 *dst = reinterpret_cast<int4 *>(o.col4 + w4);
        dst[0] = make_int4(x[0], x[1], x[2], x[3]);
        dst[1] = make_int4(x[4], x[5], x[6], x[7]);
      } else {  // an edge given more than once
        int len = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i < d && ((reps >> i) & 1u)) drop_repeat((int32_t)v, x[i], o);
          else if (i < d) o.col4[w4 + len++] = x[i];
        }
        for (int i = len; i < 8; ++i) o.col4[w4 + i] = -1;
        o.dlen[v] = len;
      }
    }
    uint32_t todo = __ballot_sync(kFull, d > 8 && d <= kWarpSortMax);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int32_t lb = __shfl_sync(kFull, b, src), ld = __shfl_sync(kFull, d, src);
      const long long lw = __shfl_sync(kFull, w4, src);
      const int32_t lv = (int32_t)(c * 32u) + src;
      if (ld <= 32) warp_sort_list<1>(col, lb, ld, lw, lv, o);
      else if (ld <= 64) warp_sort_list<2>(col, lb, ld, lw, lv, o);
      else if (ld <= 128) warp_sort_list<4>(col, lb, ld, lw, lv, o);
      else if (ld <= 256) warp_sort_list<8>(col, lb, ld, lw, lv, o);
      else warp_sort_list<16>(col, lb, ld, lw, lv, o);
    }
    const bool is_long = d > kWarpSortMax;
    const uint32_t bl = __ballot_sync(kFull, is_long);
    if (bl) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&ctrl->n_long_lists, (uint32_t)__popc(bl));
      base = __shfl_sync(kFull, base, 0);
      if (is_long) long_lists[base + __popc(bl & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

// Lists of kWarpSortMax + 1 to 2 kWarpSortMax entries: one warp each, 32
// keys per lane in registers.
constexpr int kWarpLongMax = 2 * kWarpSortMax;

__global__ void __launch_bounds__(kListThreads)
k_sort_long_lists_warp(const int32_t *__restrict__ col, const int32_t *__restrict__ off,
                       const int32_t *__restrict__ voff, ListOut o,
                       const int32_t *__restrict__ long_lists) {
  Ctrl *ctrl = o.ctrl;
  if (aborted(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t count = ctrl->n_long_lists;
  for (;;) {
    uint32_t i = 0;
    if (lane == 0) i = atomicAdd(&ctrl->next_long_list_warp, 1u);
    i = __shfl_sync(kFull, i, 0);
    if (i >= count) break;
    const int32_t v = __ldg(long_lists + i);
    const int32_t b = __ldg(off + v), d = __ldg(off + v + 1) - b;
    if (d > kWarpLongMax) continue;  // the CTA kernel's
    warp_sort_list<kWarpLongMax / 32>(col, b, d, 4ll * __ldg(voff + v), v, o);
  }
}

// Number of entries of the sorted a[0..len) below x (lower) or not above x
// (upper); plain loads (a may have been written by this kernel).
__device__ __forceinline__ int32_t count_below(const int32_t *a, int32_t len, int32_t x,
                                               bool or_equal) {
  int32_t lo = 0, hi = len;
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t y = a[mid];
    if (y < x || (or_equal && y == x)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Lists longer than kWarpLongMax: one CTA each.  Up to kCtaSortMax entries
// the list is sorted in shared memory; a longer one (only with a dense core
// of more than kCtaSortMax vertices) is sorted in chunks of kCtaSortMax,
// which are then merged pairwise in global memory, alternating between the
// list's own region of the column array and its region of col4 so that the
// last merge lands in the column array.  Then the repeats are dropped on
// the way into col4.
__global__ void __launch_bounds__(kLongListThreads, kLongListBlocks)
k_sort_long_lists(int32_t *col, const int32_t *__restrict__ off,
                  const int32_t *__restrict__ voff, ListOut o,
                  const int32_t *__restrict__ long_lists) {
  constexpr int G = kLongListThreads;
  __shared__ int32_t s_buf[kCtaSortMax];
  __shared__ uint32_t s_warp[G / 32];
  __shared__ uint32_t s_i;
  __shared__ int32_t s_len;
  Ctrl *ctrl = o.ctrl;
  if (aborted(ctrl)) return;
  const int tid = threadIdx.x;
  const uint32_t count = ctrl->n_long_lists;
  for (;;) {
    if (tid == 0) s_i = atomicAdd(&ctrl->next_long_list, 1u);
    __syncthreads();
    const uint32_t i = s_i;
    if (i >= count) break;
    const int32_t v = __ldg(long_lists + i);
    const int32_t b = __ldg(off + v), d = __ldg(off + v + 1) - b;
    if (d > kWarpLongMax) {  // shorter lists are the warp kernel's (uniform for the block)
      int32_t *dst = o.col4 + 4ll * __ldg(voff + v);
      const int r8 = (d + 7) & ~7;
      if (d <= kCtaSortMax) {
        const int P = pow2_at_least(d);
        for (int j = tid; j < P; j += G) s_buf[j] = j < d ? col[b + j] : INT32_MAX;
        __syncthreads();
        bitonic_smem<G>(s_buf, P, tid);
        cta_unique_copy<G>(s_buf, d, dst, r8, v, o, s_warp, &s_len);
      } else {
        int32_t *A = col + b;  // the list's region of the column array: d entries
        int32_t *B = dst;      // its region of col4: r8 >= d entries
        const int32_t chunks = (d + kCtaSortMax - 1) / kCtaSortMax;
        int levels = 0;
        while ((1 << levels) < chunks) ++levels;
        int32_t *src = (levels & 1) ? B : A;
        for (int32_t c0 = 0; c0 < d; c0 += kCtaSortMax) {
          const int32_t len = min(kCtaSortMax, d - c0);
          for (int j = tid; j < kCtaSortMax; j += G) s_buf[j] = j < len ? A[c0 + j] : INT32_MAX;
          __syncthreads();
          bitonic_smem<G>(s_buf, kCtaSortMax, tid);
          for (int j = tid; j < len; j += G) src[c0 + j] = s_buf[j];
          __syncthreads();
        }
        int32_t *to = src == A ? B : A;
        for (int32_t w = kCtaSortMax; w < d; w <<= 1) {
          // runs [s0, s0 + w) and [s0 + w, s0 + 2w) merged into to[s0 ..):
          // an entry's place is its place in its run plus the entries of the
          // other run before it (ties: the first run's entries first)
          for (int32_t j = tid; j < d; j += G) {
            const int32_t s0 = j / (2 * w) * (2 * w);
            const int32_t am = min(s0 + w, d), be = min(s0 + 2 * w, d);
            const int32_t x = src[j];
            const int32_t at = j < am ? (j - s0) + count_below(src + am, be - am, x, false)
                                      : (j - am) + count_below(src + s0, am - s0, x, true);
            to[s0 + at] = x;
          }
          __syncthreads();
          int32_t *t = src;
          src = to;
          to = t;
        }
        cta_unique_copy<G>(A, d, B, r8, v, o, s_warp, &s_len);
      }
    }
    __syncthreads();  // s_buf and s_i are reused
  }
}

// The row array again after repeats were dropped: row[off[v] + i] = v (off:
// the recounted node array).  One warp per vertex; only when some list held
// a repeat.
__global__ void __launch_bounds__(kListThreads)
k_fix_rows(const int32_t *__restrict__ off, int32_t n, const Ctrl *ctrl,
           int32_t *__restrict__ row) {
  if (aborted(ctrl) || *(volatile const uint32_t *)&ctrl->dups == 0u) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * kListWarps;
  for (uint32_t v = (blockIdx.x * kListThreads + threadIdx.x) >> 5; v < (uint32_t)n; v += warps) {
    const int32_t b = __ldg(off + v), e = __ldg(off + v + 1);
    for (int32_t i = b + lane; i < e; i += 32) row[i] = (int32_t)v;
  }
}

// The degrees without repeats: deg[v] -= dcorr[rank[v]] (caller ids); only
// when some list held a repeat.
__global__ void __launch_bounds__(kListThreads)
k_fix_degree(const int32_t *__restrict__ dcorr, const int32_t *__restrict__ rank, int32_t n,
             const Ctrl *ctrl, int32_t *__restrict__ deg) {
  if (aborted(ctrl) || *(volatile const uint32_t *)&ctrl->dups == 0u) return;
  const uint32_t stride = gridDim.x * kListThreads;
  for (uint32_t v = blockIdx.x * kListThreads + threadIdx.x; v < (uint32_t)n; v += stride)
    deg[v] -= __ldg(dcorr + __ldg(rank + v));
}

// heavy_ratio_pct = 100: the longer list is always the one hashed; larger
// values keep an edge at its owner unless v's list is that much longer.
__device__ __forceinline__ void split_edge(int32_t u, int32_t v, int64_t du, int64_t dv,
                                           int32_t heavy_ratio_pct, int32_t &h, int32_t &l) {
  if (dv * 100 > du * heavy_ratio_pct) {
    h = v;
    l = u;
  } else {
    h = u;
    l = v;
  }
}

// One pass over the forward edges in owner order (row[e] = u; the sorted
// list N+(u) of col4 holds v at position i = e - off[u]; row and off are
// those left after the list sort dropped repeated edges): the group key of
// every edge with the digit histograms of its h field.  When the longer
// list is v's (h = v), the intersection streams N+(u), whose entries before
// position i are all below v; N+(h) holds only ids above h = v, so those
// entries cannot match and the whole blocks among them, i >> 3, are
// skipped.  Their count rides in the key's top bits to the partner array.
// (When h = u, N+(v) is streamed and all its entries lie above v, itself
// in N+(u): nothing to skip.)
__global__ void __launch_bounds__(kGroupThreads)
k_group_keys(const int32_t *__restrict__ row, const int32_t *__restrict__ col4,
             const int32_t *__restrict__ off, const int2 *__restrict__ ldesc,
             int b, int passes, int32_t heavy_ratio_pct,
             const Ctrl *__restrict__ ctrl, uint64_t *__restrict__ gkeys,
             uint32_t *__restrict__ hist) {
  __shared__ uint32_t s_hist[kMaxGroupPasses * 256];
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out
  for (int i = threadIdx.x; i < passes * 256; i += kGroupThreads) s_hist[i] = 0;
  __syncthreads();
  const uint32_t m = ctrl->m;
  const bool carry_skip = 2 * b <= kSkipShift;
  const bool hub_on = carry_skip && ctrl->hub_on != 0u;
  const int32_t hub_lo = (int32_t)ctrl->hub_lo;
  const uint32_t stride = gridDim.x * kGroupThreads;
  // kGroupUnroll edges per thread per round, each step's loads issued for
  // all of them together: the offsets are gathers that depend on the edge
  for (uint32_t e0 = blockIdx.x * kGroupThreads + threadIdx.x; e0 < m;
       e0 += kGroupUnroll * stride) {
    int32_t u[kGroupUnroll], ub[kGroupUnroll], ue[kGroupUnroll], uw[kGroupUnroll];
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      u[q] = e < m ? __ldg(row + e) : 0;
    }
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      ub[q] = __ldg(off + u[q]);
      const int2 ld = __ldg(ldesc + u[q]);  // {first col4 word, length}
      ue[q] = ub[q] + ld.y;
      uw[q] = ld.x;
    }
    int32_t v[kGroupUnroll], vd[kGroupUnroll];
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      v[q] = e < m ? __ldg(col4 + 4ll * uw[q] + ((int32_t)e - ub[q])) : 0;
    }
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) vd[q] = __ldg(ldesc + v[q]).y;
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      if (e >= m) break;
      int32_t h, l;
      split_edge(u[q], v[q], ue[q] - ub[q], vd[q], heavy_ratio_pct, h, l);
      // an edge inside the dense hub block (owner u, hence v, of rank >=
      // hub_lo) is left to it: its stream is skipped whole
      uint64_t skip = (carry_skip && h == v[q]) ? (uint64_t)(((int32_t)e - ub[q]) >> 3) : 0ull;
      if (hub_on && u[q] >= hub_lo) skip = kSkipAll;
      gkeys[e] = (skip << kSkipShift) | ((uint64_t)(uint32_t)h << b) | (uint32_t)l;
      for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p * 256 + ((h >> (8 * p)) & 255)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += kGroupThreads)
    if (s_hist[i]) atomicAdd(&hist[i], s_hist[i]);
}

// Work of the counting phase, for instrumentation only (never on the path
// of a count): per forward edge (h, l) of group h, the entries of N+(l)
// streamed through the hash set (d+(l) less the skipped leading blocks),
// and the merge work d+(h) + d+(l) of
// Sec. II-B; per non-empty group, the list hashed once, d+(h) inserts; the
// largest d+.  Also, per hub set H = the 2^12 .. 2^15 highest ranks, the
// lookups of the edges with both endpoints in H: ranks follow (degree, id),
// so every forward neighbour of a vertex of H is in H, and those edges'
// intersections lie wholly inside H (what a dense count of the hub block
// A_HH would take over, Sec. VI).  One warp per vertex h.
__global__ void __launch_bounds__(kGroupThreads)
k_work(const int32_t *__restrict__ off, const int32_t *__restrict__ goff,
       const int32_t *__restrict__ part, const int32_t *__restrict__ pskip, int32_t n,
       Ctrl *ctrl, uint32_t shard, uint32_t shards) {
  if (aborted(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (kGroupThreads / 32);
  unsigned long long lookups = 0, inserts = 0, merge = 0, dmax = 0, hub[kHubSizes] = {};
  for (uint32_t h = (blockIdx.x * kGroupThreads + threadIdx.x) >> 5; h < (uint32_t)n;
       h += warps) {
    if (h % shards != shard) continue;  // another part's group (uniform per warp)
    const unsigned long long dh = (unsigned long long)(__ldg(off + h + 1) - __ldg(off + h));
    const int32_t pb = __ldg(goff + h), pe = __ldg(goff + h + 1);
    if (lane == 0) {
      if (pe > pb) inserts += dh;
      dmax = dh > dmax ? dh : dmax;
    }
    for (int32_t i = pb + lane; i < pe; i += 32) {
      const int32_t l = __ldg(part + i);
      const int32_t dfull = __ldg(off + l + 1) - __ldg(off + l);
      const int32_t ds = max(dfull - 8 * __ldg(pskip + i), 0);  // entries streamed
      const unsigned long long dl = (unsigned long long)ds;
      lookups += dl;
      merge += dh + (unsigned long long)dfull;
#pragma unroll
      for (int k = 0; k < kHubSizes; ++k) {
        const int64_t lo = (int64_t)n - ((int64_t)1 << (kHubLog2Min + k));
        if ((int64_t)h >= lo && (int64_t)l >= lo) hub[k] += dl;
      }
    }
  }
  for (int o = 16; o; o >>= 1) {
    lookups += __shfl_xor_sync(0xffffffffu, lookups, o);
    inserts += __shfl_xor_sync(0xffffffffu, inserts, o);
    merge += __shfl_xor_sync(0xffffffffu, merge, o);
    const unsigned long long x = __shfl_xor_sync(0xffffffffu, dmax, o);
    dmax = x > dmax ? x : dmax;
#pragma unroll
    for (int k = 0; k < kHubSizes; ++k) hub[k] += __shfl_xor_sync(0xffffffffu, hub[k], o);
  }
  if (lane == 0) {
    atomicAdd(&ctrl->work[0], lookups);
    atomicAdd(&ctrl->work[1], inserts);
    atomicAdd(&ctrl->work[2], merge);
    atomicMax(&ctrl->work[3], dmax);
#pragma unroll
    for (int k = 0; k < kHubSizes; ++k)
      if (hub[k]) atomicAdd(&ctrl->work[4 + k], hub[k]);
  }
}

uint32_t group_grid(uint32_t m_bound) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t want = (m_bound + kGroupThreads * 8 - 1) / (kGroupThreads * 8);
  return max(1u, min(want, (uint32_t)(sms > 0 ? sms : 1) * 8));
}

}  // namespace

void launch_sort_lists(int32_t *col, const int32_t *off, const int32_t *voff, int32_t n,
                       Ctrl *ctrl, int32_t *col4, int32_t *long_lists, int32_t *dlen,
                       int32_t *dcorr, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = sms > 0 ? sms : 1;
  const ListOut o{col4, dlen, dcorr, ctrl};
  const uint32_t chunks = ((uint32_t)n + 31u) / 32u;
  const uint32_t grid = max(1u, min((chunks + kListWarps - 1) / kListWarps, (uint32_t)sms * 8u));
  k_sort_lists<<<grid, kListThreads, 0, st>>>(col, off, voff, n, o, long_lists);
  k_sort_long_lists_warp<<<sms * 4, kListThreads, 0, st>>>(col, off, voff, o, long_lists);
  k_sort_long_lists<<<sms * kLongListBlocks, kLongListThreads, 0, st>>>(col, off, voff, o,
                                                                        long_lists);
  note_launch();
  note_launch();
  note_launch();
}

void launch_fix_repeats(const int32_t *off, int32_t n, const int32_t *dcorr, const int32_t *rank,
                        Ctrl *ctrl, int32_t *row, int32_t *deg, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t grid = (uint32_t)(sms > 0 ? sms : 1) * 8u;
  k_fix_rows<<<grid, kListThreads, 0, st>>>(off, n, ctrl, row);
  k_fix_degree<<<grid, kListThreads, 0, st>>>(dcorr, rank, n, ctrl, deg);
  note_launch();
  note_launch();
}

void launch_group_keys(const int32_t *row, const int32_t *col4, const int32_t *off,
                       const int2 *ldesc, uint32_t m_bound, int b,
                       int passes, int32_t heavy_ratio_pct, Ctrl *ctrl, uint64_t *gkeys,
                       uint32_t *hist, cudaStream_t st) {
  k_group_keys<<<group_grid(m_bound), kGroupThreads, 0, st>>>(row, col4, off, ldesc, b,
                                                              passes, heavy_ratio_pct, ctrl,
                                                              gkeys, hist);
  note_launch();
}

void launch_work(const int32_t *off, const int32_t *goff, const int32_t *part,
                 const int32_t *pskip, int32_t n, Ctrl *ctrl, cudaStream_t st, int32_t shard,
                 int32_t shards) {
  const uint32_t lanes = n > (1 << 28) ? (1u << 30) : (uint32_t)n * 4u;  // grid is capped anyway
  k_work<<<group_grid(lanes), kGroupThreads, 0, st>>>(off, goff, part, pskip, n, ctrl,
                                                      (uint32_t)shard, (uint32_t)shards);
  note_launch();
}

}  // namespace tc
