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

// The warp sorts the list of lane `src` (d entries from col + b) into col4
// from entry w4, with E keys per lane (32 E >= d), and records its minimum.
template <int E>
__device__ __forceinline__ void warp_sort_list(const int32_t *__restrict__ col, int32_t b,
                                               int32_t d, long long w4,
                                               int32_t *__restrict__ col4, int32_t *lmin_v) {
  const int lane = threadIdx.x & 31;
  int32_t x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    x[e] = i < d ? __ldg(col + b + i) : INT32_MAX;
  }
  warp_sort_regs<E>(x);
  const int r8 = (d + 7) & ~7;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + lane;
    if (i < r8) col4[w4 + i] = i < d ? x[e] : -1;
  }
  if (lane == 0) *lmin_v = x[0];
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

// Every forward list into col4, sorted ascending and padded with -1 to
// whole 32-byte blocks.  Warps take 32 consecutive vertices at a time: a
// list of up to 8 entries is sorted by its own lane in registers (a sorting
// network), one of up to kWarpSortMax entries by the warp in registers
// (bitonic, up to 16 keys per lane); longer lists go to k_sort_long_lists.
__global__ void __launch_bounds__(kListThreads)
k_sort_lists(const int32_t *__restrict__ col, const int32_t *__restrict__ off,
             const int32_t *__restrict__ voff, int32_t n, Ctrl *ctrl, int32_t *__restrict__ col4,
             int32_t *__restrict__ lmin, int32_t *__restrict__ long_lists) {
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t warps = gridDim.x * kListWarps;
  // lists of the dense hub block need no order: the hash path skips their
  // streams whole and hashes them as they come
  const uint32_t unsorted_from = ctrl->hub_on ? ctrl->hub_lo : 0xffffffffu;
  for (uint32_t c = blockIdx.x * kListWarps + warp; c * 32u < (uint32_t)n; c += warps) {
    const uint32_t v = c * 32u + lane;
    int32_t b = 0, d = 0;
    long long w4 = 0;  // first col4 entry of the list
    if (v < (uint32_t)n) {
      b = __ldg(off + v);
      d = __ldg(off + v + 1) - b;
      w4 = 4ll * __ldg(voff + v);
      if (d == 0) lmin[v] = INT32_MAX;
    }
    if (c * 32u >= unsorted_from) {  // a whole chunk of hub lists: copied as they are
      const uint32_t copy = __ballot_sync(kFull, d > 0);
      for (uint32_t todo = copy; todo; todo &= todo - 1) {
        const int src = __ffs(todo) - 1;
        const int32_t lb = __shfl_sync(kFull, b, src), ld = __shfl_sync(kFull, d, src);
        const long long lw = __shfl_sync(kFull, w4, src);
        const int r8 = (ld + 7) & ~7;
        for (int i = lane; i < r8; i += 32) col4[lw + i] = i < ld ? __ldg(col + lb + i) : -1;
      }
      if (d > 0) lmin[v] = INT32_MIN;  // unsorted
      continue;
    }
    if (d > 0 && d <= 8) {
      int32_t x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = i < d ? __ldg(col + b + i) : INT32_MAX;
      sort8(x);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i >= d) x[i] = -1;
      int4 *dst = reinterpret_cast<int4 *>(col4 + w4);
      dst[0] = make_int4(x[0], x[1], x[2], x[3]);
      dst[1] = make_int4(x[4], x[5], x[6], x[7]);
      lmin[v] = x[0];
    }
    uint32_t todo = __ballot_sync(kFull, d > 8 && d <= kWarpSortMax);
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int32_t lb = __shfl_sync(kFull, b, src), ld = __shfl_sync(kFull, d, src);
      const long long lw = __shfl_sync(kFull, w4, src);
      int32_t *lm = lmin + c * 32u + src;
      if (ld <= 32) warp_sort_list<1>(col, lb, ld, lw, col4, lm);
      else if (ld <= 64) warp_sort_list<2>(col, lb, ld, lw, col4, lm);
      else if (ld <= 128) warp_sort_list<4>(col, lb, ld, lw, col4, lm);
      else if (ld <= 256) warp_sort_list<8>(col, lb, ld, lw, col4, lm);
      else warp_sort_list<16>(col, lb, ld, lw, col4, lm);
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
                       const int32_t *__restrict__ voff, Ctrl *ctrl, int32_t *__restrict__ col4,
                       int32_t *__restrict__ lmin, const int32_t *__restrict__ long_lists) {
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
    warp_sort_list<kWarpLongMax / 32>(col, b, d, 4ll * __ldg(voff + v), col4, lmin + v);
  }
}

// Lists longer than kWarpLongMax: one CTA each, sorted in shared memory up
// to kCtaSortMax entries; longer lists are copied unsorted and flagged in
// lmin (their streams then skip nothing).
__global__ void __launch_bounds__(kLongListThreads, kLongListBlocks)
k_sort_long_lists(const int32_t *__restrict__ col, const int32_t *__restrict__ off,
                  const int32_t *__restrict__ voff, Ctrl *ctrl, int32_t *__restrict__ col4,
                  int32_t *__restrict__ lmin, const int32_t *__restrict__ long_lists) {
  __shared__ int32_t s_buf[kCtaSortMax];
  __shared__ int32_t s_min[kLongListThreads / 32];
  __shared__ uint32_t s_i;
  if (aborted(ctrl)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t count = ctrl->n_long_lists;
  for (;;) {
    if (tid == 0) s_i = atomicAdd(&ctrl->next_long_list, 1u);
    __syncthreads();
    const uint32_t i = s_i;
    if (i >= count) break;
    const int32_t v = __ldg(long_lists + i);
    const int32_t b = __ldg(off + v), d = __ldg(off + v + 1) - b;
    if (d > kWarpLongMax) {  // shorter lists are the warp kernel's (uniform for the block)
      int32_t *dst = col4 + 4ll * __ldg(voff + v);
      const int r8 = (d + 7) & ~7;
      if (d <= kCtaSortMax) {
        const int P = pow2_at_least(d);
        for (int j = tid; j < P; j += kLongListThreads) s_buf[j] = j < d ? __ldg(col + b + j) : INT32_MAX;
        __syncthreads();
        bitonic_smem<kLongListThreads>(s_buf, P, tid);
        for (int j = tid; j < r8; j += kLongListThreads) dst[j] = j < d ? s_buf[j] : -1;
        if (tid == 0) lmin[v] = s_buf[0];
      } else {
        int32_t mn = INT32_MAX;
        for (int j = tid; j < r8; j += kLongListThreads) {
          const int32_t x = j < d ? __ldg(col + b + j) : -1;
          dst[j] = x;
          if (j < d) mn = min(mn, x);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(kFull, mn, o));
        if (lane == 0) s_min[warp] = mn;
        __syncthreads();
        if (tid == 0) {
          for (int w = 1; w < kLongListThreads / 32; ++w) mn = min(mn, s_min[w]);
          lmin[v] = -1 - mn;  // unsorted
        }
      }
    }
    __syncthreads();  // s_buf and s_i are reused
  }
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
// list N+(u) of col4 holds v at position i = e - off[u]): the group key of
// every edge with the digit histograms of its h field.  When the longer
// list is v's (h = v), the intersection streams N+(u), whose entries before
// position i are all below v; N+(h) holds only ids above h = v, so those
// entries cannot match and the whole blocks among them, i >> 3, are
// skipped.  Their count rides in the key's top bits to the partner array.
// (When h = u, N+(v) is streamed and all its entries lie above v, itself
// in N+(u): nothing to skip.)
__global__ void __launch_bounds__(kGroupThreads)
k_group_keys(const int32_t *__restrict__ row, const int32_t *__restrict__ col4,
             const int32_t *__restrict__ off, const int32_t *__restrict__ voff,
             const int32_t *__restrict__ lmin, int b, int passes, int32_t heavy_ratio_pct,
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
    int32_t um[kGroupUnroll];
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      u[q] = e < m ? __ldg(row + e) : 0;
    }
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      ub[q] = __ldg(off + u[q]);
      ue[q] = __ldg(off + u[q] + 1);
      uw[q] = __ldg(voff + u[q]);
      um[q] = __ldg(lmin + u[q]);
    }
    int32_t v[kGroupUnroll], vd[kGroupUnroll];
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      v[q] = e < m ? __ldg(col4 + 4ll * uw[q] + ((int32_t)e - ub[q])) : 0;
    }
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) vd[q] = __ldg(off + v[q] + 1) - __ldg(off + v[q]);
#pragma unroll
    for (int q = 0; q < kGroupUnroll; ++q) {
      const uint32_t e = e0 + q * stride;
      if (e >= m) break;
      int32_t h, l;
      split_edge(u[q], v[q], ue[q] - ub[q], vd[q], heavy_ratio_pct, h, l);
      // the list of u is sorted unless it was too long to sort (um < 0); an
      // edge inside the dense hub block (owner u, hence v, of rank >=
      // hub_lo) is left to it: its stream is skipped whole
      uint64_t skip = (carry_skip && h == v[q] && um[q] >= 0)
                          ? (uint64_t)(((int32_t)e - ub[q]) >> 3) : 0ull;
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

void launch_sort_lists(const int32_t *col, const int32_t *off, const int32_t *voff, int32_t n,
                       Ctrl *ctrl, int32_t *col4, int32_t *lmin, int32_t *long_lists,
                       cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  sms = sms > 0 ? sms : 1;
  const uint32_t chunks = ((uint32_t)n + 31u) / 32u;
  const uint32_t grid = max(1u, min((chunks + kListWarps - 1) / kListWarps, (uint32_t)sms * 8u));
  k_sort_lists<<<grid, kListThreads, 0, st>>>(col, off, voff, n, ctrl, col4, lmin, long_lists);
  k_sort_long_lists_warp<<<sms * 4, kListThreads, 0, st>>>(col, off, voff, ctrl, col4, lmin,
                                                            long_lists);
  k_sort_long_lists<<<sms * kLongListBlocks, kLongListThreads, 0, st>>>(col, off, voff, ctrl,
                                                                        col4, lmin, long_lists);
  note_launch();
  note_launch();
  note_launch();
}

void launch_group_keys(const int32_t *row, const int32_t *col4, const int32_t *off,
                       const int32_t *voff, const int32_t *lmin, uint32_t m_bound, int b,
                       int passes, int32_t heavy_ratio_pct, Ctrl *ctrl, uint64_t *gkeys,
                       uint32_t *hist, cudaStream_t st) {
  k_group_keys<<<group_grid(m_bound), kGroupThreads, 0, st>>>(row, col4, off, voff, lmin, b,
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
