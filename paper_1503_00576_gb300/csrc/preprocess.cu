// preprocess.cu -- preprocessing of the forward algorithm on sm_103a.
//
// Sec. III-B of the paper builds, from an edge array, the sorted forward
// adjacency lists: sort the edges (as 64-bit integers, Sec. III-D), build the
// node array, mark and remove backward edges, unzip, rebuild the node array.
// Here the same lists are reached in this order, each step one kernel:
//
//   canon          validate ids (Sec. III-B computes n = max id + 1; here n
//                  is given and any id >= n is an error), drop self-loops,
//                  write the undirected key min(u,v) << b | max(u,v) with
//                  b = bits of n, and add one to the degree of both ends
//                  (a global atomic each).  An edge given more than once is
//                  counted as often as it is given; the list sort drops
//                  the repeats later and takes their counts back.
//   rank keys      the (degree, id) order of Sec. II-B as a permutation:
//                  a stable radix sort of deg(v) << b | v whose last pass
//                  scatters rank[v]; the rest of the pipeline runs on ranks.
//                  Any total order of the vertices counts every triangle
//                  exactly once (from its lowest vertex), so the repeats in
//                  these degrees change how the work is split, never a
//                  count; without repeats the order is the paper's.
//   orient         compact the keys (dropping self-loops; tile scan +
//                  look-back) and emit each as owner << b | neighbour in
//                  rank space, the owner being the endpoint of lower rank --
//                  marking and removing backward edges of Sec. III-B in one
//                  pass; also the digit histograms of the owner field.
//   radix passes   stable LSD passes over the owner bits only.  The last
//                  pass writes the neighbour (the column array: the
//                  "unzip"), the owner (the row array) and counts the
//                  out-degrees.
//   offsets        exclusive scan of the out-degrees = node array (CSR
//                  offsets).  The last sort pass also wrote the row of
//                  every entry, so (row[], col[]) is the paper's unzipped
//                  structure-of-arrays edge array.
//
// The paper sorts all 2m keys first (which also brings repeated edges
// together); here no global sort of the undirected keys is needed: each
// forward list is sorted on its own afterwards (group.cu), which is where
// repeated edges meet and are dropped.
#include <cstdio>

#include "tc_common.cuh"

namespace tc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Bound of every spin-wait of this file, and the radix-pass tile that never
// publishes (none by default).  Only the failure-path tests change them.
__device__ uint32_t g_spin_limit = kSpinLimit;
__device__ uint32_t g_unpublished_tile = 0xffffffffu;

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long *p, unsigned long long v) {
  *(volatile unsigned long long *)p = v;
}

// Exclusive scan of one uint32 per thread over the first 256 threads of the
// block; returns the thread's exclusive prefix, *total gets the sum.  All
// threads of the block must call it.  `scratch` holds >= 8 words.
__device__ __forceinline__ uint32_t scan256_exclusive(uint32_t v, uint32_t *scratch,
                                                      uint32_t *total) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t x = (tid < 256) ? v : 0u;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (tid < 256 && lane == 31) scratch[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    uint32_t s = scratch[w];
    if (w < warp) before += s;
    all += s;
  }
  *total = all;
  return before + incl - x;
}

// Generic block exclusive scan of one uint32 per thread (any block size that
// is a multiple of 32, up to 1024).  scratch holds >= 32 words.
template <int THREADS>
__device__ __forceinline__ uint32_t block_scan_exclusive(uint32_t x, uint32_t *scratch,
                                                         uint32_t *total) {
  constexpr int WARPS = THREADS / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  uint32_t before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    uint32_t s = scratch[w];
    if (w < warp) before += s;
    all += s;
  }
  *total = all;
  return before + incl - x;
}

// Decoupled look-back for one running sum, by one warp.  Publishes the
// tile's aggregate (unless the caller already did: `published`, see
// publish_aggregate), then reads the statuses of 32 predecessors at once (lane
// k reads tile j - k): once all 32 have published something, it adds the
// values up to the nearest inclusive prefix, or all 32 and moves on; so a
// walk back over many tiles costs one memory latency per 32 tiles.
// Publishes the tile's inclusive prefix and returns the exclusive one (in
// every lane).  If a wait runs out, or a predecessor is poisoned, the tile's
// prefix is unknown: it publishes a poisoned status, sets *bad (in every
// lane) and the caller must write nothing.  All 32 lanes of the warp must
// call it.
__device__ uint64_t lookback_warp(unsigned long long *status, uint32_t tile, uint64_t agg,
                                  Ctrl *ctrl, bool *bad, bool published = false) {
  const int lane = threadIdx.x & 31;
  *bad = false;
  if (tile == 0) {
    if (lane == 0 && !published) st_volatile_u64(&status[0], kFlagInclusive | agg);
    return 0;
  }
  if (lane == 0 && !published) st_volatile_u64(&status[tile], kFlagAggregate | agg);
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  uint32_t spins = 0;
  const uint32_t limit = g_spin_limit;
  for (;;) {
    const int64_t idx = j - lane;
    // before tile 0 nothing is added: an inclusive zero
    const unsigned long long s = idx >= 0 ? ld_volatile_u64(&status[idx]) : kFlagInclusive;
    const unsigned long long flag = s & ~kValueMask;
    if (__any_sync(kFull, flag == kFlagPoison)) {
      *bad = true;
      break;
    }
    if (__any_sync(kFull, flag == 0)) {  // a predecessor in the window has not published
      if (++spins > limit) {
        if (lane == 0) atomicOr(&ctrl->err, kErrTimeout);
        *bad = true;
        break;
      }
      if (spins > 8) __nanosleep(32);
      continue;
    }
    const uint32_t inc = __ballot_sync(kFull, flag == kFlagInclusive);
    const int last = inc ? __ffs(inc) - 1 : 31;  // lanes 0 .. last contribute
    uint64_t v = lane <= last ? (s & kValueMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    excl += v;
    if (inc) break;
    j -= 32;
  }
  if (lane == 0) st_volatile_u64(&status[tile], *bad ? kFlagPoison : kFlagInclusive | (excl + agg));
  return excl;
}

// A tile that starts after the call has failed publishes a poisoned status
// (so that no successor waits on it) and does nothing else.  One word per
// tile; called by one thread.
__device__ __forceinline__ void poison_tile(unsigned long long *status, uint32_t tile) {
  st_volatile_u64(&status[tile], kFlagPoison);
}

// The first half of lookback_warp, for a tile whose aggregate is known
// before the rest of its work: successors can sum past it sooner.  Called
// by one thread.
__device__ __forceinline__ void publish_aggregate(unsigned long long *status, uint32_t tile,
                                                  uint64_t agg) {
  st_volatile_u64(&status[tile], (tile == 0 ? kFlagInclusive : kFlagAggregate) | agg);
}

// ---------------------------------------------------------------------------
// canon: validate, drop loops, undirected 64-bit keys, degrees
// ---------------------------------------------------------------------------
constexpr int kCanonThreads = 256;
constexpr int kCanonUnroll = 8;

__global__ void __launch_bounds__(kCanonThreads)
k_canon(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, uint32_t m_in,
        int32_t n, int b, const BatchDesc *__restrict__ batch, uint64_t *__restrict__ keys,
        int32_t *__restrict__ deg, Ctrl *ctrl) {
  const uint64_t sentinel = (1ull << (2 * b)) - 1;  // > every valid key; 2b <= 62
  // batch: graph g owns pairs [eo[g], eo[g+1]) and union ids from vo[g]
  int32_t ng = 0;
  const int32_t *eo = nullptr, *vo = nullptr;
  uint32_t m_real = m_in;
  if (batch) {
    ng = batch->num_graphs;
    eo = batch->edge_off;
    vo = batch->voff;
    m_real = min((uint32_t)__ldg(eo + ng), m_in);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->m_in = m_real;
  bool bad = false;
  const uint32_t stride = gridDim.x * kCanonThreads;
  // pairs past m_real are batch padding: not keyed, not sorted.  The pairs
  // of kCanonUnroll rounds are loaded before any is keyed: the inputs may be
  // host memory read in place, where each load waits a long time.  Pairs and
  // keys pass through L2 marked to be evicted first (they are read or
  // written once here), so that the degree array stays in L2 for the atomics
  // (-0.27 ms of 2.55 at R-MAT scale 24).
  for (uint32_t i0 = blockIdx.x * kCanonThreads + threadIdx.x; i0 < m_real;
       i0 += kCanonUnroll * stride) {
    int32_t us[kCanonUnroll], vs[kCanonUnroll];
#pragma unroll
    for (int q = 0; q < kCanonUnroll; ++q) {
      const uint32_t i = i0 + q * stride;
      us[q] = i < m_real ? __ldcs(src + i) : 0;
      vs[q] = i < m_real ? __ldcs(dst + i) : 0;
    }
#pragma unroll
    for (int q = 0; q < kCanonUnroll; ++q) {
      const uint32_t i = i0 + q * stride;
      if (i >= m_real) break;
      const int32_t u = us[q], v = vs[q];
      int32_t lim = n, shift = 0, lo_graph = 0;
      if (batch) {
        int32_t lo = 0, hi = ng;  // the last graph g with eo[g] <= i
        while (hi - lo > 1) {
          const int32_t mid = (lo + hi) >> 1;
          if ((uint32_t)__ldg(eo + mid) <= i) lo = mid; else hi = mid;
        }
        lo_graph = lo;
        shift = __ldg(vo + lo);
        lim = __ldg(vo + lo + 1) - shift;
      }
      uint64_t key;
      if ((uint32_t)u >= (uint32_t)lim || (uint32_t)v >= (uint32_t)lim) {
        // a batch fails only the graph that holds the pair; the pair is dropped
        // so the other graphs of the union are counted exactly
        if (batch) batch->gerr[lo_graph] = 1; else bad = true;
        key = sentinel;
      } else if (u == v) {
        key = sentinel;  // self-loop: sorts last, dropped with the sentinels
      } else {
        const uint32_t lo = (uint32_t)(min(u, v) + shift), hi = (uint32_t)(max(u, v) + shift);
        key = ((uint64_t)lo << b) | hi;
        atomicAdd(&deg[lo], 1);
        atomicAdd(&deg[hi], 1);
      }
      __stcs(reinterpret_cast<unsigned long long *>(keys) + i, (unsigned long long)key);
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctrl->err, kErrIdRange);
}

// ---------------------------------------------------------------------------
// one LSD radix pass (8-bit digit at `shift`), onesweep style
// ---------------------------------------------------------------------------
struct RadixShared {
  uint64_t keys[kSortTile];                 // the tile, staged in digit order
  uint32_t whist[kSortThreads / 32][256];   // per warp and digit: count, then first position
  uint32_t gbase[256];                      // per digit: output position of staged index 0
  uint32_t scratch[32];
  uint32_t tile;
  uint32_t abort;  // some digit's look-back gave up: the tile writes nothing
};

// Writes one staged key to its output position (and, for the column pass,
// its row and the out-degree of its owner).
template <int MODE>
__device__ __forceinline__ void radix_out(uint64_t key, uint32_t pos, void *__restrict__ out,
                                          uint32_t col_mask, uint32_t *__restrict__ row_out,
                                          int owner_shift, int32_t *outdeg, uint32_t active) {
  if (MODE == kOutColRow || MODE == kOutPartSkip) {
    const uint32_t owner = MODE == kOutColRow ? (uint32_t)(key >> owner_shift)
                                              : (uint32_t)(key >> owner_shift) & col_mask;
    ((uint32_t *)out)[pos] = (uint32_t)key & col_mask;
    if (MODE == kOutPartSkip) row_out[pos] = (uint32_t)(key >> kSkipShift);
    else if (row_out) row_out[pos] = owner;
    // the staged tile is in owner order: consecutive lanes share owners,
    // and one atomic per run gives the out-degrees (the node array's counts)
    const uint32_t peers = __match_any_sync(active, owner);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&outdeg[owner], __popc(peers));
  } else if (MODE == kOutRank) {
    ((uint32_t *)out)[(uint32_t)key & col_mask] = pos;
  } else {
    __stcs(reinterpret_cast<unsigned long long *>(out) + pos, (unsigned long long)key);
  }
}

// One tile of a pass.  FULL: all TILE keys of the tile exist (every tile but
// the last), so no key needs a bounds test.  UNSTABLE: keys of equal digit
// are ranked in any order (a shared-memory atomic per key instead of the
// ballots): only for the first pass of a sort whose input order does not
// matter.
template <int MODE, bool FULL, bool UNSTABLE>
__device__ __forceinline__ void radix_tile(RadixShared &S, const uint64_t *__restrict__ in,
                                           void *__restrict__ out, uint32_t n_keys,
                                           uint32_t tile, uint32_t gofs, int shift,
                                           uint32_t col_mask, uint32_t *__restrict__ row_out,
                                           int owner_shift, int32_t *outdeg,
                                           unsigned long long *__restrict__ status, Ctrl *ctrl) {
  constexpr int WARPS = kSortThreads / 32, KPT = kSortKeysPerThread, TILE = kSortTile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile_base = tile * (uint32_t)TILE;
  const uint32_t first = tile_base + (uint32_t)(warp * 32 * KPT + lane);  // key i: first + 32 i

  // ---- rank keys within the tile (stable: warp-major, round-major, lane) ----
  // Keys are read and written once per pass: they pass through L2 marked to
  // be evicted first, which keeps the look-back words, the histograms and
  // the counters the last passes add to in L2 (-7% per pass at R-MAT scale
  // 24).
  // All 16 keys of a thread are loaded before ranking starts, and the
  // kernel is held to 64 registers so that four tiles fit on an SM: the
  // pass is latency-bound, and occupancy halves its time even though a few
  // keys spill to L1.
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint64_t k[KPT];
  uint32_t pk[KPT];  // digit << 16 | rank among the warp's keys of that digit
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    k[i] = (FULL || first + 32u * i < n_keys)
               ? (uint64_t)__ldcs(reinterpret_cast<const unsigned long long *>(in) + first + 32u * i)
               : 0ull;
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const bool valid = FULL || first + 32u * i < n_keys;
    const uint32_t d = (uint32_t)(k[i] >> shift) & 255u;
    if (UNSTABLE) {
      pk[i] = valid ? (d << 16) | atomicAdd(&S.whist[warp][d], 1u) : 0u;
      continue;
    }
    uint32_t peers = FULL ? kFull : __ballot_sync(kFull, valid);
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t bb = __ballot_sync(kFull, (d >> bit) & 1u);
      peers &= bb ^ (((d >> bit) & 1u) - 1u);  // bb where bit is set, else ~bb
    }
    const uint32_t below = __popc(peers & lt_mask);  // 0: the first lane of its digit
    const uint32_t before = S.whist[warp][d];
    __syncwarp();
    if (valid && below == 0) S.whist[warp][d] = before + __popc(peers);
    __syncwarp();
    pk[i] = (d << 16) | (before + below);
  }
  __syncthreads();

  // ---- per digit (thread tid): tile count, published at once; tile offset
  // and warp offsets; then the keys are staged, sorted by digit, before the
  // look-back waits on the tiles before this one ----
  unsigned long long *st = status + (size_t)tile * 256 + tid;
  uint32_t tile_cnt = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) tile_cnt += S.whist[w][tid];
  const bool publish = tile != g_unpublished_tile;  // always, but in a failure-path test
  if (publish) st_volatile_u64(st, (tile == 0 ? kFlagInclusive : kFlagAggregate) | tile_cnt);
  uint32_t tile_total;
  const uint32_t tstart = scan256_exclusive(tile_cnt, S.scratch, &tile_total);
  {
    // staged position of the first key of warp w with this digit
    uint32_t run = tstart;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t c = S.whist[w][tid];
      S.whist[w][tid] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < KPT; ++i)
    if (FULL || first + 32u * i < n_keys)
      S.keys[S.whist[warp][pk[i] >> 16] + (pk[i] & 0xffffu)] = k[i];
  {
    // decoupled look-back for this digit
    uint64_t excl = 0;
    if (tile > 0) {
      // the statuses of kLookback predecessors are read at once (one memory
      // latency per round), then summed back to the nearest inclusive one;
      // a round stops early at a predecessor that has not published yet
      constexpr int kLookback = 4;
      int64_t j = (int64_t)tile - 1;
      uint32_t spins = 0;
      const uint32_t limit = g_spin_limit;
      bool bad = false, done = false;
      while (!done) {
        unsigned long long s[kLookback];
#pragma unroll
        for (int q = 0; q < kLookback; ++q)
          s[q] = j - q >= 0 ? ld_volatile_u64(status + (size_t)(j - q) * 256 + tid)
                            : kFlagInclusive;  // before tile 0: an inclusive zero
        int used = 0;
#pragma unroll
        for (int q = 0; q < kLookback; ++q) {
          if (done || used < q) break;
          const unsigned long long flag = s[q] & ~kValueMask;
          if (flag == 0) break;  // not published yet: read again from here
          if (flag == kFlagPoison) {
            bad = done = true;
            break;
          }
          excl += s[q] & kValueMask;
          used = q + 1;
          if (flag == kFlagInclusive) done = true;
        }
        if (done) break;
        j -= used;
        if (used == 0) {
          if (++spins > limit) {
            atomicOr(&ctrl->err, kErrTimeout);
            bad = true;
            break;
          }
          if (spins > 64) __nanosleep(64);
        }
      }
      if (publish) st_volatile_u64(st, bad ? kFlagPoison : kFlagInclusive | (excl + tile_cnt));
      if (bad) S.abort = 1u;
    }
    // output position of the staged index i with digit d is s_gbase[d] + i
    // (mod 2^32 arithmetic; the result is < 2^31)
    S.gbase[tid] = gofs + (uint32_t)excl - tstart;
  }
  __syncthreads();
  if (S.abort) return;  // uniform for the block

  // ---- scatter: consecutive threads write consecutive positions of a run ----
  if (FULL) {
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const uint32_t i = (uint32_t)(tid + j * kSortThreads);
      const uint64_t key = S.keys[i];
      radix_out<MODE>(key, S.gbase[(uint32_t)(key >> shift) & 255u] + i, out, col_mask, row_out,
                      owner_shift, outdeg, kFull);
    }
  } else {
    const uint32_t tile_n = n_keys - tile_base;
    for (uint32_t i = tid; i < tile_n; i += kSortThreads) {
      const uint64_t key = S.keys[i];
      radix_out<MODE>(key, S.gbase[(uint32_t)(key >> shift) & 255u] + i, out, col_mask, row_out,
                      owner_shift, outdeg, __activemask());
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(kSortThreads, 4)
k_radix_pass(const uint64_t *__restrict__ in, void *__restrict__ out, uint32_t n_keys_bound,
             const uint32_t *__restrict__ n_keys_dev, int shift, uint32_t col_mask,
             uint32_t *__restrict__ row_out, int owner_shift, int32_t *outdeg,
             const uint32_t *__restrict__ hist, unsigned long long *__restrict__ status,
             uint32_t *ticket, Ctrl *ctrl, int unstable) {
  constexpr int WARPS = kSortThreads / 32, TILE = kSortTile;
  __shared__ RadixShared S;
  const int tid = threadIdx.x;
  if (tid == 0) {
    S.tile = atomicAdd(ticket, 1u);
    S.abort = aborted(ctrl) ? 1u : 0u;
  }
  for (int i = tid; i < WARPS * 256; i += kSortThreads) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t tile = S.tile;
  if (S.abort) {  // an earlier wait of this call ran out: the input is not complete
    st_volatile_u64(status + (size_t)tile * 256 + tid, kFlagPoison);
    return;
  }
  const uint32_t n_keys = n_keys_dev ? *n_keys_dev : n_keys_bound;
  const uint32_t tile_base = tile * (uint32_t)TILE;
  if (tile_base >= n_keys) return;  // uniform for the block

  // global start of every digit: exclusive scan of the pass histogram
  uint32_t dummy;
  const uint32_t gofs = scan256_exclusive(hist[tid], S.scratch, &dummy);
  const bool full = n_keys - tile_base >= (uint32_t)TILE;
  if (MODE == kOutKeys && unstable) {  // uniform for the grid
    if (full)
      radix_tile<MODE, true, true>(S, in, out, n_keys, tile, gofs, shift, col_mask, row_out,
                                   owner_shift, outdeg, status, ctrl);
    else
      radix_tile<MODE, false, true>(S, in, out, n_keys, tile, gofs, shift, col_mask, row_out,
                                    owner_shift, outdeg, status, ctrl);
  } else if (full) {
    radix_tile<MODE, true, false>(S, in, out, n_keys, tile, gofs, shift, col_mask, row_out,
                                  owner_shift, outdeg, status, ctrl);
  } else {
    radix_tile<MODE, false, false>(S, in, out, n_keys, tile, gofs, shift, col_mask, row_out,
                                   owner_shift, outdeg, status, ctrl);
  }
}

// ---------------------------------------------------------------------------
// rank keys: the order of Sec. II-B as a permutation.  Vertex v gets the key
// deg(v) << b | v; a stable LSD sort over the degree bits leaves the keys in
// (degree, id) order, and its last pass scatters rank[v] = position.  From
// here on the pipeline works on ranks: an edge is oriented from its lower
// rank, and the high-degree vertices, which fill most forward lists, get
// the highest, adjacent ids.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCanonThreads)
k_rank_keys(const int32_t *__restrict__ deg, int32_t n, int b, int passes,
            uint64_t *__restrict__ vkeys, uint32_t *__restrict__ hist) {
  __shared__ uint32_t sh[kMaxRankPasses * 256];
  for (int i = threadIdx.x; i < passes * 256; i += kCanonThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t stride = gridDim.x * kCanonThreads;
  for (uint32_t v = blockIdx.x * kCanonThreads + threadIdx.x; v < (uint32_t)n; v += stride) {
    const uint32_t d = (uint32_t)__ldg(deg + v);
    vkeys[v] = ((uint64_t)d << b) | v;
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * 256 + ((d >> (8 * p)) & 255u)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += kCanonThreads)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ---------------------------------------------------------------------------
// orient: compact the keys, orient by rank (= (degree, id) order)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kOrientThreads, 4)
k_orient(const uint64_t *__restrict__ keys, int b,
         const int32_t *__restrict__ rank, uint64_t *__restrict__ okeys,
         uint32_t *__restrict__ hist2, int passes2, unsigned long long *status, Ctrl *ctrl) {
  constexpr int KPT = kOrientKeysPerThread, TILE = kOrientTile;
  static_assert(KPT == 16, "the swizzle below assumes rows of 16 keys");
  // The tile passes through shared memory both ways: loaded and stored with
  // coalesced accesses, read and written per thread as 16 consecutive keys.
  // Row r of 16 keys has its columns XOR-ed with r mod 16, so that both
  // the column-wise and the row-wise accesses of a warp spread over the banks.
  __shared__ uint64_t s_buf[TILE];
  __shared__ uint32_t s_scratch[32];
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_excl;
  __shared__ uint32_t s_abort;
  __shared__ uint32_t s_hist[kMaxSort2Passes * 256];
  const int tid = threadIdx.x;
  const uint32_t m_in = ctrl->m_in;
  if (tid == 0) {
    s_tile = atomicAdd(&ctrl->tile_ticket[kTicketOrient], 1u);
    s_abort = aborted(ctrl) ? 1u : 0u;
  }
  for (int i = tid; i < passes2 * 256; i += kOrientThreads) s_hist[i] = 0;
  __syncthreads();
  const uint32_t tile = s_tile;
  if (s_abort) {  // an earlier wait of this call ran out
    if (tid == 0) poison_tile(status, tile);
    return;
  }
  const uint32_t tile_base = tile * (uint32_t)TILE;
  if (tile_base >= m_in) return;
  const uint64_t sentinel = (1ull << (2 * b)) - 1;
  const uint64_t mask = (1ull << b) - 1;

  auto swz = [](uint32_t j) { return (j & ~15u) | ((j ^ (j >> 4)) & 15u); };
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    const uint32_t j = (uint32_t)(i * kOrientThreads + tid);
    // keys in and out pass through L2 marked to be evicted first: the rank
    // array stays there for the gathers (-0.17 ms at R-MAT scale 24)
    s_buf[swz(j)] = tile_base + j < m_in
                        ? (uint64_t)__ldcs(reinterpret_cast<const unsigned long long *>(keys) +
                                           tile_base + j)
                        : sentinel;
  }
  __syncthreads();
  const uint32_t first = (uint32_t)tid * KPT;  // this thread's keys, within the tile
  uint64_t k[KPT];
  uint32_t flags = 0, cnt = 0;
  // every key but the sentinel is kept, repeats included: the list sort
  // drops those (and takes back the degrees they added)
#pragma unroll
  for (int i = 0; i < KPT; ++i) {
    k[i] = s_buf[swz(first + i)];
    const bool keep = k[i] != sentinel;
    flags |= (uint32_t)keep << i;
    cnt += keep;
  }
  // the tile's count is published before the gathers below, so that the
  // tiles after this one need not wait for them
  uint32_t tile_cnt;
  const uint32_t toff = block_scan_exclusive<kOrientThreads>(cnt, s_scratch, &tile_cnt);
  if (tid == 0) publish_aggregate(status, tile, tile_cnt);
  // orient the kept keys now: the rank gathers of eight keys at a time are
  // issued together, and all of it overlaps the other tiles' look-backs
  constexpr int HALF = KPT / 2;
#pragma unroll
  for (int h0 = 0; h0 < KPT; h0 += HALF) {
    uint32_t ra[HALF], rc[HALF];
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
      const bool keep = (flags >> (h0 + i)) & 1u;
      ra[i] = keep ? (uint32_t)__ldg(rank + (uint32_t)(k[h0 + i] >> b)) : 0u;
      rc[i] = keep ? (uint32_t)__ldg(rank + (uint32_t)(k[h0 + i] & mask)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
      const uint32_t owner = min(ra[i], rc[i]), nbr = max(ra[i], rc[i]);
      k[h0 + i] = ((uint64_t)owner << b) | nbr;
      if ((flags >> (h0 + i)) & 1u)
        for (int p = 0; p < passes2; ++p)
          atomicAdd(&s_hist[p * 256 + ((owner >> (8 * p)) & 255u)], 1u);
    }
  }
  {
    // the kept keys in tile order (the scan's barriers ordered all reads
    // of the loaded tile before these writes)
    uint32_t pos = toff;
#pragma unroll
    for (int i = 0; i < KPT; ++i)
      if ((flags >> i) & 1u) s_buf[swz(pos++)] = k[i];
  }
  if (tid < 32) {
    bool bad;
    const uint64_t excl = lookback_warp(status, tile, tile_cnt, ctrl, &bad, true);
    if (tid == 0) {
      s_excl = (uint32_t)excl;
      s_abort = bad ? 1u : 0u;
      if (!bad && tile_base + TILE >= m_in) ctrl->m = (uint32_t)(excl + tile_cnt);  // last tile
    }
  }
  __syncthreads();
  if (s_abort) return;  // the tile's place in the output is unknown
  const uint32_t base = s_excl;
  for (uint32_t j = tid; j < tile_cnt; j += kOrientThreads)
    __stcs(reinterpret_cast<unsigned long long *>(okeys) + base + j,
           (unsigned long long)s_buf[swz(j)]);
  __syncthreads();
  for (int i = tid; i < passes2 * 256; i += kOrientThreads)
    if (s_hist[i]) atomicAdd(&hist2[i], s_hist[i]);
}

// ---------------------------------------------------------------------------
// offsets: exclusive scan of per-vertex counts.  Used for the node array
// (counts = out-degrees), for the node array of the padded column array
// (counts = out-degrees rounded up to whole 32-byte blocks, in 16-byte words) and for
// the partner groups of the counting phase (counts = partners per group),
// where it also bins the groups that can hold a triangle (>= 1 partner,
// >= 2 entries in the hashed list) by the length of the hashed list: one
// warp, or a whole CTA.
// ---------------------------------------------------------------------------
enum { kScanPlain = 0, kScanGroups = 1, kScanWords = 2, kScanRecount = 3 };

template <int KIND>
__global__ void __launch_bounds__(kScanThreads)
k_offsets(const int32_t *__restrict__ counts, int32_t n, int32_t *__restrict__ off,
          const int32_t *__restrict__ row_off, int32_t *__restrict__ warp_list,
          int32_t *__restrict__ cta_list, int32_t *__restrict__ big_list, Tuning tune,
          unsigned long long *status, uint32_t *ticket, Ctrl *ctrl, uint32_t shard,
          uint32_t shards) {
  constexpr int IPT = kScanItemsPerThread, TILE = kScanTile;
  __shared__ uint32_t s_scratch[32];
  __shared__ uint32_t s_tile, s_excl, s_abort;
  const int tid = threadIdx.x, lane = tid & 31;
  // the recount of the node array is needed only when a list held repeats
  // (uniform for the grid: set by the list sort, before this launch)
  if (KIND == kScanRecount && *(volatile const uint32_t *)&ctrl->dups == 0u) return;
  if (tid == 0) {
    s_tile = atomicAdd(ticket, 1u);
    s_abort = aborted(ctrl) ? 1u : 0u;
  }
  __syncthreads();
  const uint32_t tile = s_tile;
  if (s_abort) {  // an earlier wait of this call ran out
    if (tid == 0) poison_tile(status, tile);
    return;
  }
  const uint32_t items = (uint32_t)n + 1;  // off[0..n]
  const uint32_t tile_base = tile * (uint32_t)TILE;
  if (tile_base >= items) return;
  const uint32_t first = tile_base + (uint32_t)tid * IPT;
  int32_t d[IPT];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t v = first + i;
    d[i] = v < (uint32_t)n ? __ldg(counts + v) : 0;
    if (KIND == kScanWords) d[i] = ((d[i] + 7) >> 3) << 1;
    sum += (uint32_t)d[i];
  }
  uint32_t tile_sum;
  const uint32_t toff = block_scan_exclusive<kScanThreads>(sum, s_scratch, &tile_sum);
  if (tid < 32) {
    bool bad;
    const uint32_t excl = (uint32_t)lookback_warp(status, tile, tile_sum, ctrl, &bad);
    if (tid == 0) {
      s_excl = excl;
      s_abort = bad ? 1u : 0u;
    }
  }
  __syncthreads();
  if (s_abort) return;  // the tile's prefix is unknown
  uint32_t run = s_excl + toff;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t v = first + i;
    if (v < items) off[v] = (int32_t)run;
    if (KIND == kScanRecount && v == (uint32_t)n) ctrl->m = run;  // edges left
    run += (uint32_t)d[i];
  }
  if constexpr (KIND == kScanGroups) {
  // bin groups: one appending atomic per warp and list
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t v = first + i;
    int32_t dh = 0;
    if (v < (uint32_t)n && d[i] > 0 && v % shards == shard)
      dh = __ldg(row_off + v + 1) - __ldg(row_off + v);
    // a warp takes a group only if both its list and its partner count are
    // short: one warp streaming thousands of partners would finish last
    const bool is_warp = dh >= 2 && dh <= tune.warp_max_list && d[i] <= tune.warp_max_partners;
    const bool is_cta = dh >= 2 && dh <= kCtaMaxRow && !is_warp;
    const bool is_big = dh > kCtaMaxRow;
    const uint32_t bw = __ballot_sync(kFull, is_warp), bc = __ballot_sync(kFull, is_cta);
    const uint32_t bb = __ballot_sync(kFull, is_big);
    uint32_t basew = 0, basec = 0, baseb = 0;
    if (lane == 0) {
      if (bw) basew = atomicAdd(&ctrl->n_warp_groups, (uint32_t)__popc(bw));
      if (bc) basec = atomicAdd(&ctrl->n_cta_groups, (uint32_t)__popc(bc));
      if (bb) baseb = atomicAdd(&ctrl->n_big_groups, (uint32_t)__popc(bb));
    }
    basew = __shfl_sync(kFull, basew, 0);
    basec = __shfl_sync(kFull, basec, 0);
    baseb = __shfl_sync(kFull, baseb, 0);
    const uint32_t lt = (1u << lane) - 1u;
    if (is_warp) warp_list[basew + __popc(bw & lt)] = (int32_t)v;
    if (is_cta) cta_list[basec + __popc(bc & lt)] = (int32_t)v;
    if (is_big) big_list[baseb + __popc(bb & lt)] = (int32_t)v;
  }
  }
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

}  // namespace

cudaError_t set_wait_hooks(uint32_t spin_limit, uint32_t unpublished_tile) {
  cudaError_t e = cudaMemcpyToSymbol(g_spin_limit, &spin_limit, sizeof(spin_limit));
  if (e == cudaSuccess)
    e = cudaMemcpyToSymbol(g_unpublished_tile, &unpublished_tile, sizeof(unpublished_tile));
  return e;
}

void launch_canon(const int32_t *src, const int32_t *dst, uint32_t m_in, int32_t n, int b,
                  const BatchDesc *batch, uint64_t *keys, int32_t *deg, Ctrl *ctrl,
                  cudaStream_t st) {
  // many pairs in flight: the degree atomics wait on L2
  const uint32_t want = (m_in + kCanonThreads * 8 - 1) / (kCanonThreads * 8);
  const uint32_t cap = (uint32_t)num_sms() * 32;
  const uint32_t grid = max(1u, min(want, cap));
  k_canon<<<grid, kCanonThreads, 0, st>>>(src, dst, m_in, n, b, batch, keys, deg, ctrl);
  note_launch();
}

void launch_radix_pass(const uint64_t *in, void *out, RadixOut mode, uint32_t *row_out,
                       int32_t *outdeg, uint32_t n_keys_bound, const uint32_t *n_keys_dev,
                       int shift, uint32_t col_mask, int owner_shift, const uint32_t *hist,
                       unsigned long long *status, uint32_t *ticket, Ctrl *ctrl,
                       cudaStream_t st, bool unstable) {
  const uint32_t grid = max(1u, (n_keys_bound + kSortTile - 1) / kSortTile);
  if (mode == kOutPartSkip)
    k_radix_pass<kOutPartSkip><<<grid, kSortThreads, 0, st>>>(
        in, out, n_keys_bound, n_keys_dev, shift, col_mask, row_out, owner_shift, outdeg, hist,
        status, ticket, ctrl, 0);
  else if (mode == kOutColRow)
    k_radix_pass<kOutColRow><<<grid, kSortThreads, 0, st>>>(
        in, out, n_keys_bound, n_keys_dev, shift, col_mask, row_out, owner_shift, outdeg, hist,
        status, ticket, ctrl, 0);
  else if (mode == kOutRank)
    k_radix_pass<kOutRank><<<grid, kSortThreads, 0, st>>>(in, out, n_keys_bound, n_keys_dev,
                                                          shift, col_mask, nullptr, 0, nullptr,
                                                          hist, status, ticket, ctrl, 0);
  else
    k_radix_pass<kOutKeys><<<grid, kSortThreads, 0, st>>>(in, out, n_keys_bound, n_keys_dev,
                                                          shift, col_mask, nullptr, 0, nullptr,
                                                          hist, status, ticket, ctrl,
                                                          unstable ? 1 : 0);
  note_launch();
}

void launch_rank_keys(const int32_t *deg, int32_t n, int b, int passes, uint64_t *vkeys,
                      uint32_t *hist, cudaStream_t st) {
  const uint32_t want = ((uint32_t)n + kCanonThreads * 8 - 1) / (kCanonThreads * 8);
  const uint32_t grid = max(1u, min(want, (uint32_t)num_sms() * 8));
  k_rank_keys<<<grid, kCanonThreads, 0, st>>>(deg, n, b, passes, vkeys, hist);
  note_launch();
}

void launch_orient(const uint64_t *keys, uint32_t m_in, int b, const int32_t *rank,
                   uint64_t *okeys, uint32_t *hist2, int passes2, unsigned long long *status,
                   Ctrl *ctrl, cudaStream_t st) {
  const uint32_t grid = max(1u, (m_in + kOrientTile - 1) / kOrientTile);
  k_orient<<<grid, kOrientThreads, 0, st>>>(keys, b, rank, okeys, hist2, passes2, status, ctrl);
  note_launch();
}

void launch_offsets(const int32_t *counts, int32_t n, int32_t *off, const int32_t *row_off,
                    int32_t *warp_list, int32_t *cta_list, int32_t *big_list, Tuning tune,
                    unsigned long long *status, uint32_t *ticket, Ctrl *ctrl, cudaStream_t st,
                    int32_t shard, int32_t shards) {
  const uint32_t items = (uint32_t)n + 1;
  const uint32_t grid = max(1u, (items + kScanTile - 1) / kScanTile);
  tune.warp_max_list = min(max(tune.warp_max_list, 0), kWarpMaxRow);  // warp table capacity
  if (row_off)
    k_offsets<kScanGroups><<<grid, kScanThreads, 0, st>>>(counts, n, off, row_off, warp_list,
                                                          cta_list, big_list, tune, status,
                                                          ticket, ctrl, (uint32_t)shard,
                                                          (uint32_t)shards);
  else
    k_offsets<kScanPlain><<<grid, kScanThreads, 0, st>>>(counts, n, off, nullptr, nullptr,
                                                         nullptr, nullptr, tune, status, ticket,
                                                         ctrl, 0u, 1u);
  note_launch();
}

void launch_recount(const int32_t *counts, int32_t n, int32_t *off, unsigned long long *status,
                    uint32_t *ticket, Ctrl *ctrl, cudaStream_t st) {
  const uint32_t items = (uint32_t)n + 1;
  const uint32_t grid = max(1u, (items + kScanTile - 1) / kScanTile);
  k_offsets<kScanRecount><<<grid, kScanThreads, 0, st>>>(counts, n, off, nullptr, nullptr,
                                                         nullptr, nullptr, kDefaultTuning, status,
                                                         ticket, ctrl, 0u, 1u);
  note_launch();
}

void launch_word_offsets(const int32_t *counts, int32_t n, int32_t *voff,
                         unsigned long long *status, uint32_t *ticket, Ctrl *ctrl,
                         cudaStream_t st) {
  const uint32_t items = (uint32_t)n + 1;
  const uint32_t grid = max(1u, (items + kScanTile - 1) / kScanTile);
  k_offsets<kScanWords><<<grid, kScanThreads, 0, st>>>(counts, n, voff, nullptr, nullptr,
                                                       nullptr, nullptr, kDefaultTuning, status,
                                                       ticket, ctrl, 0u, 1u);
  note_launch();
}

}  // namespace tc
