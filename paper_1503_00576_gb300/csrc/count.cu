// count.cu -- counting phase of the forward algorithm on sm_103a.
//
// Sec. III-C of the paper counts with one thread per forward edge (u, v),
// each running a two-pointer merge of N+(u) and N+(v) from global memory,
// and then sums the per-thread counts (thrust::reduce).  The result is the
// sum over forward edges of |N+(u) & N+(v)|.  Here the same sum is computed
// over the partner groups built in group.cu (group h: the edges whose
// longer forward list is N+(h); partners l: their other endpoints):
//
//  * N+(h) is staged once in shared memory as an open-addressing hash set
//    (multiplicative hashing, linear probing, load <= 1/32 where it fits),
//    by one warp when the group is small, else by a whole CTA whose warps
//    claim chunks of partners from a shared counter;
//  * the lists N+(l) of a chunk of <= 32 partners are read as one flat
//    sequence of aligned 32-byte blocks of the padded column array (each
//    list padded with -1 to whole blocks, group.cu): lane p takes block p of
//    each window of 32 blocks (one 32-byte load; the warp reads 1 KB),
//    finds the block's list by a warp vote over the list ends, and loads
//    kWindows / 2 blocks before it probes any;
//  * counts stay in registers and are reduced per warp (shuffles) into one
//    uint64 atomic per warp at the end (the paper's reduction, fused).
//
// Per-vertex counts t(v) (Sec. I: the numerator of the clustering
// coefficient): a triangle found in group h, partner l, element w adds one
// to t(h), t(l) and t(w).  t(h) is summed over the group, t(l) per block
// (shared counters per partner) and t(w) in a counter beside w's hash slot,
// so global atomics scale with the number of forward edges, not with the
// number of triangles.
//
// A hashed list longer than half the table (never seen in the workloads,
// but allowed by |N+(v)| <= sqrt(2m)) is hashed in segments.  No step needs
// the lists in sorted order: membership is by hashing, not by merging.
#include "tc_common.cuh"

namespace tc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGroupChunk = 8;  // warp groups per atomic
constexpr int kMinChunk = 8;    // fewest partners a warp of a CTA group claims
constexpr int kWindows = 4;     // 16-byte words per lane loaded before probing (two blocks)
constexpr int kBigWindows = 4;  // ... in the long-list kernel

// Main kernel: 256-thread CTAs; one table per CTA for CTA groups (lists of
// up to kCtaMaxRow entries), carved into one table per warp for warp
// groups.  Per-vertex mode adds a 32-bit counter per slot, and 6144 slots
// keep four CTAs on an SM.
constexpr int kMainThreads = 256;
constexpr int kMainWarps = kMainThreads / 32;
constexpr int kMainMinBlocks = 4;  // 64 registers per thread
template <bool PV> __host__ __device__ constexpr int main_slots() { return PV ? 6144 : 8192; }
// Long-list kernel: 512-thread CTAs, 8192 slots (lists up to 4096 entries
// at once; longer lists in segments).
constexpr int kBigThreads = 512;
constexpr int kBigWarps = kBigThreads / 32;
constexpr int kBigSlots = 8192;
constexpr int kBigMinBlocks = 2;
static_assert(main_slots<true>() >= 4 * kCtaMaxRow, "CTA lists must fit at load <= 1/4");
static_assert(main_slots<true>() / kMainWarps >= 4 * kWarpMaxRow,
              "warp lists must fit at load <= 1/4");

// Hash-set slots.  Ids are < 2^31 - 1, so 0x7fffffff marks an empty slot and
// bit 31 of an occupied slot records that some key whose home is this slot
// was displaced further along (linear probing).  A lookup whose home slot is
// neither the key nor flagged is a miss after one read: about a^2 / 2 of the
// slots are flagged at load a (0.05% at 1/32, 1.4% at the load 1/6 of the
// longest lists of a table).  The padding id -1 never matches: a slot's
// low 31 bits are non-negative.
constexpr int32_t kEmpty = 0x7fffffff;
constexpr uint32_t kDisplaced = 0x80000000u;
constexpr uint32_t kHashMul = 0x9E3779B1u;

// Home slot of x in a table of `slots` slots (any size): the high word of
// the multiplicative hash scaled to the table.
__device__ __forceinline__ uint32_t hash_slot(uint32_t x, uint32_t slots) {
  return __umulhi(x * kHashMul, slots);
}

__device__ __forceinline__ uint32_t next_slot(uint32_t h, uint32_t slots) {
  return h + 1u == slots ? 0u : h + 1u;
}

// Table size for a list of len entries: load 1/32 where it fits, else the
// whole capacity (callers keep len <= capacity / 2).  A lower load flags
// fewer home slots (misses there probe on); emptying costs in proportion to
// the list, not to the table (measured against load 1/16 at R-MAT scale 24:
// -0.4 ms total-only, -0.15 ms per vertex).
__device__ __forceinline__ uint32_t table_slots(int32_t len, uint32_t capacity) {
  return min(32u * (uint32_t)max(len, 1), capacity);
}

// Read-only view of the forward lists and partner groups.
struct Lists {
  const int32_t *__restrict__ off;   // node array (rank space): list lengths
  const int32_t *__restrict__ voff;  // node array of col4, in 16-byte words (even)
  const int32_t *__restrict__ col4;  // forward lists, sorted, each padded with -1 to whole 32-byte blocks
  const int32_t *__restrict__ goff;  // partner-group offsets
  const int32_t *__restrict__ part;   // partners
  const int32_t *__restrict__ pskip;  // per partner: leading blocks of its list skipped
  const int2 *__restrict__ desc;      // per-vertex mode, per partner: its stream
                                      //   {first col4 word, entries} (k_stream_desc)
  const int2 *__restrict__ ldesc;     // per vertex: its list {voff[v], d+(v)}, one
                                      //   8-byte gather instead of three 4-byte ones
};

// One hash set in shared memory.
struct Table {
  int32_t *tab;      // slots
  uint32_t *cnt;     // per-vertex mode: match counter of each slot
  uint32_t cnt_sa;   // shared-window address of cnt
  uint32_t slots;    // size in use
};

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ uint32_t shared_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Adds v to the shared word at saddr when c holds (predicated, no branch).
__device__ __forceinline__ void red_add_if(uint32_t saddr, uint32_t v, bool c) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t@p red.shared.add.u32 [%0], %1;\n\t}"
      ::"r"(saddr), "r"(v), "r"((uint32_t)c));
}

// Per-warp description of the chunk being probed: the non-empty partner
// lists r = 0 .. k-1 in flat order.
struct WarpScratch {
  union {
    int2 bn[32];  // block mode: {col4 word of flat position 0 of list r, flat start of r+1}
    struct {
      long long eb[32];   // element mode: col4 element of flat position 0 of list r
      int32_t enext[32];  // element mode: flat start of list r+1
    };
  };
  int32_t l[32];    // the partner owning list r (per-vertex mode)
  uint32_t lc[32];  // triangles found through that partner
};

// Empties tab[0..slots) and the counters.
template <bool PV>
__device__ __forceinline__ void clear_table(int32_t *tab, uint32_t *cnt, int slots, int rank,
                                            int group) {
  for (int i = rank; i < slots; i += group) {
    tab[i] = kEmpty;
    if (PV) cnt[i] = 0u;
  }
}

// Inserts list[0..len) (distinct ids) into the empty hash set; the slot of
// list[i] goes to slot_of[i].
__device__ __forceinline__ void fill_table(const int32_t *__restrict__ list, int32_t len,
                                           const Table &tb, uint16_t *slot_of, int rank,
                                           int group) {
  for (int32_t i = rank; i < len; i += group) {
    const int32_t x = __ldg(list + i);
    const uint32_t home = hash_slot((uint32_t)x, tb.slots);
    uint32_t h = home;
    for (;;) {
      const int32_t old = atomicCAS(&tb.tab[h], kEmpty, x);
      if (old == kEmpty) break;
      if (h == home && !((uint32_t)old & kDisplaced))
        atomicOr((unsigned *)&tb.tab[h], kDisplaced);
      h = next_slot(h, tb.slots);
    }
    slot_of[i] = (uint16_t)h;
  }
}

// Per-vertex mode: adds the counter of each of the len filled slots to t(w)
// of its key and zeroes it.
__device__ __forceinline__ void flush_counts(const Table &tb, const uint16_t *slot_of,
                                             int32_t len, int rank, int group, int64_t *t) {
  for (int32_t i = rank; i < len; i += group) {
    const uint32_t s = slot_of[i];
    const uint32_t c = tb.cnt[s];
    if (c) {
      atomicAdd((unsigned long long *)&t[tb.tab[s] & 0x7fffffff], (unsigned long long)c);
      tb.cnt[s] = 0u;
    }
  }
}

// Empties the len filled slots again (work in proportion to the list, not
// to the table).
__device__ __forceinline__ void empty_table(const Table &tb, const uint16_t *slot_of,
                                            int32_t len, int rank, int group) {
  for (int32_t i = rank; i < len; i += group) tb.tab[slot_of[i]] = kEmpty;
}

// Slot of x along the probe sequence after its flagged home slot h, or -1.
__device__ __forceinline__ int32_t probe_past(int32_t x, uint32_t h, const Table &tb) {
  for (;;) {
    h = next_slot(h, tb.slots);
    const int32_t y = tb.tab[h];
    if ((y & 0x7fffffff) == x) return (int32_t)h;
    if (y == kEmpty) return -1;
  }
}

// Looks up N entries.  Each lookup reads its home slot; only a miss at a
// flagged home slot probes on (the rare part).  Per-vertex mode bumps the
// counter beside each matched slot (t(w)).  Returns the number of matches.
//
// Per-vertex mode, N = 8 (block mode; all 32 lanes call it together): the
// misses at flagged home slots are gathered in a mask over the 8 entries and
// probed on in a warp-uniform loop, one per lane and round, so the rare part
// costs rounds in proportion to the most such misses in one lane (usually
// one), instead of a divergent branch per entry that nearly every window
// took (a window makes 256 lookups, so a flag rate of even 0.1% reaches
// most windows).  Measured at R-MAT scale 24: -1.2 ms per vertex, +0.4 ms
// without counters, so the total-only count keeps the branches.  N = 1
// (element mode; lanes may have left): the plain test.
template <bool PV, int N>
__device__ __forceinline__ uint32_t lookup(const int32_t (&x)[N], const Table &tb) {
  uint32_t h[N];
  int32_t y[N];
#pragma unroll
  for (int i = 0; i < N; ++i) h[i] = hash_slot((uint32_t)x[i], tb.slots);
#pragma unroll
  for (int i = 0; i < N; ++i) y[i] = tb.tab[h[i]];
  uint32_t hits = 0;
  if constexpr (PV && N == 8) {
    uint32_t fm = 0;  // bit i: entry i missed at a flagged home slot
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const bool mi = (y[i] & 0x7fffffff) == x[i];
      if (PV) red_add_if(tb.cnt_sa + 4u * h[i], 1u, mi);  // the counter beside the match
      hits += mi ? 1u : 0u;
      fm |= (uint32_t)(!mi && y[i] < 0) << i;
    }
    while (__any_sync(kFull, fm != 0u)) {
      if (fm) {
        const int i = __ffs(fm) - 1;
        fm &= fm - 1;
        int32_t xi = x[0];
        uint32_t hi = h[0];
#pragma unroll
        for (int j = 1; j < N; ++j) {
          xi = i == j ? x[j] : xi;
          hi = i == j ? h[j] : hi;
        }
        const int32_t slot = probe_past(xi, hi, tb);
        if (slot >= 0) {
          if (PV) red_add_if(tb.cnt_sa + 4u * (uint32_t)slot, 1u, true);
          ++hits;
        }
      }
    }
  } else {
    bool m[N];
    int32_t flagged = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      m[i] = (y[i] & 0x7fffffff) == x[i];
      flagged |= y[i];
    }
    if constexpr (PV) {
      if (flagged < 0) {  // some home slot is flagged: misses there probe on
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (!m[i] && y[i] < 0) {
            const int32_t slot = probe_past(x[i], h[i], tb);
            m[i] = slot >= 0;
            h[i] = (uint32_t)slot;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        red_add_if(tb.cnt_sa + 4u * h[i], 1u, m[i]);  // the counter beside the match
        hits += m[i] ? 1u : 0u;
      }
    } else {
      // without counters the slow path only counts: m and h need not change
      if (flagged < 0) {
#pragma unroll
        for (int i = 0; i < N; ++i)
          if (!m[i] && y[i] < 0) hits += probe_past(x[i], h[i], tb) >= 0 ? 1u : 0u;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) hits += m[i] ? 1u : 0u;
    }
  }
  return hits;
}

// Inclusive warp scan of one int32 per lane.
__device__ __forceinline__ int32_t warp_incl_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// One 32-byte block (two words) of col4 at 16-byte word a (even).
__device__ __forceinline__ void ld_block(const int32_t *col4, int32_t a, int32_t (&x)[8]) {
  asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]),
        "=r"(x[7])
      : "l"(col4 + 4 * (size_t)a));
}

// Block mode of probe_chunk: windows w .. w+NQ-1 of 32 blocks (64 words) of
// the chunk's flat sequence, lane p taking block p of each.  Lists occupy
// whole blocks, so a block lies in one list: the number of lists ending at
// or before it, i.e. those ending at or before the window (one vote) plus
// those whose last block lies in the window before this lane's (a bit mask
// OR-reduced over the lanes).  Lane r holds list r's {base, end} in bn_r.
// TAIL: the window reaches past total_v, and the blocks beyond it are -1.
template <bool PV, int NQ, bool TAIL>
__device__ __forceinline__ void probe_windows(const Lists &g, int32_t w, int32_t total_v,
                                              int2 bn_r, const Table &tb, uint32_t lc_sa,
                                              uint32_t &found) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int32_t x[NQ][8];
  int rq[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int32_t P = 64 * (w + q);
    const int c0 = __popc(__ballot_sync(kFull, bn_r.y <= P));
    const uint32_t o = (uint32_t)(bn_r.y - P - 2) >> 1;  // list r's last block in the window
    const uint32_t ends = __reduce_or_sync(kFull, o < 31u ? 1u << o : 0u);
    const int r = c0 + __popc(ends & lt);
    const int32_t a = __shfl_sync(kFull, bn_r.x, r & 31) + P + 2 * lane;
    if (TAIL) {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[q][i] = -1;
      if (P + 2 * lane < total_v) ld_block(g.col4, a, x[q]);
    } else {
      ld_block(g.col4, a, x[q]);
    }
    rq[q] = r;
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const uint32_t hits = lookup<PV, 8>(x[q], tb);
    found += hits;
    if (PV) red_add_if(lc_sa + 4u * (uint32_t)rq[q], hits, hits != 0u);
  }
}

// Streams N+(l) for the partners l = part[c0 .. c0+cs) (of np, cs <= 32)
// through the hash set of the group's list.  The chunk's non-empty lists
// are concatenated into one flat sequence.  Two granularities, chosen per
// chunk by which needs fewer warp steps:
//  * blocks: a position is one aligned 32-byte block of the padded column
//    array, eight entries probed per load; padding entries are -1 and never
//    match.  Lane p takes block p of each 32-block window (coalesced
//    loads); the list of each block comes from a warp vote over the list
//    ends, with no per-lane cursor and no branch;
//  * elements: a position is one list entry (one 4-byte load); lane p takes
//    positions p, p+32, ... with a cursor on the list holding its position.
//    For chunks of a few short lists, where whole blocks would be mostly
//    padding.
// Matches are counted in registers; per partner they go to a shared counter
// (per block, or when an element-mode lane leaves the partner's list), per w
// to the counter beside w's slot.
template <bool PV, int W>
__device__ __forceinline__ void probe_chunk(const Lists &g, const int32_t *__restrict__ part,
                                            const int32_t *__restrict__ pskip,
                                            const int2 *__restrict__ desc, int32_t np,
                                            int32_t c0, int32_t cs, const Table &tb,
                                            WarpScratch &ws, int64_t *t, uint64_t &found_total,
                                            uint64_t &found_group) {
  const int lane = threadIdx.x & 31;
  const int32_t j = c0 + lane;
  int32_t l = 0, dl = 0, vb = 0;
  if (lane < cs && j < np) {
    l = __ldg(part + j);
    if (PV) {
      // the partner's stream, written before the counting (k_stream_desc):
      // no gathers in the chunk's set-up, whose registers the per-vertex
      // counters need (measured: 1.6 ms of 31 at R-MAT scale 24; without
      // counters the separate pass costs more than it saves)
      const int2 ds = __ldg(desc + j);
      vb = ds.x;
      dl = ds.y;
    } else {
      const int32_t skip = __ldg(pskip + j);
      const int2 ld = __ldg(g.ldesc + l);
      dl = ld.y;
      vb = ld.x;
      // the leading blocks of N+(l) below the hashed list's smallest id
      // cannot meet it: stream from the first block that can
      vb += 2 * skip;
      dl = max(dl - 8 * skip, 0);
    }
  }
  const uint32_t nonempty = __ballot_sync(kFull, dl > 0);
  if (nonempty == 0) return;
  const int k = __popc(nonempty);
  const int rank = __popc(nonempty & ((1u << lane) - 1u));
  const int32_t nv = ((dl + 7) >> 3) << 1;  // 16-byte words: whole 32-byte blocks
  const int32_t incl_e = warp_incl_scan(dl);
  const int32_t incl_v = warp_incl_scan(nv);
  const int32_t total_e = __shfl_sync(kFull, incl_e, 31);
  const int32_t total_v = __shfl_sync(kFull, incl_v, 31);
  // a block step probes eight entries, an element step one: cost ~4:1
  // (measured: 4 beats 5 and 7 on R-MAT and random geometric graphs)
  const bool blocks = 4 * ((total_v + 63) >> 6) < ((total_e + 31) >> 5);
  // list r+1 starts where list r ends (empty lists add nothing to the scans)
  const bool last = rank == k - 1;
  if (dl > 0) {
    if (blocks) {
      ws.bn[rank] = make_int2(vb - (incl_v - nv), last ? INT32_MAX : incl_v);
    } else {
      ws.eb[rank] = 4ll * vb - (incl_e - dl);
      ws.enext[rank] = last ? INT32_MAX : incl_e;
    }
    if (PV) {
      ws.l[rank] = l;
      ws.lc[rank] = 0u;
    }
  }
  __syncwarp();
  uint32_t found = 0;  // matches of this lane in this chunk
  uint32_t run = 0;    // matches of this lane in list run_r not yet in ws.lc
  int run_r = 0;
  const uint32_t lc_sa = shared_addr(ws.lc);
  if (blocks) {
    // lane r holds list r's base and end (flat start of list r+1)
    const int2 bn_r = lane < k ? ws.bn[lane] : make_int2(0, INT32_MAX);
    const int32_t full = total_v >> 6;  // windows of 64 words inside the sequence
    constexpr int NQ = W / 2;           // windows per step: W words per lane in flight
    int32_t w = 0;
    for (; w + NQ <= full; w += NQ)
      probe_windows<PV, NQ, false>(g, w, total_v, bn_r, tb, lc_sa, found);
    for (; w < full; ++w) probe_windows<PV, 1, false>(g, w, total_v, bn_r, tb, lc_sa, found);
    if (total_v & 63) probe_windows<PV, 1, true>(g, w, total_v, bn_r, tb, lc_sa, found);
  } else {
    int r = 0;
    long long eb = ws.eb[0];
    int32_t next = ws.enext[0];
    for (int32_t p0 = lane; p0 < total_e; p0 += 32 * W) {
      int32_t x[W];
      int rq[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int32_t p = p0 + 32 * q;
        x[q] = -1;
        if (p < total_e) {
          while (p >= next) {
            ++r;
            eb = ws.eb[r];
            next = ws.enext[r];
          }
          x[q] = __ldg(g.col4 + (eb + p));
        }
        rq[q] = r;
      }
#pragma unroll
      for (int q = 0; q < W; ++q) {
        const int32_t e[1] = {x[q]};
        const uint32_t hits = lookup<PV, 1>(e, tb);
        found += hits;
        if (PV) {
          if (rq[q] != run_r) {
            red_add_if(lc_sa + 4u * run_r, run, run != 0);
            run = 0;
            run_r = rq[q];
          }
          run += hits;
        }
      }
    }
  }
  found_total += found;
  found_group += found;
  if (PV) {
    red_add_if(lc_sa + 4u * run_r, run, run != 0);
    __syncwarp();
    if (lane < k && ws.lc[lane])
      atomicAdd((unsigned long long *)&t[ws.l[lane]], (unsigned long long)ws.lc[lane]);
  }
  __syncwarp();
}

struct CtaShared {
  int32_t group;
  uint32_t chunk;
  unsigned long long groupsum;
};

// Groups of `list` counted by the whole CTA: N+(h) hashed once, warps claim
// chunks of partners, each a share of the partners left (at most 32), so
// that the warps run out of work together.  A list longer than half the table is hashed
// in equal segments, one after another, each probed by all partners:
// N+(h) & N+(l) is the disjoint union of the segments' intersections.  The
// table (SLOTS slots) is empty on entry and on exit.
template <bool PV, int THREADS, int SLOTS, int W>
__device__ __forceinline__ void cta_groups(const Lists &g, const int32_t *__restrict__ list,
                                           uint32_t n_list, uint32_t *cursor, Table tb,
                                           uint16_t *slot_of, WarpScratch *s_ws, CtaShared &sh,
                                           int64_t *t, int64_t *tg, uint64_t &found_total) {
  constexpr int WARPS = THREADS / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) {
      sh.group = (int32_t)atomicAdd(cursor, 1u);
      sh.groupsum = 0ull;
    }
    __syncthreads();  // also orders the previous group's drain before this fill
    const uint32_t gi = (uint32_t)sh.group;
    if (gi >= n_list) break;
    // lists are filled in about ascending rank, and high ranks (high
    // degrees) carry the most work: take them first to shorten the tail
    const int32_t h = __ldg(list + (n_list - 1 - gi));
    const int2 hld = __ldg(g.ldesc + h);
    const int32_t hd = hld.y;
    const int32_t *hl = g.col4 + 4 * (size_t)hld.x;
    const int32_t pb = __ldg(g.goff + h), np = __ldg(g.goff + h + 1) - pb;
    const int32_t nseg = (hd + SLOTS / 2 - 1) / (SLOTS / 2);
    const int32_t seg_len = (hd + nseg - 1) / nseg;
    tb.slots = table_slots(seg_len, SLOTS);
    uint64_t found_group = 0;
    for (int32_t s0 = 0; s0 < hd; s0 += seg_len) {
      const int32_t len = min(seg_len, hd - s0);
      if (tid == 0) sh.chunk = 0u;
      fill_table(hl + s0, len, tb, slot_of, tid, THREADS);
      __syncthreads();
      for (;;) {
        // guided chunks: a share of what is left, so that the warps finish
        // the group together (32 partners at most, 8 at least)
        uint32_t c = 0, cs = 0;
        if (lane == 0) {
          const int32_t left = np - (int32_t)*(volatile uint32_t *)&sh.chunk;
          cs = (uint32_t)max(kMinChunk, min(32, left / (2 * WARPS)));
          c = atomicAdd(&sh.chunk, cs);
        }
        c = __shfl_sync(kFull, c, 0);
        cs = __shfl_sync(kFull, cs, 0);
        if ((int32_t)c >= np) break;
        probe_chunk<PV, W>(g, g.part + pb, g.pskip + pb, g.desc + pb, np, (int32_t)c, (int32_t)cs, tb, s_ws[warp],
                           t, found_total, found_group);
      }
      __syncthreads();
      if (PV) {
        flush_counts(tb, slot_of, len, tid, THREADS, t);
        __syncthreads();  // flushes read keys from the slots emptied next
      }
      empty_table(tb, slot_of, len, tid, THREADS);
      if (s0 + seg_len < hd) __syncthreads();  // next segment refills the table
    }
    if (PV || tg) {
      found_group = warp_sum_u64(found_group);
      if (lane == 0 && found_group) atomicAdd(&sh.groupsum, (unsigned long long)found_group);
    }
    __syncthreads();
    // t(h) gains every triangle of the group; so does the group total
    if (tid == 0 && sh.groupsum) {
      if (PV) atomicAdd((unsigned long long *)&t[h], sh.groupsum);
      else if (tg) atomicAdd((unsigned long long *)&tg[h], sh.groupsum);
    }
  }
}

// Groups of `list` counted by one warp each with a private table of
// WSLOTS slots (empty on entry and on exit).
template <bool PV, int WSLOTS>
__device__ __forceinline__ void warp_groups(const Lists &g, const int32_t *__restrict__ list,
                                            uint32_t n_list, uint32_t *cursor, Table tb,
                                            uint16_t *slot_of, WarpScratch &ws, int64_t *t,
                                            int64_t *tg, uint64_t &found_total) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    uint32_t g0 = 0;
    if (lane == 0) g0 = atomicAdd(cursor, (uint32_t)kGroupChunk);
    g0 = __shfl_sync(kFull, g0, 0);
    if (g0 >= n_list) break;
    const uint32_t g1 = min(g0 + (uint32_t)kGroupChunk, n_list);
    for (uint32_t gi = g0; gi < g1; ++gi) {
      const int32_t h = __ldg(list + (n_list - 1 - gi));  // heavy (high-rank) groups first
      const int2 hld = __ldg(g.ldesc + h);
      const int32_t hd = hld.y;
      const int32_t *hl = g.col4 + 4 * (size_t)hld.x;
      const int32_t pb = __ldg(g.goff + h), np = __ldg(g.goff + h + 1) - pb;
      tb.slots = table_slots(hd, WSLOTS);
      fill_table(hl, hd, tb, slot_of, lane, 32);
      __syncwarp();
      uint64_t found_group = 0;
      for (int32_t c0 = 0; c0 < np; c0 += 32)
        probe_chunk<PV, kWindows>(g, g.part + pb, g.pskip + pb, g.desc + pb, np, c0, 32, tb, ws, t, found_total,
                                  found_group);
      if (PV || tg) {
        found_group = warp_sum_u64(found_group);
        if (lane == 0 && found_group)
          atomicAdd((unsigned long long *)(PV ? &t[h] : &tg[h]), (unsigned long long)found_group);
      }
      __syncwarp();
      if (PV) {
        flush_counts(tb, slot_of, hd, lane, 32, t);
        __syncwarp();
      }
      empty_table(tb, slot_of, hd, lane, 32);
      __syncwarp();
    }
  }
}

// Per-vertex mode: the stream of every partner, so that a chunk's set-up is
// one coalesced load and no gathers.  Partner l of an edge streams N+(l)
// from its first block that can meet the hashed list (the pskip leading
// blocks below it cannot): {col4 word voff[l] + 2 skip, d+(l) - 8 skip
// entries, at least 0}.
__global__ void __launch_bounds__(256)
k_stream_desc(const int32_t *__restrict__ part, const int32_t *__restrict__ pskip,
              const int2 *__restrict__ ldesc, const Ctrl *ctrl, int2 *__restrict__ desc) {
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out
  const uint32_t m = ctrl->m;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t e0 = blockIdx.x * blockDim.x + threadIdx.x; e0 < m; e0 += 4 * stride) {
    int32_t l[4], skip[4];
    int2 ld[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t e = e0 + q * stride;
      l[q] = e < m ? __ldg(part + e) : 0;
      skip[q] = e < m ? __ldg(pskip + e) : 0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) ld[q] = __ldg(ldesc + l[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t e = e0 + q * stride;
      if (e < m) desc[e] = make_int2(ld[q].x + 2 * skip[q], max(ld[q].y - 8 * skip[q], 0));
    }
  }
}

// ldesc[v] = {voff[v], off[v+1] - off[v]}: each list's first col4 word and
// length in one record (after the list sort's recount).
__global__ void __launch_bounds__(256)
k_list_desc(const int32_t *__restrict__ off, const int32_t *__restrict__ voff, int32_t n,
            const Ctrl *ctrl, int2 *__restrict__ ldesc) {
  if (aborted(ctrl)) return;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < (uint32_t)n; v += stride)
    ldesc[v] = make_int2(__ldg(voff + v), __ldg(off + v + 1) - __ldg(off + v));
}

// Dynamic shared memory of the counting kernels: the hash table, the slot
// counters (per-vertex mode) and the slot of every hashed entry.
constexpr size_t table_smem(int slots, int max_len, bool pv) {
  return (size_t)4 * slots * (pv ? 2 : 1) + (size_t)2 * max_len;
}
template <bool PV> constexpr size_t main_smem() {
  return table_smem(main_slots<PV>(), kCtaMaxRow, PV);
}
template <bool PV> constexpr size_t big_smem() { return table_smem(kBigSlots, kBigSlots / 2, PV); }
static_assert(kMainWarps * kWarpMaxRow <= kCtaMaxRow, "warp slot maps must fit the CTA's");

// Main counting kernel: CTA groups first (the heavy ones), then warp groups.
template <bool PV>
__global__ void __launch_bounds__(kMainThreads, kMainMinBlocks)
k_count(Lists g, const int32_t *__restrict__ warp_list, const int32_t *__restrict__ cta_list,
        int32_t n, Ctrl *ctrl, int64_t *t, int64_t *tg) {
  constexpr int SLOTS = main_slots<PV>();
  constexpr int WSLOTS = SLOTS / kMainWarps;
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *s_tab = reinterpret_cast<int32_t *>(smem);
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + 4 * SLOTS);
  uint16_t *s_slot = reinterpret_cast<uint16_t *>(smem + 4 * SLOTS * (PV ? 2 : 1));
  __shared__ WarpScratch s_ws[kMainWarps];
  __shared__ CtaShared s_sh;
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out: the lists are not complete
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  clear_table<PV>(s_tab, s_cnt, SLOTS, tid, kMainThreads);
  uint64_t found_total = 0;
  Table tb{s_tab, s_cnt, shared_addr(s_cnt), SLOTS};
  cta_groups<PV, kMainThreads, SLOTS, kWindows>(g, cta_list, ctrl->n_cta_groups,
                                                &ctrl->next_cta_group, tb, s_slot, s_ws, s_sh,
                                                t, tg, found_total);
  Table wtb{s_tab + warp * WSLOTS, s_cnt + warp * WSLOTS, shared_addr(s_cnt + warp * WSLOTS),
            WSLOTS};
  warp_groups<PV, WSLOTS>(g, warp_list, ctrl->n_warp_groups, &ctrl->next_warp_group, wtb,
                          s_slot + warp * kWarpMaxRow, s_ws[warp], t, tg, found_total);
  found_total = warp_sum_u64(found_total);
  if (lane == 0 && found_total) atomicAdd(&ctrl->total, (unsigned long long)found_total);
}

// Groups whose hashed list is longer than kCtaMaxRow (rare).
template <bool PV>
__global__ void __launch_bounds__(kBigThreads, kBigMinBlocks)
k_count_big(Lists g, const int32_t *__restrict__ big_list, int32_t n, Ctrl *ctrl, int64_t *t,
            int64_t *tg) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *tab = reinterpret_cast<int32_t *>(smem);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + 4 * kBigSlots);
  uint16_t *slot_of = reinterpret_cast<uint16_t *>(smem + 4 * kBigSlots * (PV ? 2 : 1));
  __shared__ WarpScratch s_ws[kBigWarps];
  __shared__ CtaShared s_sh;
  if (aborted(ctrl)) return;  // an earlier wait of this call ran out: the lists are not complete
  const int tid = threadIdx.x, lane = tid & 31;
  clear_table<PV>(tab, cnt, kBigSlots, tid, kBigThreads);
  uint64_t found_total = 0;
  Table tb{tab, cnt, shared_addr(cnt), kBigSlots};
  cta_groups<PV, kBigThreads, kBigSlots, kBigWindows>(g, big_list, ctrl->n_big_groups,
                                                      &ctrl->next_big_group, tb, slot_of, s_ws,
                                                      s_sh, t, tg, found_total);
  found_total = warp_sum_u64(found_total);
  if (lane == 0 && found_total) atomicAdd(&ctrl->total, (unsigned long long)found_total);
}

// ---------------------------------------------------------------------------
// clustering coefficients and the integer sums behind transitivity
// ---------------------------------------------------------------------------
constexpr int kClusterThreads = 256;

__global__ void __launch_bounds__(kClusterThreads)
k_clustering(const int64_t *__restrict__ t, const int32_t *__restrict__ deg, int32_t n,
             double *__restrict__ cc, unsigned long long *sums) {
  unsigned long long st = 0, sw = 0;
  const uint32_t stride = gridDim.x * kClusterThreads;
  for (uint32_t v = blockIdx.x * kClusterThreads + threadIdx.x; v < (uint32_t)n; v += stride) {
    const int64_t tv = __ldg(t + v);
    const int64_t d = __ldg(deg + v);
    if (cc) {
      double c = 0.0;
      if (d >= 2) c = (2.0 * (double)tv) / ((double)d * (double)(d - 1));
      cc[v] = c;
    }
    st += (unsigned long long)tv;
    sw += (unsigned long long)(d * (d - 1) / 2);
  }
  st = warp_sum_u64(st);
  sw = warp_sum_u64(sw);
  if ((threadIdx.x & 31) == 0) {
    if (st) atomicAdd(&sums[0], st);
    if (sw) atomicAdd(&sums[1], sw);
  }
}

// Per-vertex counts from rank space back to the caller's vertex ids.
__global__ void __launch_bounds__(kClusterThreads)
k_gather_counts(const int64_t *__restrict__ t_rank, const int32_t *__restrict__ rank, int32_t n,
                int64_t *__restrict__ t_out, const Ctrl *ctrl) {
  if (aborted(ctrl)) return;  // rank[] may be incomplete
  const uint32_t stride = gridDim.x * kClusterThreads;
  for (uint32_t v = blockIdx.x * kClusterThreads + threadIdx.x; v < (uint32_t)n; v += stride)
    t_out[v] = __ldg(t_rank + __ldg(rank + v));
}

// Per-graph sums over union vertex ranges: one warp per graph.
__global__ void __launch_bounds__(kClusterThreads)
k_segment_sums(const int64_t *__restrict__ vals, const BatchDesc *__restrict__ batch,
               int32_t num_graphs_bound, int32_t divisor, unsigned long long *__restrict__ out) {
  const int32_t ng = batch->num_graphs;
  const int32_t *vo = batch->voff;
  const int lane = threadIdx.x & 31;
  const int32_t warps = gridDim.x * (kClusterThreads / 32);
  for (int32_t gi = (blockIdx.x * kClusterThreads + threadIdx.x) >> 5; gi < num_graphs_bound;
       gi += warps) {
    unsigned long long s = 0;
    if (gi < ng) {
      const int32_t b = __ldg(vo + gi), e = __ldg(vo + gi + 1);
      for (int32_t v = b + lane; v < e; v += 32) s += (unsigned long long)__ldg(vals + v);
    }
    s = warp_sum_u64(s);
    if (lane == 0) {
      unsigned long long r = 0ull;
      if (gi < ng) r = batch->gerr[gi] ? ~0ull : s / (unsigned long long)divisor;
      out[gi] = r;  // ~0: the graph had an id out of range (TC_COUNT_ERROR)
    }
  }
}

// transitivity = 3T / wedges with T = (sum t) / 3: one float64 division.
__global__ void k_transitivity(const unsigned long long *sums, double *out) {
  const unsigned long long three_t = sums[0];  // sum of t(v) is exactly 3T
  const unsigned long long wedges = sums[1];
  out[0] = wedges ? (double)three_t / (double)wedges : 0.0;
}

constexpr int kMaxDevices = 64;

struct CountGrid {
  int main_blocks, big_blocks;
};

template <bool PV>
cudaError_t count_grid_t(int dev, CountGrid *out) {
  cudaError_t e = cudaFuncSetAttribute(k_count<PV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)main_smem<PV>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_count_big<PV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)big_smem<PV>());
  if (e != cudaSuccess) return e;
  int sms = 0, per_main = 0, per_big = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_main, k_count<PV>, kMainThreads,
                                                    main_smem<PV>());
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_big, k_count_big<PV>, kBigThreads,
                                                      big_smem<PV>());
  if (e != cudaSuccess) return e;
  sms = sms > 0 ? sms : 1;
  *out = CountGrid{sms * (per_main > 0 ? per_main : 1), sms * (per_big > 0 ? per_big : 1)};
  return cudaSuccess;
}

cudaError_t count_grid(bool pv, CountGrid *out) {
  static CountGrid cache[kMaxDevices][2];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices && cache[dev][pv].main_blocks) {
    *out = cache[dev][pv];
    return cudaSuccess;
  }
  CountGrid g{};
  e = pv ? count_grid_t<true>(dev, &g) : count_grid_t<false>(dev, &g);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices) cache[dev][pv] = g;
  *out = g;
  return cudaSuccess;
}

}  // namespace

cudaError_t prepare_count_kernels() {
  CountGrid cg;
  cudaError_t e = count_grid(true, &cg);
  if (e == cudaSuccess) e = count_grid(false, &cg);
  return e;
}

cudaError_t launch_count(const int32_t *off, const int32_t *voff, const int2 *ldesc,
                         const int32_t *col4,
                         const int32_t *goff, const int32_t *part, const int32_t *pskip,
                         int2 *desc, const int32_t *warp_groups,
                         const int32_t *cta_groups, const int32_t *big_groups, int32_t n,
                         Ctrl *ctrl, int64_t *t, int64_t *tg, cudaStream_t st) {
  const bool pv = t != nullptr;
  CountGrid cg;
  cudaError_t e = count_grid(pv, &cg);
  if (e != cudaSuccess) return e;
  if (pv) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_stream_desc<<<(sms > 0 ? sms : 1) * 16, 256, 0, st>>>(part, pskip, ldesc, ctrl, desc);
    note_launch();
  }
  const Lists g{off, voff, col4, goff, part, pskip, desc, ldesc};
  // the long lists first, on their own wide CTAs
  if (pv) {
    k_count_big<true><<<cg.big_blocks, kBigThreads, big_smem<true>(), st>>>(g, big_groups, n, ctrl,
                                                                          t, nullptr);
    k_count<true><<<cg.main_blocks, kMainThreads, main_smem<true>(), st>>>(g, warp_groups,
                                                                         cta_groups, n, ctrl, t,
                                                                         nullptr);
  } else {
    k_count_big<false><<<cg.big_blocks, kBigThreads, big_smem<false>(), st>>>(g, big_groups, n,
                                                                            ctrl, nullptr, tg);
    k_count<false><<<cg.main_blocks, kMainThreads, main_smem<false>(), st>>>(g, warp_groups,
                                                                           cta_groups, n, ctrl,
                                                                           nullptr, tg);
  }
  note_launch();
  note_launch();
  return cudaGetLastError();
}

void launch_list_desc(const int32_t *off, const int32_t *voff, int32_t n, const Ctrl *ctrl,
                      int2 *ldesc, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t want = ((uint32_t)n + 255u) / 256u;
  const uint32_t grid = max(1u, min(want, (uint32_t)(sms > 0 ? sms : 1) * 8u));
  k_list_desc<<<grid, 256, 0, st>>>(off, voff, n, ctrl, ldesc);
  note_launch();
}

void launch_clustering(const int64_t *t, const int32_t *deg, int32_t n, double *cc,
                       unsigned long long *sums, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t want = ((uint32_t)n + kClusterThreads * 4 - 1) / (kClusterThreads * 4);
  const uint32_t grid = max(1u, min(want, (uint32_t)(sms > 0 ? sms : 1) * 8));
  k_clustering<<<grid, kClusterThreads, 0, st>>>(t, deg, n, cc, sums);
  note_launch();
}

void launch_gather_counts(const int64_t *t_rank, const int32_t *rank, int32_t n, int64_t *t_out,
                          const Ctrl *ctrl, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t want = ((uint32_t)n + kClusterThreads * 4 - 1) / (kClusterThreads * 4);
  const uint32_t grid = max(1u, min(want, (uint32_t)(sms > 0 ? sms : 1) * 8));
  k_gather_counts<<<grid, kClusterThreads, 0, st>>>(t_rank, rank, n, t_out, ctrl);
  note_launch();
}

void launch_segment_sums(const int64_t *vals, const BatchDesc *batch, int32_t num_graphs,
                         int32_t divisor, unsigned long long *out, cudaStream_t st) {
  const uint32_t warps_per_block = kClusterThreads / 32;
  const uint32_t grid =
      max(1u, min(((uint32_t)num_graphs + warps_per_block - 1) / warps_per_block, 4096u));
  k_segment_sums<<<grid, kClusterThreads, 0, st>>>(vals, batch, num_graphs, divisor, out);
  note_launch();
}

void launch_transitivity(const unsigned long long *sums, double *out, cudaStream_t st) {
  k_transitivity<<<1, 1, 0, st>>>(sums, out);
  note_launch();
}

}  // namespace tc
