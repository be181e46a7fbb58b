// tc_common.cuh -- definitions shared by the library's CUDA translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

// Device-side error bits (Ctrl::err).
enum : uint32_t { kErrIdRange = 1u, kErrTimeout = 2u, kErrInternal = 4u };

// Upper bound on iterations of any spin-wait in a kernel.  Every wait in this
// library is on a predecessor tile that is already resident (tiles are handed
// out in launch order through an atomic ticket), so the bound is a safety
// net: if it is ever reached the kernel records kErrTimeout, stops waiting
// and the host reports TC_ERR_TIMEOUT.  What a timed-out tile would have
// written is not trusted: the tile publishes a poisoned status instead of its
// prefix and writes nothing, every tile that reads a poisoned status does the
// same, and every later kernel of the call returns at entry once kErrTimeout
// is set (see aborted()), so no kernel runs on incomplete data.
constexpr uint32_t kSpinLimit = 1u << 24;

// Sorted forward lists (the padded column array col4).  Lists of up to
// kWarpSortMax entries are sorted by one warp, up to kCtaSortMax by a CTA in
// shared memory; longer ones (never met in the workloads: they need a dense
// core of more than 8192 vertices) by a CTA in sorted chunks of kCtaSortMax
// merged in global memory.  Every list is sorted, and repeated entries (an
// edge given more than once) are dropped there.
constexpr int kWarpSortMax = 512;
constexpr int kCtaSortMax = 8192;
// Group keys carry, above the 2b bits of h and l, the number of leading
// 32-byte blocks of the streamed list that the intersection skips; there is
// room for it when 2b <= kSkipShift.
constexpr int kSkipShift = 48;
// Skip value of an edge whose triangles the dense hub block counts: the
// streamed list is skipped whole.
constexpr uint32_t kSkipAll = 0xFFFFu;

// Dense hub block (hub.cu): the kHubSize vertices of highest rank, counted
// on the tensor cores when they hold at least kHubMinEdges edges.  Only for
// single graphs with n >= kHubMinVertices and ids of at most 24 bits (the
// group keys must carry the skips).
constexpr int32_t kHubSize = 1 << 14;     // default size of the hub set
constexpr int32_t kHubMaxSize = 1 << 15;  // largest allowed (a multiple of 128)
constexpr int32_t kHubMinVertices = 1 << 17;
constexpr int64_t kHubMinEdges = 1 << 21;

constexpr int kMaxSort2Passes = 4;  // 31 owner bits / 8-bit digits
constexpr int kMaxRankPasses = 4;   // 31 degree bits / 8-bit digits
constexpr int kMaxGroupPasses = 4;  // 31 group bits / 8-bit digits
constexpr int kMaxPasses = kMaxSort2Passes + kMaxRankPasses + kMaxGroupPasses;
// First histogram slot of each sort.
constexpr int kSort2Slot = 0;
constexpr int kRankSlot = kMaxSort2Passes;
constexpr int kGroupSlot = kMaxSort2Passes + kMaxRankPasses;

// Hub sets of the work instrumentation: the 2^(kHubLog2Min + i) highest
// ranks, i < kHubSizes.
constexpr int kHubSizes = 4;
constexpr int kHubLog2Min = 12;

// Control block: zeroed at the start of every call.
struct Ctrl {
  uint32_t err;                    // kErr* bits
  uint32_t m;                      // oriented edges: set by orient (repeats included), then,
                                   //   if any list held repeats, by the recount of its node array
  uint32_t tile_ticket[24];        // per look-back kernel: next tile to hand out
  uint32_t n_warp_groups;          // partner groups counted by one warp each
  uint32_t n_cta_groups;           // ... by a 256-thread CTA each
  uint32_t n_big_groups;           // ... by a 512-thread CTA with a large table
  uint32_t next_warp_group;        // work cursors of the counting kernels
  uint32_t next_cta_group;
  uint32_t next_big_group;
  unsigned long long total;        // triangle count T
  uint32_t m_in;                   // input pairs that are real (not batch padding)
  uint32_t n_long_lists;           // forward lists sorted by the long-list kernels
  uint32_t next_long_list;         // work cursor of the CTA-per-list kernel
  uint32_t next_long_list_warp;    // work cursor of the warp-per-list kernel
  uint32_t hub_on;                 // the hub block is counted densely (hub.cu)
  uint32_t hub_lo;                 // its first rank
  uint32_t hub_size;               // its number of vertices (hub_lo + hub_size = n)
  uint32_t dups;                   // some forward list held a repeated edge (set by the list sort)
  unsigned long long hub_triangles;  // triangles the dense block counted
  unsigned long long hub_est[4];   // hash lookups inside each candidate hub set (hub.cu)
  // work of the counting phase (filled only when asked for; see launch_work):
  // hash lookups, hash inserts, merge work W, max out-degree, then the
  // lookups of edges with both endpoints among the 2^12 .. 2^15 top ranks
  unsigned long long work[4 + kHubSizes];
};
static_assert(sizeof(Ctrl) % 16 == 0, "Ctrl must keep 16-byte alignment");

// Ticket slots in Ctrl::tile_ticket.
enum {
  kTicketSort = 0 /* .. kMaxPasses-1, one per radix pass */,
  kTicketOrient = kMaxPasses,
  kTicketScan = kMaxPasses + 1,
  kTicketGroupScan = kMaxPasses + 2,
  kTicketVecScan = kMaxPasses + 3,
  kTicketRecount = kMaxPasses + 4
};
static_assert(kTicketRecount < 24, "ticket slots");

// Look-back status words: value in the low 62 bits, flag in the top 2.
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagInclusive = 2ull << 62;
constexpr unsigned long long kFlagPoison = 3ull << 62;  // the tile gave up: its prefix is unknown
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

#ifdef __CUDACC__
// True once some kernel of this call has recorded a wait that ran out: the
// data it left behind is incomplete, so later kernels must not read it.
__device__ __forceinline__ bool aborted(const Ctrl *ctrl) {
  return (*(const volatile uint32_t *)&ctrl->err & kErrTimeout) != 0u;
}

#endif

// Partner groups whose hashed forward list has at most kWarpMaxRow entries
// are counted by one warp, up to kCtaMaxRow by a 256-thread CTA, and longer
// ones by a 512-thread CTA with a larger table.
constexpr int kWarpMaxRow = 128;
constexpr int kWarpMaxPartners = 64;
constexpr int kCtaMaxRow = 1024;

// Runtime tuning of the counting layout (what an autotuner varies).
struct Tuning {
  int32_t warp_max_list;      // a group goes to one warp if its hashed list has
  int32_t warp_max_partners;  //   at most this many entries and partners
  int32_t heavy_ratio_pct;    // edge (u,v) is grouped at v when |N+(v)| * 100 >
                              //   |N+(u)| * heavy_ratio_pct, else at its owner u
  int64_t hub_min_edges;      // the dense hub block runs when it holds at least
                              //   this many edges (< 0: never)
  int32_t hub_vertices;       // size of the hub set: a multiple of 128, <= kHubMaxSize
};
constexpr Tuning kDefaultTuning = {128, 64, 100, kHubMinEdges, kHubSize};

// A batch of graphs counted as one disjoint union (device-side descriptor).
// Graph g owns input pairs [edge_off[g], edge_off[g+1]) and union vertex ids
// [voff[g], voff[g+1]); pairs at or beyond edge_off[num_graphs] are padding
// and are dropped like self-loops.
struct BatchDesc {
  int32_t num_graphs;
  int32_t pad_;
  const int32_t *edge_off;  // [num_graphs + 1]
  const int32_t *voff;      // [num_graphs + 1]
  int32_t *gerr;            // [num_graphs], zero on entry; set: an id outside its graph
};

// Workspace layout for an input of m_in pairs and n vertices.  All offsets
// are 256-byte aligned.
struct Layout {
  size_t ctrl, hist, st_sort, st_orient, st_scan, st_scan2, st_scan3, st_scan4;
  size_t keys_a, keys_b, deg, outdeg, off, voff, goff, warp_groups, cta_groups, big_groups;
  size_t col4;
  size_t rank, vkeys_a, vkeys_b, t_rank;
  size_t hub;  // dense hub block (0 bytes unless the layout asked for it)
  bool has_hub;
  int32_t hub_vertices;  // size of the hub set the hub region was laid out for
  size_t total;
  uint32_t sort_tiles, orient_tiles, scan_tiles;
  size_t st_sort_words_per_pass;
};

// Radix sort tiles: 256 threads x 16 keys.
constexpr int kSortThreads = 256;
constexpr int kSortKeysPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortKeysPerThread;
// Orientation/compaction tiles.
constexpr int kOrientThreads = 256;
constexpr int kOrientKeysPerThread = 16;
constexpr int kOrientTile = kOrientThreads * kOrientKeysPerThread;
// Offset-scan tiles.
constexpr int kScanThreads = 256;
constexpr int kScanItemsPerThread = 16;
constexpr int kScanTile = kScanThreads * kScanItemsPerThread;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Number of bits that hold any id in [0, n): at least 1.
inline int id_bits(int32_t n) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
  return b;
}

// Radix passes of one run over ids of b bits: the rank keys (degree <
// 2^b), the oriented keys (owner bits) and the group keys (group bits).
inline int radix_passes(int b) { return 3 * ((b + 7) / 8); }

// Whether a single-graph run of n vertices has the dense hub block.
inline bool hub_enabled(int32_t n, int b) { return n >= kHubMinVertices && 2 * b <= kSkipShift; }

inline Layout make_layout(int64_t m_in, int32_t n, bool with_hub = false,
                          int32_t hub_vertices = kHubSize) {
  Layout L{};
  size_t p = 0;
  auto take = [&](size_t bytes) {
    size_t at = p;
    p = align256(p + bytes);
    return at;
  };
  const uint64_t m = (uint64_t)(m_in > 0 ? m_in : 1);
  const uint64_t nv = (uint64_t)(n > 0 ? n : 1);
  const uint64_t keys_max = m > nv ? m : nv;  // the rank sort has n keys
  L.sort_tiles = (uint32_t)((keys_max + kSortTile - 1) / kSortTile);
  L.orient_tiles = (uint32_t)((m + kOrientTile - 1) / kOrientTile);
  L.scan_tiles = (uint32_t)((nv + 1 + kScanTile - 1) / kScanTile);
  L.st_sort_words_per_pass = (size_t)L.sort_tiles * 256;
  L.ctrl = take(sizeof(Ctrl));
  L.hist = take(sizeof(uint32_t) * 256 * kMaxPasses);
  // look-back status words for the passes that ids of [0, n) need (a run
  // with fewer vertices needs no more)
  L.st_sort = take(sizeof(unsigned long long) * L.st_sort_words_per_pass *
                   (size_t)radix_passes(id_bits(n > 0 ? n : 1)));
  L.st_orient = take(sizeof(unsigned long long) * L.orient_tiles);
  L.st_scan = take(sizeof(unsigned long long) * L.scan_tiles);
  L.st_scan2 = take(sizeof(unsigned long long) * L.scan_tiles);
  L.st_scan3 = take(sizeof(unsigned long long) * L.scan_tiles);
  L.st_scan4 = take(sizeof(unsigned long long) * L.scan_tiles);
  L.keys_a = take(sizeof(uint64_t) * m);
  L.keys_b = take(sizeof(uint64_t) * m);
  L.deg = take(sizeof(int32_t) * nv);
  L.outdeg = take(sizeof(int32_t) * nv);
  L.off = take(sizeof(int32_t) * (nv + 1));
  L.voff = take(sizeof(int32_t) * (nv + 1));
  L.goff = take(sizeof(int32_t) * (nv + 1));
  L.warp_groups = take(sizeof(int32_t) * nv);
  L.cta_groups = take(sizeof(int32_t) * nv);
  L.big_groups = take(sizeof(int32_t) * nv);
  L.rank = take(sizeof(int32_t) * nv);
  L.vkeys_a = take(sizeof(uint64_t) * nv);
  L.vkeys_b = take(sizeof(uint64_t) * nv);
  L.t_rank = take(sizeof(int64_t) * nv);
  // forward lists padded to whole 32-byte blocks: at most m + 7 min(n, m)
  // elements, since each non-empty list adds at most 7
  L.col4 = take(sizeof(int32_t) * (m + 7 * (nv < m ? nv : m)));
  const bool hub = with_hub && hub_enabled(n, id_bits(n > 0 ? n : 1));
  const size_t H = (size_t)hub_vertices;
  L.hub = take(hub ? H * H + 4 * H : 0);
  L.has_hub = hub;
  L.hub_vertices = hub_vertices;
  L.total = p;
  return L;
}


// Kernel-launch bookkeeping (defined in tc_api.cu).
void note_launch();

// Test hooks of the wait paths (preprocess.cu), on the current device:
// spin_limit bounds every spin-wait (kSpinLimit by default); the radix-pass
// tile numbered unpublished_tile (UINT32_MAX: none) never publishes its
// status, so the tiles after it wait on a word that nothing sets.
cudaError_t set_wait_hooks(uint32_t spin_limit, uint32_t unpublished_tile);

// ---- launchers (preprocess.cu) ----
// Undirected keys min << b | max of the pairs (self-loops and pairs with an
// id out of range: the sentinel 2^(2b) - 1) and deg[v] += 1 at both ends of
// every other pair (the degree with repeats; deg must be zero on entry).
// batch == nullptr: one graph on ids [0, n).  Otherwise ids of pair i are
// local to its graph, checked against that graph's vertex count, and
// shifted by the graph's first union id.
void launch_canon(const int32_t *src, const int32_t *dst, uint32_t m_in, int32_t n, int b,
                  const BatchDesc *batch, uint64_t *keys, int32_t *deg, Ctrl *ctrl,
                  cudaStream_t st);
// Output of a radix pass: the keys themselves; the column array (low bits,
// to `out`) plus the row array (key >> owner_shift, to `row_out`) with the
// out-degrees added to `outdeg`; or the rank scatter rank[low bits] =
// sorted position (to `out`).
// kOutPartSkip: the group sort's last pass: low bits to `out` (partners),
// key >> kSkipShift to `row_out` (skipped blocks) and the group sizes (the
// field at owner_shift, under col_mask) added to `outdeg`.
enum RadixOut { kOutKeys = 0, kOutColRow = 1, kOutRank = 2, kOutPartSkip = 4 };
// unstable: keys of equal digit may leave in any order (kOutKeys only; the
// first pass of a sort whose input order does not matter).
void launch_radix_pass(const uint64_t *in, void *out, RadixOut mode, uint32_t *row_out,
                       int32_t *outdeg, uint32_t n_keys_bound, const uint32_t *n_keys_dev,
                       int shift, uint32_t col_mask, int owner_shift, const uint32_t *hist,
                       unsigned long long *status, uint32_t *ticket, Ctrl *ctrl,
                       cudaStream_t st, bool unstable = false);
// Keys deg(v) << b | v for every vertex, with the digit histograms of the
// degree field (the rank sort).
void launch_rank_keys(const int32_t *deg, int32_t n, int b, int passes, uint64_t *vkeys,
                      uint32_t *hist, cudaStream_t st);
// Every non-sentinel key (in any order) as (lower rank) << b | (higher
// rank), compacted, with the digit histograms of the owner field; sets
// ctrl->m to the number written.
void launch_orient(const uint64_t *keys, uint32_t m_in, int b, const int32_t *rank,
                   uint64_t *okeys, uint32_t *hist2, int passes2, unsigned long long *status,
                   Ctrl *ctrl, cudaStream_t st);
// Exclusive scan counts[0..n) -> off[0..n].  With row_off != nullptr the
// entries are partner groups and are binned into warp_list / cta_list /
// big_list by the length of their hashed list; only the groups h with
// h mod shards = shard are binned (the share of the counting work this run
// does; shards = 1 bins them all).
void launch_offsets(const int32_t *counts, int32_t n, int32_t *off, const int32_t *row_off,
                    int32_t *warp_list, int32_t *cta_list, int32_t *big_list, Tuning tune,
                    unsigned long long *status, uint32_t *ticket, Ctrl *ctrl, cudaStream_t st,
                    int32_t shard = 0, int32_t shards = 1);
// The node array again, from the list lengths left after the list sort
// dropped repeated edges, and ctrl->m = their sum; nothing (the kernel
// returns at once) when no list held a repeat.
void launch_recount(const int32_t *counts, int32_t n, int32_t *off, unsigned long long *status,
                    uint32_t *ticket, Ctrl *ctrl, cudaStream_t st);
// Exclusive scan of 2 ceil(counts / 8) -> voff[0..n]: the node array of the
// padded column array (lists in whole 32-byte blocks), in 16-byte words.
void launch_word_offsets(const int32_t *counts, int32_t n, int32_t *voff,
                         unsigned long long *status, uint32_t *ticket, Ctrl *ctrl,
                         cudaStream_t st);
// ---- launchers (hub.cu) ----
// Workspace of the dense hub block of H vertices: the H x H fp8 matrix and
// the per-vertex sums.
size_t hub_bytes(int32_t H);
// Decides on the device (into ctrl->hub_on, hub_size, hub_lo) whether, and
// with how many of the top ranks (a candidate up to Hmax), the hub block is
// counted densely; needs the node array and the column array (any order
// within a list).
void launch_hub_decide(const int32_t *off, const int32_t *col, int32_t n, int32_t Hmax,
                       int64_t min_edges, bool per_vertex, Ctrl *ctrl, cudaStream_t st);
// Counts the triangles inside the hub block (if ctrl->hub_on): adds them to
// ctrl->total and, if t != nullptr, to the per-vertex counts t (rank space).
// Needs the forward lists; region: hub_bytes(Hmax) bytes, 256-byte aligned.
cudaError_t launch_hub_count(const int32_t *off, const int32_t *voff, const int32_t *col4,
                             int32_t n, int32_t Hmax, uint8_t *region, Ctrl *ctrl, int64_t *t,
                             cudaStream_t st);
// ---- launchers (group.cu) ----
// Sorts every forward list (the column array col, grouped by owner, node
// array off) into the padded column array col4 (list v from 16-byte word
// voff[v], padded with -1 to whole 32-byte blocks).  A
// repeated entry (an edge given more than once) is dropped: the list's
// length goes to dlen[v] (written only for such lists; dlen holds the
// lengths with repeats on entry), each dropped copy adds one to dcorr at
// both its ends (rank space; zero on entry) and ctrl->dups is set.
// long_lists: scratch of n entries; col is scratch for lists longer than
// kCtaSortMax.
void launch_sort_lists(int32_t *col, const int32_t *off, const int32_t *voff, int32_t n,
                       Ctrl *ctrl, int32_t *col4, int32_t *long_lists, int32_t *dlen,
                       int32_t *dcorr, cudaStream_t st);
// After the list sort, if some list held repeats: the row array again
// (row[off[v] + i] = v, from the recounted node array) and the degrees
// without repeats (deg[v] -= dcorr[rank[v]], caller ids).  Both return at
// once otherwise.
void launch_fix_repeats(const int32_t *off, int32_t n, const int32_t *dcorr, const int32_t *rank,
                        Ctrl *ctrl, int32_t *row, int32_t *deg, cudaStream_t st);
// Group keys s << kSkipShift | h << b | l of every forward edge (h: the
// endpoint with the longer forward list, l: the other one, s: the leading
// blocks of N+(l) the intersection skips, 0 when 2b > kSkipShift), with the
// digit histograms of the h field for the group sort.  Reads the sorted
// lists (col4; their first words and lengths from ldesc, see
// launch_list_desc) in owner order (row, node array off).
void launch_group_keys(const int32_t *row, const int32_t *col4, const int32_t *off,
                       const int2 *ldesc, uint32_t m_bound, int b,
                       int passes, int32_t heavy_ratio_pct, Ctrl *ctrl, uint64_t *gkeys,
                       uint32_t *hist, cudaStream_t st);
// Instrumentation: adds the counting phase's work into ctrl->work (from the
// partner groups, the node array and the skipped blocks), over the groups h
// with h mod shards = shard (the share one part counts).
void launch_work(const int32_t *off, const int32_t *goff, const int32_t *part,
                 const int32_t *pskip, int32_t n, Ctrl *ctrl, cudaStream_t st,
                 int32_t shard = 0, int32_t shards = 1);
// ---- launchers (count.cu) ----
// t != nullptr: per-vertex counts (rank space).  Otherwise, if tg is not
// nullptr, tg[h] += triangles found in group h (their sum per graph is the
// graph's count).  desc: scratch of 8 bytes per partner (each partner's
// stream, written first).
// ldesc[v] = {voff[v], off[v+1] - off[v]} for every vertex (the lists' first
// col4 word and length in one record), for the counting kernels.
void launch_list_desc(const int32_t *off, const int32_t *voff, int32_t n, const Ctrl *ctrl,
                      int2 *ldesc, cudaStream_t st);
cudaError_t launch_count(const int32_t *off, const int32_t *voff, const int2 *ldesc,
                         const int32_t *col4,
                         const int32_t *goff, const int32_t *part, const int32_t *pskip,
                         int2 *desc, const int32_t *warp_groups,
                         const int32_t *cta_groups, const int32_t *big_groups, int32_t n,
                         Ctrl *ctrl, int64_t *t, int64_t *tg, cudaStream_t st);
// Sets the counting kernels' attributes and occupancy for the current
// device (done lazily otherwise; needed before capturing a CUDA graph).
cudaError_t prepare_count_kernels();
// out[g] = (sum of vals over graph g's union ids) / divisor.
void launch_segment_sums(const int64_t *vals, const BatchDesc *batch, int32_t num_graphs,
                         int32_t divisor, unsigned long long *out, cudaStream_t st);
// ---- clustering (count.cu) ----
void launch_clustering(const int64_t *t, const int32_t *deg, int32_t n, double *cc,
                       unsigned long long *sums /* [2]: sum t, sum C(deg,2) */, cudaStream_t st);
void launch_transitivity(const unsigned long long *sums, double *out, cudaStream_t st);
// t_out[v] = t_rank[rank[v]]: per-vertex counts back to the caller's ids.
void launch_gather_counts(const int64_t *t_rank, const int32_t *rank, int32_t n, int64_t *t_out,
                          const Ctrl *ctrl, cudaStream_t st);

}  // namespace tc
