// tc_api.cu -- the C ABI of include/tc.h: argument checks, workspace,
// phase sequence, host-buffer variants, errors and instrumentation.
#include <atomic>
#include <cstdarg>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tc.h"
#include "tc_common.cuh"
#include "tc_debug.h"

namespace tc {

static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace tc

using namespace tc;

namespace {

thread_local tc_status t_last = TC_OK;
thread_local char t_detail[256] = "";

tc_status set_status(tc_status s, const char *fmt = nullptr, ...) {
  t_last = s;
  if (fmt) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_detail, sizeof(t_detail), fmt, ap);
    va_end(ap);
  } else {
    t_detail[0] = 0;
  }
  return s;
}

tc_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();  // a failed runtime call is not charged to the next call
  if (e == cudaErrorMemoryAllocation)
    return set_status(TC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return set_status(TC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define TC_CUDA(call, what)                     \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ---- allocation-failure injection (tc_debug_fail_allocations) ----
std::atomic<bool> g_inject_on{false};
std::mutex g_inject_mu;
int64_t g_inject_skip = 0, g_inject_fail = 0;

// Whether this device allocation is to fail as if the device were out of
// memory (only ever true in the allocation-failure tests).
bool injected_alloc_failure() {
  if (!g_inject_on.load(std::memory_order_relaxed)) return false;
  std::lock_guard<std::mutex> lk(g_inject_mu);
  if (g_inject_fail <= 0) return false;
  if (g_inject_skip > 0) {
    --g_inject_skip;
    return false;
  }
  if (--g_inject_fail == 0) g_inject_on.store(false);
  return true;
}

// Every device allocation of the library goes through these two.
cudaError_t dev_alloc_async(void **p, size_t bytes, cudaStream_t st) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, st);
}
cudaError_t dev_alloc(void **p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

// ---- instrumentation ----
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
double g_prof_ms[TC_NUM_PHASES];
uint64_t g_prof_launches[TC_NUM_PHASES];

const char *const kPhaseNames[TC_NUM_PHASES] = {"canon",   "rank",  "orient", "sort",
                                                "offsets", "lists", "groups", "count"};

// Events around each phase of one call, folded into the global totals after
// the call has synchronised its stream.
struct PhaseTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  cudaEvent_t beg[TC_NUM_PHASES] = {}, end[TC_NUM_PHASES] = {};
  uint64_t launches[TC_NUM_PHASES] = {};
  uint64_t at = 0;
  bool used[TC_NUM_PHASES] = {};

  PhaseTimer(cudaStream_t s, bool allowed) : st(s) {
    on = allowed && g_prof_on.load() != 0;
    if (!on) return;
    for (int i = 0; i < TC_NUM_PHASES; ++i) {
      cudaEventCreate(&beg[i]);
      cudaEventCreate(&end[i]);
    }
  }
  void start(int p) {
    at = g_launches.load();
    if (!on) return;
    cudaEventRecord(beg[p], st);
  }
  void stop(int p) {
    if (!on) return;
    cudaEventRecord(end[p], st);
    launches[p] += g_launches.load() - at;
    used[p] = true;
  }
  // call after the stream has been synchronised
  void fold() {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < TC_NUM_PHASES; ++i) {
      if (!used[i]) continue;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, beg[i], end[i]) == cudaSuccess) g_prof_ms[i] += ms;
      g_prof_launches[i] += launches[i];
    }
  }
  ~PhaseTimer() {
    if (!on) return;
    for (int i = 0; i < TC_NUM_PHASES; ++i) {
      cudaEventDestroy(beg[i]);
      cudaEventDestroy(end[i]);
    }
  }
};

// Keep freed stream-ordered allocations cached in the device's default pool
// (release threshold = unlimited) so repeated calls do not return memory to
// the driver and fetch it again.
void keep_pool_memory() {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  const uint64_t bit = 1ull << dev;
  if (done_mask.load() & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_mask.fetch_or(bit);
}

Ctrl *host_ctrl() {
  static thread_local Ctrl *h = nullptr;
  if (!h && cudaMallocHost((void **)&h, sizeof(Ctrl)) != cudaSuccess) h = nullptr;
  return h;
}

// Largest m (pairs) and n (vertices) a run accepts: 2^31 less a margin, so
// that no int32 index a warp advances past the end of a list, a partner
// range or a graph's vertex range (by at most a few hundred) can wrap.
constexpr int64_t kMaxItems = ((int64_t)1 << 31) - ((int64_t)1 << 10);

// The padded column array holds at most m + 7 min(n, m) entries, indexed
// by int32 16-byte words.
bool padded_fits(int64_t m, int64_t n) {
  return m + 7 * (n < m ? n : m) < ((int64_t)1 << 33);
}

tc_status check_args(const int32_t *src, const int32_t *dst, int64_t m, int32_t n) {
  if (m < 0 || n < 0) return set_status(TC_ERR_INVALID_ARG, "m=%lld n=%d", (long long)m, n);
  if (m > kMaxItems || (int64_t)n > kMaxItems)
    return set_status(TC_ERR_OVERFLOW, "m=%lld, n=%d: beyond 2^31 - 2^10 pairs or vertices",
                      (long long)m, n);
  if (!padded_fits(m, n))
    return set_status(TC_ERR_OVERFLOW, "m=%lld, n=%d: padded lists exceed 2^31 16-byte words",
                      (long long)m, n);
  if (m > 0 && (!src || !dst)) return set_status(TC_ERR_INVALID_ARG, "src/dst is NULL");
  return TC_OK;
}

// Extra inputs and outputs of a batched run (several graphs counted as one
// disjoint union).
struct BatchRun {
  const BatchDesc *desc;        // device descriptor of the graphs
  int32_t num_graphs_bound;     // grid bound of the per-graph sums
  unsigned long long *totals;   // device: triangles per graph
};

// Enqueues every phase on `st` using workspace `ws` laid out by L, ending
// with a copy of the control block into `staging` (host).  Nothing here
// synchronises or allocates, so the whole sequence can be captured in a
// CUDA graph.  t_out == nullptr counts the total only (per graph with a
// batch: group totals, summed per graph).
tc_status enqueue_core(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                       cudaStream_t st, unsigned char *ws, const Layout &L, int64_t *t_out,
                       int32_t *deg_out, const BatchRun *batch, const Tuning &tune,
                       PhaseTimer &pt, Ctrl *staging, bool work_stats = false,
                       int32_t shard = 0, int32_t shards = 1) {
  const uint32_t m = (uint32_t)m_in;
  const int b = id_bits(n);
  // radix passes: rank keys (degree bits < 2^b), oriented keys (owner bits)
  const int passes_r = (b + 7) / 8, passes2 = (b + 7) / 8;
  const int passes3 = (b + 7) / 8;  // group keys: the h field
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
  auto *st_sort = reinterpret_cast<unsigned long long *>(ws + L.st_sort);
  auto *st_orient = reinterpret_cast<unsigned long long *>(ws + L.st_orient);
  auto *st_scan = reinterpret_cast<unsigned long long *>(ws + L.st_scan);
  auto *st_scan2 = reinterpret_cast<unsigned long long *>(ws + L.st_scan2);
  auto *st_scan3 = reinterpret_cast<unsigned long long *>(ws + L.st_scan3);
  auto *st_scan4 = reinterpret_cast<unsigned long long *>(ws + L.st_scan4);
  uint64_t *keys_a = reinterpret_cast<uint64_t *>(ws + L.keys_a);
  uint64_t *keys_b = reinterpret_cast<uint64_t *>(ws + L.keys_b);
  uint64_t *vkeys_a = reinterpret_cast<uint64_t *>(ws + L.vkeys_a);
  uint64_t *vkeys_b = reinterpret_cast<uint64_t *>(ws + L.vkeys_b);
  int32_t *deg = deg_out ? deg_out : reinterpret_cast<int32_t *>(ws + L.deg);
  int32_t *outdeg = reinterpret_cast<int32_t *>(ws + L.outdeg);
  int32_t *off = reinterpret_cast<int32_t *>(ws + L.off);
  int32_t *voff = reinterpret_cast<int32_t *>(ws + L.voff);
  int32_t *col4 = reinterpret_cast<int32_t *>(ws + L.col4);
  int32_t *goff = reinterpret_cast<int32_t *>(ws + L.goff);
  int32_t *warp_groups = reinterpret_cast<int32_t *>(ws + L.warp_groups);
  int32_t *cta_groups = reinterpret_cast<int32_t *>(ws + L.cta_groups);
  int32_t *big_groups = reinterpret_cast<int32_t *>(ws + L.big_groups);
  int32_t *rank = reinterpret_cast<int32_t *>(ws + L.rank);
  // per rank: repeated edges dropped by the list sort (the rank keys are
  // free by then)
  int32_t *dcorr = reinterpret_cast<int32_t *>(ws + L.vkeys_a);
  // per vertex: its list's first col4 word and length (the second rank-key
  // buffer, free after the rank sort)
  int2 *ldesc = reinterpret_cast<int2 *>(ws + L.vkeys_b);
  // per-vertex counts, or per-group totals of a batch, in rank space
  int64_t *t_rank = (t_out || batch) ? reinterpret_cast<int64_t *>(ws + L.t_rank) : nullptr;
  // group totals back in union ids (the rank keys are free by then)
  int64_t *tg_union = reinterpret_cast<int64_t *>(ws + L.vkeys_a);
  const size_t words = L.st_sort_words_per_pass;
  // look-back status and tile tickets: one slot per radix pass, in the order
  // the passes run (rank sort, sort by owner, group sort)
  int slot = 0;
  auto next_pass = [&](unsigned long long **status, uint32_t **ticket) {
    *status = st_sort + words * (size_t)slot;
    *ticket = &ctrl->tile_ticket[kTicketSort + slot];
    ++slot;
  };

  // zero the control block, histograms and the look-back status words in use
  TC_CUDA(cudaMemsetAsync(ws, 0, L.st_sort + sizeof(unsigned long long) * words *
                                                  (size_t)radix_passes(b), st),
          "memset control");
  TC_CUDA(cudaMemsetAsync(ws + L.st_orient, 0, L.keys_a - L.st_orient, st), "memset status");
  TC_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)n, st), "memset deg");
  TC_CUDA(cudaMemsetAsync(outdeg, 0, sizeof(int32_t) * (size_t)n, st), "memset outdeg");
  if (t_rank) TC_CUDA(cudaMemsetAsync(t_rank, 0, sizeof(int64_t) * (size_t)n, st), "memset t");

  // undirected keys and the degrees (repeated edges counted as often as
  // they are given; the list sort takes them back)
  pt.start(TC_PHASE_CANON);
  launch_canon(src, dst, m, n, b, batch ? batch->desc : nullptr, keys_a, deg, ctrl, st);
  pt.stop(TC_PHASE_CANON);

  // rank of every vertex in the (degree, id) order
  pt.start(TC_PHASE_RANK);
  const uint32_t id_mask = (uint32_t)((1ull << b) - 1);
  launch_rank_keys(deg, n, b, passes_r, vkeys_a, hist + 256 * kRankSlot, st);
  {
    uint64_t *vin = vkeys_a, *vout = vkeys_b;
    for (int p = 0; p < passes_r; ++p) {
      unsigned long long *status;
      uint32_t *ticket;
      next_pass(&status, &ticket);
      const bool last = p == passes_r - 1;
      launch_radix_pass(vin, last ? (void *)rank : (void *)vout, last ? kOutRank : kOutKeys,
                        nullptr, nullptr, (uint32_t)n, nullptr, b + 8 * p, id_mask, 0,
                        hist + 256 * (kRankSlot + p), status, ticket, ctrl, st);
      uint64_t *x = vin;
      vin = vout;
      vout = x;
    }
  }
  pt.stop(TC_PHASE_RANK);

  pt.start(TC_PHASE_ORIENT);
  launch_orient(keys_a, m, b, rank, keys_b, hist + 256 * kSort2Slot, passes2, st_orient, ctrl,
                st);
  pt.stop(TC_PHASE_ORIENT);

  pt.start(TC_PHASE_SORT);
  uint64_t *in = keys_b, *out = keys_a;
  // the last pass writes the column array to `out` (first 4m bytes) and the
  // row array to the second half of the same buffer.  The order within a
  // list does not matter (each list is sorted on its own later), so the
  // first pass ranks equal digits in any order.
  for (int p = 0; p < passes2; ++p) {
    unsigned long long *status;
    uint32_t *ticket;
    next_pass(&status, &ticket);
    const bool last = p == passes2 - 1;
    uint32_t *row_target = last ? reinterpret_cast<uint32_t *>(out) + m : nullptr;
    launch_radix_pass(in, out, last ? kOutColRow : kOutKeys, row_target, last ? outdeg : nullptr,
                      m, &ctrl->m, b + 8 * p, id_mask, b, hist + 256 * (kSort2Slot + p), status,
                      ticket, ctrl, st, /*unstable=*/p == 0);
    if (!last) {
      uint64_t *x = in;
      in = out;
      out = x;
    }
  }
  int32_t *col = reinterpret_cast<int32_t *>(out);
  int32_t *row = reinterpret_cast<int32_t *>(out) + m;
  pt.stop(TC_PHASE_SORT);

  pt.start(TC_PHASE_OFFSETS);
  launch_offsets(outdeg, n, off, nullptr, nullptr, nullptr, nullptr, tune, st_scan,
                 &ctrl->tile_ticket[kTicketScan], ctrl, st);
  launch_word_offsets(outdeg, n, voff, st_scan3, &ctrl->tile_ticket[kTicketVecScan], ctrl, st);
  // whether the top ranks are counted densely (their edges are then left
  // out of the partner groups)
  const bool hub = L.has_hub && tune.hub_min_edges >= 0;
  const int32_t H = L.hub_vertices;  // the size the workspace was laid out for
  if (hub) launch_hub_decide(off, col, n, H, tune.hub_min_edges, t_out != nullptr, ctrl, st);
  pt.stop(TC_PHASE_OFFSETS);

  // every forward list sorted into the padded column array col4 (the
  // warp-group list is free scratch until the binning), repeated edges
  // dropped: their lists' new lengths overwrite the out-degrees, and only if
  // there were any, the node array, the edge count, the row array and the
  // degrees are made right again
  pt.start(TC_PHASE_LISTS);
  TC_CUDA(cudaMemsetAsync(dcorr, 0, sizeof(int32_t) * (size_t)n, st), "memset repeats");
  launch_sort_lists(col, off, voff, n, ctrl, col4, warp_groups, outdeg, dcorr, st);
  launch_recount(outdeg, n, off, st_scan4, &ctrl->tile_ticket[kTicketRecount], ctrl, st);
  launch_fix_repeats(off, n, dcorr, rank, ctrl, row, deg, st);
  launch_list_desc(off, voff, n, ctrl, ldesc, st);
  pt.stop(TC_PHASE_LISTS);

  // partner groups: each forward edge goes to the endpoint with the longer
  // forward list.  Group keys, read from the sorted lists, go to `in` (the
  // owner sort's input, free now); a radix sort over the group bits then
  // gathers every group's partners, its last pass counting the group sizes
  // into gcnt (the out-degree array's space) and writing the skipped blocks
  // of each partner's stream beside the partner array.
  pt.start(TC_PHASE_GROUPS);
  launch_group_keys(row, col4, off, ldesc, m, b, passes3, tune.heavy_ratio_pct, ctrl, in,
                    hist + 256 * kGroupSlot, st);
  int32_t *gcnt = outdeg;
  TC_CUDA(cudaMemsetAsync(gcnt, 0, sizeof(int32_t) * (size_t)n, st), "memset groups");
  const bool skip_in_key = 2 * b <= kSkipShift;
  uint64_t *gin = in, *gout = out;  // row and col are dead after the group keys
  for (int p = 0; p < passes3; ++p) {
    unsigned long long *status;
    uint32_t *ticket;
    next_pass(&status, &ticket);
    const bool last = p == passes3 - 1;
    // the last pass writes the partners l (first half of gout) and the
    // blocks their streams skip (second half); the order of a group's
    // partners does not matter, so the first pass ranks equal digits in
    // any order
    const RadixOut mode = !last ? kOutKeys : skip_in_key ? kOutPartSkip : kOutColRow;
    uint32_t *skip_target = last && skip_in_key ? reinterpret_cast<uint32_t *>(gout) + m : nullptr;
    launch_radix_pass(gin, gout, mode, skip_target, last ? gcnt : nullptr, m, &ctrl->m, b + 8 * p,
                      id_mask, b, hist + 256 * (kGroupSlot + p), status, ticket, ctrl, st,
                      /*unstable=*/p == 0);
    if (!last) {
      uint64_t *x = gin;
      gin = gout;
      gout = x;
    }
  }
  const int32_t *part = reinterpret_cast<const int32_t *>(gout);
  const int32_t *pskip = reinterpret_cast<const int32_t *>(gout) + m;
  if (!skip_in_key)  // ids of more than 24 bits leave no room for the skip: stream lists whole
    TC_CUDA(cudaMemsetAsync(reinterpret_cast<int32_t *>(gout) + m, 0, sizeof(int32_t) * (size_t)m,
                            st),
            "memset skips");
  // only this run's share of the groups is binned (all of them unless the
  // counting is split over several devices, Sec. III-E)
  launch_offsets(gcnt, n, goff, off, warp_groups, cta_groups, big_groups, tune, st_scan2,
                 &ctrl->tile_ticket[kTicketGroupScan], ctrl, st, shard, shards);
  pt.stop(TC_PHASE_GROUPS);
  if (work_stats) launch_work(off, goff, part, pskip, n, ctrl, st, shard, shards);

  pt.start(TC_PHASE_COUNT);
  // the dense block's triangles belong to the first share alone (every share
  // leaves the block's edges off its hash path)
  if (hub && shard == 0) {
    TC_CUDA(launch_hub_count(off, voff, col4, n, H, ws + L.hub, ctrl,
                             t_out ? t_rank : nullptr, st),
            "dense hub block");
  }
  // each partner's stream goes to the group sort's other buffer (free now)
  int2 *desc = reinterpret_cast<int2 *>(gin);
  cudaError_t e = launch_count(off, voff, ldesc, col4, goff, part, pskip, desc, warp_groups,
                               cta_groups,
                               big_groups, n, ctrl, t_out ? t_rank : nullptr,
                               t_out ? nullptr : t_rank, st);
  if (e == cudaSuccess && t_out) launch_gather_counts(t_rank, rank, n, t_out, ctrl, st);
  if (e == cudaSuccess && batch) {
    if (t_out) {  // per graph: (sum of t) / 3
      launch_segment_sums(t_out, batch->desc, batch->num_graphs_bound, 3, batch->totals, st);
    } else {      // per graph: sum of the group totals
      launch_gather_counts(t_rank, rank, n, tg_union, ctrl, st);
      launch_segment_sums(tg_union, batch->desc, batch->num_graphs_bound, 1, batch->totals, st);
    }
  }
  pt.stop(TC_PHASE_COUNT);
  if (e != cudaSuccess) return cuda_fail(e, "count kernel");
  TC_CUDA(cudaGetLastError(), "kernel launch");
  TC_CUDA(cudaMemcpyAsync(staging, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st), "read result");
  return TC_OK;
}

// Status of a run from its control block (after the stream has synchronised).
tc_status finish_core(const Ctrl *h, int32_t n, uint64_t *total) {
  if (h->err & kErrTimeout)
    return set_status(TC_ERR_TIMEOUT, "a device-side wait reached its iteration limit");
  if (h->err & kErrInternal)
    return set_status(TC_ERR_CUDA, "the dense hub block failed its consistency check");
  if (h->err & kErrIdRange)
    return set_status(TC_ERR_ID_RANGE, "a vertex id is outside [0, %d) of its graph", n);
  if (total) *total = (uint64_t)h->total;
  return set_status(TC_OK);
}

Tuning g_tuning = kDefaultTuning;
std::mutex g_tuning_mu;

Tuning current_tuning() {
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  return g_tuning;
}

// One synchronous single-graph run: enqueue, synchronise, read the status.
tc_status run_core(const int32_t *src, const int32_t *dst, int64_t m_in, int32_t n,
                   cudaStream_t st, unsigned char *ws, const Layout &L, int64_t *t_out,
                   int32_t *deg_out, uint64_t *total, Ctrl *staging = nullptr,
                   bool profile = true, int32_t shard = 0, int32_t shards = 1) {
  PhaseTimer pt(st, profile);
  Ctrl *h = staging ? staging : host_ctrl();
  if (!h) return set_status(TC_ERR_OOM, "pinned staging buffer");
  tc_status s = enqueue_core(src, dst, m_in, n, st, ws, L, t_out, deg_out, nullptr,
                             current_tuning(), pt, h, false, shard, shards);
  if (s != TC_OK) return s;
  TC_CUDA(cudaStreamSynchronize(st), "synchronize");
  pt.fold();
  return finish_core(h, n, total);
}

tc_status count_impl(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                     cudaStream_t st, void *ws_user, size_t ws_bytes, int64_t *t_out,
                     int32_t *deg_out, uint64_t *total, int32_t shard = 0,
                     int32_t shards = 1) {
  tc_status s = check_args(src, dst, m, n);
  if (s != TC_OK) return s;
  if (shards < 1 || shard < 0 || shard >= shards)
    return set_status(TC_ERR_INVALID_ARG, "shard %d of %d", shard, shards);
  if (m > 0 && n == 0) return set_status(TC_ERR_ID_RANGE, "n = 0 but m > 0");
  if (m == 0) {
    if (n > 0 && t_out)
      TC_CUDA(cudaMemsetAsync(t_out, 0, sizeof(int64_t) * (size_t)n, st), "memset t");
    if (n > 0 && deg_out)
      TC_CUDA(cudaMemsetAsync(deg_out, 0, sizeof(int32_t) * (size_t)n, st), "memset deg");
    TC_CUDA(cudaStreamSynchronize(st), "synchronize");
    *total = 0;
    return set_status(TC_OK);
  }
  const Layout L = make_layout(m, n, true, current_tuning().hub_vertices);
  if (ws_user) {
    if (ws_bytes < L.total)
      return set_status(TC_ERR_INVALID_ARG, "workspace has %zu bytes, needs %zu", ws_bytes,
                        L.total);
    if ((uintptr_t)ws_user & 255)
      return set_status(TC_ERR_INVALID_ARG, "workspace is not 256-byte aligned");
    return run_core(src, dst, m, n, st, (unsigned char *)ws_user, L, t_out, deg_out, total,
                    nullptr, true, shard, shards);
  }
  keep_pool_memory();
  void *ws = nullptr;
  TC_CUDA(dev_alloc_async(&ws, L.total, st), "workspace allocation");
  s = run_core(src, dst, m, n, st, (unsigned char *)ws, L, t_out, deg_out, total, nullptr, true,
               shard, shards);
  const tc_status keep = s;
  char detail[256];
  memcpy(detail, t_detail, sizeof(detail));
  cudaError_t e = cudaFreeAsync(ws, st);
  if (keep != TC_OK) {
    t_last = keep;
    memcpy(t_detail, detail, sizeof(detail));
    return keep;
  }
  if (e != cudaSuccess) return cuda_fail(e, "workspace release");
  return keep;
}

// Whether a kernel may read any host buffer in place: true where the device
// reads pageable memory through the host's page tables (address translation
// services, as on Grace), false elsewhere (then inputs are copied in).
bool kernels_read_host_memory() {
  static const bool yes = [] {
    int dev = 0, pageable = 0, page_tables = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&page_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables,
                               dev) != cudaSuccess)
      return false;
    return pageable == 1 && page_tables == 1;
  }();
  return yes;
}

// Host-buffer driver: copy in, count, copy out, on a private stream.  Only
// the first kernel reads the input pairs, once each, so where kernels can
// read host memory the pairs are read in place instead of copied first.
tc_status host_impl(const int32_t *src_h, const int32_t *dst_h, int64_t m, int32_t n,
                    int64_t *t_h, int32_t *deg_h, uint64_t *total, bool per_vertex) {
  tc_status s = check_args(src_h, dst_h, m, n);
  if (s != TC_OK) return s;
  if (per_vertex && n > 0 && !t_h) return set_status(TC_ERR_INVALID_ARG, "t_host is NULL");
  static thread_local cudaStream_t st = nullptr;
  if (!st) TC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
  keep_pool_memory();
  const size_t in_bytes = sizeof(int32_t) * (size_t)m;
  int32_t *d_src = nullptr, *d_dst = nullptr, *d_deg = nullptr;
  int64_t *d_t = nullptr;
  const bool in_place = kernels_read_host_memory();
  // what was allocated is released on every path below, failed ones included
  cudaError_t e = cudaSuccess;
  const char *what = nullptr;
  if (m > 0 && !in_place) {
    if ((e = dev_alloc_async((void **)&d_src, in_bytes, st)) != cudaSuccess ||
        (e = dev_alloc_async((void **)&d_dst, in_bytes, st)) != cudaSuccess)
      what = "input allocation";
    else if ((e = cudaMemcpyAsync(d_src, src_h, in_bytes, cudaMemcpyHostToDevice, st)) !=
                 cudaSuccess ||
             (e = cudaMemcpyAsync(d_dst, dst_h, in_bytes, cudaMemcpyHostToDevice, st)) !=
                 cudaSuccess)
      what = "copy in";
  }
  if (!what && per_vertex && n > 0) {
    if ((e = dev_alloc_async((void **)&d_t, sizeof(int64_t) * (size_t)n, st)) != cudaSuccess)
      what = "t allocation";
    else if (deg_h &&
             (e = dev_alloc_async((void **)&d_deg, sizeof(int32_t) * (size_t)n, st)) !=
                 cudaSuccess)
      what = "deg allocation";
  }
  uint64_t T = 0;
  if (what)
    s = cuda_fail(e, what);
  else
    s = count_impl(in_place ? src_h : d_src, in_place ? dst_h : d_dst, m, n, st, nullptr, 0,
                   per_vertex ? d_t : nullptr, d_deg, &T);
  if (s == TC_OK && per_vertex && n > 0) {
    cudaError_t e = cudaMemcpyAsync(t_h, d_t, sizeof(int64_t) * (size_t)n,
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && deg_h)
      e = cudaMemcpyAsync(deg_h, d_deg, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = cuda_fail(e, "copy out");
  }
  if (d_src) cudaFreeAsync(d_src, st);
  if (d_dst) cudaFreeAsync(d_dst, st);
  if (d_t) cudaFreeAsync(d_t, st);
  if (d_deg) cudaFreeAsync(d_deg, st);
  e = cudaStreamSynchronize(st);
  if (s != TC_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  if (total) *total = T;
  return set_status(TC_OK);
}

// ---------------------------------------------------------------------------
// Allocation-free counting (tc_count_noalloc).
//
// Some callers cannot allocate device memory when they count: a host process
// that hands all device memory to its own pool allocator at start-up and
// forbids driver allocations afterwards, or a service whose memory budget is
// fixed when it starts.  For them the whole workspace lives in this
// file-scope array, held by every GPU that has loaded it until the process
// exits.  When the array comes into being on a device depends on how CUDA
// loads modules: eagerly (CUDA_MODULE_LOADING=EAGER) when the library's
// context is set up there, lazily (the default) on the first use of this
// file's module on that device -- which is the first tc_count_noalloc call
// there, since no kernel lives in this file.  So the first call on each
// device may reserve the 32 MiB; callers that reserve all device memory
// later should make that first call at start-up, before they do.
//
// Host code cannot pass the array's name to a kernel (on the host it is only
// a stand-in symbol), so every call looks up its device address on the
// current device with cudaGetSymbolAddress (cheap once the module is
// loaded).  Nothing is cached, so a context torn down and set up again
// (cudaDeviceReset) gets the array's new address.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[TC_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.
tc_status noalloc_scratch(unsigned char **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e == cudaErrorMemoryAllocation)
    return cuda_fail(e, "loading the static scratch array on this device (the first "
                        "tc_count_noalloc call on a device reserves it; make that call "
                        "before device memory runs out)");
  if (e != cudaSuccess) return cuda_fail(e, "scratch symbol address");
  *out = static_cast<unsigned char *>(p);
  return TC_OK;
}

// ---------------------------------------------------------------------------
// Batches: several graphs counted as one disjoint union.
// ---------------------------------------------------------------------------
// Host-side check of a batch and the int32 offset block the device needs:
// edge offsets [G+1] followed by union vertex offsets [G+1].
struct BatchPlan {
  int32_t graphs = 0;
  int64_t pairs = 0;
  int64_t vertices = 0;
  std::vector<int32_t> block;
};

tc_status plan_batch(int32_t G, const int64_t *eo, const int32_t *vn, int64_t max_pairs,
                     int64_t max_vertices, BatchPlan *p) {
  if (G < 0 || (G > 0 && (!eo || !vn)))
    return set_status(TC_ERR_INVALID_ARG, "num_graphs < 0 or a NULL offset array");
  p->graphs = G;
  p->block.assign(2 * (size_t)(G + 1), 0);
  if (G == 0) return TC_OK;
  if (eo[0] != 0) return set_status(TC_ERR_INVALID_ARG, "edge_offsets[0] must be 0");
  int64_t nv = 0;
  for (int32_t g = 0; g < G; ++g) {
    if (eo[g + 1] < eo[g]) return set_status(TC_ERR_INVALID_ARG, "edge_offsets decrease at %d", g);
    if (vn[g] < 0) return set_status(TC_ERR_INVALID_ARG, "vertex_counts[%d] < 0", g);
    nv += vn[g];
  }
  if (eo[G] > max_pairs || nv > max_vertices)
    return set_status(TC_ERR_OVERFLOW, "batch of %lld pairs and %lld vertices exceeds %lld / %lld",
                      (long long)eo[G], (long long)nv, (long long)max_pairs,
                      (long long)max_vertices);
  nv = 0;
  for (int32_t g = 0; g <= G; ++g) {
    p->block[g] = (int32_t)eo[g];
    p->block[G + 1 + g] = (int32_t)nv;
    if (g < G) nv += vn[g];
  }
  p->pairs = eo[G];
  p->vertices = nv;
  return TC_OK;
}

// Device batch region: descriptor, offset block, per-graph totals.
// Device region of a batch: descriptor, offsets block (edge_off then voff,
// max_graphs + 1 each), per-graph error flags, per-graph totals.  Everything
// before `totals` is one host-to-device copy per batch (the flags travel as
// zeros), the totals one copy back.
struct BatchRegion {
  size_t desc, block, gerr, totals, bytes;
};
BatchRegion batch_region(int32_t max_graphs) {
  BatchRegion r;
  r.desc = 0;
  r.block = align256(sizeof(BatchDesc));
  r.gerr = align256(r.block + sizeof(int32_t) * 2 * ((size_t)max_graphs + 1));
  r.totals = align256(r.gerr + sizeof(int32_t) * (size_t)max_graphs);
  r.bytes = align256(r.totals + sizeof(unsigned long long) * (size_t)max_graphs);
  return r;
}

// Graphs of a finished batch whose total is TC_COUNT_ERROR had an id out
// of range: the batch status is TC_ERR_ID_RANGE, every other total is exact.
tc_status batch_id_status(const uint64_t *totals, int32_t G) {
  int32_t first = -1, bad = 0;
  for (int32_t g = 0; g < G; ++g)
    if (totals[g] == TC_COUNT_ERROR) {
      if (first < 0) first = g;
      ++bad;
    }
  if (!bad) return set_status(TC_OK);
  return set_status(TC_ERR_ID_RANGE, "graph %d (%d of %d graphs) has an id outside [0, n_g)",
                    first, bad, G);
}

tc_status batch_impl(const int32_t *src, const int32_t *dst, int32_t G, const int64_t *eo,
                     const int32_t *vn, cudaStream_t st, uint64_t *totals_out) {
  BatchPlan p;
  tc_status s = plan_batch(G, eo, vn, kMaxItems, kMaxItems, &p);
  if (s != TC_OK) return s;
  if (G > 0 && !totals_out) return set_status(TC_ERR_INVALID_ARG, "totals_out is NULL");
  if (p.pairs > 0 && (!src || !dst)) return set_status(TC_ERR_INVALID_ARG, "src/dst is NULL");
  if (p.pairs == 0) {
    for (int32_t g = 0; g < G; ++g) totals_out[g] = 0;
    return set_status(TC_OK);
  }
  if (p.vertices == 0) return set_status(TC_ERR_ID_RANGE, "edges but no vertices");
  const Layout L = make_layout(p.pairs, (int32_t)p.vertices);
  const BatchRegion R = batch_region(G);
  keep_pool_memory();
  unsigned char *ws = nullptr;
  TC_CUDA(dev_alloc_async((void **)&ws, L.total + R.bytes, st), "workspace allocation");
  unsigned char *bd = ws + L.total;
  std::vector<unsigned char> staging(R.totals);
  BatchDesc desc{G, 0, reinterpret_cast<int32_t *>(bd + R.block),
                 reinterpret_cast<int32_t *>(bd + R.block) + (G + 1),
                 reinterpret_cast<int32_t *>(bd + R.gerr)};
  memcpy(staging.data(), &desc, sizeof(desc));
  memcpy(staging.data() + R.block, p.block.data(), sizeof(int32_t) * p.block.size());
  auto *totals_dev = reinterpret_cast<unsigned long long *>(bd + R.totals);
  s = TC_OK;
  cudaError_t e = cudaMemcpyAsync(bd, staging.data(), staging.size(), cudaMemcpyHostToDevice, st);
  Ctrl *h = host_ctrl();
  PhaseTimer pt(st, true);
  if (e != cudaSuccess) s = cuda_fail(e, "batch descriptor copy");
  else if (!h) s = set_status(TC_ERR_OOM, "pinned staging buffer");
  if (s == TC_OK) {
    const BatchRun br{reinterpret_cast<const BatchDesc *>(bd), G, totals_dev};
    s = enqueue_core(src, dst, p.pairs, (int32_t)p.vertices, st, ws, L, nullptr, nullptr, &br,
                     current_tuning(), pt, h);
  }
  if (s == TC_OK) {
    e = cudaMemcpyAsync(totals_out, totals_dev, sizeof(uint64_t) * G, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = cuda_fail(e, "totals copy");
  }
  cudaFreeAsync(ws, st);
  e = cudaStreamSynchronize(st);
  if (s != TC_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  pt.fold();
  s = finish_core(h, (int32_t)p.vertices, nullptr);
  if (s != TC_OK) return s;
  return batch_id_status(totals_out, G);
}

}  // namespace

// A persistent batch engine: device buffers sized once, and the whole batch
// pipeline captured once as a CUDA graph.  Every batch runs with the same
// shape -- capacity pairs and vertices, the pairs past the batch's end being
// padding that is never keyed -- so one instantiated graph is replayed for
// all of them; the batch's offsets reach the device through a copy node that
// reads a pinned staging block rewritten before each launch.
struct tc_engine {
  int device = -1;
  int64_t max_pairs = 0;
  int32_t max_vertices = 0, max_graphs = 0;
  Tuning tune = kDefaultTuning;
  cudaStream_t st = nullptr;
  unsigned char *dbuf = nullptr;   // device: src, dst, workspace, batch region
  unsigned char *hbuf = nullptr;   // pinned: descriptor + offsets, control block, totals
  int32_t *src = nullptr, *dst = nullptr;
  unsigned char *ws = nullptr, *bd = nullptr;
  Layout L{};
  BatchRegion R{};
  Ctrl *ctrl_h = nullptr;
  unsigned long long *totals_h = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool busy = false;
  int32_t pending_graphs = 0;
  int32_t pending_vertices = 0;
};

namespace {

void engine_release(tc_engine *e) {
  if (!e) return;
  if (e->st) cudaStreamSynchronize(e->st);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  if (e->dbuf) cudaFree(e->dbuf);
  if (e->hbuf) cudaFreeHost(e->hbuf);
  if (e->st) cudaStreamDestroy(e->st);
  delete e;
}

tc_status engine_build(tc_engine *e) {
  TC_CUDA(cudaGetDevice(&e->device), "current device");
  TC_CUDA(prepare_count_kernels(), "count kernel attributes");
  TC_CUDA(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking), "stream");
  e->L = make_layout(e->max_pairs, e->max_vertices);
  e->R = batch_region(e->max_graphs);
  const size_t in_bytes = align256(sizeof(int32_t) * (size_t)e->max_pairs);
  TC_CUDA(dev_alloc((void **)&e->dbuf, 2 * in_bytes + e->L.total + e->R.bytes),
          "engine device memory");
  e->src = reinterpret_cast<int32_t *>(e->dbuf);
  e->dst = reinterpret_cast<int32_t *>(e->dbuf + in_bytes);
  e->ws = e->dbuf + 2 * in_bytes;
  e->bd = e->ws + e->L.total;
  const size_t h_ctrl = align256(e->R.totals);
  const size_t h_totals = align256(h_ctrl + sizeof(Ctrl));
  TC_CUDA(cudaMallocHost((void **)&e->hbuf, h_totals + sizeof(unsigned long long) *
                                                           (size_t)e->max_graphs),
          "engine pinned memory");
  e->ctrl_h = reinterpret_cast<Ctrl *>(e->hbuf + h_ctrl);
  e->totals_h = reinterpret_cast<unsigned long long *>(e->hbuf + h_totals);
  BatchDesc desc{0, 0, reinterpret_cast<int32_t *>(e->bd + e->R.block),
                 reinterpret_cast<int32_t *>(e->bd + e->R.block) + (e->max_graphs + 1),
                 reinterpret_cast<int32_t *>(e->bd + e->R.gerr)};
  memcpy(e->hbuf, &desc, sizeof(desc));
  memset(e->hbuf + e->R.block, 0, e->R.totals - e->R.block);  // offsets; error flags stay 0

  // capture: offsets in, the pipeline, control block and totals out
  TC_CUDA(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  PhaseTimer pt(e->st, false);
  auto *totals_dev = reinterpret_cast<unsigned long long *>(e->bd + e->R.totals);
  const BatchRun br{reinterpret_cast<const BatchDesc *>(e->bd), e->max_graphs, totals_dev};
  cudaError_t ce = cudaMemcpyAsync(e->bd, e->hbuf, e->R.totals, cudaMemcpyHostToDevice, e->st);
  tc_status s = TC_OK;
  if (ce == cudaSuccess)
    s = enqueue_core(e->src, e->dst, e->max_pairs, e->max_vertices, e->st, e->ws, e->L, nullptr,
                     nullptr, &br, e->tune, pt, e->ctrl_h);
  if (ce == cudaSuccess && s == TC_OK)
    ce = cudaMemcpyAsync(e->totals_h, totals_dev, sizeof(unsigned long long) * e->max_graphs,
                         cudaMemcpyDeviceToHost, e->st);
  cudaGraph_t g = nullptr;
  const cudaError_t end = cudaStreamEndCapture(e->st, &g);
  e->graph = g;
  if (s != TC_OK) return s;
  if (ce != cudaSuccess) return cuda_fail(ce, "capture");
  if (end != cudaSuccess) return cuda_fail(end, "end capture");
  TC_CUDA(cudaGraphInstantiate(&e->exec, e->graph, 0), "graph instantiate");
  return TC_OK;
}

}  // namespace

extern "C" {

uint64_t tc_count(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                  tc_stream_t stream) {
  uint64_t T = 0;
  tc_status s = count_impl(src, dst, m, n, (cudaStream_t)stream, nullptr, 0, nullptr, nullptr, &T);
  return s == TC_OK ? T : TC_COUNT_ERROR;
}

tc_status tc_count_per_vertex(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                              tc_stream_t stream, int64_t *t_out, int32_t *deg_out,
                              uint64_t *total_out) {
  if (n > 0 && !t_out) return set_status(TC_ERR_INVALID_ARG, "t_out is NULL");
  uint64_t T = 0;
  tc_status s =
      count_impl(src, dst, m, n, (cudaStream_t)stream, nullptr, 0, t_out, deg_out, &T);
  if (s == TC_OK && total_out) *total_out = T;
  return s;
}

tc_status tc_count_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                        int32_t part, int32_t parts, tc_stream_t stream, uint64_t *total_out) {
  if (!total_out) return set_status(TC_ERR_INVALID_ARG, "total_out is NULL");
  return count_impl(src, dst, m, n, (cudaStream_t)stream, nullptr, 0, nullptr, nullptr,
                    total_out, part, parts);
}

tc_status tc_count_per_vertex_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                                   int32_t part, int32_t parts, tc_stream_t stream,
                                   int64_t *t_out, int32_t *deg_out, uint64_t *total_out) {
  if (n > 0 && !t_out) return set_status(TC_ERR_INVALID_ARG, "t_out is NULL");
  uint64_t T = 0;
  tc_status s = count_impl(src, dst, m, n, (cudaStream_t)stream, nullptr, 0, t_out, deg_out, &T,
                           part, parts);
  if (s == TC_OK && total_out) *total_out = T;
  return s;
}

tc_status tc_clustering(const int64_t *t, const int32_t *deg, int32_t n, tc_stream_t stream,
                        double *cc_out, double *transitivity_out) {
  if (n < 0) return set_status(TC_ERR_INVALID_ARG, "n < 0");
  if (n > 0 && (!t || !deg)) return set_status(TC_ERR_INVALID_ARG, "t/deg is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    if (transitivity_out) *transitivity_out = 0.0;
    return set_status(TC_OK);
  }
  keep_pool_memory();
  unsigned char *buf = nullptr;
  TC_CUDA(dev_alloc_async((void **)&buf, 32, st), "scratch allocation");
  auto *sums = reinterpret_cast<unsigned long long *>(buf);
  double *dev_out = reinterpret_cast<double *>(buf + 16);
  TC_CUDA(cudaMemsetAsync(buf, 0, 32, st), "memset");
  launch_clustering(t, deg, n, cc_out, sums, st);
  launch_transitivity(sums, dev_out, st);
  double h = 0.0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && transitivity_out)
    e = cudaMemcpyAsync(&h, dev_out, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(buf, st);
  if (e == cudaSuccess && transitivity_out) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "clustering");
  if (transitivity_out) *transitivity_out = h;
  return set_status(TC_OK);
}

tc_status tc_count_host(const int32_t *src_host, const int32_t *dst_host, int64_t m, int32_t n,
                        uint64_t *total_out) {
  return host_impl(src_host, dst_host, m, n, nullptr, nullptr, total_out, false);
}

tc_status tc_count_per_vertex_host(const int32_t *src_host, const int32_t *dst_host, int64_t m,
                                   int32_t n, int64_t *t_host, int32_t *deg_host,
                                   uint64_t *total_out) {
  return host_impl(src_host, dst_host, m, n, t_host, deg_host, total_out, true);
}

size_t tc_workspace_bytes(int64_t m, int32_t n) {
  if (m < 0 || n < 0 || m > kMaxItems || (int64_t)n > kMaxItems) return 0;
  return make_layout(m, n, true, current_tuning().hub_vertices).total;
}

tc_status tc_count_ws(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                      tc_stream_t stream, void *ws, size_t ws_bytes, uint64_t *total_out) {
  if (!ws || !total_out) return set_status(TC_ERR_INVALID_ARG, "ws/total_out is NULL");
  return count_impl(src, dst, m, n, (cudaStream_t)stream, ws, ws_bytes, nullptr, nullptr,
                    total_out);
}

tc_status tc_count_noalloc(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                           tc_stream_t stream, uint64_t *total_out) {
  if (!total_out) return set_status(TC_ERR_INVALID_ARG, "total_out is NULL");
  tc_status s = check_args(src, dst, m, n);
  if (s != TC_OK) return s;
  if (m > 0 && n == 0) return set_status(TC_ERR_ID_RANGE, "n = 0 but m > 0");
  if (m == 0) {
    *total_out = 0;
    return set_status(TC_OK);
  }
  // no dense hub block here: its matrix alone would not fit the scratch
  const Layout L = make_layout(m, n);
  if (L.total > (size_t)TC_NOALLOC_SCRATCH_BYTES)
    return set_status(TC_ERR_OVERFLOW,
                      "m=%lld, n=%d needs %zu bytes of scratch; the static scratch holds %zu",
                      (long long)m, n, L.total, (size_t)TC_NOALLOC_SCRATCH_BYTES);
  unsigned char *ws = nullptr;
  s = noalloc_scratch(&ws);
  if (s != TC_OK) return s;
  Ctrl staging;  // pageable host memory: no pinned allocation either
  return run_core(src, dst, m, n, (cudaStream_t)stream, ws, L, nullptr, nullptr, total_out,
                  &staging, false);
}

tc_status tc_count_batch(const int32_t *src, const int32_t *dst, int32_t num_graphs,
                         const int64_t *edge_offsets, const int32_t *vertex_counts,
                         tc_stream_t stream, uint64_t *totals_out) {
  return batch_impl(src, dst, num_graphs, edge_offsets, vertex_counts, (cudaStream_t)stream,
                    totals_out);
}

tc_status tc_engine_create(int64_t max_pairs, int32_t max_vertices, int32_t max_graphs,
                           const tc_tuning *tuning, tc_engine **out) {
  if (!out) return set_status(TC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_pairs < 1 || max_vertices < 1 || max_graphs < 1)
    return set_status(TC_ERR_INVALID_ARG, "capacities must be positive");
  if (max_pairs > kMaxItems || (int64_t)max_vertices > kMaxItems)
    return set_status(TC_ERR_OVERFLOW, "max_pairs or max_vertices beyond 2^31 - 2^10");
  if (!padded_fits(max_pairs, max_vertices))
    return set_status(TC_ERR_OVERFLOW, "padded lists of the capacities exceed 2^31 words");
  tc_engine *e = new tc_engine;
  e->max_pairs = max_pairs;
  e->max_vertices = max_vertices;
  e->max_graphs = max_graphs;
  e->tune = tuning ? Tuning{tuning->warp_max_list, tuning->warp_max_partners,
                            max(tuning->heavy_ratio_pct, 100), tuning->hub_min_edges,
                            tuning->hub_vertices}
                   : current_tuning();
  tc_status s = engine_build(e);
  if (s != TC_OK) {
    const tc_status keep = s;
    char detail[256];
    memcpy(detail, t_detail, sizeof(detail));
    engine_release(e);
    t_last = keep;
    memcpy(t_detail, detail, sizeof(detail));
    return keep;
  }
  *out = e;
  return set_status(TC_OK);
}

tc_status tc_engine_submit(tc_engine *e, const int32_t *src, const int32_t *dst,
                           int32_t inputs_on_host, int32_t num_graphs,
                           const int64_t *edge_offsets, const int32_t *vertex_counts) {
  if (!e) return set_status(TC_ERR_INVALID_ARG, "engine is NULL");
  if (e->busy) return set_status(TC_ERR_INVALID_ARG, "engine busy: wait for the last batch");
  if (num_graphs > e->max_graphs)
    return set_status(TC_ERR_OVERFLOW, "%d graphs exceed the engine's %d", num_graphs,
                      e->max_graphs);
  BatchPlan p;
  tc_status s = plan_batch(num_graphs, edge_offsets, vertex_counts, e->max_pairs,
                           e->max_vertices, &p);
  if (s != TC_OK) return s;
  if (p.pairs > 0 && (!src || !dst)) return set_status(TC_ERR_INVALID_ARG, "src/dst is NULL");
  int dev = -1;
  TC_CUDA(cudaGetDevice(&dev), "current device");
  if (dev != e->device) return set_status(TC_ERR_INVALID_ARG, "engine belongs to device %d", e->device);
  const cudaMemcpyKind kind = inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const size_t bytes = sizeof(int32_t) * (size_t)p.pairs;
  if (bytes) {
    TC_CUDA(cudaMemcpyAsync(e->src, src, bytes, kind, e->st), "copy src");
    TC_CUDA(cudaMemcpyAsync(e->dst, dst, bytes, kind, e->st), "copy dst");
  }
  // the staging block keeps its layout: edge offsets then vertex offsets,
  // max_graphs + 1 slots each; the graph's copy node moves it to the device
  reinterpret_cast<BatchDesc *>(e->hbuf)->num_graphs = num_graphs;
  memcpy(e->hbuf + e->R.block, p.block.data(), sizeof(int32_t) * (size_t)(num_graphs + 1));
  memcpy(e->hbuf + e->R.block + sizeof(int32_t) * ((size_t)e->max_graphs + 1),
         p.block.data() + num_graphs + 1, sizeof(int32_t) * (size_t)(num_graphs + 1));
  TC_CUDA(cudaGraphLaunch(e->exec, e->st), "graph launch");
  note_launch();
  e->busy = true;
  e->pending_graphs = num_graphs;
  e->pending_vertices = (int32_t)p.vertices;
  return set_status(TC_OK);
}

tc_status tc_engine_submit_parts(tc_engine *e, int32_t num_graphs, const int32_t *const *srcs,
                                 const int32_t *const *dsts, const int64_t *pair_counts,
                                 const int32_t *vertex_counts, int32_t inputs_on_host) {
  if (!e) return set_status(TC_ERR_INVALID_ARG, "engine is NULL");
  if (e->busy) return set_status(TC_ERR_INVALID_ARG, "engine busy: wait for the last batch");
  if (num_graphs < 0 || num_graphs > e->max_graphs)
    return set_status(TC_ERR_OVERFLOW, "%d graphs for an engine of %d", num_graphs,
                      e->max_graphs);
  if (num_graphs > 0 && (!srcs || !dsts || !pair_counts))
    return set_status(TC_ERR_INVALID_ARG, "NULL part arrays");
  std::vector<int64_t> eo((size_t)num_graphs + 1, 0);
  for (int32_t g = 0; g < num_graphs; ++g) {
    if (pair_counts[g] < 0) return set_status(TC_ERR_INVALID_ARG, "pair_counts[%d] < 0", g);
    if (pair_counts[g] > 0 && (!srcs[g] || !dsts[g]))
      return set_status(TC_ERR_INVALID_ARG, "part %d is NULL", g);
    eo[g + 1] = eo[g] + pair_counts[g];
  }
  BatchPlan p;
  tc_status s = plan_batch(num_graphs, eo.data(), vertex_counts, e->max_pairs, e->max_vertices, &p);
  if (s != TC_OK) return s;
  int dev = -1;
  TC_CUDA(cudaGetDevice(&dev), "current device");
  if (dev != e->device)
    return set_status(TC_ERR_INVALID_ARG, "engine belongs to device %d", e->device);
  const cudaMemcpyKind kind = inputs_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int32_t g = 0; g < num_graphs; ++g) {
    const size_t bytes = sizeof(int32_t) * (size_t)pair_counts[g];
    if (!bytes) continue;
    TC_CUDA(cudaMemcpyAsync(e->src + eo[g], srcs[g], bytes, kind, e->st), "copy src part");
    TC_CUDA(cudaMemcpyAsync(e->dst + eo[g], dsts[g], bytes, kind, e->st), "copy dst part");
  }
  reinterpret_cast<BatchDesc *>(e->hbuf)->num_graphs = num_graphs;
  memcpy(e->hbuf + e->R.block, p.block.data(), sizeof(int32_t) * (size_t)(num_graphs + 1));
  memcpy(e->hbuf + e->R.block + sizeof(int32_t) * ((size_t)e->max_graphs + 1),
         p.block.data() + num_graphs + 1, sizeof(int32_t) * (size_t)(num_graphs + 1));
  TC_CUDA(cudaGraphLaunch(e->exec, e->st), "graph launch");
  note_launch();
  e->busy = true;
  e->pending_graphs = num_graphs;
  e->pending_vertices = (int32_t)p.vertices;
  return set_status(TC_OK);
}

int32_t tc_engine_poll(tc_engine *e) {
  if (!e || !e->busy) return 1;
  return cudaStreamQuery(e->st) == cudaErrorNotReady ? 0 : 1;
}

tc_status tc_engine_wait(tc_engine *e, uint64_t *totals_out) {
  if (!e) return set_status(TC_ERR_INVALID_ARG, "engine is NULL");
  if (!e->busy) return set_status(TC_ERR_INVALID_ARG, "no batch submitted");
  const cudaError_t ce = cudaStreamSynchronize(e->st);
  e->busy = false;
  if (ce != cudaSuccess) return cuda_fail(ce, "synchronize");
  tc_status s = finish_core(e->ctrl_h, e->pending_vertices, nullptr);
  if (s != TC_OK) return s;
  if (totals_out)
    for (int32_t g = 0; g < e->pending_graphs; ++g) totals_out[g] = e->totals_h[g];
  return batch_id_status(reinterpret_cast<const uint64_t *>(e->totals_h), e->pending_graphs);
}

tc_status tc_engine_count(tc_engine *e, const int32_t *src, const int32_t *dst,
                          int32_t inputs_on_host, int32_t num_graphs,
                          const int64_t *edge_offsets, const int32_t *vertex_counts,
                          uint64_t *totals_out) {
  tc_status s = tc_engine_submit(e, src, dst, inputs_on_host, num_graphs, edge_offsets,
                                 vertex_counts);
  if (s != TC_OK) return s;
  return tc_engine_wait(e, totals_out);
}

tc_status tc_count_work_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                             int32_t part, int32_t parts, tc_stream_t stream, tc_work *out) {
  if (!out) return set_status(TC_ERR_INVALID_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  tc_status s = check_args(src, dst, m, n);
  if (s != TC_OK) return s;
  if (parts < 1 || part < 0 || part >= parts)
    return set_status(TC_ERR_INVALID_ARG, "part %d of %d", part, parts);
  if (m > 0 && n == 0) return set_status(TC_ERR_ID_RANGE, "n = 0 but m > 0");
  out->vertices = n;
  if (m == 0) return set_status(TC_OK);
  cudaStream_t st = (cudaStream_t)stream;
  const Layout L = make_layout(m, n, true, current_tuning().hub_vertices);
  keep_pool_memory();
  unsigned char *ws = nullptr;
  TC_CUDA(dev_alloc_async((void **)&ws, L.total, st), "workspace allocation");
  Ctrl *h = host_ctrl();
  PhaseTimer pt(st, false);
  if (!h) s = set_status(TC_ERR_OOM, "pinned staging buffer");
  else s = enqueue_core(src, dst, m, n, st, ws, L, nullptr, nullptr, nullptr, current_tuning(), pt,
                        h, true, part, parts);
  cudaFreeAsync(ws, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s != TC_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  uint64_t T = 0;
  s = finish_core(h, n, &T);
  if (s != TC_OK) return s;
  out->edges = h->m;
  out->triangles = T;
  out->lookups = (int64_t)h->work[0];
  out->inserts = (int64_t)h->work[1];
  out->merge_work = (int64_t)h->work[2];
  out->max_out_degree = (int32_t)h->work[3];
  for (int k = 0; k < kHubSizes; ++k) out->hub_lookups[k] = (int64_t)h->work[4 + k];
  out->dense_vertices = h->hub_on ? (int32_t)h->hub_size : 0;
  out->dense_triangles = h->hub_triangles;
  return set_status(TC_OK);
}

tc_status tc_count_work(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                        tc_stream_t stream, tc_work *out) {
  return tc_count_work_part(src, dst, m, n, 0, 1, stream, out);
}

tc_status tc_engine_destroy(tc_engine *e) {
  engine_release(e);
  return set_status(TC_OK);
}

tc_status tc_set_tuning(const tc_tuning *t) {
  if (t && (t->warp_max_list < 0 || t->warp_max_partners < 0 || t->heavy_ratio_pct < 100 ||
            t->hub_vertices < 128 || t->hub_vertices > kHubMaxSize || t->hub_vertices % 128))
    return set_status(TC_ERR_INVALID_ARG, "tuning values out of range");
  std::lock_guard<std::mutex> lk(g_tuning_mu);
  g_tuning = t ? Tuning{t->warp_max_list, t->warp_max_partners, t->heavy_ratio_pct,
                        t->hub_min_edges, t->hub_vertices}
               : kDefaultTuning;
  return set_status(TC_OK);
}

tc_status tc_get_tuning(tc_tuning *out) {
  if (!out) return set_status(TC_ERR_INVALID_ARG, "out is NULL");
  const Tuning t = current_tuning();
  out->warp_max_list = t.warp_max_list;
  out->warp_max_partners = t.warp_max_partners;
  out->heavy_ratio_pct = t.heavy_ratio_pct;
  out->hub_min_edges = t.hub_min_edges;
  out->hub_vertices = t.hub_vertices;
  return set_status(TC_OK);
}

tc_status tc_debug_set_wait_limit(uint32_t spin_limit, int32_t unpublished_tile) {
  TC_CUDA(cudaDeviceSynchronize(), "synchronize");
  TC_CUDA(set_wait_hooks(spin_limit, unpublished_tile < 0 ? 0xffffffffu : (uint32_t)unpublished_tile),
          "wait hooks");
  return set_status(TC_OK);
}

tc_status tc_debug_fail_allocations(int32_t skip, int32_t count) {
  std::lock_guard<std::mutex> lk(g_inject_mu);
  g_inject_skip = skip > 0 ? skip : 0;
  g_inject_fail = count > 0 ? count : 0;
  g_inject_on.store(g_inject_fail > 0);
  return set_status(TC_OK);
}

tc_status tc_debug_reset(void) {
  tc_debug_fail_allocations(0, 0);
  return tc_debug_set_wait_limit(kSpinLimit, -1);
}

tc_status tc_last_error(void) { return t_last; }

const char *tc_last_error_detail(void) { return t_detail; }

const char *tc_status_string(tc_status s) {
  switch (s) {
    case TC_OK: return "ok";
    case TC_ERR_INVALID_ARG: return "invalid argument";
    case TC_ERR_ID_RANGE: return "vertex id out of range";
    case TC_ERR_OOM: return "out of device memory";
    case TC_ERR_CUDA: return "CUDA error";
    case TC_ERR_TIMEOUT: return "device wait timed out";
    case TC_ERR_OVERFLOW: return "size beyond limits";
  }
  return "unknown status";
}

uint64_t tc_launch_count(void) { return g_launches.load(); }

void tc_profile_enable(int on) { g_prof_on.store(on ? 1 : 0); }

void tc_profile_read(double *ms_out, uint64_t *launches_out, int reset) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int i = 0; i < TC_NUM_PHASES; ++i) {
    if (ms_out) ms_out[i] = g_prof_ms[i];
    if (launches_out) launches_out[i] = g_prof_launches[i];
    if (reset) {
      g_prof_ms[i] = 0.0;
      g_prof_launches[i] = 0;
    }
  }
}

const char *tc_phase_name(int phase) {
  return (phase >= 0 && phase < TC_NUM_PHASES) ? kPhaseNames[phase] : "?";
}

}  // extern "C"
