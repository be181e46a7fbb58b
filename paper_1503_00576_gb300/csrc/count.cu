// count.cu -- counting phase of the forward algorithm on sm_103a.
//
// Sec. III-C of the paper counts with one thread per forward edge (u, v),
// each running a two-pointer merge of N+(u) and N+(v) from global memory,
// and then sums the per-thread counts (thrust::reduce).  The result is
// sum over forward edges of |N+(u) & N+(v)|.  The same sum is computed here
// row by row, which suits a GB300 SM better than a per-thread merge:
//
//  * a row u (its forward list N+(u), sorted, length du) is staged once in
//    shared memory as an open-addressing hash set (multiplicative hashing,
//    linear probing, load <= 1/2), by one warp for du <= 256 or by a whole
//    CTA for longer rows;
//  * for the <= 32 forward neighbours v of one chunk of N+(u), the lists
//    N+(v) are read back to back as one flat sequence: in each 32-wide window
//    lane p takes flat element p, finds its list by a ballot over the list
//    starts plus an OR-reduction of the starts inside the window, and tests
//    membership in the hash set.  Loads of N+(v) are coalesced and every lane
//    does useful work however short the lists are;
//  * counts stay in registers and are reduced per warp (shuffles) into one
//    uint64 atomic per warp at the end (the paper's reduction, fused).
//
// Per-vertex counts t(v) (Sec. I: the numerator of the clustering
// coefficient): a triangle found at row u, neighbour v, element w adds one
// to t(u), t(v) and t(w).  t(u) is summed over the row, t(v) over the chunk
// (shared-memory counters per neighbour) and t(w) in a 16-bit counter beside
// w's hash slot, so global atomics scale with the number of forward edges,
// not with the number of triangles.
//
// Rows longer than the CTA table (du > 8192, never seen in the workloads but
// allowed by the bound du <= sqrt(2m)) fall back to a binary search of
// N+(u) in global memory for membership.
#include "tc_common.cuh"

namespace tc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCountThreads = 512;
constexpr int kCountWarps = kCountThreads / 32;
constexpr int kCtaSlots = 16384;                      // hash slots per CTA
constexpr int kWarpSlots = kCtaSlots / kCountWarps;   // per warp in warp mode
constexpr int kRowChunk = 4;                          // rows grabbed per atomic
static_assert(kWarpSlots >= 4 * kWarpMaxRow, "warp tables must keep load <= 1/4");

__device__ __forceinline__ uint32_t hash_slot(uint32_t x, int log_slots) {
  return (x * 0x9E3779B1u) >> (32 - log_slots);
}

__device__ __forceinline__ int ceil_log2(uint32_t x) {
  return x <= 1 ? 0 : 32 - __clz(x - 1);
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

struct WarpScratch {
  int32_t start[32];  // flat start of each non-empty list of the chunk
  int32_t base[32];   // col index of flat position 0 of that list
  int32_t v[32];      // the neighbour owning the list (per-vertex mode)
  uint32_t vc[32];    // triangles found through that neighbour
};

// Empties the hash set tab[0..2^log_slots) (and its 16-bit counters in
// per-vertex mode).  The calling group (a warp or the whole CTA) must
// synchronise before filling it.
template <bool PV>
__device__ __forceinline__ void clear_table(int32_t *tab, uint32_t *cnt, int log_slots, int rank,
                                            int group) {
  const uint32_t slots = 1u << log_slots;
  for (uint32_t i = rank; i < slots; i += group) tab[i] = -1;
  if (PV)
    for (uint32_t i = rank; i < (slots + 1) / 2; i += group) cnt[i] = 0u;
}

// Inserts col[beg..beg+du) (distinct ids) into the emptied hash set.
__device__ __forceinline__ void fill_table(const int32_t *__restrict__ col, int32_t beg,
                                           int32_t du, int32_t *tab, int log_slots, int rank,
                                           int group) {
  const uint32_t msk = (1u << log_slots) - 1u;
  for (int32_t i = rank; i < du; i += group) {
    const int32_t x = __ldg(col + beg + i);
    uint32_t h = hash_slot((uint32_t)x, log_slots);
    while (atomicCAS(&tab[h], -1, x) != -1) h = (h + 1u) & msk;
  }
}

// Adds each slot's triangle count to t(w) for the w stored in that slot.
__device__ __forceinline__ void flush_table(const int32_t *tab, const uint32_t *cnt,
                                            int log_slots, int rank, int group, int64_t *t) {
  const uint32_t slots = 1u << log_slots;
  for (uint32_t i = rank; i < slots; i += group) {
    const uint32_t c = (cnt[i >> 1] >> (16 * (i & 1))) & 0xffffu;
    if (c) atomicAdd((unsigned long long *)&t[tab[i]], (unsigned long long)c);
  }
}

// Intersections of N+(u) (in the table, or in global memory when TABLE is
// false) with N+(v) for the forward neighbours v = col[beg+c0 .. beg+c0+32).
template <bool PV, bool TABLE>
__device__ __forceinline__ void probe_chunk(const int32_t *__restrict__ off,
                                            const int32_t *__restrict__ col, int32_t beg,
                                            int32_t du, int32_t c0, const int32_t *tab,
                                            uint32_t *cnt, int log_slots, WarpScratch &ws,
                                            int64_t *t, uint64_t &found_total,
                                            uint64_t &found_row) {
  const int lane = threadIdx.x & 31;
  const int32_t j = c0 + lane;
  int32_t v = 0, vb = 0, dv = 0;
  if (j < du) {
    v = __ldg(col + beg + j);
    vb = __ldg(off + v);
    dv = __ldg(off + v + 1) - vb;
  }
  const uint32_t nonempty = __ballot_sync(kFull, dv > 0);
  if (nonempty == 0) return;
  const int k = __popc(nonempty);
  const int rank = __popc(nonempty & ((1u << lane) - 1u));
  int32_t incl = dv;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  const int32_t total = __shfl_sync(kFull, incl, 31);
  if (dv > 0) {
    ws.start[rank] = incl - dv;
    ws.base[rank] = vb - (incl - dv);
    if (PV) {
      ws.v[rank] = v;
      ws.vc[rank] = 0u;
    }
  }
  __syncwarp();
  const int32_t my_start = lane < k ? ws.start[lane] : INT32_MAX;
  const int32_t my_base = lane < k ? ws.base[lane] : 0;
  const uint32_t msk = (1u << log_slots) - 1u;
  for (int32_t w0 = 0; w0 < total; w0 += 32) {
    const int r0 = __popc(__ballot_sync(kFull, my_start <= w0)) - 1;
    const uint32_t bit =
        (my_start > w0 && my_start < w0 + 32) ? (1u << (my_start - w0)) : 0u;
    const uint32_t starts = __reduce_or_sync(kFull, bit);
    const int r = r0 + __popc(starts & ((2u << lane) - 1u));
    const int32_t base = __shfl_sync(kFull, my_base, r);
    const int32_t p = w0 + lane;
    if (p < total) {
      const int32_t x = __ldg(col + base + p);
      bool found = false;
      uint32_t h = 0;
      if (TABLE) {
        h = hash_slot((uint32_t)x, log_slots);
        for (;;) {
          const int32_t y = tab[h];
          if (y == x) { found = true; break; }
          if (y < 0) break;
          h = (h + 1u) & msk;
        }
      } else {
        int32_t lo = beg, hi = beg + du;
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (__ldg(col + mid) < x) lo = mid + 1; else hi = mid;
        }
        found = lo < beg + du && __ldg(col + lo) == x;
      }
      if (found) {
        ++found_total;
        if (PV) {
          ++found_row;
          atomicAdd(&ws.vc[r], 1u);
          if (TABLE)
            atomicAdd(&cnt[h >> 1], 1u << (16 * (h & 1u)));
          else
            atomicAdd((unsigned long long *)&t[x], 1ull);
        }
      }
    }
  }
  if (PV) {
    __syncwarp();
    if (lane < k && ws.vc[lane])
      atomicAdd((unsigned long long *)&t[ws.v[lane]], (unsigned long long)ws.vc[lane]);
  }
  __syncwarp();
}

template <bool PV>
__global__ void __launch_bounds__(kCountThreads)
k_count(const int32_t *__restrict__ off, const int32_t *__restrict__ col,
        const int32_t *__restrict__ warp_rows, const int32_t *__restrict__ cta_rows, Ctrl *ctrl,
        int64_t *t) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t *tab = reinterpret_cast<int32_t *>(smem);                    // kCtaSlots
  uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + 4 * kCtaSlots);   // kCtaSlots/2 (PV)
  __shared__ WarpScratch s_ws[kCountWarps];
  __shared__ int32_t s_row;
  __shared__ unsigned long long s_rowsum;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n_cta = ctrl->n_cta_rows, n_warp = ctrl->n_warp_rows;
  uint64_t found_total = 0;

  // ---- long rows: a whole CTA per row ----
  for (;;) {
    if (tid == 0) {
      s_row = (int32_t)atomicAdd(&ctrl->next_cta_row, 1u);
      s_rowsum = 0ull;
    }
    __syncthreads();
    const uint32_t r = (uint32_t)s_row;
    if (r >= n_cta) break;
    const int32_t u = __ldg(cta_rows + r);
    const int32_t beg = __ldg(off + u), du = __ldg(off + u + 1) - beg;
    int log_slots = ceil_log2(4u * (uint32_t)du);
    if ((1 << log_slots) > kCtaSlots) log_slots = ceil_log2(2u * (uint32_t)du);
    const bool use_table = (1 << log_slots) <= kCtaSlots;
    if (use_table) {
      clear_table<PV>(tab, cnt, log_slots, tid, kCountThreads);
      __syncthreads();
      fill_table(col, beg, du, tab, log_slots, tid, kCountThreads);
    }
    __syncthreads();
    uint64_t found_row = 0;
    for (int32_t c0 = warp * 32; c0 < du; c0 += kCountThreads) {
      if (use_table)
        probe_chunk<PV, true>(off, col, beg, du, c0, tab, cnt, log_slots, s_ws[warp], t,
                              found_total, found_row);
      else
        probe_chunk<PV, false>(off, col, beg, du, c0, tab, cnt, 1, s_ws[warp], t, found_total,
                               found_row);
    }
    if (PV) {
      found_row = warp_sum_u64(found_row);
      if (lane == 0 && found_row) atomicAdd(&s_rowsum, (unsigned long long)found_row);
    }
    __syncthreads();
    if (PV) {
      if (tid == 0 && s_rowsum) atomicAdd((unsigned long long *)&t[u], s_rowsum);
      if (use_table) flush_table(tab, cnt, log_slots, tid, kCountThreads, t);
    }
    __syncthreads();
  }

  // ---- short rows: one warp per row, private table ----
  int32_t *wtab = tab + warp * kWarpSlots;
  uint32_t *wcnt = cnt + warp * (kWarpSlots / 2);
  for (;;) {
    uint32_t r0 = 0;
    if (lane == 0) r0 = atomicAdd(&ctrl->next_warp_row, (uint32_t)kRowChunk);
    r0 = __shfl_sync(kFull, r0, 0);
    if (r0 >= n_warp) break;
    const uint32_t r1 = min(r0 + (uint32_t)kRowChunk, n_warp);
    for (uint32_t r = r0; r < r1; ++r) {
      const int32_t u = __ldg(warp_rows + r);
      const int32_t beg = __ldg(off + u), du = __ldg(off + u + 1) - beg;
      const int log_slots = ceil_log2(4u * (uint32_t)du);
      clear_table<PV>(wtab, wcnt, log_slots, lane, 32);
      __syncwarp();
      fill_table(col, beg, du, wtab, log_slots, lane, 32);
      __syncwarp();
      uint64_t found_row = 0;
      for (int32_t c0 = 0; c0 < du; c0 += 32)
        probe_chunk<PV, true>(off, col, beg, du, c0, wtab, wcnt, log_slots, s_ws[warp], t,
                              found_total, found_row);
      if (PV) {
        found_row = warp_sum_u64(found_row);
        if (lane == 0 && found_row) atomicAdd((unsigned long long *)&t[u], found_row);
        __syncwarp();
        flush_table(wtab, wcnt, log_slots, lane, 32, t);
      }
      __syncwarp();
    }
  }

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

// transitivity = 3T / wedges with T = (sum t) / 3: one float64 division.
__global__ void k_transitivity(const unsigned long long *sums, double *out) {
  const unsigned long long three_t = sums[0];  // sum of t(v) is exactly 3T
  const unsigned long long wedges = sums[1];
  out[0] = wedges ? (double)three_t / (double)wedges : 0.0;
}

constexpr int kMaxDevices = 64;

}  // namespace

cudaError_t launch_count(const int32_t *off, const int32_t *col, const int32_t *warp_rows,
                         const int32_t *cta_rows, Ctrl *ctrl, int64_t *t, cudaStream_t st) {
  const bool pv = t != nullptr;
  const size_t smem = (size_t)4 * kCtaSlots + (pv ? (size_t)2 * kCtaSlots : 0);
  static int grid_cache[kMaxDevices][2];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int grid = (dev >= 0 && dev < kMaxDevices) ? grid_cache[dev][pv] : 0;
  if (grid == 0) {
    e = pv ? cudaFuncSetAttribute(k_count<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem)
           : cudaFuncSetAttribute(k_count<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (pv)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count<true>, kCountThreads, smem);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count<false>, kCountThreads,
                                                        smem);
    if (e != cudaSuccess) return e;
    grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < kMaxDevices) grid_cache[dev][pv] = grid;
  }
  if (pv)
    k_count<true><<<grid, kCountThreads, smem, st>>>(off, col, warp_rows, cta_rows, ctrl, t);
  else
    k_count<false><<<grid, kCountThreads, smem, st>>>(off, col, warp_rows, cta_rows, ctrl, t);
  note_launch();
  return cudaGetLastError();
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

void launch_transitivity(const unsigned long long *sums, double *out, cudaStream_t st) {
  k_transitivity<<<1, 1, 0, st>>>(sums, out);
  note_launch();
}

}  // namespace tc
