// hub.cu -- dense counting of the hub block on the tensor cores (sm_103a).
//
// The paper closes (Sec. VI) with matrix-multiplication methods for the
// densest part of a graph.  Here that part is the hub set H: the |H|
// vertices highest in the (degree, id) order of Sec. II-B, ranks
// [lo, n) with lo = n - |H|.  Every forward neighbour of a vertex of H
// ranks higher, so it is in H too: the forward lists of H hold exactly the
// edges inside H, and every triangle with its lowest vertex in H lies
// wholly inside H.  Those triangles are counted densely and exactly:
//
//   A      the |H| x |H| adjacency matrix of H (0/1, symmetric), in fp8
//          e4m3 (1.0 = 0x38; 0/1 operands and fp32 sums below 2^24 are exact)
//   C = A A, and for every vertex i of H
//   r(i) = sum_j C(i,j) A(i,j) = 2 t_H(i)   (t_H(i): triangles of H at i)
//   sum_i r(i) = 6 T_H.
//
// The hash-set counting (count.cu) skips the edges with both endpoints in
// H (group.cu marks them), so every triangle is counted once: by the dense
// block if its lowest vertex is in H, by the hash path otherwise.
//
// The product runs on 128 x 128 tiles of C, only those with row block
// I <= column block J (C and A are symmetric: an off-diagonal tile stands
// for its mirror, its column sums being the mirror's row sums).  Both
// operands are K-major row blocks of the same matrix (A^T = A), brought in
// by TMA with 128-byte swizzling and fed to tcgen05.mma (kind::f8f6f4,
// M = N = 128, K = 32 per instruction) accumulating in tensor memory; the
// epilogue reads the accumulator with tcgen05.ld, masks it by A, and adds
// row sums (and, off the diagonal, column sums by a warp butterfly) into
// r with one atomic per row or column.
#include <cuda.h>

#include <climits>

#include "tc_common.cuh"

namespace tc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kHubTile = 128;                 // rows / columns of a C tile
constexpr int kHubKStep = 128;                // bytes (fp8 entries) of K per stage
constexpr int kHubStages = 3;                 // pipeline depth
constexpr int kHubThreads = 128;              // 4 warps: all read the accumulator
constexpr int kStageBytes = kHubTile * kHubKStep;  // one operand block, 16 KB
constexpr int kSuper = 8;                     // tiles per side of a scheduling block
constexpr uint32_t kMbarLimit = 1u << 26;     // try_wait polls before giving up
constexpr uint8_t kOne = 0x38;                // 1.0 in fp8 e4m3

// Shared memory of one CTA (dynamic, aligned to 1024 bytes in the kernel).
struct HubSmem {
  uint8_t a[kHubStages][kStageBytes];         // row block I, K slice
  uint8_t b[kHubStages][kStageBytes];         // row block J, K slice
  unsigned long long full[kHubStages];        // TMA -> MMA
  unsigned long long empty[kHubStages];       // MMA -> TMA
  unsigned long long done;                    // last MMA -> epilogue
  int32_t col[4][kHubTile];                   // per-warp column sums
  uint32_t tmem;                              // accumulator address
  uint32_t abort;                             // a wait gave up
};
constexpr size_t kHubSmemBytes = sizeof(HubSmem) + 1024;  // + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Waits until the phase of parity `parity` of *bar has completed; false if
// it does not within kMbarLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t i = 0; i < kMbarLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// 2-D TMA load of a box (128 bytes of K, 128 rows) at (x, y) into smem,
// completing on *bar.
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int32_t x, int32_t y,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand block written by TMA
// with 128-byte swizzling: rows of 128 bytes, core matrices of 8 rows
// (1024 bytes apart), descriptor version 1, swizzle mode 128 bytes.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
  const uint64_t addr = smem_u32(p);
  return ((addr & 0x3FFFFull) >> 4)            // start address
         | (1ull << 16)                        // leading byte offset (unused here)
         | ((uint64_t)(1024 >> 4) << 32)       // stride byte offset: 8 rows x 128 B
         | (1ull << 46)                        // descriptor version
         | (2ull << 61);                       // 128-byte swizzle
}

// Instruction descriptor: kind::f8f6f4, A and B e4m3, D f32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4)          // D format f32
                            | (0u << 7)        // A format e4m3
                            | (0u << 10)       // B format e4m3
                            | ((uint32_t)(kHubTile >> 3) << 17)   // N >> 3
                            | ((uint32_t)(kHubTile >> 4) << 24);  // M >> 4

__device__ __forceinline__ void mma_f8(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Tile t of the upper triangle (row block I <= column block J of T x T),
// enumerated by scheduling blocks of kSuper x kSuper tiles so that the
// tiles in flight at once share their row and column blocks in L2.
__device__ __forceinline__ void tile_of(uint32_t t, int T, int *I, int *J) {
  const int S = (T + kSuper - 1) / kSuper;
  for (int p = 0; p < S; ++p) {
    for (int q = p; q < S; ++q) {
      const int i0 = p * kSuper, j0 = q * kSuper;
      const int ni = min(kSuper, T - i0), nj = min(kSuper, T - j0);
      uint32_t cnt = 0;
      if (p < q) {
        cnt = (uint32_t)(ni * nj);
        if (t < cnt) {
          *I = i0 + (int)(t / nj);
          *J = j0 + (int)(t % nj);
          return;
        }
      } else {  // diagonal block: rows i, columns j >= i
        cnt = (uint32_t)(ni * (ni + 1) / 2);
        if (t < cnt) {
          int i = 0;
          uint32_t left = t;
          while (left >= (uint32_t)(ni - i)) {
            left -= (uint32_t)(ni - i);
            ++i;
          }
          *I = i0 + i;
          *J = i0 + i + (int)left;
          return;
        }
      }
      t -= cnt;
    }
  }
  *I = 0;
  *J = 0;  // not reached for t < T (T + 1) / 2
}

// Adds 32 column values of 32 rows (one row per lane) so that lane j ends
// with the sum of column j: five butterfly steps, 31 shuffles.
__device__ __forceinline__ int32_t column_sums32(int32_t (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const int32_t send = upper ? v[i] : v[i + h];
      const int32_t recv = __shfl_xor_sync(kFull, send, h);
      v[i] = (upper ? v[i + h] : v[i]) + recv;
    }
  }
  return v[0];
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Which hub set, if any, is worth its cost.  The candidates are the top
// Hmax/4, Hmax/2, 3Hmax/4 and Hmax ranks (multiples of 128).  For every
// edge inside the largest one, the hash lookups it would cost
// (min(d+(u), d+(v)), before skipping) are added to the smallest candidate
// that holds it: one warp per owner u.
__device__ __forceinline__ int32_t hub_candidate(int32_t Hmax, int k) {
  return ((Hmax * (k + 1) / 4) / 128) * 128;
}

__global__ void __launch_bounds__(256)
k_hub_estimate(const int32_t *__restrict__ off, const int32_t *__restrict__ col, int32_t n,
               int32_t Hmax, Ctrl *ctrl) {
  if (aborted(ctrl)) return;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  unsigned long long acc[4] = {0, 0, 0, 0};
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (uint32_t)Hmax;
       w += warps) {
    const int32_t u = n - Hmax + (int32_t)w;
    const int32_t du = __ldg(off + u + 1) - __ldg(off + u);
    // the smallest candidate holding u (and so every forward neighbour)
    int k = 3;
    while (k > 0 && n - hub_candidate(Hmax, k - 1) <= u) --k;
    unsigned long long sum = 0;
    for (int32_t i = lane; i < du; i += 32) {
      const int32_t v = __ldg(col + __ldg(off + u) + i);
      const int32_t dv = __ldg(off + v + 1) - __ldg(off + v);
      sum += (unsigned long long)min(du, dv);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += q == k ? sum : 0ull;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], o);
    if (lane == 0 && acc[q]) atomicAdd(&ctrl->hub_est[q], acc[q]);
  }
}

// Cost model (GB300, measured on R-MAT scale 20 and 24 over hub sizes of
// 8192 to 24576): a lookup taken off the hash path saves about 0.63 ps of
// the whole GPU's time when only T is counted and 1.03 ps with per-vertex
// counts (whose match counters go too); one figure between the two, 0.85
// ps, serves both, so that a graph gets the same hub set in either mode
// (and tc_count_work reports the work of the run it describes).  The dense
// block costs about 0.15 ms plus 1.55 ms (H / 16384)^3.
// The candidate with the largest saving is used if it saves anything.
// force (hub_min_edges == 0): the largest candidate, whatever the model.
__global__ void k_hub_decide(const int32_t *__restrict__ off, int32_t n, int32_t Hmax,
                             int64_t min_edges, int per_vertex, Ctrl *ctrl) {
  if (aborted(ctrl)) return;
  (void)per_vertex;
  const double ms_per_lookup = 0.85e-9;
  double best = 0.0;
  int32_t H = 0;
  unsigned long long inside = 0;
  for (int k = 0; k < 4; ++k) {
    inside += ctrl->hub_est[k];  // lookups inside candidate k (cumulative)
    const int32_t h = hub_candidate(Hmax, k);
    const double x = (double)h / 16384.0;
    const double gain = (double)inside * ms_per_lookup - (0.15 + 1.55 * x * x * x);
    const int64_t edges = (int64_t)ctrl->m - (int64_t)__ldg(off + (n - h));
    if (h > 0 && edges >= min_edges && gain > best) {
      best = gain;
      H = h;
    }
  }
  if (min_edges == 0) H = Hmax;
  ctrl->hub_on = H > 0 ? 1u : 0u;
  ctrl->hub_size = (uint32_t)H;
  ctrl->hub_lo = (uint32_t)(n - H);
}

// Zeroes the H x H corner (row pitch Hmax) of the hub matrix.
__global__ void __launch_bounds__(256)
k_hub_zero(uint8_t *__restrict__ A, int32_t Hmax, const Ctrl *ctrl) {
  if (aborted(ctrl) || !ctrl->hub_on) return;
  const uint32_t H = ctrl->hub_size;
  const uint32_t words = H / 16;  // uint4 per row
  const uint64_t total = (uint64_t)H * words;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t row = i / words, w = i % words;
    reinterpret_cast<uint4 *>(A + row * (uint64_t)Hmax)[w] = make_uint4(0, 0, 0, 0);
  }
}

// A(u - lo, v - lo) = A(v - lo, u - lo) = 1 for every forward edge of H
// (the matrix was zeroed before).  One warp per vertex of H.
__global__ void __launch_bounds__(256)
k_hub_scatter(const int32_t *__restrict__ off, const int32_t *__restrict__ voff,
              const int32_t *__restrict__ col4, int32_t n, int32_t pitch, const Ctrl *ctrl,
              uint8_t *__restrict__ A) {
  if (aborted(ctrl) || !ctrl->hub_on) return;
  const int32_t H = (int32_t)ctrl->hub_size, lo = n - H;
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < (uint32_t)H; w += warps) {
    const int32_t u = lo + (int32_t)w;
    const int32_t d = __ldg(off + u + 1) - __ldg(off + u);
    const int32_t *list = col4 + 4ll * __ldg(voff + u);
    for (int32_t i = lane; i < d; i += 32) {
      const int32_t v = __ldg(list + i) - lo;  // > u - lo >= 0
      A[(size_t)w * pitch + v] = kOne;
      A[(size_t)v * pitch + w] = kOne;
    }
  }
}

// C tiles of the upper triangle, one per CTA; r(i) += masked row (and
// column) sums.  Warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the
// MMAs; all four warps read the accumulator back.
__global__ void __launch_bounds__(kHubThreads, 2)
k_hub_gemm(const __grid_constant__ CUtensorMap amap, const uint8_t *__restrict__ A,
           int32_t pitch, Ctrl *ctrl, uint32_t *__restrict__ r) {
  extern __shared__ uint8_t smem_raw[];
  if (!ctrl->hub_on || aborted(ctrl)) return;  // uniform for the block
  const int32_t H = (int32_t)ctrl->hub_size;
  {
    const uint32_t T = (uint32_t)H / kHubTile;
    if (blockIdx.x >= T * (T + 1) / 2) return;  // a tile of a larger hub set
  }
  HubSmem &S = *reinterpret_cast<HubSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = H / kHubTile, KT = H / kHubKStep;
  int I, J;
  tile_of(blockIdx.x, T, &I, &J);

  if (tid == 0) {
    for (int s = 0; s < kHubStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // accumulator: 128 lanes x 128 fp32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem)),
                 "r"(kHubTile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = S.tmem;

  if (warp == 0 && lane == 0) {  // producer
    int issued = 0;
    for (int k = 0; k < KT; ++k) {
      const int s = k % kHubStages;
      if (k >= kHubStages && !mbar_wait(&S.empty[s], ((k / kHubStages) & 1) ^ 1)) {
        S.abort = 1;
        break;
      }
      mbar_expect_tx(&S.full[s], 2 * kStageBytes);
      tma_load(S.a[s], &amap, k * kHubKStep, I * kHubTile, &S.full[s]);
      tma_load(S.b[s], &amap, k * kHubKStep, J * kHubTile, &S.full[s]);
      issued = k + 1;
    }
    // the loads still in flight land before the block may exit
    for (int k = max(issued - kHubStages, 0); k < issued; ++k)
      mbar_wait(&S.full[k % kHubStages], (k / kHubStages) & 1);
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    for (int k = 0; k < KT; ++k) {
      const int s = k % kHubStages;
      if (!mbar_wait(&S.full[s], (k / kHubStages) & 1)) {
        S.abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = smem_desc(S.a[s]), bd = smem_desc(S.b[s]);
#pragma unroll
      for (int kk = 0; kk < kHubKStep / 32; ++kk)  // K = 32 bytes per instruction
        mma_f8(tmem, ad + 2 * kk, bd + 2 * kk, (k > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&S.empty[s]);  // the stage is free once these MMAs have read it
    }
    mma_commit(&S.done);  // arrives when every MMA issued above is complete
  }
  __syncwarp();

  // epilogue: thread tid owns row i = tid of the tile (tensor-memory lane tid)
  const bool ok = mbar_wait(&S.done, 0) && !S.abort;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int i = tid;
  const uint8_t *arow = A + (size_t)(I * kHubTile + i) * pitch + (size_t)J * kHubTile;
  int32_t rowsum = 0;
#pragma unroll 1
  for (int c = 0; c < kHubTile / 32; ++c) {
    uint32_t x[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]),
          "=r"(x[7]), "=r"(x[8]), "=r"(x[9]), "=r"(x[10]), "=r"(x[11]), "=r"(x[12]),
          "=r"(x[13]), "=r"(x[14]), "=r"(x[15]), "=r"(x[16]), "=r"(x[17]), "=r"(x[18]),
          "=r"(x[19]), "=r"(x[20]), "=r"(x[21]), "=r"(x[22]), "=r"(x[23]), "=r"(x[24]),
          "=r"(x[25]), "=r"(x[26]), "=r"(x[27]), "=r"(x[28]), "=r"(x[29]), "=r"(x[30]),
          "=r"(x[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const uint4 m0 = *reinterpret_cast<const uint4 *>(arow + 32 * c);
    const uint4 m1 = *reinterpret_cast<const uint4 *>(arow + 32 * c + 16);
    const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
    int32_t v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const bool edge = ((mw[j >> 2] >> (8 * (j & 3))) & 0xffu) != 0u;
      v[j] = (ok && edge) ? (int32_t)__float2int_rn(__uint_as_float(x[j])) : 0;
      rowsum += v[j];
    }
    if (I != J) S.col[warp][32 * c + lane] = column_sums32(v);
  }
  if (rowsum) atomicAdd(r + I * kHubTile + i, (uint32_t)rowsum);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (I != J) {
    const int32_t cs = S.col[0][tid] + S.col[1][tid] + S.col[2][tid] + S.col[3][tid];
    if (cs) atomicAdd(r + J * kHubTile + tid, (uint32_t)cs);
  }
  if (!ok && tid == 0) atomicOr(&ctrl->err, kErrTimeout);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kHubTile));
  }
}

// t(v) += r(v) / 2 for v in H (per-vertex counts, rank space) and
// T += (sum of r) / 6; r must be even and its sum a multiple of 6.  One
// block.
__global__ void __launch_bounds__(1024)
k_hub_finish(const uint32_t *__restrict__ r, Ctrl *ctrl, int64_t *t) {
  __shared__ unsigned long long s_sum[32];
  __shared__ uint32_t s_odd;
  if (aborted(ctrl) || !ctrl->hub_on) return;
  const int32_t lo = (int32_t)ctrl->hub_lo, H = (int32_t)ctrl->hub_size;
  if (threadIdx.x == 0) s_odd = 0;
  __syncthreads();
  unsigned long long sum = 0;
  uint32_t odd = 0;
  for (int32_t v = threadIdx.x; v < H; v += blockDim.x) {
    const uint32_t x = __ldg(r + v);
    sum += x;
    odd |= x & 1u;
    if (t && x) t[lo + v] += (int64_t)(x >> 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
  if (odd) atomicOr(&s_odd, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long all = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) all += s_sum[w];
    if (s_odd || all % 6ull) atomicOr(&ctrl->err, kErrInternal);
    ctrl->total += all / 6ull;
    ctrl->hub_triangles = all / 6ull;
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

}  // namespace

size_t hub_bytes(int32_t H) { return (size_t)H * (size_t)H + 4 * (size_t)H; }

void launch_hub_decide(const int32_t *off, const int32_t *col, int32_t n, int32_t Hmax,
                       int64_t min_edges, bool per_vertex, Ctrl *ctrl, cudaStream_t st) {
  k_hub_estimate<<<(Hmax + 7) / 8, 256, 0, st>>>(off, col, n, Hmax, ctrl);
  k_hub_decide<<<1, 1, 0, st>>>(off, n, Hmax, min_edges, per_vertex ? 1 : 0, ctrl);
  note_launch();
  note_launch();
}

cudaError_t launch_hub_count(const int32_t *off, const int32_t *voff, const int32_t *col4,
                             int32_t n, int32_t Hmax, uint8_t *region, Ctrl *ctrl, int64_t *t,
                             cudaStream_t st) {
  uint8_t *A = region;
  uint32_t *r = reinterpret_cast<uint32_t *>(region + (size_t)Hmax * Hmax);
  EncodeTiled enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_hub_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kHubSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  // the matrix has row pitch Hmax; the chosen set uses its top-left corner
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)Hmax, (cuuint64_t)Hmax};
  const cuuint64_t strides[1] = {(cuuint64_t)Hmax};
  const cuuint32_t box[2] = {kHubKStep, kHubTile};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, A, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(r, 0, 4 * (size_t)Hmax, st);
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_hub_zero<<<(sms > 0 ? sms : 1) * 8, 256, 0, st>>>(A, Hmax, ctrl);
  k_hub_scatter<<<(Hmax + 7) / 8, 256, 0, st>>>(off, voff, col4, n, Hmax, ctrl, A);
  const int T = Hmax / kHubTile;
  k_hub_gemm<<<T * (T + 1) / 2, kHubThreads, kHubSmemBytes, st>>>(map, A, Hmax, ctrl, r);
  k_hub_finish<<<1, 1024, 0, st>>>(r, ctrl, t);
  for (int i = 0; i < 4; ++i) note_launch();
  return cudaGetLastError();
}

}  // namespace tc
