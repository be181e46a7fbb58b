/*
 * tc.h -- exact triangle counting on GB300 (sm_103a): the C ABI.
 *
 * Method: the forward algorithm of A. Polak, "Counting Triangles in Large
 * Graphs on GPU" (arXiv 1503.00576), Sec. II-B/II-C: order the vertices by
 * (degree, id), keep each undirected edge only in the forward list N+(u) of
 * its lower endpoint, sort every forward list, and add |N+(u) & N+(v)| for
 * every forward edge (u, v).  Preprocessing reaches the sorted forward lists
 * of Sec. III-B by its own steps (degrees by atomics, backward edges dropped
 * while orienting, one sort of the oriented 64-bit keys by owner whose last
 * pass unzips, node arrays by scans, every list then sorted on its own);
 * counting computes the sum of Sec. III-C by hashing.  The order uses the
 * degree with repeated pairs counted as given (any order counts every
 * triangle once; without repeats it is the paper's).  All arithmetic is
 * exact integer.
 *
 * Input format (Sec. III-A, relaxed): an edge array given as two int32 arrays
 * src[0..m) and dst[0..m), pair i being the edge {src[i], dst[i]}.  The paper
 * assumes no self-loops, no repeated edges and every edge listed in both
 * directions; this library accepts any pairs: each pair is undirected,
 * self-loops are dropped and repeats (in either direction) collapse to one
 * edge.  So the paper's format (each edge twice) and a list with each edge
 * once give the same counts.  Vertex ids must satisfy 0 <= id < n.
 *
 * Memory: unless a function says "host", every pointer is a device pointer
 * on the current CUDA device.  Inputs are read-only and caller-owned; outputs
 * are caller-allocated.  Scratch space comes from the stream-ordered
 * allocator (cudaMallocAsync on the given stream) and is released before the
 * call returns, except in tc_count_ws, which uses the caller's workspace.
 *
 * Streams: `stream` is a cudaStream_t (0 = the legacy default stream).  All
 * work is enqueued on it.  Every function that returns a host value
 * synchronises that stream before returning.
 *
 * Errors: every call sets a thread-local status readable with
 * tc_last_error(); tc_status_string() names it.  Limits: n <= 2^31 - 2^10
 * vertices and m <= 2^31 - 2^10 pairs (beyond them TC_ERR_OVERFLOW; the
 * margin keeps every int32 index a warp advances past an end from wrapping).
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, without pulling in the CUDA headers. */
typedef struct CUstream_st *tc_stream_t;

typedef enum tc_status {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1, /* m < 0, n < 0, a required pointer is NULL, ws too small */
  TC_ERR_ID_RANGE = 2,    /* some src[i] or dst[i] is outside [0, n) */
  TC_ERR_OOM = 3,         /* the stream-ordered allocator failed */
  TC_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  TC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (never expected) */
  TC_ERR_OVERFLOW = 6     /* m or n beyond the documented limits */
} tc_status;

/* Value tc_count returns on error (no graph within the limits has this many
 * triangles: T < m^1.5 / 3 < 2^47). */
#define TC_COUNT_ERROR UINT64_MAX

/*
 * Number of triangles T of the graph, by the forward algorithm (Sec. II-C:
 * preprocessing of Sec. III-B, counting of Sec. III-C, reduction of the
 * per-thread counts).
 *   src, dst  device int32[m], read-only
 *   m         number of pairs (>= 0; 0 gives T = 0)
 *   n         number of vertices; every id must be < n
 * Returns T, or TC_COUNT_ERROR with tc_last_error() set.  Synchronises.
 */
uint64_t tc_count(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                  tc_stream_t stream);

/*
 * Per-vertex triangle counts t(v) (the number of triangles containing v; the
 * numerator of the local clustering coefficient, Sec. I) plus T and the
 * degrees of the cleaned simple graph.
 *   t_out      device int64[n], written (required when n > 0)
 *   deg_out    device int32[n], written if not NULL
 *   total_out  HOST uint64, written if not NULL (sum of t_out is 3T)
 * Synchronises (the device-side error word is read back before return).
 */
tc_status tc_count_per_vertex(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                              tc_stream_t stream, int64_t *t_out, int32_t *deg_out,
                              uint64_t *total_out);

/*
 * One share of the counting work, for counting one graph on several GPUs
 * (Sec. III-E: every device holds the edge and node arrays and counts its
 * allotted subset of the edges; the shares add up to the whole).  Here
 * every device runs the preprocessing itself (it is deterministic, so the
 * arrays agree without a copy) and counts the partner groups of the vertices
 * h of degree rank h = part mod parts (consecutive ranks have like degrees
 * and alternate between the shares, so the shares carry like work; the
 * dealing depends on the graph alone, so separate calls agree on it).
 * Summing total_out over the parts gives T,
 * and summing t_out element-wise gives the per-vertex counts; deg_out is
 * complete in every part.  The dense hub block (tc_tuning), if a graph uses
 * it, is counted by part 0 alone.  parts = 1 is tc_count /
 * tc_count_per_vertex.
 *   part, parts  0 <= part < parts, else TC_ERR_INVALID_ARG
 *   t_out        device int64[n], this part's share of t (required when n > 0)
 *   deg_out      device int32[n], written if not NULL
 *   total_out    HOST uint64, this part's share of T (required for tc_count_part)
 * Both synchronise.
 */
tc_status tc_count_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                        int32_t part, int32_t parts, tc_stream_t stream, uint64_t *total_out);
tc_status tc_count_per_vertex_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                                   int32_t part, int32_t parts, tc_stream_t stream,
                                   int64_t *t_out, int32_t *deg_out, uint64_t *total_out);

/*
 * Local clustering coefficients and the transitivity ratio from per-vertex
 * counts and degrees (Sec. I names both as the reason to count triangles):
 *   cc(v) = 2 t(v) / (deg(v) (deg(v) - 1)) in float64, 0 where deg(v) < 2
 *   transitivity = 3T / sum_v deg(v)(deg(v)-1)/2, T = sum_v t(v) / 3, with
 *                  both integers exact and one float64 division; 0 if the
 *                  denominator is 0.
 *   t, deg            device int64[n], int32[n] (as written by
 *                     tc_count_per_vertex)
 *   cc_out            device float64[n], written if not NULL
 *   transitivity_out  HOST double, written if not NULL (synchronises)
 */
tc_status tc_clustering(const int64_t *t, const int32_t *deg, int32_t n, tc_stream_t stream,
                        double *cc_out, double *transitivity_out);

/*
 * Host-buffer variants: the same computations as tc_count /
 * tc_count_per_vertex with inputs and outputs in HOST memory.  The
 * transfers are part of the call: the edge array moves to the device, is
 * counted on a stream private to the calling thread, and the results are
 * copied back before return (the paper's end-to-end timing, Sec. IV, covers
 * the same span).  Where the device reads host memory through the host's
 * page tables (Grace), the first kernel reads src_host and dst_host in
 * place, once each, instead of a copy to device memory first; elsewhere
 * they are copied (page-locked buffers transfer fastest; pageable ones
 * work).  The caller must not modify the inputs during the call.  Both
 * synchronise.
 *   src_host, dst_host  host int32[m]
 *   t_host              host int64[n] (required when n > 0)
 *   deg_host            host int32[n] or NULL
 */
tc_status tc_count_host(const int32_t *src_host, const int32_t *dst_host, int64_t m, int32_t n,
                        uint64_t *total_out);
tc_status tc_count_per_vertex_host(const int32_t *src_host, const int32_t *dst_host, int64_t m,
                                   int32_t n, int64_t *t_host, int32_t *deg_host,
                                   uint64_t *total_out);

/*
 * Caller-provided workspace.  tc_workspace_bytes(m, n) is the size that
 * tc_count_ws needs for an input of m pairs and n vertices (0 on bad
 * arguments); ws must be a device allocation of at least that many bytes,
 * 256-byte aligned.  tc_count_ws allocates nothing and otherwise behaves
 * like tc_count, writing T to the HOST uint64 *total_out.  Calls sharing a
 * workspace must be ordered (same stream, or synchronised).
 */
size_t tc_workspace_bytes(int64_t m, int32_t n);
tc_status tc_count_ws(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                      tc_stream_t stream, void *ws, size_t ws_bytes, uint64_t *total_out);

/*
 * Tuning of the counting layout (process-wide default for the calls above;
 * engines take their own).  An autotuner varies these; counts never depend
 * on them.
 *   warp_max_list, warp_max_partners: a partner group (the edges whose longer
 *     forward list is N+(h)) is counted by one warp when |N+(h)| and its
 *     partner count are at most these (warp_max_list is capped at 128),
 *     otherwise by a CTA.  Defaults 128 and 64.
 *   heavy_ratio_pct (>= 100): the intersection strategy switch.  Edge (u,v)
 *     with owner u is counted by hashing N+(v) and streaming N+(u) when
 *     |N+(v)| * 100 > |N+(u)| * heavy_ratio_pct, else by hashing N+(u) and
 *     streaming N+(v).  100 (default) always streams the shorter list.
 *   hub_min_edges, hub_vertices: single graphs of at least 2^17 vertices
 *     (ids of at most 24 bits) count the triangles among their hub_vertices
 *     highest-ranked vertices (the hub block: every forward neighbour of
 *     such a vertex is one too) as a dense 0/1 matrix product on the tensor
 *     cores when that block holds at least hub_min_edges edges; < 0 never.
 *     hub_vertices is a multiple of 128 from 128 to 32768 (the workspace
 *     grows by its square in bytes).  Defaults 2^21 and 16384.  Batches and
 *     engines never use it.
 * tc_set_tuning(NULL) restores the defaults.
 */
typedef struct tc_tuning {
  int32_t warp_max_list;
  int32_t warp_max_partners;
  int32_t heavy_ratio_pct;
  int64_t hub_min_edges;
  int32_t hub_vertices;
} tc_tuning;
tc_status tc_set_tuning(const tc_tuning *tuning);
tc_status tc_get_tuning(tc_tuning *out);

/*
 * Batched counting: the triangle counts of G graphs in one pass.  The paper
 * counts one graph per run; a batch is counted as the disjoint union of its
 * graphs (ids shifted per graph), which has exactly the union of their
 * triangles, so every per-graph count equals the graph's count alone.
 *   src, dst        device int32 pairs of all graphs, graph g's pairs at
 *                   [edge_offsets[g], edge_offsets[g+1]) with ids local to
 *                   the graph, 0 <= id < vertex_counts[g]
 *   edge_offsets    HOST int64[G+1], edge_offsets[0] = 0, non-decreasing
 *   vertex_counts   HOST int32[G]
 *   totals_out      HOST uint64[G]: triangles of each graph
 * Limits: total pairs and total vertices <= 2^31 - 2^10 (TC_ERR_OVERFLOW).  An
 * id out of range fails only the graph that holds it: the call returns
 * TC_ERR_ID_RANGE, that graph's total is TC_COUNT_ERROR and every other
 * total is still written and exact.  Synchronises.
 */
tc_status tc_count_batch(const int32_t *src, const int32_t *dst, int32_t num_graphs,
                         const int64_t *edge_offsets, const int32_t *vertex_counts,
                         tc_stream_t stream, uint64_t *totals_out);

/*
 * Persistent batch engine: device buffers for max_pairs pairs, max_vertices
 * union vertices and max_graphs graphs, allocated once, and the whole batch
 * pipeline captured once as a CUDA graph and replayed for every batch
 * (padding pairs past a batch's end are skipped, so the shape never changes).
 *   tc_engine_create   tuning NULL: the process default at creation;
 *                      max_pairs and max_vertices at most 2^31 - 2^10.
 *   tc_engine_submit   copies the batch's pairs (host or device memory, per
 *                      inputs_on_host) into the engine and launches the graph
 *                      on the engine's own stream; returns without waiting.
 *                      Host inputs must stay valid until tc_engine_wait;
 *                      page-locked ones overlap with other work.
 *   tc_engine_wait     waits for the submitted batch; totals_out HOST
 *                      uint64[G] (may be NULL).  As with tc_count_batch,
 *                      a graph with an id out of range gets TC_COUNT_ERROR
 *                      and the status TC_ERR_ID_RANGE; the others are exact.
 *   tc_engine_count    submit + wait.
 * One batch in flight per engine; an engine is used by one thread at a time
 * and on the device that was current at creation.  Two engines overlap.
 */
typedef struct tc_engine tc_engine;
tc_status tc_engine_create(int64_t max_pairs, int32_t max_vertices, int32_t max_graphs,
                           const tc_tuning *tuning, tc_engine **out);
tc_status tc_engine_submit(tc_engine *engine, const int32_t *src, const int32_t *dst,
                           int32_t inputs_on_host, int32_t num_graphs,
                           const int64_t *edge_offsets, const int32_t *vertex_counts);
tc_status tc_engine_wait(tc_engine *engine, uint64_t *totals_out);
/* Like tc_engine_submit, for graphs held in separate arrays: graph g has
 * pair_counts[g] pairs at srcs[g], dsts[g] (all in host memory, or all on the
 * device, per inputs_on_host), each copied straight into the engine. */
tc_status tc_engine_submit_parts(tc_engine *engine, int32_t num_graphs,
                                 const int32_t *const *srcs, const int32_t *const *dsts,
                                 const int64_t *pair_counts, const int32_t *vertex_counts,
                                 int32_t inputs_on_host);
/* 1 if the engine has no batch running (tc_engine_wait will not block), 0 if
 * its last batch is still running. */
int32_t tc_engine_poll(tc_engine *engine);
tc_status tc_engine_count(tc_engine *engine, const int32_t *src, const int32_t *dst,
                          int32_t inputs_on_host, int32_t num_graphs,
                          const int64_t *edge_offsets, const int32_t *vertex_counts,
                          uint64_t *totals_out);
tc_status tc_engine_destroy(tc_engine *engine);

/*
 * Work of the counting phase (instrumentation; the paper reports running
 * times only).  Runs the same pipeline as tc_count with the current tuning,
 * plus one reduction kernel over the forward edges, and reports what the
 * counting phase does for this graph:
 *   edges          m, distinct undirected edges = forward edges (Sec. II-B)
 *   lookups        sum over forward edges {u, v} of the forward-list length
 *                  streamed through the hash set (the shorter of N+(u),
 *                  N+(v) under the default tuning)
 *   inserts        sum over partner groups of the hashed list length
 *   merge_work     W = sum over forward edges of d+(u) + d+(v): the elements
 *                  a sorted-list merge of Sec. II-B would read
 *   max_out_degree the largest d+(v), at most sqrt(2m) (Sec. II-B; sqrt of
 *                  twice the input pairs when some pair is repeated)
 *   triangles      T
 *   hub_lookups[i] the lookups of the forward edges whose endpoints both
 *                  lie in the hub set H_i of the 2^(12+i) vertices highest
 *                  in the (degree, id) order; H_i is closed under forward
 *                  edges, so these edges' triangles lie wholly in H_i and a
 *                  dense count of the block A_{H_i H_i} (the matrix methods
 *                  of Sec. VI) could replace exactly this share of lookups
 *   dense_vertices the size of the hub set this run counted on the tensor
 *                  cores (its highest-ranked vertices; 0: none, see tc_tuning)
 *   dense_triangles the triangles counted there (all three vertices in it);
 *                  the hash intersections counted triangles - dense_triangles
 * Same arguments and errors as tc_count; synchronises `stream`.
 */
typedef struct tc_work {
  int64_t edges;
  int64_t lookups;
  int64_t inserts;
  int64_t merge_work;
  uint64_t triangles;
  int32_t max_out_degree;
  int32_t vertices;
  int64_t hub_lookups[4];
  uint64_t dense_triangles;
  int32_t dense_vertices;
  int32_t pad_;
} tc_work;
tc_status tc_count_work(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                        tc_stream_t stream, tc_work *out);
/* The same counters over the share that tc_count_part(part, parts) counts:
 * lookups, inserts, merge work, hub lookups and triangles of its partner
 * groups (edges, max_out_degree and vertices stay those of the whole
 * graph).  Summing one of those counters over the parts gives
 * tc_count_work's. */
tc_status tc_count_work_part(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                             int32_t part, int32_t parts, tc_stream_t stream, tc_work *out);

/*
 * Allocation-free count, for callers that cannot allocate device memory
 * while they run: for example a process whose own pool allocator reserves
 * all device memory at start-up and forbids driver allocations afterwards,
 * or a service whose memory budget is fixed when it starts.  The paper has
 * no counterpart; this is a deployment variant of tc_count.
 *
 * It computes exactly what tc_count computes, on the caller's device
 * pointers and stream, but its scratch space is a static device array of
 * TC_NOALLOC_SCRATCH_BYTES bytes that is part of the library image: every
 * GPU on which it has been loaded holds it until the process exits.  The
 * call itself allocates nothing (no cudaMalloc*, cudaFree*, pinned host
 * buffers or events).
 *   src, dst   device int32[m], read-only
 *   total_out  HOST uint64, receives T
 * Returns TC_ERR_OVERFLOW, with a message stating the bytes needed, when
 * tc_workspace_bytes(m, n) exceeds TC_NOALLOC_SCRATCH_BYTES (about
 * 24.5 m + 92 n bytes: up to about 1.1 million pairs with n = 2^16).
 *
 * First call on a device: under CUDA's lazy module loading (the default)
 * the array and the library's kernels are loaded onto a device when they
 * are first used there, i.e. by the first call on that device, so that
 * call may take device memory (the 32 MiB array plus kernel code).  A caller
 * that later reserves all device memory should make one call (on any small
 * graph) at start-up first; with CUDA_MODULE_LOADING=EAGER they are loaded
 * with the context instead.  If loading fails for lack of memory the call
 * returns TC_ERR_OOM.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress), synchronises `stream` and reads the result back
 * with a plain copy, so it cannot be called while a stream is being
 * captured into a CUDA graph.  All calls share the one array and it keeps
 * the previous call's contents (each call clears what must start at zero),
 * so calls that overlap on the GPU -- from two threads or on two streams --
 * race: order them.
 */
#define TC_NOALLOC_SCRATCH_BYTES (32u << 20)
tc_status tc_count_noalloc(const int32_t *src, const int32_t *dst, int64_t m, int32_t n,
                           tc_stream_t stream, uint64_t *total_out);

/* Status of the calling thread's most recent call, and its name. */
tc_status tc_last_error(void);
const char *tc_status_string(tc_status status);
/* Human-readable detail of the last error of this thread ("" if none). */
const char *tc_last_error_detail(void);

/*
 * Instrumentation.
 *   tc_launch_count     number of kernels this library has launched in this
 *                       process (monotonic).
 *   tc_profile_enable   1: record CUDA events around every phase of every
 *                       subsequent call (on the call's stream); 0: stop.
 *   tc_profile_read     copies the accumulated per-phase device time in ms
 *                       and launch counts since the last reset into
 *                       ms_out[0..TC_NUM_PHASES) / launches_out (either may
 *                       be NULL); reset != 0 clears them.
 *   tc_phase_name       name of phase i.
 */
enum {
  TC_PHASE_CANON = 0,   /* validate ids, drop loops, 64-bit keys, degrees */
  TC_PHASE_RANK = 1,    /* vertex ranks in (degree, id) order */
  TC_PHASE_ORIENT = 2,  /* compact + orient from the lower rank + owner histograms */
  TC_PHASE_SORT = 3,    /* LSD radix sort by owner, unzip to the column array */
  TC_PHASE_OFFSETS = 4, /* node array by exclusive scan */
  TC_PHASE_LISTS = 5,   /* every forward list sorted, repeated edges dropped */
  TC_PHASE_GROUPS = 6,  /* each forward edge to the endpoint with the longer list */
  TC_PHASE_COUNT = 7,   /* intersections, reductions, counts back to caller ids */
  TC_NUM_PHASES = 8
};
uint64_t tc_launch_count(void);
void tc_profile_enable(int on);
void tc_profile_read(double *ms_out, uint64_t *launches_out, int reset);
const char *tc_phase_name(int phase);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
