/*
 * graph.h -- C ABI of the GB300 BSP graph library.
 *
 * The library runs the bulk-synchronous superstep of the TOTEM engine (Section 4.1) on one
 * GPU: a compute phase over each partition's CSR, a communication phase that moves boundary
 * messages from outbox to inbox buffers (Section 4.3.2), and a termination vote. Breadth-
 * first search (Section 6.3.2, Figure 11), pull PageRank (Section 7.1, Figure 14) and
 * Bellman-Ford shortest paths (Section 7.3, Figure 20) run on it.
 *
 * Conventions shared by every call:
 *  - Vertex ids are uint32 in [0, n), n < 2^31 (bit 31 of a partitioned edge marks a
 *    boundary edge, Section 4.3.1). Edge offsets are int64.
 *  - INF (GRAPH_INF = 0xFFFFFFFF) marks unreached vertices in levels, parents and distances.
 *  - Results are written in the caller's global vertex order, into caller-owned arrays of
 *    length n, in host or device memory as the attribute `out_mem` says. Host output arrays
 *    should be pinned for full copy speed; any host memory works.
 *  - Every call returns a graph_status (0 = success, negative = error) and never aborts.
 *    graph_strerror() names a status; graph_last_error() gives the detail of the most
 *    recent failure on the calling thread.
 *  - Work is issued on the stream given at load time (graph_runtime.stream) and the call
 *    returns after its results are complete. Calls on one handle must not overlap; distinct
 *    handles are independent. Handles are not thread-safe.
 */
#ifndef GB300_GRAPH_H
#define GB300_GRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct graph graph_t; /* opaque; owns device copies of the graph and workspaces */
typedef int graph_status;

#define GRAPH_OK 0
#define GRAPH_EINVAL (-1)   /* bad argument: NULL pointer, id out of range, bad CSR, ... */
#define GRAPH_ENOMEM (-2)   /* device or pinned-host allocation failed */
#define GRAPH_ECUDA (-3)    /* a CUDA runtime call failed; see graph_last_error() */
#define GRAPH_ETIMEOUT (-4) /* a bounded device wait or the superstep cap ran out */
#define GRAPH_ERANGE (-5)   /* a result does not fit its type (distance >= 2^32 - 1) */
#define GRAPH_ESTATE (-6)   /* call out of order (e.g. an algorithm before partitioning) */

#define GRAPH_INF 0xFFFFFFFFu

#define GRAPH_MEM_HOST 0
#define GRAPH_MEM_DEVICE 1

/* Device memory and stream used by a graph handle. alloc/free may be NULL (then the
 * library uses cudaMalloc/cudaFree). alloc must return memory aligned to at least 256 bytes
 * or NULL; free receives the pointer and the size that alloc was asked for. stream is a
 * cudaStream_t (NULL = the legacy default stream). The struct is copied at load time. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* ctx;
  void* stream;
} graph_runtime;

/* ---------------------------------------------------------------------------------------
 * graph_load_csr -- copy a CSR graph into device memory (the graph representation of
 * Section 4.3.1: V = offsets, E = destination ids).
 *   n        number of vertices, 0 < n < 2^31
 *   m        number of directed edge entries (offsets[n] must equal m)
 *   offsets  int64[n+1], non-decreasing, offsets[0] = 0
 *   cols     uint32[m], each < n. Undirected graphs store both directions. BFS parents
 *            and the SSSP certificate assume the stored graph is symmetric; PageRank
 *            pulls along the stored entries (in-neighbours = stored neighbours).
 *   weights  uint32[m] edge weights >= 1 for SSSP, or NULL
 *   mem      GRAPH_MEM_HOST or GRAPH_MEM_DEVICE: where offsets/cols/weights live
 *   rt       allocator and stream, or NULL for cudaMalloc and the default stream
 *   out      receives the new handle
 * The inputs are validated on the device (monotone offsets, ids < n) and copied; the
 * caller keeps ownership of its arrays. Errors: EINVAL (bad sizes, NULL, invalid CSR),
 * ENOMEM, ECUDA. The graph starts unpartitioned: call graph_partition before algorithms.
 * ------------------------------------------------------------------------------------- */
graph_status graph_load_csr(uint32_t n, int64_t m, const int64_t* offsets,
                            const uint32_t* cols, const uint32_t* weights, int mem,
                            const graph_runtime* rt, graph_t** out);

/* Partition strategies (Section 6.2-6.3.1). */
#define GRAPH_PART_NONE 0     /* one partition: every vertex in partition 1, none in 0 */
#define GRAPH_PART_DEGREE 1   /* HIGH: partition 0 = vertices with degree >= T (hubs),  \
                                 partition 1 = the rest (leaves) */
#define GRAPH_PART_EXPLICIT 2 /* caller-given partition id per vertex (e.g. RAND) */

typedef struct {
  int strategy;
  uint32_t degree_threshold; /* DEGREE: T, used when edge_share <= 0 */
  double edge_share;         /* DEGREE: if > 0, T = largest t such that the vertices of
                                degree >= t hold at least edge_share * m edge entries */
  const uint8_t* assignment; /* EXPLICIT: n host bytes, each 0 or 1 */
} graph_partition_attr;

/* ---------------------------------------------------------------------------------------
 * graph_partition -- split the vertices into two partitions and build, on the device,
 * each partition's data structures (Section 4.3.1-4.3.2, Figure 6):
 *  - local ids 0..|V_p|-1, ordered by degree class (bit length of the degree) descending,
 *    then by global id; l2g maps local to global ids (used to collect results);
 *  - CSR per partition, each vertex's local neighbours first (Section 4.3.1), then its
 *    boundary neighbours, original order within each group;
 *  - a boundary edge stores 0x80000000 | (index into the partition's outbox);
 *  - the outbox lists the distinct remote targets in ascending local id of their owner,
 *    which makes it element-for-element the owner's inbox (messages are reduced at the
 *    source: one slot per remote vertex, Section 3.4).
 * Re-partitioning replaces the previous partition. Errors: EINVAL (bad strategy,
 * assignment values > 1, missing assignment), ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
graph_status graph_partition(graph_t* g, const graph_partition_attr* attr);

typedef struct {
  uint32_t n;
  int64_t m;
  uint32_t threshold;   /* T used by DEGREE (0 otherwise) */
  uint32_t nv[2];       /* |V_p| */
  int64_t ne[2];        /* |E_p| */
  uint32_t nout[2];     /* |V_o| of partition p = |V_i| of the other partition */
  uint32_t cls_end[2][34]; /* local ids of degree class c are [cls_end[c+1], cls_end[c]) */
  int64_t bytes_graph;  /* device bytes of the partitioned graph per the space formula of
                           Section 4.3.3 (offsets, edges, weights, in/outbox vertex ids) */
} graph_partition_info;

/* Sizes of the current partition. Errors: EINVAL, ESTATE (not partitioned). */
graph_status graph_get_partition_info(const graph_t* g, graph_partition_info* info);

/* Copies partition p's arrays to host buffers sized from graph_get_partition_info: l2g
 * [nv], off [nv+1], E [ne], W [ne] (NULL to skip; requires weights), outbox [nout],
 * g2l [n] ((p << 31) | local id; NULL to skip). Any other pointer may be NULL to skip.
 * Meant for inspection and tests. Errors: EINVAL, ESTATE, ECUDA. */
graph_status graph_export_partition(const graph_t* g, int p, uint32_t* l2g, int64_t* off,
                                    uint32_t* E, uint32_t* W, uint32_t* outbox,
                                    uint32_t* g2l);

/* ---------------------------------------------------------------------------------------
 * graph_set_edge_memory -- where the edge arrays live: device memory (the default) or
 * page-locked host memory mapped into the device's address space, which the kernels then
 * read over the host link (Section 4.3.4 (iii), Section 8: immutable, sequentially read
 * edge arrays of a partition kept in mapped host memory so that graphs larger than the
 * GPU's memory can be processed; GB300's link to the Grace host carries about 190 GB/s).
 *   which  bit 0: partition 0's edge ids and weights; bit 1: partition 1's; bit 2: the
 *          loaded CSR's column and weight arrays (read again only by graph_partition and
 *          by pagerank_multi's first call). 1 ... 7.
 *   mem    GRAPH_MEM_HOST or GRAPH_MEM_DEVICE.
 * Every algorithm works with either placement and gives the same results; offsets, vertex
 * state and messages stay in device memory. The call copies the arrays (blocking), frees
 * their old copies and drops the algorithms' workspaces, which the next calls rebuild.
 * Re-partitioning puts the new partitions' edge arrays in device memory. Errors: EINVAL
 * (bad which or mem), ESTATE (bits 0-1 before graph_partition), ENOMEM (no page-locked
 * host memory, or no device memory to move back to), ECUDA.
 * ------------------------------------------------------------------------------------- */
graph_status graph_set_edge_memory(graph_t* g, int which, int mem);

/* Current placement: bit 0 / 1 / 2 set when partition 0's / partition 1's / the loaded
 * CSR's edge arrays are in host memory. Errors: EINVAL. */
graph_status graph_get_edge_memory(const graph_t* g, int* placement);

/* Per-call statistics (all optional; pass NULL). Times are CUDA-event times on the
 * handle's stream, filled when the attribute `timing` is non-zero. */
typedef struct {
  int supersteps;          /* BSP rounds executed (BFS levels, SSSP rounds, PR iterations) */
  int topdown_steps;       /* BFS: rounds run top-down */
  int bottomup_steps;      /* BFS: rounds run bottom-up */
  int64_t edges_traversed; /* TEPS numerator (Section 5): BFS/SSSP the degree sum of the
                              reached vertices; PageRank m * iterations */
  int64_t edges_inspected; /* edge entries the compute kernels actually read */
  int64_t messages;        /* outbox entries delivered through the exchange */
  double residual;         /* PageRank: L1 change of the last iteration (FP64) */
  double ms_total;         /* whole call, including result copy-out */
  double ms_compute;       /* compute-phase kernels */
  double ms_exchange;      /* communication-phase kernels (outbox -> inbox) */
  int64_t launches;        /* CUDA kernels the call launched */
} graph_stats;

/* ---------------------------------------------------------------------------------------
 * bfs -- level-synchronous breadth-first search from `source` (Section 6.3.2, Figure 11;
 * the Appendix's entry point takes a graph, a source and an output level array).
 *   levels   n uint32: hop distance from source, INF if unreached (required)
 *   parents  n uint32: a BFS tree, parent[source] = source, INF if unreached, or NULL.
 *            Parents are one valid choice among the neighbours one level up.
 * Each round expands the frontier top-down (push through the visited bitmap, boundary
 * discoveries reduced in the outbox) or bottom-up (unvisited vertices look for a frontier
 * neighbour; the owner publishes its frontier to the other partition's ghost bitmap), as
 * the direction-optimising rule of Beamer et al. selects. Errors: EINVAL (source >= n,
 * NULL levels), ESTATE (not partitioned), ETIMEOUT (max_supersteps reached), ENOMEM,
 * ECUDA.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_BFS_AUTO 0      /* direction-optimising */
#define GRAPH_BFS_TOPDOWN 1   /* top-down every round */
#define GRAPH_BFS_BOTTOMUP 2  /* bottom-up every round after the first */

typedef struct {
  int out_mem;        /* GRAPH_MEM_HOST or GRAPH_MEM_DEVICE for levels/parents */
  int direction;      /* GRAPH_BFS_* */
  double alpha;       /* top-down -> bottom-up when frontier edges > unexplored edges /
                         alpha (<= 0: 15) */
  double beta;        /* bottom-up -> top-down when the frontier shrinks below n / beta
                         (<= 0: 18) */
  int max_supersteps; /* <= 0: no cap other than n + 1 */
  int timing;         /* fill per-phase times in graph_stats */
} bfs_attr;

graph_status bfs(graph_t* g, uint32_t source, uint32_t* levels, uint32_t* parents,
                 const bfs_attr* attr, graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * bfs_batch -- k <= 64 breadth-first searches in one sequence of supersteps. The paper
 * runs one search per call (Section 6.3.2, Figure 11); here every vertex carries a 64-bit
 * frontier mask and a 64-bit seen mask, bit s belonging to search s (multi-source BFS as
 * bit lanes, Then et al., VLDB 2014), so the edges of a level are read once for all k
 * searches. Each superstep has the same three phases as bfs: compute (push: a frontier
 * vertex ORs its mask, less what the neighbour has seen, into the neighbour's next mask,
 * boundary neighbours into their outbox slot; or pull: a vertex ORs the frontier masks of
 * its neighbours until every search it has not seen is covered, boundary neighbours read
 * from the ghost masks the owner published), communication (push: outbox masks are ORed
 * into the owner's next masks; pull: publication of the frontier masks) and termination
 * (no search found a new vertex).
 *   sources  k uint32 source ids in host memory (duplicates allowed), each < n
 *   k        1 <= k <= GRAPH_BATCH_MAX (other values: EINVAL)
 *   levels   k * n uint32, row s (levels + s * n) = hop distances from sources[s] in global
 *            vertex order, INF if unreached: exactly what bfs returns for sources[s].
 *            Host or device memory per attr->out_mem; caller-owned.
 * attr: out_mem, direction (GRAPH_BFS_AUTO picks push or pull per superstep by comparing
 * the frontier's edges with the edges of vertices some search has not reached, weighted
 * by alpha), alpha, max_supersteps and timing as for bfs; beta is unused. No parents.
 * stats->edges_traversed is the sum over the k searches of each search's TEPS numerator.
 * Superstep loop: with attr->timing == 0 the supersteps run as one CUDA graph launch, a
 * conditional while loop whose body holds two supersteps; a one-thread control kernel after
 * each superstep applies the termination vote, the max_supersteps cap and the direction
 * rule on the device and sets the loop condition, so the host waits once per call instead
 * of once per superstep. The graph is captured on the first call and replayed while the
 * graph, k, direction, alpha and cap stay the same. With attr->timing != 0 the host drives
 * the supersteps (one round trip each) so that the phases can be timed; both loops give
 * the same levels and statistics except stats->launches.
 * Device workspace: 24 bytes per vertex, 16 per outbox slot and 4 * roundup(k, 4) per
 * vertex of level lanes, kept with the graph until it is re-partitioned or freed.
 * Errors: EINVAL, ESTATE (not partitioned), ETIMEOUT (max_supersteps), ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_BATCH_MAX 64u

graph_status bfs_batch(graph_t* g, const uint32_t* sources, uint32_t k, uint32_t* levels,
                       const bfs_attr* attr, graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * sssp -- single-source shortest paths by Bellman-Ford with an active set (Section 7.3,
 * Figure 20): each round relaxes the edges of the vertices whose distance improved,
 * atomic minimum on the target (boundary targets reduce into their outbox slot), and the
 * exchange applies the outbox minima to the owner. Rounds end when no vertex is active.
 *   dist   n uint32: shortest distance, INF if unreachable. Requires weights.
 *   attr->delta  0: every improved vertex is active in the next round (Figure 20).
 *          > 0: near-far order, an extension not in the paper: only improved vertices with
 *          distance below a threshold are active; the others wait, and when no vertex is
 *          active the threshold becomes the smallest waiting distance + delta. Same
 *          distances, fewer wasted relaxations.
 * Sums saturate below INF; if a true distance would reach 2^32 - 1 the call returns
 * ERANGE. Errors: EINVAL (source >= n, NULL dist, no weights), ESTATE, ETIMEOUT, ERANGE,
 * ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int out_mem;
  int max_supersteps; /* <= 0: no cap other than n + 1 */
  int timing;
  uint32_t delta;     /* 0: plain active-set rounds; > 0: near-far bucket width */
} sssp_attr;

graph_status sssp(graph_t* g, uint32_t source, uint32_t* dist, const sssp_attr* attr,
                  graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * sssp_batch -- k <= GRAPH_SSSP_BATCH_MAX shortest-path searches in one sequence of
 * Bellman-Ford supersteps (Section 7.3, Figure 20). The paper runs one
 * search per call; here every vertex carries a row of 8 distances (one 32-byte sector,
 * lane s belonging to search s), a vertex is queued for the searches whose distance
 * improved, and one relaxation pass reads each of its edge ids and weights once for all of
 * them; boundary targets reduce into an outbox row, which the exchange applies to the
 * owner's row.
 *   sources  k uint32 source ids in host memory (duplicates allowed), each < n
 *   k        1 <= k <= GRAPH_SSSP_BATCH_MAX (other values: EINVAL)
 *   dist     k * n uint32, row s (dist + s * n) = the distances sssp returns for
 *            sources[s], global order, INF unreachable. Host or device per attr->out_mem.
 * attr: out_mem, max_supersteps and timing as for sssp; delta > 0 runs the near-far order
 * with one threshold for all k searches (a lane is queued while its distance is below
 * it; when nothing is queued it moves to the smallest waiting distance + delta). The
 * threshold staggers the lanes, so a vertex reads its edges once per group of lanes
 * activated together instead of once: on RMAT it relaxes more edges than plain rounds
 * (delta = 0), which is the faster choice for batches.
 * stats->edges_traversed is the sum over the k searches of each search's TEPS numerator;
 * edges_inspected counts edge entries read (once per pass, whatever the number of lanes).
 * Superstep loop: with attr->timing == 0 the rounds run as one CUDA graph launch (a
 * conditional while loop; one-thread control kernels move the near-far threshold, build
 * each round's relax plan from the queue tails, apply the termination vote and the cap,
 * and set the loop condition), so the host waits once per call; the graph is captured on
 * the first call after a partition and replayed. With attr->timing != 0 the host drives
 * the rounds so that the phases can be timed. Both give the same distances and statistics
 * except stats->launches.
 * Device workspace: about 76 bytes per vertex (distance and queued rows, lane mask, queues)
 * and 32 per outbox slot, kept with the graph until it is re-partitioned or freed.
 * Errors: EINVAL, ESTATE, ETIMEOUT, ERANGE, ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_SSSP_BATCH_MAX 8u

graph_status sssp_batch(graph_t* g, const uint32_t* sources, uint32_t k, uint32_t* dist,
                        const sssp_attr* attr, graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * betweenness -- betweenness centrality summed over a list of sources (Section 7.2,
 * Figure 18; Brandes' algorithm). Per source, a forward BSP cycle finds BFS levels and the
 * number of shortest paths sigma (each new vertex sums sigma over its neighbours one level
 * up; boundary neighbours through published ghost copies), and a backward cycle from the
 * deepest level up accumulates the dependency delta(v) = sum over neighbours w one level
 * further of sigma(v) / sigma(w) * (1 + delta(w)).
 *   sources  k uint32 source ids in host memory, each < n (k >= 1, repeats allowed)
 *   scores   n doubles, global order: sum over the sources s of delta_s(v), v != s (host
 *            or device per attr->out_mem). Scores of ordered pairs: an undirected
 *            graph's textbook betweenness (unordered pairs) is half of the all-source sum.
 * The stored graph must be symmetric (successors are taken from the same adjacency that
 * gives predecessors). Path counts are FP64; they are exact while below 2^53.
 * A forward level whose frontier's edges, times 2, exceed the edges of the vertices not yet
 * discovered is pulled: every undiscovered vertex sums the path counts of its neighbours at
 * the frontier level and is discovered by a non-zero sum (same levels and path counts).
 * stats->edges_traversed: twice the degree sum of the vertices each source reaches
 * (Section 5: forward and backward phases), summed over the sources; stats->bottomup_steps:
 * the pulled forward levels.
 * Errors: EINVAL, ESTATE, ETIMEOUT, ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int out_mem;
  int timing;
} bc_attr;

graph_status betweenness(graph_t* g, const uint32_t* sources, uint32_t k, double* scores,
                         const bc_attr* attr, graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * connected_components -- label propagation (Section 9.4's connected components, with the
 * minimum label reduced at the source as Section 3.4 describes): every vertex starts with
 * its own global id as label; each superstep, vertices whose label dropped send it to
 * their neighbours (atomic minimum; boundary neighbours through their outbox slot,
 * applied to the owner in the exchange); it ends when no label changes.
 *   labels  n uint32, global order: the smallest vertex id of the vertex's component.
 * The stored graph must be symmetric. Weights are not needed. stats->edges_traversed = m.
 * Errors: EINVAL, ESTATE, ETIMEOUT (max_supersteps), ENOMEM, ECUDA.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int out_mem;
  int max_supersteps; /* <= 0: no cap other than n + 1 */
  int timing;
} cc_attr;

graph_status connected_components(graph_t* g, uint32_t* labels, const cc_attr* attr,
                                  graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * pagerank -- pull PageRank (Section 7.1, Figure 14). Each iteration every vertex sums
 * its neighbours' contributions x[u] = r[u] / deg(u) and sets
 *     r'[v] = (1 - d)/n + d * (sum + D/n)
 * where D is the rank held by degree-zero vertices (dangling = 1) or 0 (dangling = 0,
 * Figure 14 taken literally). Ranks start at 1/n. Boundary contributions are read from
 * ghost slots the owner publishes in the communication phase (pull direction, Section
 * 4.3.2). D and the L1 residual sum |r' - r| are reduced in FP64 on the device.
 * Precision of the stored contributions and of the per-vertex sum:
 *   GRAPH_PR_FP32  FP32 x, FP32 accumulation, FP32 ranks
 *   GRAPH_PR_FP64  FP64 throughout
 *   GRAPH_PR_FP16  x stored as FP16 scaled by n (n*r/deg), FP32 accumulation, FP32 ranks
 *   ranks   n doubles: the ranks after the last iteration
 * Runs max_iter iterations, or stops after the first iteration whose residual < tol
 * (tol <= 0: never).
 * How the neighbour sum is formed (method; the result is the same sum up to FP32 rounding
 * order):
 *   GRAPH_PR_AUTO       GATHER (measured faster than SEGMENTED on RMAT graphs here)
 *   GRAPH_PR_GATHER     every edge entry gathers its neighbour's contribution from global
 *                       memory (per-vertex work items by degree class)
 *   GRAPH_PR_SEGMENTED  FP32 / FP16 only: the source ids of each partition are cut into
 *                       segments of 2^seg_log2 whose contributions fit in shared memory; a
 *                       first pass sums every destination's entries of one segment from
 *                       shared memory into a partial sum, a second pass adds each
 *                       destination's partial sums and updates the vertex. The layout (the
 *                       plan: 2 bytes per edge entry, about 6 bytes per partial sum) is
 *                       built on the device by the first call after graph_partition and kept
 *                       until the next partition, graph_free or a call with other seg_*
 *                       values. Limits: at most 2,047 partial sums per vertex, at most 2,378
 *                       segments per partition and fewer than 2^31 edge entries per
 *                       partition; a graph beyond them returns EINVAL.
 *   seg_log2   6 ... 15 (0: 15), seg_chunk 64 ... 8176 entries per first-pass chunk (0:
 *              8176), seg_bin 64 ... 14336 partial sums per second-pass bin (0: 12288, and
 *              at most 14336 - 6 * segments of the partition); ignored by GATHER.
 *              pagerank_hybrid and pagerank_multi always gather.
 * Errors: EINVAL (damping outside [0,1], max_iter < 1, NULL ranks, bad precision, method
 * or seg_* value), ESTATE, ENOMEM, ECUDA, ETIMEOUT.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_PR_FP32 0
#define GRAPH_PR_FP64 1
#define GRAPH_PR_FP16 2

#define GRAPH_PR_AUTO 0
#define GRAPH_PR_GATHER 1
#define GRAPH_PR_SEGMENTED 2

typedef struct {
  double damping; /* d, e.g. 0.85 */
  int max_iter;
  double tol;
  int precision;  /* GRAPH_PR_FP32 / FP64 / FP16 */
  int dangling;   /* 1 = spread degree-zero rank uniformly, 0 = drop it */
  int out_mem;
  int timing;
  int method;     /* GRAPH_PR_AUTO / GATHER / SEGMENTED */
  int seg_log2;   /* SEGMENTED layout parameters, 0 = default (see above) */
  int seg_chunk;
  int seg_bin;
} pagerank_attr;

/* Layout of the segmented plan that pagerank() last built for g's current partition
 * (inspection; all zero before the first segmented call). */
typedef struct {
  int built;           /* 1 after a segmented call on the current partition */
  int usable;          /* 0: the graph exceeded a limit; calls gather instead */
  int seg_log2, seg_chunk, seg_bin;
  uint64_t partials;   /* partial sums per iteration (rows of the first pass) */
  uint32_t chunks;     /* first-pass chunks */
  uint32_t bins;       /* second-pass bins */
  double build_ms;     /* wall-clock time of the plan build */
} pagerank_plan_info;

graph_status pagerank_plan_get(const graph_t* g, pagerank_plan_info* info);

graph_status pagerank(graph_t* g, const pagerank_attr* attr, double* ranks,
                      graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * pagerank_hybrid -- PageRank with the paper's hybrid placement (Section 4.1, Figure 6;
 * Section 6.2, HIGH): partition 0 (with the DEGREE strategy, the vertices of degree >= T,
 * or of the edge share chosen by edge_share) is updated by cpu_threads host threads from
 * host copies of its arrays, partition 1 by the GPU, at the same time. Each iteration is one
 * superstep: the communication phase copies only message arrays across the host/device
 * boundary (Section 4.3.2): partition 0's ghost slots (contributions of its partition-1
 * neighbours) go from device to host, and partition 1's ghost slots, gathered on the host,
 * go from host to device. Then both processors compute their partition, and the residual
 * is the FP64 sum of both parts. The result is the PageRank of pagerank() (same
 * attributes and readings) up to the order of the FP32 / FP64 neighbour sums.
 *   attr         as for pagerank; precision GRAPH_PR_FP32 or GRAPH_PR_FP64 (FP16: EINVAL)
 *   cpu_threads  host threads, 1 ... GRAPH_HYBRID_MAX_THREADS; <= 0: the host's hardware
 *                threads (capped at GRAPH_HYBRID_MAX_THREADS)
 *   ranks        n doubles in global order (host or device per attr->out_mem)
 *   info         per-processor sizes and times, or NULL
 * The first call after graph_partition copies partition 0's offsets and edge ids and
 * partition 1's outbox to host memory (kept with the PageRank workspace until re-partition,
 * a change of precision or graph_free) and allocates pinned message buffers. Host times
 * are wall-clock; GPU compute times are CUDA-event times on the handle's stream. Errors:
 * EINVAL, ESTATE (not partitioned), ENOMEM (host or device), ECUDA, ETIMEOUT.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_HYBRID_MAX_THREADS 1024

typedef struct {
  int cpu_threads;         /* host threads used */
  uint32_t cpu_vertices;   /* vertices of partition 0 (host) */
  uint32_t gpu_vertices;   /* vertices of partition 1 (GPU) */
  int64_t cpu_edges;       /* edge entries of partition 0 */
  int64_t gpu_edges;       /* edge entries of partition 1 */
  double ms_cpu_compute;   /* host partition updates, summed over iterations (wall clock) */
  double ms_gpu_compute;   /* GPU partition kernels, summed over iterations (CUDA events) */
  double ms_exchange;      /* communication phase on the stream: publication, device-to-host
                              and host-to-device copies (includes the host's gather when
                              the stream waits for it), summed over iterations */
} pagerank_hybrid_info;

graph_status pagerank_hybrid(graph_t* g, const pagerank_attr* attr, int cpu_threads,
                             double* ranks, graph_stats* stats, pagerank_hybrid_info* info);

/* ---------------------------------------------------------------------------------------
 * bfs_hybrid, sssp_hybrid -- BFS and SSSP with the paper's hybrid placement (Section 4.1,
 * Figure 6; Section 6.2-6.3 for BFS, Section 7.3 for SSSP): partition 0 (with the DEGREE
 * strategy, the high-degree vertices) is processed by cpu_threads host threads from host
 * copies of its arrays, partition 1 by the GPU, in the same superstep. BFS: both sides
 * expand their own frontier top-down (Figure 11); SSSP: both run the Bellman-Ford round of
 * Figure 20 on their own active vertices (plain rounds). The communication phase moves only
 * messages (Section 4.3.2): the claims (BFS: target, level, parent) or lowered outbox minima
 * (SSSP: target, distance) each side produced for the other's vertices, as compact lists
 * across the host/device boundary, applied with the same claim / minimum the GPU-only calls
 * use. Results equal those of bfs() (levels; parents valid) and sssp() (distances).
 *   source, levels, parents, dist, stats   as for bfs / sssp
 *   attr         as for bfs (direction AUTO or TOPDOWN: top-down only) / sssp (delta = 0)
 *   cpu_threads  as for pagerank_hybrid
 *   info         per-processor sizes and times (the pagerank_hybrid report), or NULL
 * The first call after graph_partition copies partition 0's offsets, edge ids (weights for
 * SSSP), local-to-global ids (BFS) and outbox to host memory (kept with the BFS / SSSP
 * workspace until re-partition or graph_free) and allocates pinned message buffers.
 * Errors: EINVAL, ESTATE, ENOMEM (host or device), ECUDA, ETIMEOUT, ERANGE (SSSP overflow).
 * ------------------------------------------------------------------------------------- */
graph_status bfs_hybrid(graph_t* g, uint32_t source, uint32_t* levels, uint32_t* parents,
                        const bfs_attr* attr, int cpu_threads, graph_stats* stats,
                        pagerank_hybrid_info* info);
graph_status sssp_hybrid(graph_t* g, uint32_t source, uint32_t* dist, const sssp_attr* attr,
                         int cpu_threads, graph_stats* stats, pagerank_hybrid_info* info);

/* ---------------------------------------------------------------------------------------
 * pagerank_multi -- PageRank of many independent graphs in one pass of supersteps. The
 * paper ranks one graph per run (Section 7.1, Figure 14); here the loaded graph is the
 * disjoint union of ngraphs components, component c owning global vertex ids
 * [vbase[c], vbase[c+1]), and each component gets exactly the iteration pagerank gives
 * that graph alone: r_0 = 1/n_c, r' = (1-d)/n_c + d (sum + D_c/n_c) with its own dangling
 * mass D_c. Every iteration is one launch over the work items of all components; the
 * max_iter iterations are captured once as a CUDA graph and replayed by later calls with
 * the same layout, iteration count, damping and dangling mode.
 *   ngraphs    >= 1 components
 *   vbase      ngraphs + 1 uint32 in host memory: 0 = vbase[0] <= vbase[1] <= ... <=
 *              vbase[ngraphs] = n (empty components allowed). Every edge must join two
 *              vertices of one component (checked on the device; else EINVAL).
 *   attr       as for pagerank, with tol = 0 (a fixed count of max_iter iterations)
 *   ranks      n doubles in global order, each component's ranks summing to 1 (host or
 *              device per attr->out_mem)
 *   residuals  ngraphs doubles in host memory: each component's L1 change in the last
 *              iteration, or NULL
 * The first call for a layout validates it and counts each component's degree-zero
 * vertices (one pass over the edges); the layout, the per-vertex component ids and the
 * captured graph are kept with the PageRank workspace (freed on re-partition or
 * graph_free). Errors: EINVAL, ESTATE (not partitioned), ENOMEM, ECUDA, ETIMEOUT.
 * ------------------------------------------------------------------------------------- */
graph_status pagerank_multi(graph_t* g, uint32_t ngraphs, const uint32_t* vbase,
                            const pagerank_attr* attr, double* ranks, double* residuals,
                            graph_stats* stats);

/* ---------------------------------------------------------------------------------------
 * Query server -- continuous batching of BFS and SSSP queries on one resident graph. The
 * paper runs one algorithm at a time (Section 4.1); a server keeps the partitioned graph
 * resident and runs many queries at once, each advancing one BSP superstep at a time:
 *  - BFS queries take bit lanes of one resident multi-source search (as in bfs_batch): a
 *    query joins at the next superstep boundary on a free lane and leaves when a superstep
 *    adds no vertex to its search, so queries enter and leave while others run.
 *  - SSSP queries each run on an SSSP job with its own workspace and stream; up to
 *    sssp_slots jobs run at once, their supersteps overlapping on the device. With
 *    attr.sssp_batch, batched jobs are added: queries that wait together are started as
 *    one sssp_batch search of up to GRAPH_SSSP_BATCH_MAX lanes (shared edge reads, plain
 *    rounds); single-query jobs use attr.sssp_delta.
 *  - Admission is by device memory: at creation the server sizes the lanes and the job
 *    slots to mem_budget (per-query state: bfs_lanes_bytes once, sssp_job_bytes per
 *    slot) and allocates them; a query waits in FIFO order until a lane or a slot is free.
 * A worker thread inside the library issues all device work (nothing is allocated after
 * creation); results are exactly those of bfs() levels / sssp() distances for the source.
 * While a server exists the graph handle must not be used by other calls, re-partitioned
 * or freed.
 * ------------------------------------------------------------------------------------- */
typedef struct graph_server graph_server_t;

#define GRAPH_QUERY_BFS 0
#define GRAPH_QUERY_SSSP 1

typedef struct {
  uint64_t mem_budget; /* bytes for per-query state; 0: half of the free device memory */
  uint32_t bfs_lanes;  /* BFS lanes, 1..64 (0: 64) */
  uint32_t max_sssp;   /* upper bound on single-query SSSP slots (0: 64, or 16 next to
                          batched jobs); the budget may allow fewer */
  int out_mem;         /* GRAPH_MEM_HOST (pinned recommended) or _DEVICE for outputs */
  uint32_t sssp_delta; /* single-query SSSP jobs: near-far bucket width (0: plain rounds) */
  uint32_t sssp_batch; /* 0: SSSP queries run one per job; 1: also on batched jobs, where up
                          to GRAPH_SSSP_BATCH_MAX queries waiting together share one
                          sssp_batch search, taken when no single-query slot is free or at
                          least half a batch waits */
} graph_server_attr;

typedef struct {
  uint64_t ticket;     /* as returned by graph_server_submit */
  int kind;            /* GRAPH_QUERY_* */
  int status;          /* GRAPH_OK or the query's error */
  uint32_t source;
  int supersteps;      /* supersteps the query took part in */
  double t_submit_ms;  /* times since the server's creation (host steady clock) */
  double t_admit_ms;   /* lane or slot assigned, device work issued */
  double t_done_ms;    /* result complete in the output array */
} graph_completion;

typedef struct {
  uint32_t bfs_lanes, sssp_slots;
  uint64_t bytes_lanes, bytes_per_sssp, mem_budget;
  uint64_t submitted, completed, pending;
  uint32_t max_lanes_busy, max_slots_busy; /* peak concurrency seen */
  uint64_t bfs_supersteps;                  /* supersteps of the lane search */
  uint32_t sssp_batch_slots;                /* batched SSSP jobs */
  uint32_t max_batch_busy;                  /* peak batched jobs running at once */
  uint64_t bytes_per_sssp_batch;            /* device bytes per batched job */
  uint64_t sssp_batched;                    /* SSSP queries answered by batched jobs */
} graph_server_info;

/* Creates a server on g (loaded, partitioned; SSSP slots need weights, else 0 slots).
 * Errors: EINVAL, ESTATE, ENOMEM (not even one lane set or slot fits), ECUDA. */
graph_status graph_server_create(graph_t* g, const graph_server_attr* attr,
                                 graph_server_t** out);
/* Queues a query; out receives n uint32 (levels or distances, global order, INF
 * unreached) in the memory kind of attr.out_mem and must stay valid until the query's
 * completion is returned. Never blocks on the device. Errors: EINVAL (kind, source >= n,
 * NULL out, SSSP without slots). */
graph_status graph_server_submit(graph_server_t* s, int kind, uint32_t source, uint32_t* out,
                                 uint64_t* ticket);
/* Moves up to cap completions (oldest first) into done; *count receives how many. Waits up
 * to wait_ms milliseconds for the first one when none is ready (0: no wait). */
graph_status graph_server_poll(graph_server_t* s, graph_completion* done, uint32_t cap,
                               uint32_t* count, int wait_ms);
graph_status graph_server_info_get(graph_server_t* s, graph_server_info* info);
/* Finishes every queued and running query, then frees the server's device memory. */
graph_status graph_server_destroy(graph_server_t* s);

/* ---------------------------------------------------------------------------------------
 * bfs_csr_noalloc -- breadth-first search for callers that cannot allocate device memory.
 * The paper has no counterpart: this entry point exists for code that must not call
 * cudaMalloc at search time (host callbacks and driver hooks where allocation is forbidden
 * or could deadlock, allocators frozen after start-up, services with a fixed device-memory
 * budget). It allocates nothing: no cudaMalloc, cudaFree or allocating library call. Its
 * scratch (visited bitmap, two frontier queues, counters) lives in one fixed device array
 * of (2^21/32 + 2 * 2^21 + 64) * 4 = 17,039,616 bytes (17.0 MB, 16.25 MiB) that every GPU
 * loading this library holds until the process exits.
 *   n        number of vertices, 1 <= n <= GRAPH_NOALLOC_MAX_VERTICES (larger n: EINVAL)
 *   m        number of edge entries
 *   offsets  DEVICE int64[n+1], cols DEVICE uint32[m]: the caller's CSR, read in place
 *            and checked first (monotone offsets, offsets[n] = m, ids < n; else EINVAL)
 *   source   start vertex (< n)
 *   levels   DEVICE uint32[n]: hop distance, GRAPH_INF if unreached (required)
 *   parents  DEVICE uint32[n]: a BFS tree (parents[source] = source), or NULL
 *   stream   cudaStream_t for all work (NULL = legacy default stream); the call blocks:
 *            it synchronises the stream with the host after the CSR check and after every
 *            level, and returns after the results are complete
 * Search is level-synchronous and top-down on the unpartitioned graph; levels equal those
 * of bfs(). The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current, so make the first call before any
 * stream capture. Every call shares the scratch array and clears what must start at zero;
 * calls that overlap on the GPU race on it and must not be issued concurrently.
 * Errors: EINVAL, ETIMEOUT (more than n levels), ECUDA.
 * ------------------------------------------------------------------------------------- */
#define GRAPH_NOALLOC_MAX_VERTICES (1u << 21)

graph_status bfs_csr_noalloc(uint32_t n, int64_t m, const int64_t* offsets,
                             const uint32_t* cols, uint32_t source, uint32_t* levels,
                             uint32_t* parents, void* stream);

/* Releases every device and host resource of the handle (NULL is a no-op). Waits for the
 * handle's stream first. */
void graph_free(graph_t* g);

/* Static string naming a status. */
const char* graph_strerror(graph_status s);

/* Detail of the most recent failure on the calling thread ("" if none). */
const char* graph_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_GRAPH_H */
