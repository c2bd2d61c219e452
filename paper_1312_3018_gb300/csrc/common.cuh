// Internal definitions shared by the CUDA translation units of the graph library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/graph.h"

namespace gg {

constexpr uint32_t kRemote = 0x80000000u;   // boundary-edge flag in a partition's E array
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr int kNClass = 34;                 // degree classes 0..32 plus a sentinel
constexpr int kThreads = 256;               // threads per CTA of every edge kernel
constexpr unsigned kFull = 0xFFFFFFFFu;

// Degree-class buckets. Local ids of a partition are ordered by degree class descending, so
// every bucket is a contiguous local-id range. Group size per bucket (lanes per vertex):
//   bucket 0 "hub"    class >= kClassHub   (deg >= 2048)  one CTA per vertex / edge chunk
//   bucket 1 "warp"   class >= kClassWarp  (deg >= 32)    one warp per vertex
//   bucket 2 "sub"    class >= kClassSub   (deg >= 4)     kSubLanes lanes per vertex
//   bucket 3 "thread" class >= 1           (deg >= 1)     one lane per vertex
// Degree-zero vertices (class 0) follow the last bucket.
constexpr int kNBucket = 4;
constexpr int kClassHub = 12;
constexpr int kClassWarp = 6;
constexpr int kClassSub = 3;
constexpr int kSubShift = 2;                // 4 lanes
constexpr int kHubChunk = 2048;             // edges per hub chunk (dense work)
constexpr int kTileE = 2048;                // max edges staged per dense tile
constexpr int kTileV = 1024;                // max vertices per dense tile
constexpr int kLeafEdges = 1024;            // class-c tile holds kLeafEdges >> (c-1) vertices

// ------------------------------------------------------------------------------------
// Device views (passed by value to kernels)
// ------------------------------------------------------------------------------------
struct PartView {
  uint32_t nv;
  uint32_t nout;
  int64_t ne;
  const int64_t* off;     // [nv+1]
  const uint32_t* E;      // [ne]
  const uint32_t* W;      // [ne] or null
  const uint32_t* l2g;    // [nv]
  const uint32_t* outbox; // [nout] local ids in the other partition
  // hub chunks: chunk c covers edges [chunk_first[c], min(+kHubChunk, end of its vertex))
  // of vertex chunk_vertex[c]; hub vertex v owns chunks hub_chunk0[v] ...
  const uint32_t* chunk_vertex;
  const int64_t* chunk_first;
  const uint32_t* hub_chunk0;
  uint32_t nchunk;
  uint32_t bstart[kNBucket + 1];  // bucket b = [bstart[b], bstart[b+1]); bstart[4] = end of
                                  // vertices with edges (degree-zero vertices follow)
};

// Bucket 0..3 of a local id; 4 for degree-zero vertices (never queued).
__device__ __forceinline__ int bucket_of(const PartView& P, uint32_t lid) {
  return (lid >= P.bstart[1]) + (lid >= P.bstart[2]) + (lid >= P.bstart[3]) +
         (lid >= P.bstart[4]);
}

// One launch covers several segments of vertices; a segment is a contiguous run of blocks
// working on one bucket of one partition, either a dense local-id range (items == null:
// vertex i is v0 + i) or a queue of local ids.
constexpr int kMaxSeg = 12;
struct Seg {
  const uint32_t* items;
  uint32_t v0;
  uint32_t count;
  uint32_t blk0;
  uint8_t part;
  uint8_t gshift;   // log2 lanes per vertex: 0, kSubShift, 5, or 8 (whole CTA)
  uint8_t bucket;
  uint8_t pad;
};
struct Plan {
  Seg seg[kMaxSeg];
  int nseg;
  uint32_t nblocks;
};

__host__ __device__ inline uint32_t seg_blocks(uint32_t count, int gshift) {
  uint32_t per = (gshift >= 8) ? 1u : (uint32_t)(kThreads >> gshift);
  return (count + per - 1) / per;
}

__host__ __device__ inline void plan_add(Plan& pl, const uint32_t* items, uint32_t v0,
                                         uint32_t count, int part, int gshift, int bucket) {
  if (count == 0) return;
  Seg& s = pl.seg[pl.nseg++];
  s.items = items;
  s.v0 = v0;
  s.count = count;
  s.blk0 = pl.nblocks;
  s.part = (uint8_t)part;
  s.gshift = (uint8_t)gshift;
  s.bucket = (uint8_t)bucket;
  s.pad = 0;
  pl.nblocks += seg_blocks(count, gshift);
}

// Segment of plan block b (pl must be a __grid_constant__ kernel parameter: its address is
// taken).
__device__ __forceinline__ int find_seg(const Plan& pl, uint32_t b = blockIdx.x) {
  int s = 0;
  #pragma unroll 1
  for (int i = 1; i < pl.nseg; ++i)
    if (b >= pl.seg[i].blk0) s = i;
  return s;
}

// Grid for kernels that walk a plan's blocks with a grid stride: enough CTAs to fill the
// GPU (8 per SM), never more than the plan has.
unsigned plan_grid(uint32_t plan_blocks);

// ------------------------------------------------------------------------------------
// Warp helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Appends the chunks of hub vertex u (bucket 0) to a chunk list: push work on a hub is
// split into kHubChunk-edge pieces, one CTA each.
__device__ __forceinline__ void append_hub_chunks(const PartView& P, uint32_t u, uint32_t* tail,
                                                  uint32_t* list) {
  const int64_t deg = P.off[u + 1] - P.off[u];
  const uint32_t nch = (uint32_t)((deg + kHubChunk - 1) / kHubChunk);
  const uint32_t c0 = P.hub_chunk0[u];
  const uint32_t at = atomicAdd(tail, nch);
  for (uint32_t j = 0; j < nch; ++j) list[at + j] = c0 + j;
}

// Appends `item` (when `has`) to the next-round work of its bucket: buckets 1..3 to
// queue[bstart[bucket] + tail[bucket]++] with one atomic per (warp, bucket); bucket 0 (hub)
// as its chunks to hubq (tail[0] counts chunks); bucket 4 (degree zero) is not queued. All
// 32 lanes must call it.
__device__ __forceinline__ void warp_append_bucketed(bool has, uint32_t item, int bucket,
                                                     uint32_t* tails, uint32_t* queue,
                                                     const PartView& P, uint32_t* hubq) {
  const uint32_t* bstart = P.bstart;
  if (has && bucket == 0) append_hub_chunks(P, item, &tails[0], hubq);
  #pragma unroll
  for (int b = 1; b < kNBucket; ++b) {
    const bool mine = has && bucket == b;
    const unsigned m = __ballot_sync(kFull, mine);
    if (m) {
      const int leader = __ffs(m) - 1;
      uint32_t base = 0;
      if ((int)lane_id() == leader) base = atomicAdd(&tails[b], (uint32_t)__popc(m));
      base = __shfl_sync(kFull, base, leader);
      if (mine) queue[bstart[b] + base + __popc(m & lanemask_lt())] = item;
    }
  }
}

// warp_append_bucketed for U items per lane (has[u], item[u], bucket[u]) at once: one
// atomic per (warp, bucket) for all of them. All 32 lanes must call it.
template <int U>
__device__ __forceinline__ void warp_append_bucketed_n(const bool* has, const uint32_t* item,
                                                       const int* bucket, uint32_t* tails,
                                                       uint32_t* queue, const PartView& P,
                                                       uint32_t* hubq) {
  #pragma unroll
  for (int u = 0; u < U; ++u)
    if (has[u] && bucket[u] == 0) append_hub_chunks(P, item[u], &tails[0], hubq);
  #pragma unroll
  for (int b = 1; b < kNBucket; ++b) {
    unsigned m[U];
    uint32_t tot = 0;
    #pragma unroll
    for (int u = 0; u < U; ++u) {
      m[u] = __ballot_sync(kFull, has[u] && bucket[u] == b);
      tot += (uint32_t)__popc(m[u]);
    }
    if (tot) {
      uint32_t base = 0;
      if (lane_id() == 0) base = atomicAdd(&tails[b], tot);
      uint32_t at = P.bstart[b] + __shfl_sync(kFull, base, 0);
      #pragma unroll
      for (int u = 0; u < U; ++u) {
        if (has[u] && bucket[u] == b) queue[at + __popc(m[u] & lanemask_lt())] = item[u];
        at += (uint32_t)__popc(m[u]);
      }
    }
  }
}

__device__ __forceinline__ void warp_append(bool has, uint32_t item, uint32_t* tail,
                                            uint32_t* list) {
  const unsigned m = __ballot_sync(kFull, has);
  if (m) {
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(tail, (uint32_t)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (has) list[base + __popc(m & lanemask_lt())] = item;
  }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Sum within aligned groups of 2^gshift lanes (gshift <= 5); every lane gets its group sum.
template <class T>
__device__ __forceinline__ T group_sum(T v, int gshift) {
  for (int o = 1; o < (1 << gshift); o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Test-and-set of bit i in a word bitmap; true if this call set it.
__device__ __forceinline__ bool bitmap_claim(uint32_t* bm, uint32_t i) {
  const uint32_t bit = 1u << (i & 31u);
  if (bm[i >> 5] & bit) return false;
  return !(atomicOr(&bm[i >> 5], bit) & bit);
}
__device__ __forceinline__ bool bitmap_test(const uint32_t* bm, uint32_t i) {
  return (bm[i >> 5] >> (i & 31u)) & 1u;
}

// ------------------------------------------------------------------------------------
// Bulk (TMA engine) global -> shared copies tracked by an mbarrier
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// 1D bulk copy: dst (shared) and src (global) 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Same copy with an L2 policy that evicts the streamed bytes first, so that data reused
// across the kernel (gathered vertex state) keeps its L2 residency.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, uint32_t bytes,
                                                uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
// Read-only load of a streamed word (edge id or weight) that is not reused: L2 evicts it
// first.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t policy) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;"
               : "=r"(v)
               : "l"(p), "l"(policy));
  return v;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2^22 polls (each poll may suspend the thread for a
// hardware-chosen interval), raising the device error flag instead of hanging.
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  int* err_flag) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err_flag, 1);
  return false;
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;      // device address (for host-resident buffers: the device alias)
  size_t bytes = 0;
  void* host = nullptr;   // page-locked host allocation behind p, or null (device memory)
};

struct Part {
  uint32_t nv = 0, nout = 0;
  int64_t ne = 0;
  DevBuf off, E, W, l2g, outbox;
  uint32_t cls_end[kNClass] = {0};
  // dense hub chunk table (PageRank): per chunk (vertex, first edge), per hub vertex the
  // first chunk index; chunk k of vertex v covers [first edge, min(first + kHubChunk, end))
  uint32_t nhub = 0, nchunk = 0;
  DevBuf chunk_vertex, chunk_first, hub_chunk0;
  PartView view() const;
};

struct BfsWs;
struct SsspWs;
struct PrWs;
struct MsWs;
struct BcWs;
struct SbWs;
struct SegWs;

}  // namespace gg

struct graph {
  uint32_t n = 0;
  int64_t m = 0;
  bool weighted = false;
  graph_runtime rt{};
  cudaStream_t stream = nullptr;
  int device = 0;
  gg::DevBuf off, col, w, g2l;
  bool partitioned = false;
  int strategy = 0;
  uint32_t threshold = 0;
  gg::Part part[2];
  gg::DevBuf err;          // int device error flag
  gg::DevBuf counters;     // per-round counters (algorithm specific layout)
  void* host_counters = nullptr;  // pinned mirror
  size_t host_counters_bytes = 0;
  gg::DevBuf stage;        // device staging for host outputs
  gg::BfsWs* bfs = nullptr;
  gg::SsspWs* sssp = nullptr;
  gg::PrWs* pr = nullptr;
  gg::MsWs* ms = nullptr;     // batched BFS workspace
  gg::BcWs* bc = nullptr;     // betweenness workspace
  gg::SbWs* sb = nullptr;     // batched SSSP workspace
  gg::SegWs* seg = nullptr;   // segmented PageRank plan of the current partition
};

namespace gg {

// Thread-local detail of the last failure.
void set_error(const char* fmt, ...);
graph_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define GG_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t _e = (call);                                                   \
    if (_e != cudaSuccess) return ::gg::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define GG_TRY(call)                      \
  do {                                    \
    graph_status _s = (call);             \
    if (_s != GRAPH_OK) return _s;        \
  } while (0)

graph_status dalloc(graph* g, DevBuf& b, size_t bytes);
void dfree(graph* g, DevBuf& b);
graph_status ensure_host_counters(graph* g, size_t bytes);
graph_status ensure_stage(graph* g, size_t bytes);
graph_status check_device_error(graph* g);

// Device-wide exclusive scans (scan.cu). Input via a typed array; out may alias in.
graph_status exclusive_scan_u32(graph* g, const uint32_t* in, uint32_t* out, uint64_t n,
                                uint32_t* total_host);
graph_status exclusive_scan_u8_to_u32(graph* g, const uint8_t* in, uint32_t* out,
                                      uint64_t n, uint32_t* total_host);
graph_status exclusive_scan_i64(graph* g, const int64_t* in, int64_t* out, uint64_t n,
                                int64_t* total_host);

// Copies an n-element result from the staging/device buffer to the caller's array.
graph_status deliver(graph* g, void* dst, const void* dev_src, size_t bytes, int out_mem);
// Where a collect kernel writes a result bound for dst: dst itself for device outputs; for
// host outputs, the device address of dst when it is page-locked host memory mapped into the
// device's address space (the kernel's stores then cross the host link directly, at the
// link's rate, with no staging copy), else the staging buffer at byte offset stage_off of a
// staging area of stage_bytes (*staged = true: the caller copies it out with deliver()).
graph_status out_target(graph* g, void* dst, int out_mem, size_t stage_bytes, size_t stage_off,
                        void** target, bool* staged);

void free_bfs(graph* g);
void free_sssp(graph* g);
void free_pr(graph* g);
void free_msbfs(graph* g);
void free_bc(graph* g);
void free_ssspb(graph* g);
void free_seg(graph* g);

inline unsigned grid_for(uint64_t work, unsigned per_block) {
  uint64_t b = (work + per_block - 1) / per_block;
  if (b == 0) b = 1;
  if (b > 0x7FFFFFFFull) b = 0x7FFFFFFFull;
  return (unsigned)b;
}

// Event-based phase timer (enabled by the `timing` attribute).
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> evs;
  std::vector<int> kinds;   // 0 compute, 1 exchange, 2 other
  void start(bool enable, cudaStream_t stream) {
    on = enable;
    s = stream;
  }
  void mark(int kind) {
    if (!on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      on = false;
      return;
    }
    cudaEventRecord(e, s);
    evs.push_back(e);
    kinds.push_back(kind);
  }
  // Interval i (between mark i-1 and mark i) is attributed to kinds[i].
  void finish(graph_stats* st) {
    if (on && st && evs.size() > 1) {
      cudaEventSynchronize(evs.back());
      double c = 0, x = 0, t = 0;
      for (size_t i = 1; i < evs.size(); ++i) {
        float ms = 0;
        cudaEventElapsedTime(&ms, evs[i - 1], evs[i]);
        t += ms;
        if (kinds[i] == 0) c += ms;
        else if (kinds[i] == 1) x += ms;
      }
      st->ms_compute = c;
      st->ms_exchange = x;
      st->ms_total = t;
    }
    for (auto e : evs) cudaEventDestroy(e);
    evs.clear();
    kinds.clear();
  }
};

}  // namespace gg
