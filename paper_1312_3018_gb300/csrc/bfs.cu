// Level-synchronous BFS on the partitioned graph (Section 6.3.2, Figure 11; Appendix).
//
// One BSP superstep per level:
//  - compute: top-down (push): each frontier vertex claims unvisited neighbours in the
//    visited bitmap and writes level+1 and its parent; a boundary neighbour is claimed in
//    the outbox's own bitmap instead, so all messages to one remote vertex reduce into one
//    outbox slot (Section 3.4, the Appendix's get_dst_ptr). Or bottom-up (pull): each
//    unvisited vertex stops at its first neighbour in the frontier; boundary neighbours
//    are tested in a ghost bitmap that the owner filled in the communication phase.
//  - communication: top-down sends the outbox entries claimed this level to the owner
//    (scatter with min: only an unvisited owner vertex takes the level and parent);
//    bottom-up publishes the frontier of each partition to the other's ghost bitmap.
//  - termination: the host reads how many vertices the level discovered; zero ends the
//    search (every partition voted finished).
// Frontiers are kept both as bucketed queues (degree-class buckets, for top-down work
// dispatch) and as bitmaps (for bottom-up tests).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <memory>

#include "common.cuh"
#include "hybrid.cuh"

namespace gg {

struct BfsCounters {
  uint32_t tail[2][kNBucket];  // next-queue length per partition and bucket
  uint32_t dirty_tail[2];      // outbox entries claimed this level
  uint32_t nf;                 // vertices discovered this level
  uint32_t pad;
  unsigned long long mf;       // their degree sum
  unsigned long long inspected;
  unsigned long long messages;
};

// Host side of bfs_hybrid: partition 0's CSR and ids (host copies made once per
// partition), its search state, and pinned message arrays for both directions.
struct HbfsHost {
  std::vector<int64_t> off0;
  std::vector<uint32_t> E0, l2g0, outbox0;
  std::unique_ptr<std::atomic<uint64_t>[]> vis, oseen;   // partition 0 / its outbox slots
  std::vector<uint32_t> level, parent;
  uint32_t* pin_out = nullptr;  // [3 nout0]: (local id in partition 1, level, parent)
  uint32_t* pin_in = nullptr;   // [3 nout1]: (local id in partition 0, level, parent)
  DevBuf dmsg;                  // [3 max(nout0, nout1)] device staging of either direction
  cudaEvent_t ev[3] = {};       // GPU compute start / end, device messages ready
};

struct BfsWs {
  DevBuf level[2], parent[2], visited[2], front[2][2], queue[2][2], hubq[2][2];
  DevBuf oseen[2], olevel[2], oparent[2], dirty[2], ghost[2];
  size_t words[2] = {0, 0}, owords[2] = {0, 0};
  HbfsHost* hyb = nullptr;
};

void free_hbfs(graph* g, BfsWs* w) {
  HbfsHost* h = w->hyb;
  if (!h) return;
  if (h->pin_out) cudaFreeHost(h->pin_out);
  if (h->pin_in) cudaFreeHost(h->pin_in);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  dfree(g, h->dmsg);
  delete h;
  w->hyb = nullptr;
}

void free_bfs(graph* g) {
  if (!g->bfs) return;
  BfsWs* w = g->bfs;
  free_hbfs(g, w);
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->level[p], &w->parent[p], &w->visited[p], &w->front[p][0],
                     &w->front[p][1], &w->queue[p][0], &w->queue[p][1], &w->hubq[p][0],
                     &w->hubq[p][1], &w->oseen[p],
                     &w->olevel[p], &w->oparent[p], &w->dirty[p], &w->ghost[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->bfs = nullptr;
}

namespace {

struct BfsSide {
  PartView P;
  uint32_t* level;
  uint32_t* parent;
  uint32_t* visited;
  const uint32_t* front;  // current frontier bitmap
  uint32_t* next;         // next frontier bitmap
  const uint32_t* queue;  // current queue (bucketed)
  uint32_t* nqueue;       // next queue (bucketed)
  uint32_t* nhubq;        // next hub chunk list
  uint32_t* oseen;        // outbox claims
  uint32_t* olevel;
  uint32_t* oparent;
  uint32_t* dirty;        // outbox indices claimed this level
  uint32_t* ghost;        // frontier bits of the outbox targets (bottom-up)
};

struct BfsArgs {
  BfsSide side[2];
  BfsCounters* ctr;
  uint32_t L;  // level being expanded
};

struct LocalCounts {
  uint32_t nf = 0;
  unsigned long long mf = 0, insp = 0, msg = 0;
};

__device__ void flush_counts(LocalCounts c, BfsCounters* ctr) {
  __shared__ unsigned long long s[4];
  if (threadIdx.x < 4) s[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long nf = warp_sum((unsigned long long)c.nf), mf = warp_sum(c.mf),
                     in = warp_sum(c.insp), ms = warp_sum(c.msg);
  if (lane_id() == 0) {
    if (nf) atomicAdd(&s[0], nf);
    if (mf) atomicAdd(&s[1], mf);
    if (in) atomicAdd(&s[2], in);
    if (ms) atomicAdd(&s[3], ms);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s[0]) atomicAdd(&ctr->nf, (uint32_t)s[0]);
    if (s[1]) atomicAdd(&ctr->mf, s[1]);
    if (s[2]) atomicAdd(&ctr->inspected, s[2]);
    if (s[3]) atomicAdd(&ctr->messages, s[3]);
  }
}

// Top-down edge loop of one vertex whose adjacency starts at Ep: edges i = first,
// first + stride, ... < deg (warp-uniform trip count). The append machinery runs only when
// some lane of the warp discovered a vertex or claimed an outbox slot.
__device__ __forceinline__ void td_edges(const BfsSide& S, int p, uint32_t L, uint32_t vgid,
                                         const uint32_t* Ep, int first, int deg, int stride,
                                         BfsCounters* ctr, LocalCounts& c) {
  const uint64_t pol = l2_evict_first_policy();
  for (int i = first; __any_sync(kFull, i < deg); i += stride) {
    bool dis = false, msg = false;
    uint32_t u = 0, idx = 0;
    if (i < deg) {
      c.insp++;
      const uint32_t x = ld_stream(Ep + i, pol);
      if (!(x & kRemote)) {
        if (bitmap_claim(S.visited, x)) {
          dis = true;
          u = x;
          S.level[x] = L + 1;
          S.parent[x] = vgid;
          atomicOr(&S.next[x >> 5], 1u << (x & 31u));
          c.nf++;
          c.mf += (unsigned long long)(S.P.off[x + 1] - S.P.off[x]);
        }
      } else {
        idx = x & kIdMask;
        if (bitmap_claim(S.oseen, idx)) {
          msg = true;
          S.olevel[idx] = L + 1;
          S.oparent[idx] = vgid;
        }
      }
    }
    if (__any_sync(kFull, dis || msg)) {
      warp_append_bucketed(dis, u, dis ? bucket_of(S.P, u) : 0, ctr->tail[p], S.nqueue, S.P,
                           S.nhubq);
      warp_append(msg, idx, &ctr->dirty_tail[p], S.dirty);
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_bfs_topdown(const __grid_constant__ Plan plan, const __grid_constant__ BfsArgs A) {
  LocalCounts c;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const int p = G.part;
    const BfsSide& S = A.side[p];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      // one hub chunk per plan block
      const uint32_t ch = G.items[rel];
      const uint32_t v = S.P.chunk_vertex[ch];
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      td_edges(S, p, A.L, S.P.l2g[v], S.P.E + e0, threadIdx.x, (int)(e1 - e0), kThreads, A.ctr,
               c);
    } else {
      const int gs = G.gshift;
      const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
      int64_t s = 0, t = 0;
      uint32_t vg = 0;
      if (gi < G.count) {
        const uint32_t v = G.items[gi];
        s = S.P.off[v];
        t = S.P.off[v + 1];
        vg = S.P.l2g[v];
      }
      const int gl = threadIdx.x & ((1 << gs) - 1);
      td_edges(S, p, A.L, vg, S.P.E + s, gl, (int)(t - s), 1 << gs, A.ctr, c);
    }
  }
  flush_counts(c, A.ctr);
}

// Communication phase after a top-down level: deliver claimed outbox entries of p to the
// owner partition q = 1 - p (min-scatter through the inbox order; Appendix scatter_inbox_min).
__global__ void __launch_bounds__(kThreads) k_bfs_exchange(const __grid_constant__ BfsArgs A) {
  LocalCounts c;
  const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int p = 0; p < 2; ++p) {
    const BfsSide& S = A.side[p];
    const BfsSide& Q = A.side[1 - p];
    const int q = 1 - p;
    const uint32_t cnt = *(volatile uint32_t*)&A.ctr->dirty_tail[p];
    for (uint32_t i0 = warp_global * 32; i0 < cnt; i0 += nwarps * 32) {
      const uint32_t i = i0 + lane_id();
      bool dis = false;
      uint32_t u = 0;
      if (i < cnt) {
        const uint32_t idx = S.dirty[i];
        u = S.P.outbox[idx];
        c.msg++;
        if (bitmap_claim(Q.visited, u)) {
          dis = true;
          Q.level[u] = S.olevel[idx];
          Q.parent[u] = S.oparent[idx];
          atomicOr(&Q.next[u >> 5], 1u << (u & 31u));
          c.nf++;
          c.mf += (unsigned long long)(Q.P.off[u + 1] - Q.P.off[u]);
        }
      }
      warp_append_bucketed(dis, u, dis ? bucket_of(Q.P, u) : 0, A.ctr->tail[q], Q.nqueue, Q.P,
                           Q.nhubq);
    }
  }
  flush_counts(c, A.ctr);
}

// Communication phase before a bottom-up level: ghost bit i of p = frontier bit of
// outbox target i (pull direction, Section 4.3.2).
__global__ void k_bfs_publish_frontier(const __grid_constant__ BfsArgs A, uint32_t words0) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int p = w < words0 ? 0 : 1;
  const uint32_t word = p == 0 ? w : w - words0;
  const BfsSide& S = A.side[p];
  const BfsSide& Q = A.side[1 - p];
  if (word * 32 >= S.P.nout) return;  // warp-uniform
  const uint32_t i = word * 32 + lane_id();
  bool bit = false;
  if (i < S.P.nout) bit = bitmap_test(Q.front, S.P.outbox[i]);
  const unsigned m = __ballot_sync(kFull, bit);
  if (lane_id() == 0) S.ghost[word] = m;
}

// Bottom-up level over every unvisited vertex with edges (dense bucket segments). Leaf-
// partition vertices scan their adjacency from the end: their boundary neighbours (the
// hubs, listed after the local ones) are the likeliest frontier members.
__global__ void __launch_bounds__(kThreads)
k_bfs_bottomup(const __grid_constant__ Plan plan, const __grid_constant__ BfsArgs A) {
  LocalCounts c;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const int p = G.part;
    const BfsSide& S = A.side[p];
    const BfsSide& Q = A.side[1 - p];
    const uint32_t rel = vb - G.blk0;
    const int gs = G.gshift;  // <= 5 here
    const int gsz = 1 << gs;
    const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
    const int gl = threadIdx.x & (gsz - 1);
    const unsigned gmask = (gsz == 32) ? kFull : (((1u << gsz) - 1) << (lane_id() & ~(gsz - 1)));
    uint32_t v = 0;
    int64_t s = 0, t = 0;
    bool active = false;
    if (gi < G.count) {
      v = G.v0 + gi;
      if (!bitmap_test(S.visited, v)) {
        active = true;
        s = S.P.off[v];
        t = S.P.off[v + 1];
      }
    }
    const int deg = (int)(t - s);
    const bool rev = p == 1;
    bool found = false;
    uint32_t pg = 0;
    int i = gl;
    while (__any_sync(kFull, active)) {
      bool hit = false;
      uint32_t x = 0;
      if (active && i < deg) {
        c.insp++;
        x = S.P.E[rev ? t - 1 - i : s + i];
        hit = (x & kRemote) ? bitmap_test(S.ghost, x & kIdMask) : bitmap_test(S.front, x);
      }
      const unsigned hits = __ballot_sync(kFull, hit) & gmask;
      if (active) {
        if (hits) {
          const int src = __ffs(hits) - 1;
          const uint32_t xs = __shfl_sync(gmask, x, src);
          if (gl == 0) {
            found = true;
            pg = (xs & kRemote) ? Q.P.l2g[S.P.outbox[xs & kIdMask]] : S.P.l2g[xs];
          }
          active = false;
        } else {
          i += gsz;
          if (i - gl >= deg) active = false;
        }
      }
    }
    if (found) {
      S.level[v] = A.L + 1;
      S.parent[v] = pg;
      atomicOr(&S.visited[v >> 5], 1u << (v & 31u));
      atomicOr(&S.next[v >> 5], 1u << (v & 31u));
      c.nf++;
      c.mf += (unsigned long long)deg;
    }
    warp_append_bucketed(found, v, found ? G.bucket : 0, A.ctr->tail[p], S.nqueue, S.P, S.nhubq);
  }
  flush_counts(c, A.ctr);
}

__global__ void k_bfs_init(const __grid_constant__ BfsArgs A, const uint32_t* g2l,
                           uint32_t source, uint32_t* queue0, uint32_t* queue1, uint32_t* hubq0,
                           uint32_t* hubq1) {
  const uint32_t gl = g2l[source];
  const int p = gl >> 31;
  const uint32_t lid = gl & kIdMask;
  const BfsSide& S = A.side[p];
  S.level[lid] = 0;
  S.parent[lid] = source;
  S.visited[lid >> 5] |= 1u << (lid & 31u);
  ((uint32_t*)S.front)[lid >> 5] |= 1u << (lid & 31u);
  const int b = bucket_of(S.P, lid);
  A.ctr->nf = 1;
  A.ctr->mf = (unsigned long long)(S.P.off[lid + 1] - S.P.off[lid]);
  if (b == 0) {
    append_hub_chunks(S.P, lid, &A.ctr->tail[p][0], p == 0 ? hubq0 : hubq1);
  } else if (b < kNBucket) {
    (p == 0 ? queue0 : queue1)[S.P.bstart[b]] = lid;
    A.ctr->tail[p][b] = 1;
  }
}

// Results in global order: thread i reads vertex i's local entry through g2l, so the writes
// (possibly over the host link) are coalesced.
__global__ void k_bfs_collect(const __grid_constant__ BfsArgs A, uint32_t n, const uint32_t* g2l,
                              uint32_t* levels, uint32_t* parents) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t gl = g2l[i];
  const BfsSide& S = A.side[gl >> 31];
  const uint32_t lid = gl & kIdMask;
  levels[i] = S.level[lid];
  if (parents) parents[i] = S.parent[lid];
}

// bfs_hybrid, device to host: partition 1's outbox claims of this level as (owner's local
// id in partition 0, level, parent).
__global__ void k_hbfs_out(const __grid_constant__ BfsArgs A, uint32_t* out) {
  const BfsSide& S = A.side[1];
  const uint32_t cnt = A.ctr->dirty_tail[1];
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
    const uint32_t idx = S.dirty[k];
    out[3 * k] = S.P.outbox[idx];
    out[3 * k + 1] = S.olevel[idx];
    out[3 * k + 2] = S.oparent[idx];
  }
}

// bfs_hybrid, host to device: messages (local id in partition 1, level, parent) from the
// host's partition 0. An unvisited target takes the level and parent and joins the next
// queue (the scatter of the communication phase, as in k_bfs_exchange).
__global__ void __launch_bounds__(kThreads) k_hbfs_in(const __grid_constant__ BfsArgs A,
                                                      const uint32_t* in, uint32_t cnt) {
  LocalCounts c;
  const BfsSide& Q = A.side[1];
  const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t i0 = warp_global * 32; i0 < cnt; i0 += nwarps * 32) {
    const uint32_t i = i0 + lane_id();
    bool dis = false;
    uint32_t u = 0;
    if (i < cnt) {
      u = in[3 * i];
      c.msg++;
      if (bitmap_claim(Q.visited, u)) {
        dis = true;
        Q.level[u] = in[3 * i + 1];
        Q.parent[u] = in[3 * i + 2];
        atomicOr(&Q.next[u >> 5], 1u << (u & 31u));
        c.nf++;
        c.mf += (unsigned long long)(Q.P.off[u + 1] - Q.P.off[u]);
      }
    }
    warp_append_bucketed(dis, u, dis ? bucket_of(Q.P, u) : 0, A.ctr->tail[1], Q.nqueue, Q.P,
                         Q.nhubq);
  }
  flush_counts(c, A.ctr);
}

graph_status alloc_ws(graph* g) {
  if (g->bfs) return GRAPH_OK;
  BfsWs* w = new BfsWs();
  g->bfs = w;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    w->words[p] = (P.nv + 31) / 32;
    w->owords[p] = (P.nout + 31) / 32;
    const size_t nv = P.nv, words = w->words[p], owords = w->owords[p];
    GG_TRY(dalloc(g, w->level[p], 4 * nv));
    GG_TRY(dalloc(g, w->parent[p], 4 * nv));
    GG_TRY(dalloc(g, w->visited[p], 4 * words));
    GG_TRY(dalloc(g, w->front[p][0], 4 * words));
    GG_TRY(dalloc(g, w->front[p][1], 4 * words));
    GG_TRY(dalloc(g, w->queue[p][0], 4 * nv));
    GG_TRY(dalloc(g, w->queue[p][1], 4 * nv));
    GG_TRY(dalloc(g, w->hubq[p][0], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->hubq[p][1], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->oseen[p], 4 * owords));
    GG_TRY(dalloc(g, w->olevel[p], 4 * (size_t)P.nout));
    GG_TRY(dalloc(g, w->oparent[p], 4 * (size_t)P.nout));
    GG_TRY(dalloc(g, w->dirty[p], 4 * (size_t)P.nout));
    GG_TRY(dalloc(g, w->ghost[p], 4 * owords));
  }
  if (g->counters.bytes < sizeof(BfsCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g) {
  const graph_status s = alloc_ws(g);
  if (s != GRAPH_OK) free_bfs(g);
  return s;
}

BfsArgs make_args(graph* g, int cur, uint32_t L) {
  BfsWs* w = g->bfs;
  BfsArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    BfsSide& S = A.side[p];
    S.P = g->part[p].view();
    S.level = (uint32_t*)w->level[p].p;
    S.parent = (uint32_t*)w->parent[p].p;
    S.visited = (uint32_t*)w->visited[p].p;
    S.front = (const uint32_t*)w->front[p][cur].p;
    S.next = (uint32_t*)w->front[p][1 - cur].p;
    S.queue = (const uint32_t*)w->queue[p][cur].p;
    S.nqueue = (uint32_t*)w->queue[p][1 - cur].p;
    S.nhubq = (uint32_t*)w->hubq[p][1 - cur].p;
    S.oseen = (uint32_t*)w->oseen[p].p;
    S.olevel = (uint32_t*)w->olevel[p].p;
    S.oparent = (uint32_t*)w->oparent[p].p;
    S.dirty = (uint32_t*)w->dirty[p].p;
    S.ghost = (uint32_t*)w->ghost[p].p;
  }
  A.ctr = (BfsCounters*)g->counters.p;
  A.L = L;
  return A;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" graph_status bfs(graph_t* g, uint32_t source, uint32_t* levels, uint32_t* parents,
                            const bfs_attr* attr, graph_stats* stats) {
  if (!g || !levels) {
    set_error("graph or levels is NULL");
    return GRAPH_EINVAL;
  }
  if (source >= g->n) {
    set_error("source %u >= n %u", source, g->n);
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before bfs");
    return GRAPH_ESTATE;
  }
  bfs_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) {
    set_error("bad out_mem");
    return GRAPH_EINVAL;
  }
  const double alpha = at.alpha > 0 ? at.alpha : 15.0;
  const double beta = at.beta > 0 ? at.beta : 18.0;
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps : (int64_t)g->n + 1;
  GG_TRY(ensure_ws(g));
  BfsWs* w = g->bfs;
  cudaStream_t st = g->stream;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  // Reset state.
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->level[p].p, 0xFF, 4ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->parent[p].p, 0xFF, 4ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->visited[p].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->front[p][0].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->oseen[p].p, 0, 4 * w->owords[p], st));
  }
  GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(BfsCounters), st));
  int cur = 0;
  {
    BfsArgs A = make_args(g, cur, 0);
    k_bfs_init<<<1, 1, 0, st>>>(A, (const uint32_t*)g->g2l.p, source,
                                (uint32_t*)w->queue[0][cur].p, (uint32_t*)w->queue[1][cur].p,
                                (uint32_t*)w->hubq[0][cur].p, (uint32_t*)w->hubq[1][cur].p);
    GG_CUDA(cudaGetLastError());
  }
  BfsCounters* hc = (BfsCounters*)g->host_counters;
  GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  int64_t traversed = 0, inspected = 0, messages = 0, explored = 0, launches = 1;
  int td_steps = 0, bu_steps = 0;
  bool bottom_up = false;
  uint32_t nf_prev = 0;
  int64_t L = 0;
  for (;; ++L) {
    BfsCounters c = *hc;
    if (c.nf == 0) break;
    if (L >= cap) {
      set_error("bfs reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    traversed += (int64_t)c.mf;
    // Direction choice (Beamer et al.): edges out of the frontier vs edges left unexplored.
    const int64_t unexplored = g->m - explored - (int64_t)c.mf;
    if (at.direction == GRAPH_BFS_TOPDOWN) {
      bottom_up = false;
    } else if (at.direction == GRAPH_BFS_BOTTOMUP) {
      bottom_up = L > 0;
    } else if (!bottom_up) {
      bottom_up = L > 0 && (double)c.mf > (double)unexplored / alpha;
    } else {
      bottom_up = !((double)c.nf < (double)g->n / beta && c.nf < nf_prev);
    }
    explored += (int64_t)c.mf;
    nf_prev = c.nf;
    GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(BfsCounters), st));
    for (int p = 0; p < 2; ++p)
      GG_CUDA(cudaMemsetAsync(w->front[p][1 - cur].p, 0, 4 * w->words[p], st));
    BfsArgs A = make_args(g, cur, (uint32_t)L);
    timer.mark(2);
    if (!bottom_up) {
      Plan pl;
      memset(&pl, 0, sizeof(pl));
      const int gsh[kNBucket] = {8, 5, kSubShift, 0};
      for (int p = 0; p < 2; ++p) {
        const PartView V = g->part[p].view();
        plan_add(pl, (const uint32_t*)w->hubq[p][cur].p, 0, c.tail[p][0], p, 8, 0);  // chunks
        for (int b = 1; b < kNBucket; ++b)
          plan_add(pl, (const uint32_t*)w->queue[p][cur].p + V.bstart[b], 0, c.tail[p][b], p,
                   gsh[b], b);
      }
      if (pl.nblocks) k_bfs_topdown<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
      GG_CUDA(cudaGetLastError());
      timer.mark(0);
      k_bfs_exchange<<<152 * 4, kThreads, 0, st>>>(A);
      launches += 1 + (pl.nblocks ? 1 : 0);
      GG_CUDA(cudaGetLastError());
      timer.mark(1);
      td_steps++;
    } else {
      const uint32_t words0 = (uint32_t)((g->part[0].nout + 31) / 32);
      const uint32_t words1 = (uint32_t)((g->part[1].nout + 31) / 32);
      const uint64_t tw = (uint64_t)words0 + words1;
      if (tw) k_bfs_publish_frontier<<<grid_for(tw * 32, 256), 256, 0, st>>>(A, words0);
      launches += tw ? 1 : 0;
      GG_CUDA(cudaGetLastError());
      timer.mark(1);
      Plan pl;
      memset(&pl, 0, sizeof(pl));
      const int gsh[kNBucket] = {5, 5, kSubShift, 0};
      for (int p = 0; p < 2; ++p) {
        const PartView V = g->part[p].view();
        for (int b = 0; b < kNBucket; ++b)
          plan_add(pl, nullptr, V.bstart[b], V.bstart[b + 1] - V.bstart[b], p, gsh[b], b);
      }
      if (pl.nblocks) k_bfs_bottomup<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
      launches += pl.nblocks ? 1 : 0;
      GG_CUDA(cudaGetLastError());
      timer.mark(0);
      bu_steps++;
    }
    GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    cur = 1 - cur;
  }
  // Collect (local -> global order).
  graph_status s = GRAPH_OK;
  void *dl = nullptr, *dp = nullptr;
  bool sl = false, sp = false;
  GG_TRY(out_target(g, levels, at.out_mem, 8ull * g->n, 0, &dl, &sl));
  if (parents) GG_TRY(out_target(g, parents, at.out_mem, 8ull * g->n, 4ull * g->n, &dp, &sp));
  {
    BfsArgs A = make_args(g, cur, 0);
    k_bfs_collect<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->n, (const uint32_t*)g->g2l.p,
                                                       (uint32_t*)dl, (uint32_t*)dp);
    launches++;
    GG_CUDA(cudaGetLastError());
  }
  if (sl) GG_TRY(deliver(g, levels, dl, 4ull * g->n, GRAPH_MEM_HOST));
  if (sp) GG_TRY(deliver(g, parents, dp, 4ull * g->n, GRAPH_MEM_HOST));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)L;
    stats->topdown_steps = td_steps;
    stats->bottomup_steps = bu_steps;
    stats->edges_traversed = traversed;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
  }
  timer.finish(stats);
  return s;
}

// ---------------------------------------------------------------------------------------
// bfs_hybrid: partition 0 on host threads, partition 1 on the GPU (Section 4.1, Figure 6;
// Section 6.2-6.3). Both sides expand their own frontier top-down in the same superstep
// (Figure 11); only messages cross: the claims each side made on the other's vertices,
// as (target, level, parent) lists.
// ---------------------------------------------------------------------------------------
namespace gg {
namespace {

graph_status ensure_hbfs(graph* g, BfsWs* w) {
  if (w->hyb) return GRAPH_OK;
  const Part& P0 = g->part[0];
  const Part& P1 = g->part[1];
  cudaStream_t st = g->stream;
  HbfsHost* h = new HbfsHost();
  w->hyb = h;
  h->off0.resize((size_t)P0.nv + 1);
  h->E0.resize((size_t)P0.ne);
  h->l2g0.resize(P0.nv);
  h->outbox0.resize(P0.nout);
  h->level.resize(P0.nv);
  h->parent.resize(P0.nv);
  h->vis.reset(new std::atomic<uint64_t>[(P0.nv + 63) / 64 + 1]);
  h->oseen.reset(new std::atomic<uint64_t>[(P0.nout + 63) / 64 + 1]);
  GG_CUDA(cudaMemcpyAsync(h->off0.data(), P0.off.p, 8ull * (P0.nv + 1), cudaMemcpyDeviceToHost, st));
  if (P0.ne) GG_CUDA(cudaMemcpyAsync(h->E0.data(), P0.E.p, 4ull * P0.ne, cudaMemcpyDefault, st));
  if (P0.nv) GG_CUDA(cudaMemcpyAsync(h->l2g0.data(), P0.l2g.p, 4ull * P0.nv, cudaMemcpyDeviceToHost, st));
  if (P0.nout)
    GG_CUDA(cudaMemcpyAsync(h->outbox0.data(), P0.outbox.p, 4ull * P0.nout, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  for (cudaEvent_t& e : h->ev) GG_CUDA(cudaEventCreate(&e));
  const size_t b0 = 12ull * std::max<uint32_t>(P0.nout, 1), b1 = 12ull * std::max<uint32_t>(P1.nout, 1);
  if (cudaHostAlloc((void**)&h->pin_out, b0, cudaHostAllocDefault) != cudaSuccess) h->pin_out = nullptr;
  if (cudaHostAlloc((void**)&h->pin_in, b1, cudaHostAllocDefault) != cudaSuccess) h->pin_in = nullptr;
  if (!h->pin_out || !h->pin_in) {
    set_error("pinned host allocation of the message arrays failed");
    return GRAPH_ENOMEM;
  }
  GG_TRY(dalloc(g, h->dmsg, std::max(b0, b1)));
  return GRAPH_OK;
}

}  // namespace
}  // namespace gg

extern "C" graph_status bfs_hybrid(graph_t* g, uint32_t source, uint32_t* levels,
                                   uint32_t* parents, const bfs_attr* attr, int cpu_threads,
                                   graph_stats* stats, pagerank_hybrid_info* info) {
  using Clock = std::chrono::steady_clock;
  if (!g || !levels) {
    set_error("graph or levels is NULL");
    return GRAPH_EINVAL;
  }
  if (source >= g->n) {
    set_error("source %u >= n %u", source, g->n);
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before bfs_hybrid");
    return GRAPH_ESTATE;
  }
  bfs_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if ((at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) ||
      at.direction == GRAPH_BFS_BOTTOMUP || cpu_threads > GRAPH_HYBRID_MAX_THREADS) {
    set_error("bad bfs_hybrid attributes (top-down only; out_mem; cpu_threads)");
    return GRAPH_EINVAL;
  }
  const int nt = hybrid_threads(cpu_threads);
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps : (int64_t)g->n + 1;
  GG_TRY(ensure_ws(g));
  BfsWs* w = g->bfs;
  {
    graph_status s = GRAPH_OK;
    try {
      s = ensure_hbfs(g, w);
    } catch (const std::bad_alloc&) {
      set_error("host allocation for the host partition failed");
      s = GRAPH_ENOMEM;
    }
    if (s != GRAPH_OK) {
      free_hbfs(g, w);
      return s;
    }
  }
  HbfsHost* h = w->hyb;
  cudaStream_t st = g->stream;
  const Part& P0 = g->part[0];
  const uint32_t nv0 = P0.nv;
  const auto t_start = Clock::now();
  // Reset: the device state of partition 1, the host state of partition 0.
  {
    const Part& P1 = g->part[1];
    GG_CUDA(cudaMemsetAsync(w->level[1].p, 0xFF, 4ull * P1.nv, st));
    GG_CUDA(cudaMemsetAsync(w->parent[1].p, 0xFF, 4ull * P1.nv, st));
    GG_CUDA(cudaMemsetAsync(w->visited[1].p, 0, 4 * w->words[1], st));
    GG_CUDA(cudaMemsetAsync(w->front[1][0].p, 0, 4 * w->words[1], st));
    GG_CUDA(cudaMemsetAsync(w->oseen[1].p, 0, 4 * w->owords[1], st));
    GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(BfsCounters), st));
  }
  std::fill(h->level.begin(), h->level.end(), kInf);
  std::fill(h->parent.begin(), h->parent.end(), kInf);
  for (size_t i = 0; i < (nv0 + 63) / 64 + 1; ++i) h->vis[i].store(0, std::memory_order_relaxed);
  for (size_t i = 0; i < (P0.nout + 63) / 64 + 1; ++i) h->oseen[i].store(0, std::memory_order_relaxed);
  uint32_t gl = 0;
  GG_CUDA(cudaMemcpyAsync(&gl, (const uint32_t*)g->g2l.p + source, 4, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  int cur = 0;
  std::vector<uint32_t> F0;   // partition 0's frontier (local ids)
  int64_t traversed = 0, inspected = 0, messages = 0, launches = 0, host_mf = 0;
  if (gl & kRemote) {
    BfsArgs A = make_args(g, cur, 0);
    k_bfs_init<<<1, 1, 0, st>>>(A, (const uint32_t*)g->g2l.p, source,
                                (uint32_t*)w->queue[0][cur].p, (uint32_t*)w->queue[1][cur].p,
                                (uint32_t*)w->hubq[0][cur].p, (uint32_t*)w->hubq[1][cur].p);
    GG_CUDA(cudaGetLastError());
    launches++;
  } else {
    const uint32_t lid = gl;
    h->level[lid] = 0;
    h->parent[lid] = source;
    host_claim(h->vis.get(), lid);
    F0.push_back(lid);
    host_mf = h->off0[lid + 1] - h->off0[lid];
  }
  BfsCounters* hc = (BfsCounters*)g->host_counters;
  GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  double ms_cpu = 0, ms_gpu = 0, ms_xchg = 0;
  std::vector<std::vector<uint32_t>> disc(nt), mslot(nt), mpar(nt);
  std::vector<int64_t> tmf(nt), tin(nt);
  int64_t L = 0;
  for (;; ++L) {
    const BfsCounters c = *hc;
    if (c.nf == 0 && F0.empty()) break;
    if (L >= cap) {
      set_error("bfs_hybrid reached the superstep cap (%lld)", (long long)cap);
      return GRAPH_ETIMEOUT;
    }
    traversed += (int64_t)c.mf + host_mf;
    host_mf = 0;
    // GPU: partition 1's top-down level, then its claims on partition 0 as messages.
    GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(BfsCounters), st));
    GG_CUDA(cudaMemsetAsync(w->front[1][1 - cur].p, 0, 4 * w->words[1], st));
    BfsArgs A = make_args(g, cur, (uint32_t)L);
    GG_CUDA(cudaEventRecord(h->ev[0], st));
    {
      Plan pl;
      memset(&pl, 0, sizeof(pl));
      const int gsh[kNBucket] = {8, 5, kSubShift, 0};
      const PartView V = g->part[1].view();
      plan_add(pl, (const uint32_t*)w->hubq[1][cur].p, 0, c.tail[1][0], 1, 8, 0);
      for (int b = 1; b < kNBucket; ++b)
        plan_add(pl, (const uint32_t*)w->queue[1][cur].p + V.bstart[b], 0, c.tail[1][b], 1,
                 gsh[b], b);
      if (pl.nblocks) {
        k_bfs_topdown<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
        launches++;
      }
    }
    GG_CUDA(cudaEventRecord(h->ev[1], st));
    k_hbfs_out<<<152 * 2, 256, 0, st>>>(A, (uint32_t*)h->dmsg.p);
    launches++;
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaEventRecord(h->ev[2], st));
    // Host: partition 0's top-down level (Figure 11) while the GPU works.
    const auto tc0 = Clock::now();
    for (int k = 0; k < nt; ++k) {
      disc[k].clear();
      mslot[k].clear();
      mpar[k].clear();
      tmf[k] = 0;
      tin[k] = 0;
    }
    const uint32_t next_level = (uint32_t)L + 1;
    host_dynamic(nt, F0.size(), 1, [&](int k, uint64_t a, uint64_t b) {
      for (uint64_t i = a; i < b; ++i) {
        const uint32_t v = F0[i];
        const uint32_t vg = h->l2g0[v];
        const int64_t e1 = h->off0[v + 1];
        for (int64_t e = h->off0[v]; e < e1; ++e) {
          const uint32_t x = h->E0[e];
          if (!(x & kRemote)) {
            if (host_claim(h->vis.get(), x)) {
              h->level[x] = next_level;
              h->parent[x] = vg;
              disc[k].push_back(x);
              tmf[k] += h->off0[x + 1] - h->off0[x];
            }
          } else if (host_claim(h->oseen.get(), x & kIdMask)) {
            mslot[k].push_back(x & kIdMask);
            mpar[k].push_back(vg);
          }
        }
        tin[k] += e1 - h->off0[v];
      }
    });
    const auto tc1 = Clock::now();
    ms_cpu += std::chrono::duration<double, std::milli>(tc1 - tc0).count();
    // Exchange: the GPU's claims on partition 0 come up and are applied on the host ...
    GG_CUDA(cudaEventSynchronize(h->ev[2]));
    float gms = 0;
    GG_CUDA(cudaEventElapsedTime(&gms, h->ev[0], h->ev[1]));
    ms_gpu += gms;
    const auto tx0 = Clock::now();
    const uint32_t n1 = hc->dirty_tail[1];
    inspected += (int64_t)hc->inspected;
    if (n1) {
      GG_CUDA(cudaMemcpyAsync(h->pin_in, h->dmsg.p, 12ull * n1, cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<uint32_t> in_disc;
    for (uint32_t i = 0; i < n1; ++i) {
      const uint32_t u = h->pin_in[3 * i];
      if (host_claim(h->vis.get(), u)) {
        h->level[u] = h->pin_in[3 * i + 1];
        h->parent[u] = h->pin_in[3 * i + 2];
        in_disc.push_back(u);
        host_mf += h->off0[u + 1] - h->off0[u];
      }
    }
    // ... and the host's claims on partition 1 go down and are applied on the device.
    uint32_t n0 = 0;
    for (int k = 0; k < nt; ++k)
      for (size_t j = 0; j < mslot[k].size(); ++j) {
        h->pin_out[3 * n0] = h->outbox0[mslot[k][j]];
        h->pin_out[3 * n0 + 1] = next_level;
        h->pin_out[3 * n0 + 2] = mpar[k][j];
        ++n0;
      }
    if (n0) {
      GG_CUDA(cudaMemcpyAsync(h->dmsg.p, h->pin_out, 12ull * n0, cudaMemcpyHostToDevice, st));
      k_hbfs_in<<<std::min(grid_for(32ull * n0, kThreads), 152u * 8), kThreads, 0, st>>>(
          A, (const uint32_t*)h->dmsg.p, n0);
      launches++;
      GG_CUDA(cudaGetLastError());
    }
    // The counters now hold the level's discoveries in partition 1 from both kernels (the
    // next queue's tails, nf, mf).
    GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(BfsCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    messages += (int64_t)n1 + n0;
    ms_xchg += std::chrono::duration<double, std::milli>(Clock::now() - tx0).count();
    // Partition 0's next frontier.
    F0.clear();
    for (int k = 0; k < nt; ++k) {
      F0.insert(F0.end(), disc[k].begin(), disc[k].end());
      host_mf += tmf[k];
      inspected += tin[k];
    }
    F0.insert(F0.end(), in_disc.begin(), in_disc.end());
    cur = 1 - cur;
  }
  (void)t_start;
  // Collect: the host partition's levels and parents join the device's, then the usual
  // local -> global write.
  if (nv0) {
    GG_CUDA(cudaMemcpyAsync(w->level[0].p, h->level.data(), 4ull * nv0, cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaMemcpyAsync(w->parent[0].p, h->parent.data(), 4ull * nv0, cudaMemcpyHostToDevice, st));
  }
  void *dl = nullptr, *dp = nullptr;
  bool sl = false, sp = false;
  GG_TRY(out_target(g, levels, at.out_mem, 8ull * g->n, 0, &dl, &sl));
  if (parents) GG_TRY(out_target(g, parents, at.out_mem, 8ull * g->n, 4ull * g->n, &dp, &sp));
  {
    BfsArgs A = make_args(g, cur, 0);
    k_bfs_collect<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->n, (const uint32_t*)g->g2l.p,
                                                       (uint32_t*)dl, (uint32_t*)dp);
    launches++;
    GG_CUDA(cudaGetLastError());
  }
  if (sl) GG_TRY(deliver(g, levels, dl, 4ull * g->n, GRAPH_MEM_HOST));
  if (sp) GG_TRY(deliver(g, parents, dp, 4ull * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)L;
    stats->topdown_steps = (int)L;
    stats->edges_traversed = traversed;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
    stats->ms_compute = std::max(ms_cpu, ms_gpu);
    stats->ms_exchange = ms_xchg;
    stats->ms_total = std::chrono::duration<double, std::milli>(Clock::now() - t_start).count();
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->cpu_threads = nt;
    info->cpu_vertices = nv0;
    info->gpu_vertices = g->part[1].nv;
    info->cpu_edges = P0.ne;
    info->gpu_edges = g->part[1].ne;
    info->ms_cpu_compute = ms_cpu;
    info->ms_gpu_compute = ms_gpu;
    info->ms_exchange = ms_xchg;
  }
  return s;
}
