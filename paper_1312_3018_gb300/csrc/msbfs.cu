// Batched BFS: up to 64 level-synchronous searches share one sequence of BSP supersteps
// (Section 4.1's compute / communication / termination phases, the BFS of Section 6.3.2
// and Figure 11 run for k sources at once). Every vertex carries 64-bit masks, bit s
// belonging to search s (multi-source BFS as bit lanes, Then et al., VLDB 2014):
//   seen[v]   searches that have reached v
//   front[v]  searches for which v is in the current frontier
//   next[v]   searches that reach v in this level
// One superstep:
//  - compute, push: each frontier vertex ORs front[v] & ~seen[u] into next[u] of every
//    local neighbour u and front[v] into the outbox slot of every boundary neighbour; or
//    pull: each vertex that some search has not reached ORs the frontier masks of its
//    neighbours (boundary neighbours through the ghost masks) until every missing search
//    is covered, and keeps the covered bits in next[v].
//  - communication: push ORs each outbox slot, less what the owner has seen, into the
//    owner's next mask (the inbox side); pull publishes the owner's frontier masks into the
//    ghost masks before the compute phase (Section 4.3.2's pull direction).
//  - advance and termination: seen |= next, next becomes the frontier, the level of each
//    new (vertex, search) pair is written to the vertex's level lanes, and the host reads
//    how many vertices gained a bit; zero ends all k searches.
// Level lanes are vertex-major (K = roundup(k, 4) uint32 per vertex) so that the advance
// writes and the final transpose to the caller's search-major layout are coalesced.
#include <string.h>

#include "common.cuh"
#include "jobs.cuh"

namespace gg {

typedef unsigned long long u64;

struct MsCounters {
  u64 nf;         // vertices that gained a bit this level
  u64 mf;         // their degree sum (edges out of the next frontier)
  u64 mu;         // degree sum of vertices with edges that some search has not reached
  u64 traversed;  // sum over new (vertex, search) pairs of the vertex degree
  u64 inspected;  // edge entries read by the compute phase
  u64 messages;   // outbox slots delivered by the exchange
  u64 gained;     // searches (bits) that reached a new vertex this level
};

// Device-side control of a graph-driven bfs_batch (one superstep after another inside a
// CUDA graph while loop, no host round trip): the level, the direction of the next
// superstep, the termination vote and the statistics.
struct MsCtl {
  uint32_t L;          // level the next superstep expands
  uint32_t pull;       // direction of the next superstep
  uint32_t done;       // no search gained a vertex (or the cap was reached)
  uint32_t timeout;    // the superstep cap was reached
  uint32_t push_steps, pull_steps;
  u64 traversed, inspected, messages;
  // parameters
  u64 m;               // edge entries of the graph (the direction rule's first "unexplored")
  double alpha;
  int direction;
  int pad;
  int64_t cap;
};

// The captured superstep graph of a workspace, and what it was captured for.
struct MsGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  DevBuf ctl;
  uint32_t k = 0, K = 0;
  int direction = -1;
  double alpha = 0;
  int64_t cap_steps = 0;
  void* counters = nullptr;
};

struct MsWs {
  DevBuf seen[2], mask[2][2], lvl[2], ghost[2], omsg[2];
  uint32_t K = 0;  // level lanes per vertex the lvl buffers hold
  MsGraph graph;
};

void free_msgraph(graph* g, MsWs* w) {
  MsGraph& G = w->graph;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.cap) cudaStreamDestroy(G.cap);
  dfree(g, G.ctl);
  G = MsGraph();
}

void free_msbfs(graph* g) {
  if (!g->ms) return;
  MsWs* w = g->ms;
  free_msgraph(g, w);
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->seen[p], &w->mask[p][0], &w->mask[p][1], &w->lvl[p], &w->ghost[p],
                     &w->omsg[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->ms = nullptr;
}

namespace {

struct MsSide {
  PartView P;
  u64* seen;
  u64* front;   // current frontier masks
  u64* next;    // masks gained this level
  u64* ghost;   // [nout] frontier masks of the outbox targets (pull)
  u64* omsg;    // [nout] masks pushed to the outbox targets (push)
  uint32_t* lvl;  // [nv * K] level lanes
};

struct MsArgs {
  MsSide side[2];
  MsCounters* ctr;
  u64 full;     // bits of the k searches
  uint32_t K;
  uint32_t L;   // level being expanded (the host-driven loop)
  MsCtl* ctl;   // graph-driven loop: level, direction and termination on the device, else null
};

// Graph-driven loop: whether a compute / communication kernel of direction `pull` runs
// this superstep (the other direction's kernels return at once); CTA-uniform.
__device__ __forceinline__ bool ms_skip(const MsArgs& A, uint32_t pull) {
  if (!A.ctl) return false;
  const volatile MsCtl* c = A.ctl;
  return c->done || c->pull != pull;
}

struct MsSources {
  uint32_t id[GRAPH_BATCH_MAX];
};

struct Cnt {
  u64 nf = 0, mf = 0, mu = 0, trav = 0, insp = 0, msg = 0, gained = 0;
};

__device__ void flush(const Cnt& c, MsCounters* ctr) {
  __shared__ u64 s[7];
  if (threadIdx.x < 7) s[threadIdx.x] = 0;
  __syncthreads();
  const u64 v[6] = {warp_sum(c.nf), warp_sum(c.mf), warp_sum(c.mu), warp_sum(c.trav),
                    warp_sum(c.insp), warp_sum(c.msg)};
  const u64 gor = ((u64)__reduce_or_sync(kFull, (unsigned)(c.gained >> 32)) << 32) |
                  __reduce_or_sync(kFull, (unsigned)c.gained);
  if (lane_id() == 0) {
    for (int j = 0; j < 6; ++j)
      if (v[j]) atomicAdd(&s[j], v[j]);
    if (gor) atomicOr(&s[6], gor);
  }
  __syncthreads();
  if (threadIdx.x < 6 && s[threadIdx.x]) atomicAdd(&((u64*)ctr)[threadIdx.x], s[threadIdx.x]);
  if (threadIdx.x == 6 && s[6]) atomicOr(&ctr->gained, s[6]);
}

// OR within aligned groups of 2^gshift lanes (gshift <= 5); all 32 lanes must call.
__device__ __forceinline__ u64 group_or(u64 v, int gshift) {
  for (int o = 1; o < (1 << gshift); o <<= 1) v |= __shfl_xor_sync(kFull, v, o);
  return v;
}

// Push of one frontier vertex's mask fm over edges first, first + stride, ... < deg.
__device__ __forceinline__ void push_edges(const MsSide& S, u64 fm, const uint32_t* Ep,
                                           int first, int deg, int stride, Cnt& c) {
  const uint64_t pol = l2_evict_first_policy();
  for (int i = first; i < deg; i += stride) {
    c.insp++;
    const uint32_t x = ld_stream(Ep + i, pol);
    if (!(x & kRemote)) {
      const u64 nb = fm & ~S.seen[x];
      // next only gains bits during the compute phase, so an old copy never hides a bit
      // that still has to be set
      if (nb & ~__ldcg(&S.next[x])) atomicOr(&S.next[x], nb);
    } else {
      const uint32_t idx = x & kIdMask;
      if (fm & ~__ldcg(&S.omsg[idx])) atomicOr(&S.omsg[idx], fm);
    }
  }
}

// Compute phase, push direction, over every vertex with edges (hub vertices as one CTA
// per kHubChunk-edge chunk); vertices outside every frontier are skipped.
__global__ void __launch_bounds__(kThreads)
k_ms_push(const __grid_constant__ Plan plan, const __grid_constant__ MsArgs A) {
  if (ms_skip(A, 0)) return;
  Cnt c;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const MsSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      const uint32_t ch = G.v0 + rel;
      const uint32_t v = S.P.chunk_vertex[ch];
      const u64 fm = S.front[v];
      if (!fm) continue;  // CTA-uniform
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      push_edges(S, fm, S.P.E + e0, threadIdx.x, (int)(e1 - e0), kThreads, c);
    } else {
      const int gs = G.gshift;
      const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
      if (gi >= G.count) continue;
      const uint32_t v = G.v0 + gi;
      const u64 fm = S.front[v];
      if (!fm) continue;
      const int64_t s = S.P.off[v], t = S.P.off[v + 1];
      push_edges(S, fm, S.P.E + s, threadIdx.x & ((1 << gs) - 1), (int)(t - s), 1 << gs, c);
    }
  }
  flush(c, A.ctr);
}

// Communication phase after a push level: outbox slot i of partition p carries the
// searches that reached outbox[i] of the other partition q; ORed into q's next mask less
// what q has seen, then cleared for the next level.
__global__ void __launch_bounds__(kThreads) k_ms_exchange(const __grid_constant__ MsArgs A) {
  if (ms_skip(A, 0)) return;
  Cnt c;
  const uint64_t nout0 = A.side[0].P.nout;
  const uint64_t total = nout0 + A.side[1].P.nout;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int p = i < nout0 ? 0 : 1;
    const uint32_t idx = (uint32_t)(p == 0 ? i : i - nout0);
    const MsSide& S = A.side[p];
    const MsSide& Q = A.side[1 - p];
    const u64 msg = S.omsg[idx];
    if (!msg) continue;
    S.omsg[idx] = 0;
    c.msg++;
    const uint32_t u = S.P.outbox[idx];
    const u64 nb = msg & ~Q.seen[u];
    if (nb) atomicOr(&Q.next[u], nb);
  }
  flush(c, A.ctr);
}

// Communication phase before a pull level: ghost mask i of p = frontier mask of outbox
// target i in the other partition.
__global__ void k_ms_publish(const __grid_constant__ MsArgs A) {
  if (ms_skip(A, 1)) return;
  const uint64_t nout0 = A.side[0].P.nout;
  const uint64_t total = nout0 + A.side[1].P.nout;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int p = i < nout0 ? 0 : 1;
    const uint32_t idx = (uint32_t)(p == 0 ? i : i - nout0);
    const MsSide& S = A.side[p];
    S.ghost[idx] = A.side[1 - p].front[S.P.outbox[idx]];
  }
}

__device__ __forceinline__ u64 frontier_of(const MsSide& S, uint32_t x) {
  return (x & kRemote) ? S.ghost[x & kIdMask] : S.front[x];
}

// Compute phase, pull direction. A group of lanes scans vertex v's adjacency and stops
// once the frontier masks it has ORed cover every search v has not seen. Leaf-partition
// vertices scan from the end, where their boundary neighbours (the hubs) are listed. A hub
// vertex is scanned chunk by chunk, one CTA per chunk, each warp a contiguous slice.
__global__ void __launch_bounds__(kThreads)
k_ms_pull(const __grid_constant__ Plan plan, const __grid_constant__ MsArgs A) {
  if (ms_skip(A, 1)) return;
  Cnt c;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const int p = G.part;
    const MsSide& S = A.side[p];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      const uint32_t ch = G.v0 + rel;
      const uint32_t v = S.P.chunk_vertex[ch];
      const u64 need = A.full & ~S.seen[v];
      if (!need) continue;  // CTA-uniform
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t len = min((int64_t)kHubChunk, S.P.off[v + 1] - e0);
      const int64_t slice = (len + (kThreads / 32) - 1) / (kThreads / 32);
      const int64_t w0 = e0 + (threadIdx.x >> 5) * slice;
      const int64_t w1 = min(w0 + slice, e0 + len);
      u64 acc = 0;
      for (int64_t b = w0; b < w1; b += 32) {  // warp-uniform trip count
        const int64_t e = b + lane_id();
        if (e < w1) {
          c.insp++;
          acc |= frontier_of(S, S.P.E[e]);
        }
        acc = group_or(acc, 5);
        if ((acc & need) == need) break;
      }
      if (lane_id() == 0 && (acc & need)) atomicOr(&S.next[v], acc & need);
      continue;
    }
    const int gs = G.gshift;
    const int gsz = 1 << gs;
    const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
    const int gl = threadIdx.x & (gsz - 1);
    uint32_t v = 0;
    int64_t s = 0, t = 0;
    u64 need = 0;
    if (gi < G.count) {
      v = G.v0 + gi;
      need = A.full & ~S.seen[v];
      if (need) {
        s = S.P.off[v];
        t = S.P.off[v + 1];
      }
    }
    const int deg = (int)(t - s);
    const bool rev = p == 1;
    bool active = need != 0 && deg > 0;
    u64 acc = 0;
    int i = gl;
    while (__any_sync(kFull, active)) {
      if (active && i < deg) {
        c.insp++;
        acc |= frontier_of(S, S.P.E[rev ? t - 1 - i : s + i]);
      }
      acc = group_or(acc, gs);
      if (active) {
        i += gsz;
        if ((acc & need) == need || i - gl >= deg) active = false;
      }
    }
    if (gl == 0 && (acc & need)) S.next[v] = acc & need;
  }
  flush(c, A.ctr);
}

// Advance: seen |= next; the next masks become the frontier (the old frontier buffer is
// cleared to serve as the next level's next buffer); new (vertex, search) pairs get level
// L + 1 in the vertex's level lanes, written by the whole warp one vertex at a time.
__global__ void __launch_bounds__(256) k_ms_advance(const __grid_constant__ MsArgs A) {
  uint32_t L = A.L;
  if (A.ctl) {
    const volatile MsCtl* ctl = A.ctl;
    if (ctl->done) return;
    L = ctl->L;
  }
  Cnt c;
  const uint32_t nv0 = A.side[0].P.nv;
  const uint64_t total = (uint64_t)nv0 + A.side[1].P.nv;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
    const uint64_t i = base + threadIdx.x;
    int p = 0;
    uint32_t v = 0;
    u64 nx = 0;
    if (i < total) {
      p = i < nv0 ? 0 : 1;
      v = (uint32_t)(p == 0 ? i : i - nv0);
      const MsSide& S = A.side[p];
      nx = S.next[v];
      if (S.front[v]) S.front[v] = 0;
      const int64_t deg = S.P.off[v + 1] - S.P.off[v];
      u64 sm = S.seen[v];
      if (nx) {
        sm |= nx;
        S.seen[v] = sm;
        c.nf++;
        c.mf += (u64)deg;
        c.trav += (u64)deg * (u64)__popcll(nx);
        c.gained |= nx;
      }
      if (deg > 0 && sm != A.full) c.mu += (u64)deg;
    }
    unsigned todo = __ballot_sync(kFull, nx != 0);
    while (todo) {
      const int j = __ffs(todo) - 1;
      todo &= todo - 1;
      const int pj = __shfl_sync(kFull, p, j);
      const uint32_t vj = __shfl_sync(kFull, v, j);
      const u64 mj = __shfl_sync(kFull, nx, j);
      uint32_t* row = A.side[pj].lvl + (size_t)vj * A.K;
      const uint32_t l = lane_id();
      if ((mj >> l) & 1ull) row[l] = L + 1;
      if ((mj >> (l + 32)) & 1ull) row[l + 32] = L + 1;
    }
  }
  flush(c, A.ctr);
}

// Graph-driven loop, before the first superstep: the statistics start from the seeding
// (k_ms_init), level 0 is a push, the counters are cleared for it.
__global__ void k_ms_ctl_init(MsCounters* ctr, MsCtl* ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const MsCounters c = *ctr;
  ctl->L = 0;
  ctl->pull = 0;
  ctl->done = c.nf == 0;
  ctl->timeout = 0;
  ctl->push_steps = ctl->pull_steps = 0;
  ctl->traversed = c.traversed;
  ctl->inspected = ctl->messages = 0;
  *ctr = MsCounters{};
}

// Graph-driven loop, after each superstep: the statistics, the termination vote (no
// search gained a vertex; Section 4.1: every partition votes to finish), the cap, and the
// next level's direction by the same rule the host loop applies (Beamer et al.: pull when
// the frontier's edges times alpha exceed the edges of vertices some search has not
// reached); the counters are cleared for the next superstep. With set_cond it sets the
// while loop's condition (0 ends the loop).
__global__ void k_ms_ctl_step(MsCounters* ctr, MsCtl* ctl, cudaGraphConditionalHandle h,
                              int set_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!ctl->done) {
    const MsCounters c = *ctr;
    ctl->inspected += c.inspected;
    ctl->messages += c.messages;
    ctl->traversed += c.traversed;
    if (ctl->pull) ctl->pull_steps++;
    else ctl->push_steps++;
    if (c.nf == 0) {
      ctl->done = 1;
    } else {
      ctl->L = ctl->L + 1;
      if ((int64_t)ctl->L >= ctl->cap) {
        ctl->done = 1;
        ctl->timeout = 1;
      } else if (ctl->direction == GRAPH_BFS_TOPDOWN) {
        ctl->pull = 0;
      } else if (ctl->direction == GRAPH_BFS_BOTTOMUP) {
        ctl->pull = 1;
      } else {
        ctl->pull = (double)c.mf * ctl->alpha > (double)c.mu;
      }
    }
    *ctr = MsCounters{};
  }
  if (set_cond) cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
}

__global__ void k_ms_init(const __grid_constant__ MsArgs A, const __grid_constant__ MsSources src,
                          uint32_t k, const uint32_t* g2l) {
  const uint32_t s = threadIdx.x;
  if (s >= k) return;
  const uint32_t gl = g2l[src.id[s]];
  const int p = gl >> 31;
  const uint32_t lid = gl & kIdMask;
  const MsSide& S = A.side[p];
  const u64 bit = 1ull << s;
  const u64 old = atomicOr(&S.seen[lid], bit);
  atomicOr(&S.front[lid], bit);
  S.lvl[(size_t)lid * A.K + s] = 0;
  const u64 deg = (u64)(S.P.off[lid + 1] - S.P.off[lid]);
  atomicAdd(&A.ctr->traversed, deg);
  if (old == 0) {
    atomicAdd(&A.ctr->nf, 1ull);
    atomicAdd(&A.ctr->mf, deg);
  }
}

// Local -> global, vertex-major level lanes -> search-major rows of the caller's array.
__global__ void k_ms_collect(const __grid_constant__ MsArgs A, uint32_t n, uint32_t k,
                             const uint32_t* g2l, uint32_t* levels) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const uint32_t gl = g2l[g];
  const MsSide& S = A.side[gl >> 31];
  const uint32_t lid = gl & kIdMask;
  const u64 sm = S.seen[lid];
  const uint4* row = (const uint4*)(S.lvl + (size_t)lid * A.K);
  for (uint32_t s4 = 0; s4 * 4 < k; ++s4) {
    const uint4 q = row[s4];
    const uint32_t val[4] = {q.x, q.y, q.z, q.w};
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t s = s4 * 4 + j;
      if (s < k) levels[(size_t)s * n + g] = ((sm >> s) & 1ull) ? val[j] : kInf;
    }
  }
}

// Lanes joining at level L: search `lane[t]` starts from `src[t]` (its level counts from L).
struct MsSeeds {
  uint32_t lane[GRAPH_BATCH_MAX];
  uint32_t src[GRAPH_BATCH_MAX];
  uint32_t count;
};

__global__ void k_ms_seed(const __grid_constant__ MsArgs A, const __grid_constant__ MsSeeds S,
                          const uint32_t* g2l) {
  const uint32_t t = threadIdx.x;
  if (t >= S.count) return;
  const uint32_t gl = g2l[S.src[t]];
  const MsSide& P = A.side[gl >> 31];
  const uint32_t lid = gl & kIdMask;
  const u64 bit = 1ull << S.lane[t];
  atomicOr(&P.seen[lid], bit);
  atomicOr(&P.front[lid], bit);
  P.lvl[(size_t)lid * A.K + S.lane[t]] = A.L;
}

// Levels of the finished lanes F (relative to each lane's start level) into their output
// arrays in global order; the lanes' seen bits are cleared so that the lanes can take new
// searches.
struct MsLaneOut {
  uint32_t* out[GRAPH_BATCH_MAX];
  uint32_t start[GRAPH_BATCH_MAX];
  u64 F;
};

__global__ void k_ms_lane_collect(const __grid_constant__ MsArgs A,
                                  const __grid_constant__ MsLaneOut O, uint32_t n,
                                  const uint32_t* g2l) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const uint32_t gl = g2l[g];
  const MsSide& S = A.side[gl >> 31];
  const uint32_t lid = gl & kIdMask;
  const u64 sm = S.seen[lid];
  const uint32_t* row = S.lvl + (size_t)lid * A.K;
  for (u64 f = O.F; f; f &= f - 1) {
    const int l = __ffsll((long long)f) - 1;
    O.out[l][g] = ((sm >> l) & 1ull) ? row[l] - O.start[l] : kInf;
  }
  if (sm & O.F) S.seen[lid] = sm & ~O.F;
}

graph_status alloc_ms_into(graph* g, MsWs* w, uint32_t K) {
  if (!w->seen[0].p) {
    for (int p = 0; p < 2; ++p) {
      const Part& P = g->part[p];
      GG_TRY(dalloc(g, w->seen[p], 8ull * P.nv));
      GG_TRY(dalloc(g, w->mask[p][0], 8ull * P.nv));
      GG_TRY(dalloc(g, w->mask[p][1], 8ull * P.nv));
      GG_TRY(dalloc(g, w->ghost[p], 8ull * P.nout));
      GG_TRY(dalloc(g, w->omsg[p], 8ull * P.nout));
    }
  }
  if (w->K < K) {
    w->K = 0;
    for (int p = 0; p < 2; ++p) {
      dfree(g, w->lvl[p]);
      GG_TRY(dalloc(g, w->lvl[p], 4ull * K * g->part[p].nv));
    }
    w->K = K;
  }
  return GRAPH_OK;
}

void free_ms_buffers(graph* g, MsWs* w) {
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->seen[p], &w->mask[p][0], &w->mask[p][1], &w->lvl[p], &w->ghost[p],
                     &w->omsg[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  w->K = 0;
}

graph_status alloc_ws(graph* g, uint32_t K) {
  if (!g->ms) g->ms = new MsWs();
  GG_TRY(alloc_ms_into(g, g->ms, K));
  if (g->counters.bytes < sizeof(MsCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g, uint32_t K) {
  const graph_status s = alloc_ws(g, K);
  if (s != GRAPH_OK) free_msbfs(g);
  return s;
}

MsArgs make_args_ws(graph* g, MsWs* w, MsCounters* ctr, int cur, u64 full, uint32_t L) {
  MsArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    MsSide& S = A.side[p];
    S.P = g->part[p].view();
    S.seen = (u64*)w->seen[p].p;
    S.front = (u64*)w->mask[p][cur].p;
    S.next = (u64*)w->mask[p][1 - cur].p;
    S.ghost = (u64*)w->ghost[p].p;
    S.omsg = (u64*)w->omsg[p].p;
    S.lvl = (uint32_t*)w->lvl[p].p;
  }
  A.ctr = ctr;
  A.full = full;
  A.K = w->K;
  A.L = L;
  return A;
}

u64 lanes_mask(uint32_t k) { return k >= 64 ? ~0ull : ((1ull << k) - 1); }

MsArgs make_args(graph* g, int cur, uint32_t k, uint32_t L) {
  return make_args_ws(g, g->ms, (MsCounters*)g->counters.p, cur, lanes_mask(k), L);
}

// Both directions walk the same dense plan: hub chunks, then buckets 1..3 of each part.
Plan make_plan(graph* g) {
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  const int gsh[kNBucket] = {8, 5, kSubShift, 0};
  for (int p = 0; p < 2; ++p) {
    const PartView V = g->part[p].view();
    plan_add(pl, nullptr, 0, V.nchunk, p, 8, 0);
    for (int b = 1; b < kNBucket; ++b)
      plan_add(pl, nullptr, V.bstart[b], V.bstart[b + 1] - V.bstart[b], p, gsh[b], b);
  }
  return pl;
}

constexpr unsigned kSweepGrid = 152 * 8;

uint64_t nout_ms(const graph* g) { return (uint64_t)g->part[0].nout + g->part[1].nout; }

// One superstep (compute, communication, advance) with A's counters cleared first.
graph_status launch_superstep(graph* g, const MsArgs& A, const Plan& pl, bool pull,
                              cudaStream_t st, PhaseTimer* timer, int64_t* launches) {
  const uint64_t nout = (uint64_t)g->part[0].nout + g->part[1].nout;
  const uint64_t nvt = (uint64_t)g->part[0].nv + g->part[1].nv;
  GG_CUDA(cudaMemsetAsync(A.ctr, 0, sizeof(MsCounters), st));
  if (timer) timer->mark(2);
  if (!pull) {
    if (pl.nblocks) k_ms_push<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
    GG_CUDA(cudaGetLastError());
    if (timer) timer->mark(0);
    if (nout) k_ms_exchange<<<kSweepGrid, kThreads, 0, st>>>(A);
    GG_CUDA(cudaGetLastError());
    if (timer) timer->mark(1);
  } else {
    if (nout) k_ms_publish<<<kSweepGrid, 256, 0, st>>>(A);
    GG_CUDA(cudaGetLastError());
    if (timer) timer->mark(1);
    if (pl.nblocks) k_ms_pull<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
    GG_CUDA(cudaGetLastError());
    if (timer) timer->mark(0);
  }
  k_ms_advance<<<grid_for(nvt, 256) < kSweepGrid ? grid_for(nvt, 256) : kSweepGrid, 256, 0,
                 st>>>(A);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(2);
  *launches += (pl.nblocks ? 1 : 0) + (nout ? 1 : 0) + 1;
  return GRAPH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// BFS lanes for the query server: the 64-lane search above kept resident, lanes joining at
// any superstep boundary (continuous batching) and leaving when their search ends.
// ---------------------------------------------------------------------------------------
struct BfsLanes {
  MsWs ws;
  DevBuf ctr;                 // MsCounters (device)
  MsCounters* hc = nullptr;   // pinned mirror
  DevBuf stage;               // nlanes x n uint32: results for host destinations
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  Plan plan;
  uint32_t nlanes = 0;
  int cur = 0;
  uint32_t L = 0;             // supersteps issued so far (the level clock)
  bool in_flight = false;
  bool have_counts = false;
  u64 active = 0;             // lanes holding a search
  u64 pending = 0;            // admitted, not yet seeded
  u64 stepped = 0;            // lanes that took part in the superstep in flight
  u64 mf = 0, mu = 0;         // last superstep: next frontier's edges, unreached edges
  uint32_t src[GRAPH_BATCH_MAX] = {};
  uint32_t start[GRAPH_BATCH_MAX] = {};
  uint32_t* dst[GRAPH_BATCH_MAX] = {};
  int dst_mem[GRAPH_BATCH_MAX] = {};
};

size_t bfs_lanes_bytes(const graph* g, uint32_t nlanes) {
  const size_t K = (nlanes + 3) & ~3u;
  size_t b = 1024 + 4ull * g->n * nlanes;
  for (int p = 0; p < 2; ++p) b += (24 + 4 * K) * (size_t)g->part[p].nv + 16ull * g->part[p].nout;
  return b;
}

void bfs_lanes_destroy(graph* g, BfsLanes* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  free_ms_buffers(g, &b->ws);
  dfree(g, b->ctr);
  dfree(g, b->stage);
  if (b->hc) cudaFreeHost(b->hc);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

static graph_status lanes_alloc(graph* g, BfsLanes* b) {
  GG_TRY(alloc_ms_into(g, &b->ws, (b->nlanes + 3) & ~3u));
  GG_TRY(dalloc(g, b->ctr, 1024));
  GG_TRY(dalloc(g, b->stage, 4ull * g->n * b->nlanes));
  GG_CUDA(cudaMallocHost(&b->hc, sizeof(MsCounters)));
  GG_CUDA(cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking));
  GG_CUDA(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
  for (int p = 0; p < 2; ++p) {
    GG_CUDA(cudaMemsetAsync(b->ws.seen[p].p, 0, 8ull * g->part[p].nv, b->st));
    GG_CUDA(cudaMemsetAsync(b->ws.mask[p][0].p, 0, 8ull * g->part[p].nv, b->st));
    GG_CUDA(cudaMemsetAsync(b->ws.mask[p][1].p, 0, 8ull * g->part[p].nv, b->st));
    GG_CUDA(cudaMemsetAsync(b->ws.omsg[p].p, 0, 8ull * g->part[p].nout, b->st));
  }
  GG_CUDA(cudaStreamSynchronize(b->st));
  b->plan = make_plan(g);
  return GRAPH_OK;
}

graph_status bfs_lanes_create(graph* g, uint32_t nlanes, BfsLanes** out) {
  if (nlanes < 1 || nlanes > GRAPH_BATCH_MAX) {
    set_error("lanes %u outside 1..%u", nlanes, GRAPH_BATCH_MAX);
    return GRAPH_EINVAL;
  }
  BfsLanes* b = new BfsLanes();
  b->nlanes = nlanes;
  const graph_status s = lanes_alloc(g, b);
  if (s != GRAPH_OK) {
    bfs_lanes_destroy(g, b);
    return s;
  }
  *out = b;
  return GRAPH_OK;
}

uint64_t bfs_lanes_free(const BfsLanes* b) { return lanes_mask(b->nlanes) & ~b->active; }

bool bfs_lanes_busy(const BfsLanes* b) { return b->in_flight; }

graph_status bfs_lanes_admit(BfsLanes* b, int lane, uint32_t source, uint32_t* dst,
                             int dst_mem) {
  const u64 bit = 1ull << lane;
  if (b->in_flight || lane < 0 || lane >= (int)b->nlanes || (b->active & bit)) {
    set_error("lane %d cannot be admitted now", lane);
    return GRAPH_ESTATE;
  }
  b->active |= bit;
  b->pending |= bit;
  b->src[lane] = source;
  b->dst[lane] = dst;
  b->dst_mem[lane] = dst_mem;
  return GRAPH_OK;
}

graph_status bfs_lanes_launch(graph* g, BfsLanes* b) {
  if (b->in_flight || !b->active) return GRAPH_OK;
  if (b->pending) {
    MsSeeds S;
    memset(&S, 0, sizeof(S));
    for (u64 f = b->pending; f; f &= f - 1) {
      const int l = __builtin_ctzll(f);
      S.lane[S.count] = (uint32_t)l;
      S.src[S.count] = b->src[l];
      S.count++;
      b->start[l] = b->L;
    }
    const MsArgs A0 = make_args_ws(g, &b->ws, (MsCounters*)b->ctr.p, b->cur, b->active, b->L);
    k_ms_seed<<<1, GRAPH_BATCH_MAX, 0, b->st>>>(A0, S, (const uint32_t*)g->g2l.p);
    GG_CUDA(cudaGetLastError());
    b->pending = 0;
  }
  // Beamer's rule on the last superstep's counts (pull when the frontier's edges, weighted
  // by alpha = 15, exceed the edges of vertices some search has not reached).
  const bool pull = b->have_counts && (double)b->mf * 15.0 > (double)b->mu;
  const MsArgs A = make_args_ws(g, &b->ws, (MsCounters*)b->ctr.p, b->cur, b->active, b->L);
  int64_t launches = 0;
  GG_TRY(launch_superstep(g, A, b->plan, pull, b->st, nullptr, &launches));
  GG_CUDA(cudaMemcpyAsync(b->hc, b->ctr.p, sizeof(MsCounters), cudaMemcpyDeviceToHost, b->st));
  GG_CUDA(cudaEventRecord(b->ev, b->st));
  b->stepped = b->active;
  b->in_flight = true;
  return GRAPH_OK;
}

int bfs_lanes_poll(graph* g, BfsLanes* b, uint64_t* finished, int* steps,
                   cudaEvent_t done_ev) {
  *finished = 0;
  if (!b->in_flight) return 0;
  const cudaError_t q = cudaEventQuery(b->ev);
  if (q == cudaErrorNotReady) return 0;
  if (q != cudaSuccess) return cuda_fail(q, "bfs lanes event", __FILE__, __LINE__);
  b->in_flight = false;
  b->cur = 1 - b->cur;
  b->L++;
  b->mf = b->hc->mf;
  b->mu = b->hc->mu;
  b->have_counts = true;
  const u64 fin = b->stepped & ~b->hc->gained;
  if (fin) {
    MsLaneOut O;
    memset(&O, 0, sizeof(O));
    O.F = fin;
    for (u64 f = fin; f; f &= f - 1) {
      const int l = __builtin_ctzll(f);
      O.out[l] = b->dst_mem[l] == GRAPH_MEM_DEVICE ? b->dst[l]
                                                   : (uint32_t*)b->stage.p + (size_t)l * g->n;
      O.start[l] = b->start[l];
      steps[l] = (int)(b->L - b->start[l]);
    }
    const MsArgs A = make_args_ws(g, &b->ws, (MsCounters*)b->ctr.p, b->cur, b->active, b->L);
    k_ms_lane_collect<<<grid_for(g->n, 256), 256, 0, b->st>>>(A, O, g->n,
                                                              (const uint32_t*)g->g2l.p);
    GG_CUDA(cudaGetLastError());
    for (u64 f = fin; f; f &= f - 1) {
      const int l = __builtin_ctzll(f);
      if (b->dst_mem[l] != GRAPH_MEM_DEVICE)
        GG_CUDA(cudaMemcpyAsync(b->dst[l], O.out[l], 4ull * g->n, cudaMemcpyDeviceToHost,
                                b->st));
    }
    GG_CUDA(cudaEventRecord(done_ev, b->st));
    b->active &= ~fin;
    if (!b->active) b->have_counts = false;
  }
  *finished = fin;
  return 1;
}

}  // namespace gg

using namespace gg;

namespace gg {
namespace {

// The supersteps of bfs_batch as one CUDA graph: a while loop (conditional node) whose
// body is two supersteps (buffers of the even and odd levels), each of them the kernels of
// both directions (the one the control block did not choose returns at once), the advance
// and the control step; the second control step sets the loop condition. Captured once
// per workspace, lane count, direction rule and cap; replayed by later calls.
graph_status ensure_ms_graph(graph* g, MsWs* w, uint32_t k, int direction, double alpha,
                             int64_t cap, const Plan& pl) {
  MsGraph& G = w->graph;
  if (G.exec && G.k == k && G.K == w->K && G.direction == direction && G.alpha == alpha &&
      G.cap_steps == cap && G.counters == g->counters.p)
    return GRAPH_OK;
  free_msgraph(g, w);
  GG_TRY(dalloc(g, G.ctl, sizeof(MsCtl)));
  GG_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
  cudaGraph_t gr = nullptr;
  GG_CUDA(cudaGraphCreate(&gr, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, gr, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(G.cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gr);
    return cuda_fail(e, "building the superstep graph", __FILE__, __LINE__);
  }
  const uint64_t nout = (uint64_t)g->part[0].nout + g->part[1].nout;
  const uint64_t nvt = (uint64_t)g->part[0].nv + g->part[1].nv;
  const unsigned adv = grid_for(nvt, 256) < kSweepGrid ? grid_for(nvt, 256) : kSweepGrid;
  MsCounters* ctr = (MsCounters*)g->counters.p;
  MsCtl* ctl = (MsCtl*)G.ctl.p;
  for (int cur = 0; cur < 2; ++cur) {
    MsArgs A = make_args(g, cur, k, 0);
    A.ctl = ctl;
    if (pl.nblocks) k_ms_push<<<plan_grid(pl.nblocks), kThreads, 0, G.cap>>>(pl, A);
    if (nout) k_ms_exchange<<<kSweepGrid, kThreads, 0, G.cap>>>(A);
    if (nout) k_ms_publish<<<kSweepGrid, 256, 0, G.cap>>>(A);
    if (pl.nblocks) k_ms_pull<<<plan_grid(pl.nblocks), kThreads, 0, G.cap>>>(pl, A);
    k_ms_advance<<<adv, 256, 0, G.cap>>>(A);
    k_ms_ctl_step<<<1, 32, 0, G.cap>>>(ctr, ctl, h, cur == 1);
  }
  cudaGraph_t body = nullptr;
  e = cudaStreamEndCapture(G.cap, &body);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return cuda_fail(e, "capturing the supersteps", __FILE__, __LINE__);
  }
  G.k = k;
  G.K = w->K;
  G.direction = direction;
  G.alpha = alpha;
  G.cap_steps = cap;
  G.counters = g->counters.p;
  return GRAPH_OK;
}

}  // namespace
}  // namespace gg

extern "C" graph_status bfs_batch(graph_t* g, const uint32_t* sources, uint32_t k,
                                  uint32_t* levels, const bfs_attr* attr, graph_stats* stats) {
  if (!g || !sources || !levels) {
    set_error("graph, sources or levels is NULL");
    return GRAPH_EINVAL;
  }
  if (k < 1 || k > GRAPH_BATCH_MAX) {
    set_error("k = %u outside 1..%u", k, GRAPH_BATCH_MAX);
    return GRAPH_EINVAL;
  }
  MsSources src;
  memset(&src, 0, sizeof(src));
  for (uint32_t s = 0; s < k; ++s) {
    if (sources[s] >= g->n) {
      set_error("sources[%u] = %u >= n %u", s, sources[s], g->n);
      return GRAPH_EINVAL;
    }
    src.id[s] = sources[s];
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before bfs_batch");
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
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps : (int64_t)g->n + 1;
  const uint32_t K = (k + 3) & ~3u;
  GG_TRY(ensure_ws(g, K));
  MsWs* w = g->ms;
  cudaStream_t st = g->stream;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->seen[p].p, 0, 8ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->mask[p][0].p, 0, 8ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->mask[p][1].p, 0, 8ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->omsg[p].p, 0, 8ull * P.nout, st));
  }
  GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(MsCounters), st));
  int cur = 0;
  k_ms_init<<<1, 64, 0, st>>>(make_args(g, cur, k, 0), src, k, (const uint32_t*)g->g2l.p);
  GG_CUDA(cudaGetLastError());
  MsCounters* hc = (MsCounters*)g->host_counters;
  const Plan pl = make_plan(g);
  int64_t traversed = 0, inspected = 0, messages = 0, launches = 1;
  int push_steps = 0, pull_steps = 0;
  uint64_t mu = (uint64_t)g->m;
  int64_t L = 0;
  if (!at.timing) {
    // Graph-driven: the supersteps and their termination vote run on the device.
    const graph_status gs = ensure_ms_graph(g, w, k, at.direction, alpha, cap, pl);
    if (gs != GRAPH_OK) {
      free_msgraph(g, w);
      return gs;
    }
    MsCtl hctl;
    memset(&hctl, 0, sizeof(hctl));
    hctl.m = (u64)g->m;
    hctl.alpha = alpha;
    hctl.direction = at.direction;
    hctl.cap = cap;
    MsCtl* dctl = (MsCtl*)w->graph.ctl.p;
    GG_CUDA(cudaMemcpyAsync(dctl, &hctl, sizeof(hctl), cudaMemcpyHostToDevice, st));
    k_ms_ctl_init<<<1, 32, 0, st>>>((MsCounters*)g->counters.p, dctl);
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaGraphLaunch(w->graph.exec, st));
    GG_CUDA(cudaMemcpyAsync(&hctl, dctl, sizeof(hctl), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    if (hctl.timeout) {
      set_error("bfs_batch reached the superstep cap (%lld)", (long long)cap);
      return GRAPH_ETIMEOUT;
    }
    push_steps = (int)hctl.push_steps;
    pull_steps = (int)hctl.pull_steps;
    L = push_steps + pull_steps;
    traversed = (int64_t)hctl.traversed;
    inspected = (int64_t)hctl.inspected;
    messages = (int64_t)hctl.messages;
    // kernels: the control init, then per replay of the loop body its two supersteps, each
    // with both directions' compute and communication kernels, the advance and the control
    // step (the kernels of the direction not taken return at once)
    const int64_t per = 2 * ((pl.nblocks ? 2 : 0) + (nout_ms(g) ? 2 : 0) + 2);
    launches += 1 + per * std::max<int64_t>(1, (L + 1) / 2);
    cur = (int)(L & 1);
  }
  if (at.timing) {
  GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(MsCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  traversed = (int64_t)hc->traversed;
  for (;; ++L) {
    const MsCounters c = *hc;
    if (c.nf == 0) break;
    if (L >= cap) {
      set_error("bfs_batch reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    if (L > 0) mu = c.mu;
    bool pull;
    if (at.direction == GRAPH_BFS_TOPDOWN) pull = false;
    else if (at.direction == GRAPH_BFS_BOTTOMUP) pull = L > 0;
    else pull = L > 0 && (double)c.mf * alpha > (double)mu;
    const MsArgs A = make_args(g, cur, k, (uint32_t)L);
    GG_TRY(launch_superstep(g, A, pl, pull, st, &timer, &launches));
    if (pull) pull_steps++;
    else push_steps++;
    GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(MsCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    traversed += (int64_t)hc->traversed;
    cur = 1 - cur;
  }
  }
  uint32_t* dl = levels;
  const size_t bytes = 4ull * k * g->n;
  if (at.out_mem == GRAPH_MEM_HOST) {
    GG_TRY(ensure_stage(g, bytes));
    dl = (uint32_t*)g->stage.p;
  }
  k_ms_collect<<<grid_for(g->n, 256), 256, 0, st>>>(make_args(g, cur, k, 0), g->n, k,
                                                   (const uint32_t*)g->g2l.p, dl);
  GG_CUDA(cudaGetLastError());
  launches++;
  if (at.out_mem == GRAPH_MEM_HOST) GG_TRY(deliver(g, levels, dl, bytes, GRAPH_MEM_HOST));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)L;
    stats->topdown_steps = push_steps;
    stats->bottomup_steps = pull_steps;
    stats->edges_traversed = traversed;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
  }
  timer.finish(stats);
  return s;
}
