// Betweenness centrality (Section 7.2, Figure 18; Brandes' algorithm) on the partitioned
// graph, summed over a list of sources. Each source runs two BSP cycles:
//
// Forward cycle, one superstep per level L (the BFS of Figure 18's forward kernel, with
// the path counts gathered instead of scattered):
//  - compute (push): vertices at level L mark undiscovered neighbours with L + 1; a
//    boundary neighbour is marked in its outbox slot.
//  - communication: marked outbox slots give their owner level L + 1; then every outbox
//    slot publishes its owner's level and path count into the ghost arrays (pull).
//  - compute (pull): every vertex at level L + 1 sums the path counts sigma of its
//    neighbours at level L. Path counts are integers held in FP64, exact in any summation
//    order below 2^53, so no atomics race on them except the chunk sums of hub vertices.
//  - termination: no vertex was discovered.
// Backward cycle, one superstep per level L from the deepest down to 1 (Figure 18's
// backward kernel): every vertex at level L sums c(w) = (1 + delta(w)) / sigma(w) over its
// neighbours at level L + 1 (ghost copies for boundary neighbours, published first), sets
// delta(v) = sigma(v) * sum, c(v), and adds delta(v) to its score. Writing the dependency
// as sigma(v) times a sum of per-vertex quotients needs one division per vertex instead of
// one per edge (this GPU's FP64 rate is low).
//
// Level queues: a vertex enters its partition's level-ordered queue (by degree bucket; hub
// vertices as their chunks) when it is discovered, and the tails recorded after each
// forward level delimit the levels, so every compute kernel of either cycle walks exactly
// the vertices of its level instead of testing the level of every vertex.
//
// Direction of a forward level (after Beamer et al.'s rule for BFS): when the frontier's
// edges outnumber half of the edges of the vertices not yet discovered, the level is
// pulled instead: every undiscovered vertex sums the path counts of its neighbours at the
// frontier level (boundary neighbours through the ghost copies) and is discovered when the
// sum is non-zero, which forms discovery and path counts in one pass over the undiscovered
// vertices' edges instead of a push over the frontier's edges and a pull over the new
// vertices' edges.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace gg {

struct BcCounters {
  unsigned long long discovered;
  unsigned long long reached_degree;
  unsigned long long inspected;
  unsigned long long messages;
  uint32_t tail[2][kNBucket];  // level-queue tails (hub chunks, buckets 1..3), per source
};
constexpr size_t kBcLevelCounters = 4 * sizeof(unsigned long long);  // cleared per level
// A forward level is pulled when its frontier's edges times this factor exceed the edges
// of the vertices not yet discovered.
constexpr double kBcPullAlpha = 2.0;

struct BcWs {
  DevBuf dist[2], sigma[2], cq[2], score[2], hacc[2];
  DevBuf odist[2], gdist[2], gval[2];
  DevBuf lq[2], lh[2];  // level-ordered vertex queue (by bucket) and hub chunk queue
};

void free_bc(graph* g) {
  if (!g->bc) return;
  BcWs* w = g->bc;
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p],  &w->sigma[p], &w->cq[p],   &w->score[p], &w->hacc[p],
                     &w->odist[p], &w->gdist[p], &w->gval[p], &w->lq[p],    &w->lh[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->bc = nullptr;
}

namespace {

struct BcSide {
  PartView P;
  uint32_t* dist;
  double* sigma;
  double* cq;     // (1 + delta) / sigma of vertices whose dependency is final
  double* score;  // betweenness summed over the sources so far
  double* hacc;   // hub partial sums
  uint32_t* odist;  // level given to each outbox target by this partition (INF: none)
  uint32_t* gdist;  // published level of each outbox target
  double* gval;     // published sigma (forward) or c (backward) of each outbox target
  uint32_t* lq;     // [nv] level-ordered queue: bucket b at lq + bstart[b]
  uint32_t* lh;     // [nchunk] level-ordered hub chunks
  uint32_t* tail;   // [kNBucket] this partition's queue tails
};

struct BcArgs {
  BcSide side[2];
  BcCounters* ctr;
  uint32_t L;
};

struct Cnt {
  unsigned long long disc = 0, deg = 0, insp = 0, msg = 0;
};

__device__ void flush(const Cnt& c, BcCounters* ctr) {
  __shared__ unsigned long long s[4];
  if (threadIdx.x < 4) s[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long v[4] = {warp_sum(c.disc), warp_sum(c.deg), warp_sum(c.insp),
                                   warp_sum(c.msg)};
  if (lane_id() == 0)
    for (int j = 0; j < 4; ++j)
      if (v[j]) atomicAdd(&s[j], v[j]);
  __syncthreads();
  if (threadIdx.x < 4 && s[threadIdx.x])
    atomicAdd(&((unsigned long long*)ctr)[threadIdx.x], s[threadIdx.x]);
}

__device__ __forceinline__ double group_sum_d(double v, int gshift) {
  for (int o = 1; o < (1 << gshift); o <<= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Forward push from a vertex at level L over edges first, first + stride, ... < deg
// (warp-uniform trip count: every lane takes part in the queue appends). A discovered
// local neighbour gets level L + 1 and enters the level queue; a boundary neighbour is
// marked in its outbox slot.
__device__ __forceinline__ void discover_edges(const BcSide& S, uint32_t L, const uint32_t* Ep,
                                               int first, int deg, int stride, Cnt& c) {
  const uint64_t pol = l2_evict_first_policy();
  for (int i = first; __any_sync(kFull, i < deg); i += stride) {
    bool dis = false;
    uint32_t x = 0;
    if (i < deg) {
      c.insp++;
      x = ld_stream(Ep + i, pol);
      if (!(x & kRemote)) {
        if (S.dist[x] == kInf && atomicCAS(&S.dist[x], kInf, L + 1) == kInf) {
          dis = true;
          c.disc++;
          c.deg += (unsigned long long)(S.P.off[x + 1] - S.P.off[x]);
        }
      } else {
        const uint32_t idx = x & kIdMask;
        if (S.odist[idx] == kInf) atomicCAS(&S.odist[idx], kInf, L + 1);
      }
    }
    if (__any_sync(kFull, dis))
      warp_append_bucketed(dis, x, dis ? bucket_of(S.P, x) : 0, S.tail, S.lq, S.P, S.lh);
  }
}

__global__ void __launch_bounds__(kThreads)
k_bc_discover(const __grid_constant__ Plan plan, const __grid_constant__ BcArgs A) {
  Cnt c;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const BcSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      const uint32_t ch = G.items[rel];
      const uint32_t v = S.P.chunk_vertex[ch];
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      discover_edges(S, A.L, S.P.E + e0, threadIdx.x, (int)(e1 - e0), kThreads, c);
    } else {
      const int gs = G.gshift;
      const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
      int64_t s = 0, t = 0;
      if (gi < G.count) {
        const uint32_t v = G.items[gi];
        s = S.P.off[v];
        t = S.P.off[v + 1];
      }
      discover_edges(S, A.L, S.P.E + s, threadIdx.x & ((1 << gs) - 1), (int)(t - s), 1 << gs, c);
    }
  }
  flush(c, A.ctr);
}

// Outbox slots marked with level L + 1 this superstep give their owner that level.
// One partition at a time, a warp over 32 consecutive slots, so that the owner's queue
// appends are warp-wide.
__global__ void __launch_bounds__(kThreads) k_bc_exchange(const __grid_constant__ BcArgs A) {
  Cnt c;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < 2; ++p) {
    const BcSide& S = A.side[p];
    const BcSide& Q = A.side[1 - p];
    const uint64_t total = S.P.nout;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < total;
         base += stride) {
      const uint64_t i = base + lane_id();
      bool dis = false;
      uint32_t u = 0;
      if (i < total && S.odist[i] == A.L + 1) {
        c.msg++;
        u = S.P.outbox[i];
        if (Q.dist[u] == kInf && atomicCAS(&Q.dist[u], kInf, A.L + 1) == kInf) {
          dis = true;
          c.disc++;
          c.deg += (unsigned long long)(Q.P.off[u + 1] - Q.P.off[u]);
        }
      }
      if (__any_sync(kFull, dis))
        warp_append_bucketed(dis, u, dis ? bucket_of(Q.P, u) : 0, Q.tail, Q.lq, Q.P, Q.lh);
    }
  }
  flush(c, A.ctr);
}

// Pull publication: level and sigma (forward) or c (backward) of every outbox target.
__global__ void k_bc_publish(const __grid_constant__ BcArgs A, int backward) {
  const uint64_t n0 = A.side[0].P.nout, total = n0 + A.side[1].P.nout;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const int p = i < n0 ? 0 : 1;
    const uint32_t idx = (uint32_t)(p == 0 ? i : i - n0);
    const BcSide& S = A.side[p];
    const BcSide& Q = A.side[1 - p];
    const uint32_t u = S.P.outbox[idx];
    const uint32_t d = Q.dist[u];
    S.gdist[idx] = d;
    S.gval[idx] = backward ? Q.cq[u] : Q.sigma[u];
  }
}

// Sum over the neighbours at level `want` of sigma (forward) or c (backward).
__device__ __forceinline__ double pull_one(const BcSide& S, uint32_t x, uint32_t want,
                                           int backward) {
  if (x & kRemote) {
    const uint32_t idx = x & kIdMask;
    return S.gdist[idx] == want ? S.gval[idx] : 0.0;
  }
  return S.dist[x] == want ? (backward ? S.cq[x] : S.sigma[x]) : 0.0;
}

__device__ __forceinline__ void finish_vertex(const BcSide& S, uint32_t v, double sum,
                                              int backward) {
  if (!backward) {
    S.sigma[v] = sum;
  } else {
    const double sg = S.sigma[v];
    const double delta = sg * sum;
    S.cq[v] = (1.0 + delta) / sg;
    S.score[v] += delta;
  }
}

// Pull over the vertices at level `at`, taken from the level queue (forward: the new level,
// summing sigma of level at - 1; backward: level at, summing c of level at + 1). Hub
// vertices are summed chunk by chunk into hacc and finished by k_bc_hubs.
__global__ void __launch_bounds__(kThreads)
k_bc_pull(const __grid_constant__ Plan plan, const __grid_constant__ BcArgs A, uint32_t at,
          int backward) {
  Cnt c;
  const uint32_t want = backward ? at + 1 : at - 1;
  __shared__ double red[kThreads / 32];
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const BcSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      const uint32_t ch = G.items[rel];
      const uint32_t v = S.P.chunk_vertex[ch];
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      double s = 0;
      for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
        c.insp++;
        s += pull_one(S, S.P.E[e], want, backward);
      }
      s = group_sum_d(s, 5);
      if (lane_id() == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < kThreads / 32; ++i) t += red[i];
        if (t != 0.0) atomicAdd(&S.hacc[v], t);
      }
      __syncthreads();
      continue;
    }
    const int gs = G.gshift;
    const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
    const int gl = threadIdx.x & ((1 << gs) - 1);
    bool act = false;
    uint32_t v = 0;
    int64_t s0 = 0, t0 = 0;
    if (gi < G.count) {
      v = G.items[gi];
      act = true;
      s0 = S.P.off[v];
      t0 = S.P.off[v + 1];
    }
    double s = 0;
    for (int64_t e = s0 + gl; e < t0; e += (1 << gs)) {
      c.insp++;
      s += pull_one(S, S.P.E[e], want, backward);
    }
    s = group_sum_d(s, gs);
    if (act && gl == 0) finish_vertex(S, v, s, backward);
  }
  flush(c, A.ctr);
}

// Hub vertices at level `at`: finish from their chunk sums.
__global__ void k_bc_hubs(const __grid_constant__ BcArgs A, uint32_t at, int backward) {
  for (int p = 0; p < 2; ++p) {
    const BcSide& S = A.side[p];
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < S.P.bstart[1];
         v += gridDim.x * blockDim.x) {
      if (S.dist[v] != at) continue;
      finish_vertex(S, v, S.hacc[v], backward);
      S.hacc[v] = 0.0;
    }
  }
}

// Pulled forward level L: every vertex with dist INF (dense plan) sums sigma over its
// neighbours at level L; a non-zero sum discovers it at level L + 1 with that path count
// and queues it. Hub chunks add their partial sums into hacc; k_bc_hubs_discover finishes
// the hubs.
__global__ void __launch_bounds__(kThreads)
k_bc_pull_discover(const __grid_constant__ Plan plan, const __grid_constant__ BcArgs A) {
  Cnt c;
  const uint32_t L = A.L;
  __shared__ double red[kThreads / 32];
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const BcSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      const uint32_t ch = G.v0 + rel;
      const uint32_t v = S.P.chunk_vertex[ch];
      if (S.dist[v] != kInf) continue;  // CTA-uniform
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      double s = 0;
      for (int64_t e = e0 + threadIdx.x; e < e1; e += kThreads) {
        c.insp++;
        s += pull_one(S, S.P.E[e], L, 0);
      }
      s = group_sum_d(s, 5);
      if (lane_id() == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < kThreads / 32; ++i) t += red[i];
        if (t != 0.0) atomicAdd(&S.hacc[v], t);
      }
      __syncthreads();
      continue;
    }
    const int gs = G.gshift;
    const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
    const int gl = threadIdx.x & ((1 << gs) - 1);
    bool act = false;
    uint32_t v = 0;
    int64_t s0 = 0, t0 = 0;
    if (gi < G.count) {
      v = G.v0 + gi;
      if (S.dist[v] == kInf) {
        act = true;
        s0 = S.P.off[v];
        t0 = S.P.off[v + 1];
      }
    }
    double s = 0;
    for (int64_t e = s0 + gl; e < t0; e += (1 << gs)) {
      c.insp++;
      s += pull_one(S, S.P.E[e], L, 0);
    }
    s = group_sum_d(s, gs);
    const bool dis = act && gl == 0 && s != 0.0;
    if (dis) {
      S.dist[v] = L + 1;
      S.sigma[v] = s;
      c.disc++;
      c.deg += (unsigned long long)(t0 - s0);
    }
    warp_append_bucketed(dis, v, dis ? (int)G.bucket : 0, S.tail, S.lq, S.P, S.lh);
  }
  flush(c, A.ctr);
}

// Hub vertices after a pulled level: an undiscovered hub whose chunk sums are non-zero is
// discovered at level L + 1 with their sum as its path count, and its chunks are queued.
__global__ void k_bc_hubs_discover(const __grid_constant__ BcArgs A) {
  Cnt c;
  for (int p = 0; p < 2; ++p) {
    const BcSide& S = A.side[p];
    const uint32_t nh = S.P.bstart[1];
    for (uint32_t base = blockIdx.x * blockDim.x; base < nh; base += gridDim.x * blockDim.x) {
      const uint32_t v = base + threadIdx.x;
      if (v < nh && S.dist[v] == kInf) {
        const double h = S.hacc[v];
        if (h != 0.0) {
          S.hacc[v] = 0.0;
          S.dist[v] = A.L + 1;
          S.sigma[v] = h;
          c.disc++;
          c.deg += (unsigned long long)(S.P.off[v + 1] - S.P.off[v]);
          append_hub_chunks(S.P, v, &S.tail[0], S.lh);
        }
      }
    }
  }
  flush(c, A.ctr);
}

__global__ void k_bc_source(const __grid_constant__ BcArgs A, const uint32_t* g2l,
                            uint32_t source) {
  const uint32_t gl = g2l[source];
  const BcSide& S = A.side[gl >> 31];
  const uint32_t lid = gl & kIdMask;
  S.dist[lid] = 0;
  S.sigma[lid] = 1.0;
  A.ctr->discovered = 1;
  A.ctr->reached_degree = (unsigned long long)(S.P.off[lid + 1] - S.P.off[lid]);
  const int b = bucket_of(S.P, lid);
  if (b == 0) append_hub_chunks(S.P, lid, &S.tail[0], S.lh);
  else if (b < kNBucket) S.lq[S.P.bstart[b] + S.tail[b]++] = lid;
}

// Scores in global order (coalesced writes; each thread reads its vertex through g2l).
__global__ void k_bc_collect(const __grid_constant__ BcArgs A, uint32_t n, const uint32_t* g2l,
                             double* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t gl = g2l[i];
  out[i] = A.side[gl >> 31].score[gl & kIdMask];
}

graph_status alloc_ws(graph* g) {
  if (g->bc) return GRAPH_OK;
  BcWs* w = new BcWs();
  g->bc = w;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_TRY(dalloc(g, w->dist[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->sigma[p], 8ull * P.nv));
    GG_TRY(dalloc(g, w->cq[p], 8ull * P.nv));
    GG_TRY(dalloc(g, w->score[p], 8ull * P.nv));
    GG_TRY(dalloc(g, w->hacc[p], 8ull * P.nhub));
    GG_TRY(dalloc(g, w->odist[p], 4ull * P.nout));
    GG_TRY(dalloc(g, w->gdist[p], 4ull * P.nout));
    GG_TRY(dalloc(g, w->gval[p], 8ull * P.nout));
    GG_TRY(dalloc(g, w->lq[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->lh[p], 4ull * P.nchunk));
  }
  if (g->counters.bytes < sizeof(BcCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g) {
  const graph_status s = alloc_ws(g);
  if (s != GRAPH_OK) free_bc(g);
  return s;
}

BcArgs make_args(graph* g, uint32_t L) {
  BcWs* w = g->bc;
  BcArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    BcSide& S = A.side[p];
    S.P = g->part[p].view();
    S.dist = (uint32_t*)w->dist[p].p;
    S.sigma = (double*)w->sigma[p].p;
    S.cq = (double*)w->cq[p].p;
    S.score = (double*)w->score[p].p;
    S.hacc = (double*)w->hacc[p].p;
    S.odist = (uint32_t*)w->odist[p].p;
    S.gdist = (uint32_t*)w->gdist[p].p;
    S.gval = (double*)w->gval[p].p;
    S.lq = (uint32_t*)w->lq[p].p;
    S.lh = (uint32_t*)w->lh[p].p;
    S.tail = ((BcCounters*)g->counters.p)->tail[p];
  }
  A.ctr = (BcCounters*)g->counters.p;
  A.L = L;
  return A;
}

// Queue tails at a level boundary: [p][0] hub chunks, [p][1..3] vertices of bucket b.
struct LevelMark {
  uint32_t t[2][kNBucket];
};

// Every vertex with edges (hub chunks, buckets 1..3): the plan of a pulled level.
Plan dense_plan(graph* g) {
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

// The vertices of one level: the queue entries between two level boundaries.
Plan level_plan(graph* g, const LevelMark& a, const LevelMark& b) {
  BcWs* w = g->bc;
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  const int gsh[kNBucket] = {8, 5, kSubShift, 0};
  for (int p = 0; p < 2; ++p) {
    const PartView V = g->part[p].view();
    plan_add(pl, (const uint32_t*)w->lh[p].p + a.t[p][0], 0, b.t[p][0] - a.t[p][0], p, 8, 0);
    for (int k = 1; k < kNBucket; ++k)
      plan_add(pl, (const uint32_t*)w->lq[p].p + V.bstart[k] + a.t[p][k], 0,
               b.t[p][k] - a.t[p][k], p, gsh[k], k);
  }
  return pl;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" graph_status betweenness(graph_t* g, const uint32_t* sources, uint32_t k,
                                    double* scores, const bc_attr* attr, graph_stats* stats) {
  if (!g || !sources || !scores || k == 0) {
    set_error("graph, sources or scores is NULL, or k is 0");
    return GRAPH_EINVAL;
  }
  for (uint32_t i = 0; i < k; ++i)
    if (sources[i] >= g->n) {
      set_error("sources[%u] = %u >= n %u", i, sources[i], g->n);
      return GRAPH_EINVAL;
    }
  if (!g->partitioned) {
    set_error("graph_partition must run before betweenness");
    return GRAPH_ESTATE;
  }
  bc_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) {
    set_error("bad out_mem");
    return GRAPH_EINVAL;
  }
  GG_TRY(ensure_ws(g));
  BcWs* w = g->bc;
  cudaStream_t st = g->stream;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  const uint64_t nout = (uint64_t)g->part[0].nout + g->part[1].nout;
  const unsigned sweep = 152 * 8;
  const unsigned hub_grid = 152;
  BcCounters* hc = (BcCounters*)g->host_counters;
  BcCounters* dc = (BcCounters*)g->counters.p;
  for (int p = 0; p < 2; ++p) {
    GG_CUDA(cudaMemsetAsync(w->score[p].p, 0, 8ull * g->part[p].nv, st));
    GG_CUDA(cudaMemsetAsync(w->hacc[p].p, 0, 8ull * g->part[p].nhub, st));
  }
  int64_t launches = 0, traversed = 0, inspected = 0, messages = 0, steps = 0, pulled = 0;
  const Plan dense = dense_plan(g);
  // marks[L] .. marks[L + 1]: the queue entries of the vertices at level L
  std::vector<LevelMark> marks;
  auto mark_now = [&]() {
    LevelMark m;
    memcpy(m.t, hc->tail, sizeof(m.t));
    marks.push_back(m);
  };
  for (uint32_t si = 0; si < k; ++si) {
    for (int p = 0; p < 2; ++p) {
      const Part& P = g->part[p];
      GG_CUDA(cudaMemsetAsync(w->dist[p].p, 0xFF, 4ull * P.nv, st));
      GG_CUDA(cudaMemsetAsync(w->sigma[p].p, 0, 8ull * P.nv, st));
      GG_CUDA(cudaMemsetAsync(w->odist[p].p, 0xFF, 4ull * P.nout, st));
    }
    GG_CUDA(cudaMemsetAsync(dc, 0, sizeof(BcCounters), st));
    k_bc_source<<<1, 1, 0, st>>>(make_args(g, 0), (const uint32_t*)g->g2l.p, sources[si]);
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(BcCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    int64_t reached = (int64_t)hc->reached_degree;
    launches++;
    marks.clear();
    marks.push_back(LevelMark{});
    mark_now();
    GG_CUDA(cudaMemsetAsync(dc, 0, kBcLevelCounters, st));
    // Forward cycle. Pushed level: level L's queue entries discover level L + 1 (push, then
    // the outbox marks to their owners); the host reads the tails that now delimit level
    // L + 1, the ghosts are published and level L + 1 sums its path counts. Pulled level:
    // the ghosts are published, the undiscovered vertices pull, the host reads the tails.
    uint32_t L = 0;
    int64_t frontier = reached;  // degree sum of level L
    for (;; ++L) {
      if (L >= g->n) {
        set_error("betweenness reached the level cap");
        timer.finish(nullptr);
        return GRAPH_ETIMEOUT;
      }
      const BcArgs A = make_args(g, L);
      timer.mark(2);
      if ((double)frontier * kBcPullAlpha > (double)(g->m - reached)) {
        if (nout) k_bc_publish<<<sweep, 256, 0, st>>>(A, 0);
        GG_CUDA(cudaGetLastError());
        timer.mark(1);
        if (dense.nblocks) {
          k_bc_pull_discover<<<plan_grid(dense.nblocks), kThreads, 0, st>>>(dense, A);
          k_bc_hubs_discover<<<hub_grid, 256, 0, st>>>(A);
        }
        GG_CUDA(cudaGetLastError());
        timer.mark(0);
        launches += (nout ? 1 : 0) + (dense.nblocks ? 2 : 0);
        GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(BcCounters), cudaMemcpyDeviceToHost, st));
        GG_CUDA(cudaStreamSynchronize(st));
        inspected += (int64_t)hc->inspected;
        reached += (int64_t)hc->reached_degree;
        frontier = (int64_t)hc->reached_degree;
        steps++;
        pulled++;
        if (hc->discovered == 0) break;
        mark_now();
        GG_CUDA(cudaMemsetAsync(dc, 0, kBcLevelCounters, st));
        continue;
      }
      const Plan pd = level_plan(g, marks[L], marks[L + 1]);
      if (pd.nblocks) k_bc_discover<<<plan_grid(pd.nblocks), kThreads, 0, st>>>(pd, A);
      GG_CUDA(cudaGetLastError());
      timer.mark(0);
      if (nout) k_bc_exchange<<<sweep, kThreads, 0, st>>>(A);
      GG_CUDA(cudaGetLastError());
      timer.mark(1);
      launches += (pd.nblocks ? 1 : 0) + (nout ? 1 : 0);
      GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(BcCounters), cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      inspected += (int64_t)hc->inspected;
      messages += (int64_t)hc->messages;
      reached += (int64_t)hc->reached_degree;
      frontier = (int64_t)hc->reached_degree;
      steps++;
      if (hc->discovered == 0) break;
      mark_now();
      GG_CUDA(cudaMemsetAsync(dc, 0, kBcLevelCounters, st));
      if (nout) k_bc_publish<<<sweep, 256, 0, st>>>(A, 0);
      GG_CUDA(cudaGetLastError());
      timer.mark(1);
      const Plan pp = level_plan(g, marks[L + 1], marks[L + 2]);
      if (pp.nblocks) {
        k_bc_pull<<<plan_grid(pp.nblocks), kThreads, 0, st>>>(pp, A, L + 1, 0);
        k_bc_hubs<<<hub_grid, 256, 0, st>>>(A, L + 1, 0);
      }
      GG_CUDA(cudaGetLastError());
      timer.mark(0);
      launches += (nout ? 1 : 0) + (pp.nblocks ? 2 : 0);
    }
    // L is now the deepest level (the ghost levels published last are final). Backward
    // cycle: levels L .. 1 from their queue entries, with no host round trip; the deepest
    // level has no successors.
    GG_CUDA(cudaMemsetAsync(dc, 0, kBcLevelCounters, st));
    for (uint32_t lv = L; lv >= 1; --lv) {
      const BcArgs A = make_args(g, lv);
      timer.mark(2);
      if (nout && lv < L) k_bc_publish<<<sweep, 256, 0, st>>>(A, 1);
      GG_CUDA(cudaGetLastError());
      timer.mark(1);
      const Plan pb = level_plan(g, marks[lv], marks[lv + 1]);
      if (pb.nblocks) {
        k_bc_pull<<<plan_grid(pb.nblocks), kThreads, 0, st>>>(pb, A, lv, 1);
        k_bc_hubs<<<hub_grid, 256, 0, st>>>(A, lv, 1);
      }
      GG_CUDA(cudaGetLastError());
      timer.mark(0);
      launches += (pb.nblocks ? 2 : 0) + (nout && lv < L ? 1 : 0);
      steps++;
    }
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(BcCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    traversed += 2 * reached;
  }
  void* out = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, scores, at.out_mem, 8ull * g->n, 0, &out, &staged));
  k_bc_collect<<<grid_for(g->n, 256), 256, 0, st>>>(make_args(g, 0), g->n,
                                                   (const uint32_t*)g->g2l.p, (double*)out);
  GG_CUDA(cudaGetLastError());
  launches++;
  if (staged) GG_TRY(deliver(g, scores, out, 8ull * g->n, GRAPH_MEM_HOST));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)steps;
    stats->bottomup_steps = (int)pulled;
    stats->edges_traversed = traversed;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
  }
  timer.finish(stats);
  return s;
}
