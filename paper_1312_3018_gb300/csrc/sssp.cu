// Single-source shortest paths by Bellman-Ford over an active set (Section 7.3, Figure 20)
// on the partitioned graph.
//
// One BSP superstep per round:
//  - compute: every active vertex reads its current distance and relaxes its edges with
//    an atomic minimum on the target. A boundary target's minimum goes to its outbox
//    slot, so the messages to one remote vertex reduce at the source (Section 3.4). A
//    vertex whose distance drops joins the next round's active set (a bitmap guards
//    against duplicates; queues are bucketed by degree class for work dispatch).
//  - communication: the outbox slots lowered this round are applied to the owner with an
//    atomic minimum (the inbox scatter with min of the Appendix); an owner vertex that
//    improves becomes active.
//  - termination: the round ends the search when no vertex became active.
// Distances are uint32; a relaxation saturates at 0xFFFFFFFE and flags an overflow.
#include <string.h>

#include "common.cuh"

namespace gg {

struct SsspCounters {
  uint32_t tail[2][kNBucket];
  uint32_t dirty_tail[2];
  uint32_t overflow;
  uint32_t pad;
  unsigned long long inspected;
  unsigned long long messages;
  unsigned long long reached_degree;  // filled by the final reduction
  uint32_t clamped;                   // a final distance equals the saturation value
};

struct SsspWs {
  DevBuf dist[2], inq[2], queue[2][2], omsg[2], odirty[2], dirty[2];
  size_t words[2] = {0, 0}, owords[2] = {0, 0};
};

void free_sssp(graph* g) {
  if (!g->sssp) return;
  SsspWs* w = g->sssp;
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p], &w->inq[p], &w->queue[p][0], &w->queue[p][1],
                     &w->omsg[p], &w->odirty[p], &w->dirty[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->sssp = nullptr;
}

namespace {

struct SsspSide {
  PartView P;
  uint32_t* dist;
  uint32_t* inq;      // membership of the next active queue
  uint32_t* nqueue;   // next active queue (bucketed)
  uint32_t* omsg;     // outbox minima
  uint32_t* odirty;   // outbox slots lowered this round
  uint32_t* dirty;    // list of those slots
};

struct SsspArgs {
  SsspSide side[2];
  SsspCounters* ctr;
};

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b, bool& ovf) {
  const uint64_t s = (uint64_t)a + (uint64_t)b;
  if (s >= (uint64_t)kInf) {
    ovf = true;
    return kInf - 1;
  }
  return (uint32_t)s;
}

__device__ void flush_ssp(unsigned long long insp, unsigned long long msg, bool ovf,
                          SsspCounters* ctr) {
  __shared__ unsigned long long s[2];
  __shared__ int so;
  if (threadIdx.x == 0) {
    s[0] = s[1] = 0;
    so = 0;
  }
  __syncthreads();
  insp = warp_sum(insp);
  msg = warp_sum(msg);
  const bool any_ovf = __any_sync(kFull, ovf);
  if (lane_id() == 0) {
    if (insp) atomicAdd(&s[0], insp);
    if (msg) atomicAdd(&s[1], msg);
    if (any_ovf) so = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s[0]) atomicAdd(&ctr->inspected, s[0]);
    if (s[1]) atomicAdd(&ctr->messages, s[1]);
    if (so) atomicOr(&ctr->overflow, 1u);
  }
}

__device__ __forceinline__ void relax_edges(const SsspSide& S, int p, uint32_t dv, int64_t e,
                                            int64_t t, int stride, SsspCounters* ctr,
                                            unsigned long long& insp, bool& ovf) {
  while (__any_sync(kFull, e < t)) {
    bool act = false, msg = false;
    uint32_t u = 0, idx = 0;
    if (e < t) {
      insp++;
      const uint32_t x = S.P.E[e];
      bool o = false;
      const uint32_t nd = sat_add(dv, S.P.W[e], o);
      if (!(x & kRemote)) {
        if (nd < S.dist[x]) {
          const uint32_t old = atomicMin(&S.dist[x], nd);
          if (nd < old) {
            ovf |= o;
            if (bitmap_claim(S.inq, x)) {
              act = true;
              u = x;
            }
          }
        }
      } else {
        idx = x & kIdMask;
        if (nd < S.omsg[idx]) {
          const uint32_t old = atomicMin(&S.omsg[idx], nd);
          if (nd < old) {
            ovf |= o;
            msg = bitmap_claim(S.odirty, idx);
          }
        }
      }
    }
    warp_append_bucketed(act, u, act ? bucket_of(S.P, u) : 0, ctr->tail[p], S.nqueue, S.P);
    warp_append(msg, idx, &ctr->dirty_tail[p], S.dirty);
    e += stride;
  }
}

__global__ void __launch_bounds__(kThreads)
k_sssp_relax(const __grid_constant__ Plan plan, const __grid_constant__ SsspArgs A) {
  const Seg& G = plan.seg[find_seg(plan)];
  const int p = G.part;
  const SsspSide& S = A.side[p];
  const uint32_t rel = blockIdx.x - G.blk0;
  unsigned long long insp = 0;
  bool ovf = false;
  if (G.gshift >= 8) {
    const uint32_t v = G.items[rel];
    const uint32_t dv = __ldcg(&S.dist[v]);
    relax_edges(S, p, dv, S.P.off[v] + threadIdx.x, S.P.off[v + 1], kThreads, A.ctr, insp, ovf);
  } else {
    const int gs = G.gshift;
    const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
    int64_t s = 0, t = 0;
    uint32_t dv = 0;
    if (gi < G.count) {
      const uint32_t v = G.items[gi];
      s = S.P.off[v];
      t = S.P.off[v + 1];
      dv = __ldcg(&S.dist[v]);
    }
    const int gl = threadIdx.x & ((1 << gs) - 1);
    relax_edges(S, p, dv, s + gl, t, 1 << gs, A.ctr, insp, ovf);
  }
  flush_ssp(insp, 0, ovf, A.ctr);
}

// Communication phase: apply lowered outbox slots of p to the owner q (inbox scatter-min).
__global__ void __launch_bounds__(kThreads) k_sssp_exchange(const __grid_constant__ SsspArgs A) {
  const uint32_t warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned long long msgs = 0;
  for (int p = 0; p < 2; ++p) {
    const SsspSide& S = A.side[p];
    const SsspSide& Q = A.side[1 - p];
    const int q = 1 - p;
    const uint32_t cnt = *(volatile uint32_t*)&A.ctr->dirty_tail[p];
    for (uint32_t i0 = warp_global * 32; i0 < cnt; i0 += nwarps * 32) {
      const uint32_t i = i0 + lane_id();
      bool act = false;
      uint32_t u = 0;
      if (i < cnt) {
        const uint32_t idx = S.dirty[i];
        atomicAnd(&S.odirty[idx >> 5], ~(1u << (idx & 31u)));
        u = S.P.outbox[idx];
        const uint32_t val = S.omsg[idx];
        msgs++;
        if (val < Q.dist[u]) {
          const uint32_t old = atomicMin(&Q.dist[u], val);
          if (val < old) act = bitmap_claim(Q.inq, u);
        }
      }
      warp_append_bucketed(act, u, act ? bucket_of(Q.P, u) : 0, A.ctr->tail[q], Q.nqueue, Q.P);
    }
  }
  flush_ssp(0, msgs, false, A.ctr);
}

__global__ void k_sssp_init(const __grid_constant__ SsspArgs A, const uint32_t* g2l,
                            uint32_t source, uint32_t* queue0, uint32_t* queue1) {
  const uint32_t gl = g2l[source];
  const int p = gl >> 31;
  const uint32_t lid = gl & kIdMask;
  const SsspSide& S = A.side[p];
  S.dist[lid] = 0;
  const int b = bucket_of(S.P, lid);
  if (b < kNBucket) {
    (p == 0 ? queue0 : queue1)[S.P.bstart[b]] = lid;
    A.ctr->tail[p][b] = 1;
  }
}

__global__ void k_sssp_collect(const __grid_constant__ SsspArgs A, uint32_t nv0, uint32_t n,
                               uint32_t* dist, unsigned long long* reached_degree,
                               uint32_t* clamped) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long d = 0;
  if (i < n) {
    const int p = i < nv0 ? 0 : 1;
    const uint32_t lid = p == 0 ? i : i - nv0;
    const SsspSide& S = A.side[p];
    const uint32_t dv = S.dist[lid];
    dist[S.P.l2g[lid]] = dv;
    if (dv != kInf) d = (unsigned long long)(S.P.off[lid + 1] - S.P.off[lid]);
    if (dv == kInf - 1) atomicOr(clamped, 1u);
  }
  d = warp_sum(d);
  if (lane_id() == 0 && d) atomicAdd(reached_degree, d);
}

graph_status ensure_ws(graph* g) {
  if (g->sssp) return GRAPH_OK;
  SsspWs* w = new SsspWs();
  g->sssp = w;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    w->words[p] = (P.nv + 31) / 32;
    w->owords[p] = (P.nout + 31) / 32;
    GG_TRY(dalloc(g, w->dist[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->inq[p], 4 * w->words[p]));
    GG_TRY(dalloc(g, w->queue[p][0], 4ull * P.nv));
    GG_TRY(dalloc(g, w->queue[p][1], 4ull * P.nv));
    GG_TRY(dalloc(g, w->omsg[p], 4ull * P.nout));
    GG_TRY(dalloc(g, w->odirty[p], 4 * w->owords[p]));
    GG_TRY(dalloc(g, w->dirty[p], 4ull * P.nout));
  }
  if (g->counters.bytes < sizeof(SsspCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

SsspArgs make_args(graph* g, int cur) {
  SsspWs* w = g->sssp;
  SsspArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    SsspSide& S = A.side[p];
    S.P = g->part[p].view();
    S.dist = (uint32_t*)w->dist[p].p;
    S.inq = (uint32_t*)w->inq[p].p;
    S.nqueue = (uint32_t*)w->queue[p][1 - cur].p;
    S.omsg = (uint32_t*)w->omsg[p].p;
    S.odirty = (uint32_t*)w->odirty[p].p;
    S.dirty = (uint32_t*)w->dirty[p].p;
  }
  A.ctr = (SsspCounters*)g->counters.p;
  return A;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" graph_status sssp(graph_t* g, uint32_t source, uint32_t* dist,
                             const sssp_attr* attr, graph_stats* stats) {
  if (!g || !dist) {
    set_error("graph or dist is NULL");
    return GRAPH_EINVAL;
  }
  if (source >= g->n) {
    set_error("source %u >= n %u", source, g->n);
    return GRAPH_EINVAL;
  }
  if (!g->weighted) {
    set_error("sssp needs edge weights (load the graph with weights)");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before sssp");
    return GRAPH_ESTATE;
  }
  sssp_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) {
    set_error("bad out_mem");
    return GRAPH_EINVAL;
  }
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps : (int64_t)g->n + 1;
  GG_TRY(ensure_ws(g));
  SsspWs* w = g->sssp;
  cudaStream_t st = g->stream;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->dist[p].p, 0xFF, 4ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->omsg[p].p, 0xFF, 4ull * P.nout, st));
    GG_CUDA(cudaMemsetAsync(w->odirty[p].p, 0, 4 * w->owords[p], st));
  }
  GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(SsspCounters), st));
  int cur = 0;
  {
    SsspArgs A = make_args(g, cur);
    k_sssp_init<<<1, 1, 0, st>>>(A, (const uint32_t*)g->g2l.p, source,
                                 (uint32_t*)w->queue[0][cur].p, (uint32_t*)w->queue[1][cur].p);
    GG_CUDA(cudaGetLastError());
  }
  SsspCounters* hc = (SsspCounters*)g->host_counters;
  GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  int64_t inspected = 0, messages = 0, launches = 1;
  bool overflow = false;
  int64_t rounds = 0;
  for (;; ++rounds) {
    SsspCounters c = *hc;
    uint64_t active = 0;
    for (int p = 0; p < 2; ++p)
      for (int b = 0; b < kNBucket; ++b) active += c.tail[p][b];
    if (active == 0) break;
    if (rounds >= cap) {
      set_error("sssp reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    GG_CUDA(cudaMemsetAsync(g->counters.p, 0, sizeof(SsspCounters), st));
    for (int p = 0; p < 2; ++p) GG_CUDA(cudaMemsetAsync(w->inq[p].p, 0, 4 * w->words[p], st));
    SsspArgs A = make_args(g, cur);
    Plan pl;
    memset(&pl, 0, sizeof(pl));
    const int gsh[kNBucket] = {8, 5, kSubShift, 0};
    for (int p = 0; p < 2; ++p) {
      const PartView V = g->part[p].view();
      for (int b = 0; b < kNBucket; ++b)
        plan_add(pl, (const uint32_t*)w->queue[p][cur].p + V.bstart[b], 0, c.tail[p][b], p,
                 gsh[b], b);
    }
    timer.mark(2);
    if (pl.nblocks) k_sssp_relax<<<pl.nblocks, kThreads, 0, st>>>(pl, A);
    GG_CUDA(cudaGetLastError());
    timer.mark(0);
    k_sssp_exchange<<<152 * 4, kThreads, 0, st>>>(A);
    launches += 1 + (pl.nblocks ? 1 : 0);
    GG_CUDA(cudaGetLastError());
    timer.mark(1);
    GG_CUDA(cudaMemcpyAsync(hc, g->counters.p, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    overflow |= hc->overflow != 0;
    cur = 1 - cur;
  }
  uint32_t* dd = dist;
  if (at.out_mem == GRAPH_MEM_HOST) {
    GG_TRY(ensure_stage(g, 4ull * g->n + 64));
    dd = (uint32_t*)g->stage.p;
  }
  SsspCounters* dc = (SsspCounters*)g->counters.p;
  GG_CUDA(cudaMemsetAsync(dc, 0, sizeof(SsspCounters), st));
  {
    SsspArgs A = make_args(g, cur);
    k_sssp_collect<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->part[0].nv, g->n, dd,
                                                         &dc->reached_degree, &dc->clamped);
    launches++;
    GG_CUDA(cudaGetLastError());
  }
  if (at.out_mem == GRAPH_MEM_HOST) GG_TRY(deliver(g, dist, dd, 4ull * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  graph_status s = check_device_error(g);
  const unsigned long long reached_degree = hc->reached_degree;
  if (!hc->clamped) overflow = false;  // a clamped relaxation was later improved upon
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)rounds;
    stats->edges_traversed = (int64_t)reached_degree;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
  }
  timer.finish(stats);
  if (s == GRAPH_OK && overflow) {
    set_error("a shortest distance reached 2^32 - 1");
    return GRAPH_ERANGE;
  }
  return s;
}
