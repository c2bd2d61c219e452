// Batched SSSP: up to kSbLanes single-source shortest-path searches share one sequence of
// Bellman-Ford supersteps (Section 7.3, Figure 20, run for k sources at once). Every vertex
// carries a row of kSbLanes distances (one 32-byte sector, vertex-major), so a relaxation
// pass reads an edge id and its weight once for every search in which the source vertex is
// active, and the target's row costs the same sector a single distance would.
//   dist[v][l]   distance of v in search l
//   snap[v][l]   distance v was last queued (and relaxed) with in search l (INF: never)
//   tbits        vertices lowered (in some search) this round, a bitmap
//   amask[v]     searches v was queued for in the current round
// One superstep:
//  - compute: every queued vertex relaxes its edges lane by lane (hub chunks with the
//    distances the hub was queued with, other vertices with their newest distances):
//    a lower candidate is written with an atomic minimum (a reduction no thread waits for)
//    and marks the target's lane; a boundary target reduces into its outbox row.
//  - communication: dirty outbox rows are applied to their owners the same way.
//  - filter and termination: a touched vertex is queued for the lanes whose distance is
//    below their queued value; the searches end when no vertex is queued.
//  - optional near-far order (delta > 0), one threshold tau for all lanes: a lane is queued
//    only while its distance is below tau; a vertex with improved lanes at or above tau
//    stays touched, and when nothing is queued tau moves to the smallest such distance +
//    delta (every lane starts at 0, so their frontiers stay at similar distances).
// Results equal those of k separate sssp() calls (plain rounds): shortest distances are
// unique.
#include <string.h>

#include "common.cuh"

namespace gg {

constexpr int kSbLanes = 8;  // distances per vertex row (one 32-byte sector)

struct SbCounters {
  uint32_t tail[2][kNBucket];  // next-round work: [0] hub chunks, [1..3] vertices
  uint32_t overflow;
  uint32_t far;                // (vertex, lane) pairs left waiting at or above the threshold
  uint32_t far_key;            // max of ~dist over them (zero-initialised counters work)
  uint32_t pad;
  unsigned long long inspected;
  unsigned long long messages;
  unsigned long long reached_degree[kSbLanes];  // filled by the collect
  uint32_t clamped;
};

// Device-side control of a graph-driven sssp_batch (the rounds inside one CUDA graph while
// loop, no host round trip): the near-far threshold, the termination vote, the cap, the
// statistics and the round's relax plan, which a one-thread kernel builds from the queue
// tails the filter left.
struct SbCtl {
  uint32_t done;       // nothing queued and nothing waiting (or the cap was reached)
  uint32_t timeout;    // the superstep cap was reached
  uint32_t refilter;   // this half of the loop body moves the near-far threshold first
  uint32_t round;      // this half of the loop body runs a round
  uint32_t tau, delta;
  uint32_t overflow;
  uint32_t bodies;     // loop body executions
  int64_t rounds, cap;
  unsigned long long inspected, messages;
  Plan plan;
};

// The captured round graph of a workspace and the counters it was captured with.
struct SbGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  DevBuf ctl;
  void* counters = nullptr;
};

struct SbWs {
  DevBuf dist[2], snap[2], tbits[2], amask[2], queue[2][2], hubq[2][2], omsg[2], odirty[2];
  size_t words[2] = {0, 0}, owords[2] = {0, 0};
  SbGraph graph;
};

void free_sbgraph(graph* g, SbWs* w) {
  SbGraph& G = w->graph;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.cap) cudaStreamDestroy(G.cap);
  dfree(g, G.ctl);
  G = SbGraph();
}

void free_ssspb(graph* g) {
  if (!g->sb) return;
  SbWs* w = g->sb;
  free_sbgraph(g, w);
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p],     &w->snap[p],     &w->tbits[p],    &w->amask[p],
                     &w->queue[p][0], &w->queue[p][1], &w->hubq[p][0],  &w->hubq[p][1],
                     &w->omsg[p],     &w->odirty[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->sb = nullptr;
}

namespace {

struct SbSide {
  PartView P;
  uint32_t* dist;    // [nv][kSbLanes]
  uint32_t* snap;    // [nv][kSbLanes]
  uint32_t* tbits;   // [words]
  uint32_t* amask;   // [nv]
  uint32_t* nqueue;  // next active queue (bucketed)
  uint32_t* nhubq;   // next hub chunk list
  uint32_t* omsg;    // [nout][kSbLanes] outbox minima
  uint32_t* odirty;  // [owords] outbox rows lowered this round
};

struct SbArgs {
  SbSide side[2];
  SbCounters* ctr;
  SbCtl* ctl;   // graph-driven loop, else null
  int slot;     // graph-driven loop: 1 the threshold move's filter, 2 the round's kernels
};

// Graph-driven loop: whether this kernel's slot is idle in this half of the loop body (the
// other kernels of the body then return at once); CTA-uniform.
__device__ __forceinline__ bool sb_skip(const SbArgs& A) {
  if (!A.ctl) return false;
  const volatile SbCtl* c = A.ctl;
  if (c->done) return true;
  return A.slot == 1 ? !c->refilter : !c->round;
}

__device__ __forceinline__ uint32_t sb_sat_add(uint32_t a, uint32_t b, bool& ovf) {
  const uint64_t s = (uint64_t)a + (uint64_t)b;
  if (s >= (uint64_t)kInf) {
    ovf = true;
    return kInf - 1;
  }
  return (uint32_t)s;
}
__device__ __forceinline__ void sb_red_min(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v));
}
__device__ __forceinline__ void sb_red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v));
}

// A 32-byte distance row (two 16-byte loads; rows are 32-byte aligned).
struct Row {
  uint32_t d[kSbLanes];
};
__device__ __forceinline__ Row load_row(const uint32_t* p) {
  const uint4 a = __ldcg(reinterpret_cast<const uint4*>(p));
  const uint4 b = __ldcg(reinterpret_cast<const uint4*>(p) + 1);
  Row r;
  r.d[0] = a.x; r.d[1] = a.y; r.d[2] = a.z; r.d[3] = a.w;
  r.d[4] = b.x; r.d[5] = b.y; r.d[6] = b.z; r.d[7] = b.w;
  return r;
}

__device__ void sb_flush(unsigned long long insp, unsigned long long msg, bool ovf,
                         SbCounters* ctr) {
  insp = warp_sum(insp);
  msg = warp_sum(msg);
  const bool any_ovf = __any_sync(kFull, ovf);
  if (lane_id() == 0) {
    if (insp) atomicAdd(&ctr->inspected, insp);
    if (msg) atomicAdd(&ctr->messages, msg);
    if (any_ovf) atomicOr(&ctr->overflow, 1u);
  }
}

// Lowers the target row `row` with candidates dv[l] + w for the lanes in m; returns the
// lanes lowered.
__device__ __forceinline__ uint32_t relax_row(uint32_t* row, const uint32_t* dv, uint32_t m,
                                              uint32_t w, bool& ovf) {
  const Row t = load_row(row);
  uint32_t low = 0;
  #pragma unroll
  for (int l = 0; l < kSbLanes; ++l) {
    if (!((m >> l) & 1u)) continue;
    bool o = false;
    const uint32_t nd = sb_sat_add(dv[l], w, o);
    if (nd < t.d[l]) {
      ovf |= o;
      sb_red_min(row + l, nd);
      low |= 1u << l;
    }
  }
  return low;
}

__device__ __forceinline__ void relax_edges_b(const SbSide& S, const uint32_t* dv, uint32_t m,
                                              const uint32_t* Ep, const uint32_t* Wp, int first,
                                              int deg, int stride, unsigned long long& insp,
                                              bool& ovf) {
  const uint64_t pol = l2_evict_first_policy();
  for (int i = first; i < deg; i += 2 * stride) {
    const bool two = i + stride < deg;
    insp += two ? 2 : 1;
    const uint32_t xa = ld_stream(Ep + i, pol), wa = ld_stream(Wp + i, pol);
    const uint32_t xb = two ? ld_stream(Ep + i + stride, pol) : 0u;
    const uint32_t wb = two ? ld_stream(Wp + i + stride, pol) : 0u;
    uint32_t* ra = (xa & kRemote) ? S.omsg + (size_t)(xa & kIdMask) * kSbLanes
                                  : S.dist + (size_t)xa * kSbLanes;
    uint32_t* rb = (xb & kRemote) ? S.omsg + (size_t)(xb & kIdMask) * kSbLanes
                                  : S.dist + (size_t)xb * kSbLanes;
    const Row ta = load_row(ra);
    const Row tb = two ? load_row(rb) : ta;
    uint32_t la = 0, lb = 0;
    #pragma unroll
    for (int l = 0; l < kSbLanes; ++l) {
      if (!((m >> l) & 1u)) continue;
      bool o = false;
      const uint32_t na = sb_sat_add(dv[l], wa, o);
      if (na < ta.d[l]) { ovf |= o; sb_red_min(ra + l, na); la |= 1u << l; }
      if (two) {
        bool o2 = false;
        const uint32_t nb = sb_sat_add(dv[l], wb, o2);
        if (nb < tb.d[l]) { ovf |= o2; sb_red_min(rb + l, nb); lb |= 1u << l; }
      }
    }
    if (la) {
      if (!(xa & kRemote)) sb_red_or(&S.tbits[xa >> 5], 1u << (xa & 31u));
      else sb_red_or(&S.odirty[(xa & kIdMask) >> 5], 1u << ((xa & kIdMask) & 31u));
    }
    if (lb) {
      if (!(xb & kRemote)) sb_red_or(&S.tbits[xb >> 5], 1u << (xb & 31u));
      else sb_red_or(&S.odirty[(xb & kIdMask) >> 5], 1u << ((xb & kIdMask) & 31u));
    }
  }
}

__device__ __forceinline__ void sb_relax(const Plan& plan, const SbArgs& A) {
  unsigned long long insp = 0;
  bool ovf = false;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const SbSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    uint32_t v, m;
    int64_t e0, e1;
    int first, stride;
    bool have = false, hub = false;
    if (G.gshift >= 8) {  // one hub chunk per plan block
      const uint32_t ch = G.items[rel];
      v = S.P.chunk_vertex[ch];
      e0 = S.P.chunk_first[ch];
      e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      first = threadIdx.x;
      stride = kThreads;
      have = true;
      hub = true;
    } else {
      const int gs = G.gshift;
      const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
      first = threadIdx.x & ((1 << gs) - 1);
      stride = 1 << gs;
      if (gi < G.count) {
        v = G.items[gi];
        e0 = S.P.off[v];
        e1 = S.P.off[v + 1];
        have = true;
      }
    }
    if (have) {
      m = __ldcg(&S.amask[v]);
      // A hub's chunks all relax with the distances it was queued with; a vertex handled by
      // one lane group relaxes with its newest distances (lowered since it was queued, they
      // are better candidates) and records them as its queued values, so the filter does
      // not queue it again for the same values (the paper's same-round activation).
      uint32_t* sp = S.snap + (size_t)v * kSbLanes;
      Row q = load_row(hub ? sp : S.dist + (size_t)v * kSbLanes);
      if (!hub && first == 0) {
        #pragma unroll
        for (int l = 0; l < kSbLanes; ++l)
          if ((m >> l) & 1u) sp[l] = q.d[l];
      }
      relax_edges_b(S, q.d, m, S.P.E + e0, S.P.W + e0, first, (int)(e1 - e0), stride, insp,
                    ovf);
    }
  }
  sb_flush(insp, 0, ovf, A.ctr);
}

__global__ void __launch_bounds__(kThreads)
k_sb_relax(const __grid_constant__ Plan plan, const __grid_constant__ SbArgs A) {
  sb_relax(plan, A);
}

// The graph-driven loop's relax: the plan the control kernel built, copied to shared
// memory; a fixed grid walks its blocks.
__global__ void __launch_bounds__(kThreads)
k_sb_relax_dev(const Plan* plan, const __grid_constant__ SbArgs A) {
  if (sb_skip(A)) return;
  __shared__ Plan sp;
  constexpr int kWords = (int)(sizeof(Plan) / 4);
  static_assert(sizeof(Plan) % 4 == 0, "plan copied as words");
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    reinterpret_cast<uint32_t*>(&sp)[i] = reinterpret_cast<const volatile uint32_t*>(plan)[i];
  __syncthreads();
  sb_relax(sp, A);
}

// A warp's 32 bitmap words (one per lane) are walked in bit order (every lane its own
// word's set bits, a step's rows on 32 different lines) or in word order (the warp's
// non-empty words one per step, lane b on bit b, a step's rows contiguous); word order
// where the words are dense, bit order where they are sparse, chosen per warp.
__device__ __forceinline__ bool sb_word_order(uint32_t nz, uint32_t bits) {
  return (uint32_t)__popc(nz) <= 2u * __reduce_max_sync(kFull, (uint32_t)__popc(bits));
}

// Communication phase: apply the dirty outbox rows of p to their owners in q.
__device__ __forceinline__ void sb_exchange_slot(const SbSide& S, const SbSide& Q, uint32_t idx,
                                                 unsigned long long& msgs, bool& ovf) {
  const uint32_t u = S.P.outbox[idx];
  const Row mv = load_row(S.omsg + (size_t)idx * kSbLanes);
  msgs++;
  uint32_t fin = 0;  // lanes that carry a message
  #pragma unroll
  for (int l = 0; l < kSbLanes; ++l) fin |= (mv.d[l] != kInf ? 1u : 0u) << l;
  const uint32_t low = relax_row(Q.dist + (size_t)u * kSbLanes, mv.d, fin, 0u, ovf);
  if (low) sb_red_or(&Q.tbits[u >> 5], 1u << (u & 31u));
}

__global__ void __launch_bounds__(kThreads) k_sb_exchange(const __grid_constant__ SbArgs A,
                                                          uint32_t words0) {
  if (sb_skip(A)) return;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = i < words0 ? 0 : 1;  // warps never straddle: words0 is a multiple of 32
  const uint32_t word = p == 0 ? i : i - words0;
  const SbSide& S = A.side[p];
  const SbSide& Q = A.side[1 - p];
  unsigned long long msgs = 0;
  bool ovf = false;
  uint32_t bits = 0;
  if (word * 32 < S.P.nout) {
    bits = S.odirty[word];
    if (bits) S.odirty[word] = 0;
  }
  const uint32_t nz = __ballot_sync(kFull, bits != 0);
  if (nz && sb_word_order(nz, bits)) {
    const uint32_t w0 = word - lane_id();
    for (uint32_t r = nz; r; r &= r - 1) {
      const int l = __ffs(r) - 1;
      const uint32_t wb = __shfl_sync(kFull, bits, l);
      if ((wb >> lane_id()) & 1u) sb_exchange_slot(S, Q, (w0 + l) * 32 + lane_id(), msgs, ovf);
    }
  } else {
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      sb_exchange_slot(S, Q, word * 32 + b, msgs, ovf);
    }
  }
  sb_flush(0, msgs, ovf, A.ctr);
}

// Filter: a touched vertex is queued for the lanes whose distance is below their queued
// value (which then becomes that distance) and below tau; lanes at or above tau keep the
// vertex touched and are counted with their smallest distance. One lane per bitmap word,
// the warp's words walked in bit or word order; every step appends warp-aggregated.
__device__ __forceinline__ bool sb_filter_vertex(const SbSide& S, uint32_t x, uint32_t tau,
                                                 bool& wait, uint32_t& nfar, uint32_t& key) {
  const Row d = load_row(S.dist + (size_t)x * kSbLanes);
  uint32_t* sp = S.snap + (size_t)x * kSbLanes;
  const Row q = load_row(sp);
  uint32_t am = 0;
  #pragma unroll
  for (int l = 0; l < kSbLanes; ++l) {
    if (!(d.d[l] < q.d[l])) continue;
    if (d.d[l] < tau) {
      sp[l] = d.d[l];
      am |= 1u << l;
    } else {
      wait = true;
      nfar++;
      key = max(key, ~d.d[l]);
    }
  }
  if (am) S.amask[x] = am;
  return am != 0;
}

__global__ void __launch_bounds__(kThreads) k_sb_filter(const __grid_constant__ SbArgs A,
                                                        uint32_t words0, uint32_t words,
                                                        uint32_t tau) {
  if (sb_skip(A)) return;
  if (A.ctl) tau = ((const volatile SbCtl*)A.ctl)->tau;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = i < words0 ? 0 : 1;  // warps never straddle: words0 is a multiple of 32
  const uint32_t word = p == 0 ? i : i - words0;
  const SbSide& S = A.side[p];
  uint32_t bits = 0, keep = 0, nfar = 0, key = 0;
  if (i < words) {
    bits = S.tbits[word];
    if (bits) S.tbits[word] = 0;
  }
  const uint32_t nz = __ballot_sync(kFull, bits != 0);
  if (!nz) return;
  if (sb_word_order(nz, bits)) {
    const uint32_t w0 = word - lane_id();
    for (uint32_t r = nz; r; r &= r - 1) {
      const int l = __ffs(r) - 1;
      const uint32_t wb = __shfl_sync(kFull, bits, l);
      const uint32_t x = (w0 + l) * 32 + lane_id();
      bool wait = false, act = false;
      if ((wb >> lane_id()) & 1u) act = sb_filter_vertex(S, x, tau, wait, nfar, key);
      const uint32_t km = __ballot_sync(kFull, wait);
      if ((int)lane_id() == l) keep = km;
      warp_append_bucketed(act, x, act ? bucket_of(S.P, x) : 0, A.ctr->tail[p], S.nqueue, S.P,
                           S.nhubq);
    }
  } else {
    while (__any_sync(kFull, bits != 0)) {
      bool act = false, wait = false;
      uint32_t x = 0;
      if (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        x = word * 32 + b;
        act = sb_filter_vertex(S, x, tau, wait, nfar, key);
        if (wait) keep |= 1u << b;
      }
      warp_append_bucketed(act, x, act ? bucket_of(S.P, x) : 0, A.ctr->tail[p], S.nqueue, S.P,
                           S.nhubq);
    }
  }
  if (keep) S.tbits[word] = keep;
  nfar = warp_sum(nfar);
  key = __reduce_max_sync(kFull, key);
  if (lane_id() == 0 && nfar) {
    atomicAdd(&A.ctr->far, nfar);
    atomicMax(&A.ctr->far_key, key);
  }
}

__device__ __forceinline__ uint64_t sb_active(const SbCounters& c) {
  uint64_t a = 0;
  for (int p = 0; p < 2; ++p)
    for (int b = 0; b < kNBucket; ++b) a += c.tail[p][b];
  return a;
}

// Graph-driven loop, first kernel of each half of the body: when nothing is queued but
// lanes wait at or above the near-far threshold, the threshold moves to their smallest
// distance + delta and the counters are cleared for the filter that queues what now lies
// below it.
__global__ void k_sb_ctl_pre(SbCounters* ctr, SbCtl* ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->refilter = 0;
  if (ctl->done) return;
  const SbCounters c = *ctr;
  if (sb_active(c) == 0 && c.far != 0) {
    const uint64_t t = (uint64_t)(~c.far_key) + ctl->delta;
    ctl->tau = t >= kInf ? kInf : (uint32_t)t;
    ctl->refilter = 1;
    *ctr = SbCounters();
  }
}

// The round's queues of one parity, for the plan the control kernel builds.
struct SbQueues {
  const uint32_t* hubq[2];
  const uint32_t* queue[2];
  uint32_t bstart[2][kNBucket];
};

// Graph-driven loop, before the round: the termination vote (nothing queued and nothing
// waiting: every search has converged, Section 4.1), the cap, and the relax plan from the
// queue tails (hub chunks, then the vertex buckets of each partition); the counters are
// cleared for the round. Nothing queued while lanes still wait leaves the threshold move
// to the next half of the body.
__global__ void k_sb_ctl_plan(SbCounters* ctr, SbCtl* ctl, const __grid_constant__ SbQueues q) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->round = 0;
  if (ctl->done) return;
  const SbCounters c = *ctr;
  if (sb_active(c) == 0) {
    if (c.far == 0) ctl->done = 1;
    return;
  }
  if (ctl->rounds >= ctl->cap) {
    ctl->done = 1;
    ctl->timeout = 1;
    return;
  }
  Plan pl;
  pl.nseg = 0;
  pl.nblocks = 0;
  const int gsh[kNBucket] = {8, 5, kSubShift, 0};
  for (int p = 0; p < 2; ++p) {
    plan_add(pl, q.hubq[p], 0, c.tail[p][0], p, 8, 0);
    for (int b = 1; b < kNBucket; ++b)
      plan_add(pl, q.queue[p] + q.bstart[p][b], 0, c.tail[p][b], p, gsh[b], b);
  }
  ctl->plan = pl;
  *ctr = SbCounters();
  ctl->round = 1;
}

// Graph-driven loop, after the round: statistics, and the vote for the next round taken
// at once when nothing is queued or waiting. With set_cond it sets the while loop's
// condition (0 ends the loop).
__global__ void k_sb_ctl_post(SbCounters* ctr, SbCtl* ctl, cudaGraphConditionalHandle h,
                              int set_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!ctl->done && ctl->round) {
    const SbCounters c = *ctr;
    ctl->inspected += c.inspected;
    ctl->messages += c.messages;
    ctl->overflow |= c.overflow;
    ctl->rounds++;
    ctl->round = 0;
    if (sb_active(c) == 0 && c.far == 0) ctl->done = 1;
  }
  if (set_cond) {
    ctl->bodies++;
    cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
  }
}

// Sources: distance 0 in their lane, touched for the first filter.
struct SbSources {
  uint32_t id[kSbLanes];
};
__global__ void k_sb_init(const __grid_constant__ SbArgs A, const uint32_t* g2l,
                          const __grid_constant__ SbSources src, uint32_t k) {
  const uint32_t l = threadIdx.x;
  if (l >= k) return;
  const uint32_t gl = g2l[src.id[l]];
  const int p = gl >> 31;
  const uint32_t v = gl & kIdMask;
  const SbSide& S = A.side[p];
  S.dist[(size_t)v * kSbLanes + l] = 0;
  atomicOr(&S.tbits[v >> 5], 1u << (v & 31u));
}

// Output rows of the collect: lane l's distances go to rows.p[l] (n uint32, global order).
struct OutRows {
  uint32_t* p[kSbLanes];
};

// Each lane's reached degree sum and the clamped flag, in local order (coalesced reads).
__global__ void k_sb_reached(const __grid_constant__ SbArgs A, uint32_t nv0, uint32_t n,
                             uint32_t k, SbCounters* ctr) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long d[kSbLanes] = {0};
  if (i < n) {
    const int p = i < nv0 ? 0 : 1;
    const uint32_t v = p == 0 ? i : i - nv0;
    const SbSide& S = A.side[p];
    const Row r = load_row(S.dist + (size_t)v * kSbLanes);
    const unsigned long long deg = (unsigned long long)(S.P.off[v + 1] - S.P.off[v]);
    #pragma unroll
    for (int l = 0; l < kSbLanes; ++l) {
      if ((uint32_t)l >= k) break;
      if (r.d[l] != kInf) d[l] = deg;
      if (r.d[l] == kInf - 1) atomicOr(&ctr->clamped, 1u);
    }
  }
  #pragma unroll
  for (int l = 0; l < kSbLanes; ++l) {
    if ((uint32_t)l >= k) break;
    const unsigned long long s = warp_sum(d[l]);
    if (lane_id() == 0 && s) atomicAdd(&ctr->reached_degree[l], s);
  }
}

// Lane l's distances into rows.p[l] in global order: thread i reads vertex i's row through
// g2l, so the writes of every lane's row (possibly over the host link) are coalesced.
__global__ void k_sb_collect(const __grid_constant__ SbArgs A, uint32_t n, const uint32_t* g2l,
                             uint32_t k, const __grid_constant__ OutRows rows) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t gl = g2l[i];
  const Row r = load_row(A.side[gl >> 31].dist + (size_t)(gl & kIdMask) * kSbLanes);
  #pragma unroll
  for (int l = 0; l < kSbLanes; ++l) {
    if ((uint32_t)l >= k) break;
    rows.p[l][i] = r.d[l];
  }
}

graph_status alloc_ws_into(graph* g, SbWs* w) {
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    // bitmap words rounded to whole warps (the filter assigns one lane per word)
    w->words[p] = ((P.nv + 31) / 32 + 31) & ~(size_t)31;
    w->owords[p] = ((P.nout + 31) / 32 + 31) & ~(size_t)31;
    GG_TRY(dalloc(g, w->dist[p], 4ull * kSbLanes * P.nv));
    GG_TRY(dalloc(g, w->snap[p], 4ull * kSbLanes * P.nv));
    GG_TRY(dalloc(g, w->tbits[p], 4 * w->words[p]));
    GG_TRY(dalloc(g, w->amask[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->queue[p][0], 4ull * P.nv));
    GG_TRY(dalloc(g, w->queue[p][1], 4ull * P.nv));
    GG_TRY(dalloc(g, w->hubq[p][0], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->hubq[p][1], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->omsg[p], 4ull * kSbLanes * P.nout));
    GG_TRY(dalloc(g, w->odirty[p], 4 * w->owords[p]));
  }
  return GRAPH_OK;
}

void free_ws_buffers(graph* g, SbWs* w) {
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p],     &w->snap[p],     &w->tbits[p],    &w->amask[p],
                     &w->queue[p][0], &w->queue[p][1], &w->hubq[p][0],  &w->hubq[p][1],
                     &w->omsg[p],     &w->odirty[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
}

graph_status alloc_ws(graph* g) {
  if (g->sb) return GRAPH_OK;
  SbWs* w = new SbWs();
  g->sb = w;
  GG_TRY(alloc_ws_into(g, w));
  if (g->counters.bytes < sizeof(SbCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g) {
  const graph_status s = alloc_ws(g);
  if (s != GRAPH_OK) free_ssspb(g);
  return s;
}

SbArgs make_args(graph* g, SbWs* w, SbCounters* ctr, int cur) {
  SbArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    SbSide& S = A.side[p];
    S.P = g->part[p].view();
    S.dist = (uint32_t*)w->dist[p].p;
    S.snap = (uint32_t*)w->snap[p].p;
    S.tbits = (uint32_t*)w->tbits[p].p;
    S.amask = (uint32_t*)w->amask[p].p;
    S.nqueue = (uint32_t*)w->queue[p][1 - cur].p;
    S.nhubq = (uint32_t*)w->hubq[p][1 - cur].p;
    S.omsg = (uint32_t*)w->omsg[p].p;
    S.odirty = (uint32_t*)w->odirty[p].p;
  }
  A.ctr = ctr;
  return A;
}

uint64_t active_count(const SbCounters& c) {
  uint64_t a = 0;
  for (int p = 0; p < 2; ++p)
    for (int b = 0; b < kNBucket; ++b) a += c.tail[p][b];
  return a;
}

// Resets a workspace, puts each source at distance 0 in its lane and queues the sources
// (round 0's active set) into queues 0.
graph_status launch_start(graph* g, SbWs* w, SbCounters* ctr, const uint32_t* sources,
                          uint32_t k, cudaStream_t st) {
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->dist[p].p, 0xFF, 4ull * kSbLanes * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->snap[p].p, 0xFF, 4ull * kSbLanes * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->tbits[p].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->omsg[p].p, 0xFF, 4ull * kSbLanes * P.nout, st));
    GG_CUDA(cudaMemsetAsync(w->odirty[p].p, 0, 4 * w->owords[p], st));
  }
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SbCounters), st));
  SbSources src;
  memset(&src, 0, sizeof(src));
  for (uint32_t l = 0; l < k; ++l) src.id[l] = sources[l];
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  const SbArgs A = make_args(g, w, ctr, 1);  // the filter appends into queues 0
  k_sb_init<<<1, 32, 0, st>>>(A, (const uint32_t*)g->g2l.p, src, k);
  GG_CUDA(cudaGetLastError());
  k_sb_filter<<<grid_for(words, kThreads), kThreads, 0, st>>>(A, words0, words, kInf);
  GG_CUDA(cudaGetLastError());
  return GRAPH_OK;
}

// One round: relax the active set c describes (queues `cur`), apply the outbox, filter.
graph_status launch_round(graph* g, SbWs* w, SbCounters* ctr, const SbCounters& c, int cur,
                          cudaStream_t st, PhaseTimer* timer, int64_t* launches,
                          uint32_t tau) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SbCounters), st));
  const SbArgs A = make_args(g, w, ctr, cur);
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  const int gsh[kNBucket] = {8, 5, kSubShift, 0};
  for (int p = 0; p < 2; ++p) {
    const PartView V = g->part[p].view();
    plan_add(pl, (const uint32_t*)w->hubq[p][cur].p, 0, c.tail[p][0], p, 8, 0);
    for (int b = 1; b < kNBucket; ++b)
      plan_add(pl, (const uint32_t*)w->queue[p][cur].p + V.bstart[b], 0, c.tail[p][b], p,
               gsh[b], b);
  }
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  const uint32_t owords0 = (uint32_t)w->owords[0], owords = owords0 + (uint32_t)w->owords[1];
  if (timer) timer->mark(2);
  if (pl.nblocks) k_sb_relax<<<plan_grid(pl.nblocks), kThreads, 0, st>>>(pl, A);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(0);
  if (owords) k_sb_exchange<<<grid_for(owords, kThreads), kThreads, 0, st>>>(A, owords0);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(1);
  k_sb_filter<<<grid_for(words, kThreads), kThreads, 0, st>>>(A, words0, words, tau);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(0);
  *launches += 1 + (owords ? 1 : 0) + (pl.nblocks ? 1 : 0);
  return GRAPH_OK;
}

// Near-far: nothing is queued but lanes wait at or above the threshold. The next threshold
// is their smallest distance + delta; the filter alone then queues what lies below it for
// the round that reads queues `cur`.
uint32_t next_threshold(const SbCounters& c, uint32_t delta) {
  const uint64_t t = (uint64_t)(~c.far_key) + delta;
  return t >= kInf ? kInf : (uint32_t)t;
}

graph_status launch_refilter(graph* g, SbWs* w, SbCounters* ctr, int cur, uint32_t tau,
                             cudaStream_t st, int64_t* launches) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SbCounters), st));
  const SbArgs A = make_args(g, w, ctr, 1 - cur);  // appends into queues `cur`
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  k_sb_filter<<<grid_for(words, kThreads), kThreads, 0, st>>>(A, words0, words, tau);
  GG_CUDA(cudaGetLastError());
  *launches += 1;
  return GRAPH_OK;
}

graph_status launch_collect(graph* g, SbWs* w, SbCounters* ctr, int cur, const OutRows& rows,
                            uint32_t k, cudaStream_t st) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SbCounters), st));
  const SbArgs A = make_args(g, w, ctr, cur);
  k_sb_reached<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->part[0].nv, g->n, k, ctr);
  k_sb_collect<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->n, (const uint32_t*)g->g2l.p, k, rows);
  GG_CUDA(cudaGetLastError());
  return GRAPH_OK;
}

// The rounds of sssp_batch as one CUDA graph: a while loop (conditional node) whose body is
// two halves, one per queue parity, each: threshold move (control kernel, then the filter
// appending into the queues this half reads), plan (control kernel), relax, exchange,
// filter (appending into the other parity's queues) and the post-round control kernel; the
// second half's control kernel sets the loop condition. Kernels whose slot is idle return
// at once. Captured once per workspace and counters buffer.
graph_status ensure_sb_graph(graph* g, SbWs* w) {
  SbGraph& G = w->graph;
  if (G.exec && G.counters == g->counters.p) return GRAPH_OK;
  free_sbgraph(g, w);
  GG_TRY(dalloc(g, G.ctl, sizeof(SbCtl)));
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
    return cuda_fail(e, "building the round graph", __FILE__, __LINE__);
  }
  SbCounters* ctr = (SbCounters*)g->counters.p;
  SbCtl* ctl = (SbCtl*)G.ctl.p;
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  const uint32_t owords0 = (uint32_t)w->owords[0], owords = owords0 + (uint32_t)w->owords[1];
  for (int cur = 0; cur < 2; ++cur) {
    SbArgs R = make_args(g, w, ctr, 1 - cur);  // the threshold move queues into `cur`
    R.ctl = ctl;
    R.slot = 1;
    SbArgs A = make_args(g, w, ctr, cur);
    A.ctl = ctl;
    A.slot = 2;
    SbQueues q;
    memset(&q, 0, sizeof(q));
    for (int p = 0; p < 2; ++p) {
      const PartView V = g->part[p].view();
      q.hubq[p] = (const uint32_t*)w->hubq[p][cur].p;
      q.queue[p] = (const uint32_t*)w->queue[p][cur].p;
      for (int b = 0; b < kNBucket; ++b) q.bstart[p][b] = V.bstart[b];
    }
    k_sb_ctl_pre<<<1, 32, 0, G.cap>>>(ctr, ctl);
    k_sb_filter<<<grid_for(words, kThreads), kThreads, 0, G.cap>>>(R, words0, words, kInf);
    k_sb_ctl_plan<<<1, 32, 0, G.cap>>>(ctr, ctl, q);
    k_sb_relax_dev<<<plan_grid(~0u), kThreads, 0, G.cap>>>(&ctl->plan, A);
    if (owords) k_sb_exchange<<<grid_for(owords, kThreads), kThreads, 0, G.cap>>>(A, owords0);
    k_sb_filter<<<grid_for(words, kThreads), kThreads, 0, G.cap>>>(A, words0, words, kInf);
    k_sb_ctl_post<<<1, 32, 0, G.cap>>>(ctr, ctl, h, cur == 1);
  }
  cudaGraph_t body = nullptr;
  e = cudaStreamEndCapture(G.cap, &body);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return cuda_fail(e, "capturing the rounds", __FILE__, __LINE__);
  }
  G.counters = g->counters.p;
  return GRAPH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Stepwise batched SSSP jobs for the query server: the rounds of sssp_batch issued one at
// a time on the job's own stream and advanced when the round's event has completed.
// ---------------------------------------------------------------------------------------
struct SbJob {
  SbWs ws;
  DevBuf ctr;                  // SbCounters (device)
  SbCounters* hc = nullptr;    // pinned mirror
  DevBuf stage;                // result staging for host destinations (kSbLanes rows)
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint32_t* dst[kSbLanes] = {};
  uint32_t k = 0;
  int dst_mem = 0;
  int cur = 0;
  int phase = 0;               // 0 idle, 1 round in flight, 2 collect in flight
  int64_t rounds = 0;
  bool overflow = false;
  uint32_t delta = 0;          // near-far bucket width (0: plain rounds)
  uint32_t tau = kInf;         // current near-far threshold
};

uint32_t sb_job_lanes() { return (uint32_t)kSbLanes; }

size_t sb_job_bytes(const graph* g) {
  size_t b = 1024 + 4ull * kSbLanes * g->n;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    const size_t words = ((P.nv + 31) / 32 + 31) & ~(size_t)31;
    const size_t owords = ((P.nout + 31) / 32 + 31) & ~(size_t)31;
    b += (8ull * kSbLanes + 12) * P.nv + 4 * words + 8ull * P.nchunk +
         4ull * kSbLanes * P.nout + 4 * owords;
  }
  return b;
}

void sb_job_destroy(graph* g, SbJob* j) {
  if (!j) return;
  if (j->st) cudaStreamSynchronize(j->st);
  free_ws_buffers(g, &j->ws);
  dfree(g, j->ctr);
  dfree(g, j->stage);
  if (j->hc) cudaFreeHost(j->hc);
  if (j->ev) cudaEventDestroy(j->ev);
  if (j->st) cudaStreamDestroy(j->st);
  delete j;
}

static graph_status sb_job_alloc(graph* g, SbJob* j) {
  GG_TRY(alloc_ws_into(g, &j->ws));
  GG_TRY(dalloc(g, j->ctr, 1024));
  GG_TRY(dalloc(g, j->stage, 4ull * kSbLanes * g->n));
  GG_CUDA(cudaMallocHost(&j->hc, sizeof(SbCounters)));
  GG_CUDA(cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking));
  GG_CUDA(cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming));
  return GRAPH_OK;
}

graph_status sb_job_create(graph* g, SbJob** out) {
  SbJob* j = new SbJob();
  const graph_status s = sb_job_alloc(g, j);
  if (s != GRAPH_OK) {
    sb_job_destroy(g, j);
    return s;
  }
  *out = j;
  return GRAPH_OK;
}

graph_status sb_job_start(graph* g, SbJob* j, const uint32_t* sources, uint32_t k,
                          uint32_t* const* dst, int dst_mem, uint32_t delta) {
  if (k < 1 || k > (uint32_t)kSbLanes) {
    set_error("a batched SSSP job takes 1..%d searches", kSbLanes);
    return GRAPH_EINVAL;
  }
  j->k = k;
  j->delta = delta;
  j->tau = delta ? delta : kInf;
  for (uint32_t l = 0; l < k; ++l) j->dst[l] = dst[l];
  j->dst_mem = dst_mem;
  j->cur = 0;
  j->rounds = 0;
  j->overflow = false;
  SbCounters* dc = (SbCounters*)j->ctr.p;
  GG_TRY(launch_start(g, &j->ws, dc, sources, k, j->st));
  GG_CUDA(cudaMemcpyAsync(j->hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, j->st));
  GG_CUDA(cudaEventRecord(j->ev, j->st));
  j->phase = 1;
  return GRAPH_OK;
}

static int sb_job_fail(SbJob* j, graph_status s) {
  j->phase = 0;
  return s;
}

int sb_job_poll(graph* g, SbJob* j, int* rounds) {
  if (j->phase == 0) return 0;
  const cudaError_t q = cudaEventQuery(j->ev);
  if (q == cudaErrorNotReady) return 0;
  if (q != cudaSuccess) return sb_job_fail(j, cuda_fail(q, "sssp batch job event", __FILE__, __LINE__));
  if (rounds) *rounds = (int)j->rounds;
  SbCounters* dc = (SbCounters*)j->ctr.p;
  if (j->phase == 2) {
    j->phase = 0;
    if (j->overflow && j->hc->clamped) {
      set_error("a shortest distance reached 2^32 - 1");
      return GRAPH_ERANGE;
    }
    return 1;
  }
  const SbCounters c = *j->hc;
  j->overflow |= c.overflow != 0;
  if (active_count(c) == 0 && c.far != 0) {
    // near-far: raise the threshold and queue the waiting lanes below it
    int64_t launches = 0;
    j->tau = next_threshold(c, j->delta);
    graph_status s = launch_refilter(g, &j->ws, dc, j->cur, j->tau, j->st, &launches);
    if (s != GRAPH_OK) return sb_job_fail(j, s);
    cudaError_t e = cudaMemcpyAsync(j->hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
    if (e != cudaSuccess)
      return sb_job_fail(j, cuda_fail(e, "sssp batch job refilter", __FILE__, __LINE__));
    return 0;
  }
  if (active_count(c) == 0) {
    OutRows rows;
    memset(&rows, 0, sizeof(rows));
    for (uint32_t l = 0; l < j->k; ++l)
      rows.p[l] = j->dst_mem == GRAPH_MEM_DEVICE ? j->dst[l]
                                                 : (uint32_t*)j->stage.p + (size_t)l * g->n;
    graph_status s = launch_collect(g, &j->ws, dc, j->cur, rows, j->k, j->st);
    if (s != GRAPH_OK) return sb_job_fail(j, s);
    cudaError_t e = cudaSuccess;
    if (j->dst_mem != GRAPH_MEM_DEVICE)
      for (uint32_t l = 0; l < j->k && e == cudaSuccess; ++l)
        e = cudaMemcpyAsync(j->dst[l], rows.p[l], 4ull * g->n, cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(j->hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
    if (e != cudaSuccess)
      return sb_job_fail(j, cuda_fail(e, "sssp batch job collect", __FILE__, __LINE__));
    j->phase = 2;
    return 0;
  }
  if (j->rounds >= ((int64_t)g->n + 1) * (j->delta ? j->k : 1)) {
    set_error("sssp batch job reached the superstep cap");
    return sb_job_fail(j, GRAPH_ETIMEOUT);
  }
  int64_t launches = 0;
  graph_status s = launch_round(g, &j->ws, dc, c, j->cur, j->st, nullptr, &launches, j->tau);
  if (s != GRAPH_OK) return sb_job_fail(j, s);
  cudaError_t e = cudaMemcpyAsync(j->hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, j->st);
  if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
  if (e != cudaSuccess) return sb_job_fail(j, cuda_fail(e, "sssp batch job round", __FILE__, __LINE__));
  j->cur = 1 - j->cur;
  j->rounds++;
  return 0;
}

}  // namespace gg

using namespace gg;

extern "C" graph_status sssp_batch(graph_t* g, const uint32_t* sources, uint32_t k,
                                   uint32_t* dist, const sssp_attr* attr, graph_stats* stats) {
  if (!g || !sources || !dist) {
    set_error("graph, sources or dist is NULL");
    return GRAPH_EINVAL;
  }
  if (k < 1 || k > (uint32_t)kSbLanes) {
    set_error("k = %u searches; 1 <= k <= %d", k, kSbLanes);
    return GRAPH_EINVAL;
  }
  for (uint32_t l = 0; l < k; ++l)
    if (sources[l] >= g->n) {
      set_error("source %u >= n %u", sources[l], g->n);
      return GRAPH_EINVAL;
    }
  if (!g->weighted) {
    set_error("sssp_batch needs edge weights (load the graph with weights)");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before sssp_batch");
    return GRAPH_ESTATE;
  }
  sssp_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) {
    set_error("bad out_mem");
    return GRAPH_EINVAL;
  }
  // Plain rounds end within n + 1 rounds (Bellman-Ford); with one near-far threshold a
  // round can advance some lanes while others wait, so up to k (n + 1).
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps
                                            : ((int64_t)g->n + 1) * (at.delta ? k : 1);
  GG_TRY(ensure_ws(g));
  SbWs* w = g->sb;
  cudaStream_t st = g->stream;
  SbCounters* dc = (SbCounters*)g->counters.p;
  SbCounters* hc = (SbCounters*)g->host_counters;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  GG_TRY(launch_start(g, w, dc, sources, k, st));
  int64_t inspected = 0, messages = 0, launches = 2, rounds = 0;
  bool overflow = false;
  int cur = 0;
  uint32_t tau = at.delta ? at.delta : kInf;  // the sources have distance 0 < delta
  if (!at.timing) {
    // Graph-driven: the rounds, the threshold moves and the termination vote run on the
    // device; the host waits once.
    const graph_status gs = ensure_sb_graph(g, w);
    if (gs != GRAPH_OK) {
      free_sbgraph(g, w);
      return gs;
    }
    SbCtl hctl;
    memset(&hctl, 0, sizeof(hctl));
    hctl.tau = tau;
    hctl.delta = at.delta;
    hctl.cap = cap;
    SbCtl* dctl = (SbCtl*)w->graph.ctl.p;
    GG_CUDA(cudaMemcpyAsync(dctl, &hctl, sizeof(hctl), cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaGraphLaunch(w->graph.exec, st));
    GG_CUDA(cudaMemcpyAsync(&hctl, dctl, sizeof(hctl), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    if (hctl.timeout) {
      set_error("sssp_batch reached the superstep cap (%lld)", (long long)cap);
      return GRAPH_ETIMEOUT;
    }
    rounds = hctl.rounds;
    inspected = (int64_t)hctl.inspected;
    messages = (int64_t)hctl.messages;
    overflow = hctl.overflow != 0;
    // per body execution: two halves of pre, filter, plan, relax, exchange, filter, post
    const uint64_t owords = w->owords[0] + w->owords[1];
    launches += (int64_t)hctl.bodies * 2 * (owords ? 7 : 6);
  } else {
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  for (;; ++rounds) {
    SbCounters c = *hc;
    while (active_count(c) == 0 && c.far != 0) {
      // near-far: nothing below the threshold; move it up to the waiting lanes
      tau = next_threshold(c, at.delta);
      GG_TRY(launch_refilter(g, w, dc, cur, tau, st, &launches));
      GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      c = *hc;
    }
    if (active_count(c) == 0) break;
    if (rounds >= cap) {
      set_error("sssp_batch reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    GG_TRY(launch_round(g, w, dc, c, cur, st, &timer, &launches, tau));
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    overflow |= hc->overflow != 0;
    cur = 1 - cur;
  }
  }
  void* ddv = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, dist, at.out_mem, 4ull * k * g->n + 64, 0, &ddv, &staged));
  uint32_t* dd = (uint32_t*)ddv;
  OutRows rows;
  memset(&rows, 0, sizeof(rows));
  for (uint32_t l = 0; l < k; ++l) rows.p[l] = dd + (size_t)l * g->n;
  GG_TRY(launch_collect(g, w, dc, cur, rows, k, st));
  launches += 2;
  if (staged) GG_TRY(deliver(g, dist, dd, 4ull * k * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SbCounters), cudaMemcpyDeviceToHost, st));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  graph_status s = check_device_error(g);
  if (!hc->clamped) overflow = false;  // a clamped relaxation was later improved upon
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)rounds;
    int64_t trav = 0;
    for (uint32_t l = 0; l < k; ++l) trav += (int64_t)hc->reached_degree[l];
    stats->edges_traversed = trav;
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
