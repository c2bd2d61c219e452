// Single-source shortest paths by Bellman-Ford over an active set (Section 7.3, Figure 20)
// on the partitioned graph.
//
// One BSP superstep per round:
//  - compute: every active vertex relaxes its edges with a distance dv and records dv as the
//    value it was relaxed with (a vertex handled by one lane group reads its newest
//    distance; the chunks of a hub all use the distance it was queued with, so that every
//    chunk relaxes with the same value): for a target whose distance exceeds dv + w,
//    an atomic minimum (a reduction: no thread waits for it) lowers the distance and marks
//    the target in a "touched" bitmap. A boundary target's minimum goes to its outbox slot
//    (messages to one remote vertex reduce at the source, Section 3.4) and marks the slot
//    in a dirty bitmap.
//  - communication: the dirty outbox slots are applied to their owners with the same
//    minimum-and-mark (the inbox scatter with min of the Appendix).
//  - filter and termination: a touched vertex whose distance is now below the value it was
//    last relaxed with joins the next round's active set (queues bucketed by degree class,
//    hubs as edge chunks); the search ends when that set is empty. A non-hub vertex lowered
//    while it waits in the current round is relaxed with its newest distance and not
//    re-queued, the paper's same-round activation.
//  - optional near-far order (delta > 0): only improved vertices with distance below a
//    threshold are activated; the others wait in a far bitmap. When the active set runs
//    dry the threshold moves to the smallest waiting distance + delta and the filter
//    rescans the far bitmap. Every improved vertex is still relaxed with its final
//    distance, so the distances are the same; fewer relaxations are wasted on distances
//    that later improve.
// Distances are uint32; a relaxation saturates at 0xFFFFFFFE and flags an overflow.
#include <string.h>

#include <chrono>
#include <memory>

#include "common.cuh"
#include "hybrid.cuh"
#include "jobs.cuh"

namespace gg {

struct SsspCounters {
  uint32_t tail[2][kNBucket];  // next-round work: [0] hub chunks, [1..3] vertices
  uint32_t overflow;
  uint32_t clamped;                   // a final distance equals the saturation value
  unsigned long long inspected;
  unsigned long long messages;
  unsigned long long reached_degree;  // filled by the final reduction
  // Near-far, kept across rounds and cleared at a threshold move, after which the rescan
  // of the waiting set sets them exactly: far is nonzero when a vertex joined the waiting
  // set since (so zero only when the set is empty), far_key the max of ~dist over them.
  uint32_t far;
  uint32_t far_key;
};
// Bytes a round clears: everything but the near-far fields.
constexpr size_t kRoundCounterBytes = offsetof(SsspCounters, far);

// Host side of sssp_hybrid: partition 0's CSR, weights and ids (host copies made once per
// partition), its search state and outbox minima, and pinned message arrays.
struct HsspHost {
  std::vector<int64_t> off0;
  std::vector<uint32_t> E0, W0, outbox0;
  std::unique_ptr<std::atomic<uint32_t>[]> dist, omsg;
  std::unique_ptr<std::atomic<uint8_t>[]> touched, odirty;
  std::vector<uint32_t> snap;
  uint32_t* pin_out = nullptr;  // [2 nout0]: (local id in partition 1, distance)
  uint32_t* pin_in = nullptr;   // [2 nout1 + 4]: count, then (local id in partition 0, distance)
  DevBuf dmsg;                  // device staging of either direction (same layout as pin_in)
  cudaEvent_t ev[3] = {};
};

struct SsspWs {
  DevBuf dist[2], snap[2], touched[2], farb[2], queue[2][2], hubq[2][2], omsg[2], odirty[2];
  size_t words[2] = {0, 0}, owords[2] = {0, 0};
  HsspHost* hyb = nullptr;
};

void free_hsssp(graph* g, SsspWs* w) {
  HsspHost* h = w->hyb;
  if (!h) return;
  if (h->pin_out) cudaFreeHost(h->pin_out);
  if (h->pin_in) cudaFreeHost(h->pin_in);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  dfree(g, h->dmsg);
  delete h;
  w->hyb = nullptr;
}

void free_sssp(graph* g) {
  if (!g->sssp) return;
  SsspWs* w = g->sssp;
  free_hsssp(g, w);
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p],     &w->snap[p],    &w->touched[p], &w->farb[p],
                     &w->queue[p][0], &w->queue[p][1], &w->hubq[p][0], &w->hubq[p][1],
                     &w->omsg[p],     &w->odirty[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  delete w;
  g->sssp = nullptr;
}

namespace {

struct SsspSide {
  PartView P;
  uint32_t* dist;
  uint32_t* snap;     // distance each vertex was last relaxed with (INF: never)
  uint32_t* touched;  // vertices lowered this round
  uint32_t* farb;     // near-far waiting set: improved vertices at or above the threshold
  uint32_t* nqueue;   // next active queue (bucketed)
  uint32_t* nhubq;    // next hub chunk list
  uint32_t* omsg;     // outbox minima
  uint32_t* odirty;   // outbox slots lowered this round
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

__device__ __forceinline__ void red_min(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_or(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

// Relaxes edges i = first, first + stride, ... < deg of one vertex whose adjacency starts at
// Ep / Wp. Lowering a distance is a fire-and-forget reduction plus a touched mark. CC:
// label propagation, every weight zero (Wp unused), distances are component labels.
template <bool CC>
__device__ __forceinline__ void relax_edges(const SsspSide& S, uint32_t dv, const uint32_t* Ep,
                                            const uint32_t* Wp, int first, int deg, int stride,
                                            unsigned long long& insp, bool& ovf) {
  // Four edges per step: their ids and weights, then their targets' distances, are all
  // loaded before any comparison, so each lane keeps several loads in flight.
  const uint64_t pol = l2_evict_first_policy();
  for (int i = first; i < deg; i += 4 * stride) {
    uint32_t x[4], nd[4], cur[4];
    bool o[4];
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ii = i + j * stride;
      o[j] = false;
      x[j] = ii < deg ? ld_stream(Ep + ii, pol) : kInf;
      nd[j] = CC ? dv : sat_add(dv, ii < deg ? ld_stream(Wp + ii, pol) : 0u, o[j]);
    }
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      cur[j] = 0;
      if (x[j] != kInf) {
        insp++;
        cur[j] = (x[j] & kRemote) ? S.omsg[x[j] & kIdMask] : S.dist[x[j]];
      }
    }
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (x[j] == kInf || !(nd[j] < cur[j])) continue;
      ovf |= o[j];
      if (!(x[j] & kRemote)) {
        red_min(&S.dist[x[j]], nd[j]);
        red_or(&S.touched[x[j] >> 5], 1u << (x[j] & 31u));
      } else {
        const uint32_t idx = x[j] & kIdMask;
        red_min(&S.omsg[idx], nd[j]);
        red_or(&S.odirty[idx >> 5], 1u << (idx & 31u));
      }
    }
  }
}

template <bool CC>
__global__ void __launch_bounds__(kThreads)
k_sssp_relax(const __grid_constant__ Plan plan, const __grid_constant__ SsspArgs A) {
  unsigned long long insp = 0;
  bool ovf = false;
  for (uint32_t vb = blockIdx.x; vb < plan.nblocks; vb += gridDim.x) {
    const Seg& G = plan.seg[find_seg(plan, vb)];
    const SsspSide& S = A.side[G.part];
    const uint32_t rel = vb - G.blk0;
    if (G.gshift >= 8) {
      // one hub chunk per plan block
      const uint32_t ch = G.items[rel];
      const uint32_t v = S.P.chunk_vertex[ch];
      const int64_t e0 = S.P.chunk_first[ch];
      const int64_t e1 = min(e0 + (int64_t)kHubChunk, S.P.off[v + 1]);
      const uint32_t dv = __ldcg(&S.snap[v]);  // the distance the hub was queued with
      relax_edges<CC>(S, dv, S.P.E + e0, CC ? nullptr : S.P.W + e0, threadIdx.x,
                      (int)(e1 - e0), kThreads, insp, ovf);
    } else {
      const int gs = G.gshift;
      const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
      const int gl = threadIdx.x & ((1 << gs) - 1);
      if (gi < G.count) {
        const uint32_t v = G.items[gi];
        const int64_t s = S.P.off[v], t = S.P.off[v + 1];
        const uint32_t dv = __ldcg(&S.dist[v]);
        if (gl == 0) S.snap[v] = dv;
        relax_edges<CC>(S, dv, S.P.E + s, CC ? nullptr : S.P.W + s, gl, (int)(t - s), 1 << gs,
                        insp, ovf);
      }
    }
  }
  flush_ssp(insp, 0, ovf, A.ctr);
}

// A warp's 32 bitmap words (one per lane) are walked in one of two orders. Bit order: every
// lane walks its own word's set bits, one per step, so a step's 32 loads fall on 32
// different lines; that takes as many steps as the fullest word has bits. Word order: the
// warp walks its non-empty words, one per step, lane b looking at bit b of the word, so a
// step's loads fall on one 128-byte line; that takes one step per non-empty word. Word
// order wins where the words are dense (the large middle rounds), bit order where they
// are sparse; the choice is made per warp.
__device__ __forceinline__ bool word_order(uint32_t nz, uint32_t bits) {
  return (uint32_t)__popc(nz) <= 2u * __reduce_max_sync(kFull, (uint32_t)__popc(bits));
}

// Communication phase: apply the dirty outbox slots of p to their owners in q.
__device__ __forceinline__ void exchange_slot(const SsspSide& S, const SsspSide& Q, uint32_t idx,
                                              unsigned long long& msgs) {
  const uint32_t u = S.P.outbox[idx];
  const uint32_t val = S.omsg[idx];
  msgs++;
  if (val < Q.dist[u]) {
    red_min(&Q.dist[u], val);
    red_or(&Q.touched[u >> 5], 1u << (u & 31u));
  }
}

__global__ void __launch_bounds__(kThreads) k_sssp_exchange(const __grid_constant__ SsspArgs A,
                                                            uint32_t words0) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = i < words0 ? 0 : 1;  // warps never straddle: words0 is a multiple of 32
  const uint32_t word = p == 0 ? i : i - words0;
  const SsspSide& S = A.side[p];
  const SsspSide& Q = A.side[1 - p];
  unsigned long long msgs = 0;
  uint32_t bits = 0;
  if (word * 32 < S.P.nout) {
    bits = S.odirty[word];
    if (bits) S.odirty[word] = 0;
  }
  const uint32_t nz = __ballot_sync(kFull, bits != 0);
  if (nz && word_order(nz, bits)) {
    const uint32_t w0 = word - lane_id();
    for (uint32_t r = nz; r; r &= r - 1) {
      const int l = __ffs(r) - 1;
      const uint32_t wb = __shfl_sync(kFull, bits, l);
      if ((wb >> lane_id()) & 1u) exchange_slot(S, Q, (w0 + l) * 32 + lane_id(), msgs);
    }
  } else {
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      exchange_slot(S, Q, word * 32 + b, msgs);
    }
  }
  flush_ssp(0, msgs, false, A.ctr);
}

// Filter: touched vertices whose distance dropped below the value they were last relaxed
// with form the next active set, when that distance is below tau; the others join the
// waiting set (the far bitmap) and are counted, with their smallest distance. After a
// threshold move the same kernel rescans the waiting set instead (from_far): its vertices
// below the new tau are queued, those still above stay, and those queued since they
// joined (distance equal to the value they were queued with) leave it. So a round's
// filter reads only the vertices lowered in that round. One lane per bitmap word, the
// warp's words walked in bit or word order; every step appends warp-aggregated.
__device__ __forceinline__ bool filter_vertex(const SsspSide& S, uint32_t x, uint32_t tau,
                                              bool& far, uint32_t& nfar, uint32_t& key) {
  const uint32_t d = S.dist[x];
  if (d < S.snap[x]) {
    if (d < tau) {
      S.snap[x] = d;  // queued with d
      return true;
    }
    far = true;
    nfar++;
    key = max(key, ~d);
  }
  return false;
}

__global__ void __launch_bounds__(kThreads) k_sssp_filter(const __grid_constant__ SsspArgs A,
                                                          uint32_t words0, uint32_t words,
                                                          uint32_t tau, int from_far) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = i < words0 ? 0 : 1;  // warps never straddle: words0 is a multiple of 32
  const uint32_t word = p == 0 ? i : i - words0;
  const SsspSide& S = A.side[p];
  uint32_t* src = from_far ? S.farb : S.touched;
  uint32_t bits = 0, keep = 0, nfar = 0, key = 0;
  if (i < words) {
    bits = src[word];
    if (bits) src[word] = 0;
  }
  const uint32_t nz = __ballot_sync(kFull, bits != 0);
  if (!nz) return;
  if (word_order(nz, bits)) {
    // kU non-empty words per step: their distance and snapshot loads are in flight
    // together, and one append (one atomic per bucket) serves all of them.
    constexpr int kU = 4;
    const uint32_t w0 = word - lane_id();
    for (uint32_t r = nz; r;) {
      uint32_t x[kU], d[kU], q[kU];
      int lw[kU], bk[kU];
      bool sel[kU], act[kU];
      #pragma unroll
      for (int u = 0; u < kU; ++u) {
        lw[u] = r ? __ffs(r) - 1 : -1;  // warp-uniform
        r &= r - 1;
        const int l = lw[u] < 0 ? 0 : lw[u];
        const uint32_t wb = __shfl_sync(kFull, bits, l);
        x[u] = (w0 + l) * 32 + lane_id();
        sel[u] = lw[u] >= 0 && ((wb >> lane_id()) & 1u);
        d[u] = sel[u] ? S.dist[x[u]] : 0u;
        q[u] = sel[u] ? S.snap[x[u]] : 0u;
      }
      #pragma unroll
      for (int u = 0; u < kU; ++u) {
        bool far = false;
        act[u] = false;
        if (sel[u] && d[u] < q[u]) {
          if (d[u] < tau) {
            S.snap[x[u]] = d[u];  // queued with d
            act[u] = true;
          } else {
            far = true;
            nfar++;
            key = max(key, ~d[u]);
          }
        }
        const uint32_t km = __ballot_sync(kFull, far);
        if ((int)lane_id() == lw[u]) keep = km;
        bk[u] = act[u] ? bucket_of(S.P, x[u]) : 0;
      }
      warp_append_bucketed_n<kU>(act, x, bk, A.ctr->tail[p], S.nqueue, S.P, S.nhubq);
    }
  } else {
    while (__any_sync(kFull, bits != 0)) {
      bool act = false, far = false;
      uint32_t x = 0;
      if (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        x = word * 32 + b;
        act = filter_vertex(S, x, tau, far, nfar, key);
        if (far) keep |= 1u << b;
      }
      warp_append_bucketed(act, x, act ? bucket_of(S.P, x) : 0, A.ctr->tail[p], S.nqueue, S.P,
                           S.nhubq);
    }
  }
  if (keep) S.farb[word] |= keep;  // the word's only writer in this kernel
  nfar = warp_sum(nfar);
  key = __reduce_max_sync(kFull, key);
  if (lane_id() == 0 && nfar) {
    if (!*(volatile uint32_t*)&A.ctr->far) A.ctr->far = 1u;  // every writer stores 1
    atomicMax(&A.ctr->far_key, key);
  }
}

__global__ void k_sssp_init(const __grid_constant__ SsspArgs A, const uint32_t* g2l,
                            uint32_t source, uint32_t* queue0, uint32_t* queue1,
                            uint32_t* hubq0, uint32_t* hubq1) {
  const uint32_t gl = g2l[source];
  const int p = gl >> 31;
  const uint32_t lid = gl & kIdMask;
  const SsspSide& S = A.side[p];
  S.dist[lid] = 0;
  S.snap[lid] = 0;
  const int b = bucket_of(S.P, lid);
  if (b == 0) {
    append_hub_chunks(S.P, lid, &A.ctr->tail[p][0], p == 0 ? hubq0 : hubq1);
  } else if (b < kNBucket) {
    (p == 0 ? queue0 : queue1)[S.P.bstart[b]] = lid;
    A.ctr->tail[p][b] = 1;
  }
}

// Degree sum of the reached vertices and the clamped flag, in local order (coalesced reads
// of distances and offsets).
__global__ void k_sssp_reached(const __grid_constant__ SsspArgs A, uint32_t nv0, uint32_t n,
                               unsigned long long* reached_degree, uint32_t* clamped) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long d = 0;
  if (i < n) {
    const int p = i < nv0 ? 0 : 1;
    const uint32_t lid = p == 0 ? i : i - nv0;
    const SsspSide& S = A.side[p];
    const uint32_t dv = S.dist[lid];
    if (dv != kInf) d = (unsigned long long)(S.P.off[lid + 1] - S.P.off[lid]);
    if (dv == kInf - 1) atomicOr(clamped, 1u);
  }
  d = warp_sum(d);
  if (lane_id() == 0 && d) atomicAdd(reached_degree, d);
}

// Distances in global order: thread i reads vertex i's local entry through g2l, so the
// writes (possibly over the host link) are coalesced.
__global__ void k_sssp_collect(const __grid_constant__ SsspArgs A, uint32_t n, const uint32_t* g2l,
                               uint32_t* dist) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t gl = g2l[i];
  dist[i] = A.side[gl >> 31].dist[gl & kIdMask];
}

// Connected components start: every vertex labelled with its global id, every vertex
// with edges active (queued with its label; hub vertices as all of their chunks).
__global__ void k_cc_init(const __grid_constant__ SsspArgs A, uint32_t nv0, uint32_t ntot,
                          uint32_t* queue0, uint32_t* queue1, uint32_t* hubq0,
                          uint32_t* hubq1) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const int p = i < nv0 ? 0 : 1;
  const uint32_t v = p == 0 ? i : i - nv0;
  const SsspSide& S = A.side[p];
  const uint32_t label = S.P.l2g[v];
  S.dist[v] = label;
  S.snap[v] = label;
  const int b = bucket_of(S.P, v);
  if (b == 0) {
    const int64_t deg = S.P.off[v + 1] - S.P.off[v];
    const uint32_t c0 = S.P.hub_chunk0[v];
    const uint32_t c1 = c0 + (uint32_t)((deg + kHubChunk - 1) / kHubChunk);
    for (uint32_t c = c0; c < c1; ++c) (p == 0 ? hubq0 : hubq1)[c] = c;
  } else if (b < kNBucket) {
    (p == 0 ? queue0 : queue1)[v] = v;
  }
}

__global__ void k_cc_tails(const __grid_constant__ SsspArgs A) {
  if (threadIdx.x != 0) return;
  for (int p = 0; p < 2; ++p) {
    const PartView& P = A.side[p].P;
    A.ctr->tail[p][0] = P.nchunk;
    for (int b = 1; b < kNBucket; ++b) A.ctr->tail[p][b] = P.bstart[b + 1] - P.bstart[b];
  }
}

// sssp_hybrid, device to host: partition 1's outbox slots lowered this round, as (owner's
// local id in partition 0, minimum); out[0] counts them. One lane per dirty word.
__global__ void k_hsssp_out(const __grid_constant__ SsspArgs A, uint32_t* out) {
  const SsspSide& S = A.side[1];
  const uint32_t word = blockIdx.x * blockDim.x + threadIdx.x;
  if (word * 32 >= S.P.nout) return;
  uint32_t bits = S.odirty[word];
  if (!bits) return;
  S.odirty[word] = 0;
  const uint32_t at = atomicAdd(out, (uint32_t)__popc(bits));
  uint32_t k = 0;
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    const uint32_t idx = word * 32 + b;
    out[4 + 2 * (at + k)] = S.P.outbox[idx];
    out[4 + 2 * (at + k) + 1] = S.omsg[idx];
    ++k;
  }
}

// sssp_hybrid, host to device: (local id in partition 1, distance) messages from the host's
// partition 0, applied with the minimum-and-mark of the communication phase.
__global__ void k_hsssp_in(const __grid_constant__ SsspArgs A, const uint32_t* in, uint32_t cnt) {
  const SsspSide& Q = A.side[1];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint32_t u = in[2 * i], val = in[2 * i + 1];
    if (val < Q.dist[u]) {
      red_min(&Q.dist[u], val);
      red_or(&Q.touched[u >> 5], 1u << (u & 31u));
    }
  }
}

graph_status alloc_ws_into(graph* g, SsspWs* w) {
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    // bitmap words rounded to whole warps (the filter assigns one lane per word)
    w->words[p] = ((P.nv + 31) / 32 + 31) & ~(size_t)31;
    w->owords[p] = ((P.nout + 31) / 32 + 31) & ~(size_t)31;
    GG_TRY(dalloc(g, w->dist[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->snap[p], 4ull * P.nv));
    GG_TRY(dalloc(g, w->touched[p], 4 * w->words[p]));
    GG_TRY(dalloc(g, w->farb[p], 4 * w->words[p]));
    GG_TRY(dalloc(g, w->queue[p][0], 4ull * P.nv));
    GG_TRY(dalloc(g, w->queue[p][1], 4ull * P.nv));
    GG_TRY(dalloc(g, w->hubq[p][0], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->hubq[p][1], 4ull * P.nchunk));
    GG_TRY(dalloc(g, w->omsg[p], 4ull * P.nout));
    GG_TRY(dalloc(g, w->odirty[p], 4 * w->owords[p]));
  }
  return GRAPH_OK;
}

void free_ws_buffers(graph* g, SsspWs* w) {
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->dist[p],     &w->snap[p],    &w->touched[p], &w->farb[p],
                     &w->queue[p][0], &w->queue[p][1], &w->hubq[p][0], &w->hubq[p][1],
                     &w->omsg[p],     &w->odirty[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
}

graph_status alloc_ws(graph* g) {
  if (g->sssp) return GRAPH_OK;
  SsspWs* w = new SsspWs();
  g->sssp = w;
  GG_TRY(alloc_ws_into(g, w));
  if (g->counters.bytes < sizeof(SsspCounters) || !g->counters.p) {
    dfree(g, g->counters);
    GG_TRY(dalloc(g, g->counters, 1024));
  }
  return ensure_host_counters(g, 1024);
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g) {
  const graph_status s = alloc_ws(g);
  if (s != GRAPH_OK) free_sssp(g);
  return s;
}

SsspArgs make_args(graph* g, SsspWs* w, SsspCounters* ctr, int cur) {
  SsspArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    SsspSide& S = A.side[p];
    S.P = g->part[p].view();
    S.dist = (uint32_t*)w->dist[p].p;
    S.snap = (uint32_t*)w->snap[p].p;
    S.touched = (uint32_t*)w->touched[p].p;
    S.farb = (uint32_t*)w->farb[p].p;
    S.nqueue = (uint32_t*)w->queue[p][1 - cur].p;
    S.nhubq = (uint32_t*)w->hubq[p][1 - cur].p;
    S.omsg = (uint32_t*)w->omsg[p].p;
    S.odirty = (uint32_t*)w->odirty[p].p;
  }
  A.ctr = ctr;
  return A;
}

// Resets a workspace and seeds the source (round 0's active set).
graph_status launch_start(graph* g, SsspWs* w, SsspCounters* ctr, uint32_t source,
                          cudaStream_t st) {
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->dist[p].p, 0xFF, 4ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->snap[p].p, 0xFF, 4ull * P.nv, st));
    GG_CUDA(cudaMemsetAsync(w->touched[p].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->farb[p].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->omsg[p].p, 0xFF, 4ull * P.nout, st));
    GG_CUDA(cudaMemsetAsync(w->odirty[p].p, 0, 4 * w->owords[p], st));
  }
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SsspCounters), st));
  const SsspArgs A = make_args(g, w, ctr, 0);
  k_sssp_init<<<1, 1, 0, st>>>(A, (const uint32_t*)g->g2l.p, source,
                               (uint32_t*)w->queue[0][0].p, (uint32_t*)w->queue[1][0].p,
                               (uint32_t*)w->hubq[0][0].p, (uint32_t*)w->hubq[1][0].p);
  GG_CUDA(cudaGetLastError());
  return GRAPH_OK;
}

uint64_t active_count(const SsspCounters& c) {
  uint64_t a = 0;
  for (int p = 0; p < 2; ++p)
    for (int b = 0; b < kNBucket; ++b) a += c.tail[p][b];
  return a;
}

// One round: relax the active set c describes (queues `cur`), apply the outbox, filter.
graph_status launch_round(graph* g, SsspWs* w, SsspCounters* ctr, const SsspCounters& c,
                          int cur, cudaStream_t st, PhaseTimer* timer, int64_t* launches,
                          bool cc = false, uint32_t tau = kInf) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, kRoundCounterBytes, st));
  const SsspArgs A = make_args(g, w, ctr, cur);
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
  const uint32_t owords0 = (uint32_t)w->owords[0], owords = owords0 + (uint32_t)w->owords[1];
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  if (timer) timer->mark(2);
  if (pl.nblocks) {
    // one CTA per plan block: short-lived CTAs overlap their load phases better than a
    // fixed grid walking the blocks
    if (cc) k_sssp_relax<true><<<pl.nblocks, kThreads, 0, st>>>(pl, A);
    else k_sssp_relax<false><<<pl.nblocks, kThreads, 0, st>>>(pl, A);
  }
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(0);
  if (owords) k_sssp_exchange<<<grid_for(owords, kThreads), kThreads, 0, st>>>(A, owords0);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(1);
  k_sssp_filter<<<grid_for(words, kThreads), kThreads, 0, st>>>(A, words0, words, tau, 0);
  GG_CUDA(cudaGetLastError());
  if (timer) timer->mark(0);
  *launches += 1 + (owords ? 1 : 0) + (pl.nblocks ? 1 : 0);
  return GRAPH_OK;
}

// Near-far: the active set is empty but improved vertices wait at or above the threshold.
// The next threshold is their smallest distance + delta; the filter alone then rescans
// the waiting set and queues those below it for the round that reads queues `cur`.
uint32_t next_threshold(const SsspCounters& c, uint32_t delta) {
  const uint64_t t = (uint64_t)(~c.far_key) + delta;
  return t >= kInf ? kInf : (uint32_t)t;
}

graph_status launch_refilter(graph* g, SsspWs* w, SsspCounters* ctr, int cur, uint32_t tau,
                             cudaStream_t st, int64_t* launches) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SsspCounters), st));
  const SsspArgs A = make_args(g, w, ctr, 1 - cur);  // appends into queues `cur`
  const uint32_t words0 = (uint32_t)w->words[0], words = words0 + (uint32_t)w->words[1];
  k_sssp_filter<<<grid_for(words, kThreads), kThreads, 0, st>>>(A, words0, words, tau, 1);
  GG_CUDA(cudaGetLastError());
  *launches += 1;
  return GRAPH_OK;
}

// Distances in global order into out (device) and the reached-degree / clamped reduction
// into ctr.
graph_status launch_collect(graph* g, SsspWs* w, SsspCounters* ctr, int cur, uint32_t* out,
                            cudaStream_t st) {
  GG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(SsspCounters), st));
  const SsspArgs A = make_args(g, w, ctr, cur);
  k_sssp_reached<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->part[0].nv, g->n,
                                                       &ctr->reached_degree, &ctr->clamped);
  k_sssp_collect<<<grid_for(g->n, 256), 256, 0, st>>>(A, g->n, (const uint32_t*)g->g2l.p, out);
  GG_CUDA(cudaGetLastError());
  return GRAPH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Stepwise SSSP jobs for the query server: the same rounds as sssp(), issued one at a time
// on the job's own stream and advanced when the round's event has completed.
// ---------------------------------------------------------------------------------------
struct SsspJob {
  SsspWs ws;
  DevBuf ctr;                  // SsspCounters (device)
  SsspCounters* hc = nullptr;  // pinned mirror
  DevBuf stage;                // result staging for host destinations
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  uint32_t* dst = nullptr;
  int dst_mem = 0;
  int cur = 0;
  int phase = 0;               // 0 idle, 1 round in flight, 2 collect in flight
  int64_t rounds = 0;
  bool overflow = false;
  uint32_t delta = 0;          // near-far bucket width (0: plain rounds)
  uint32_t tau = kInf;         // current near-far threshold
};

size_t sssp_job_bytes(const graph* g) {
  size_t b = 1024 + 4ull * g->n;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    const size_t words = ((P.nv + 31) / 32 + 31) & ~(size_t)31;
    const size_t owords = ((P.nout + 31) / 32 + 31) & ~(size_t)31;
    b += 16ull * P.nv + 4 * words + 8ull * P.nchunk + 4ull * P.nout + 4 * owords;
  }
  return b;
}

void sssp_job_destroy(graph* g, SsspJob* j) {
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

static graph_status job_alloc(graph* g, SsspJob* j) {
  GG_TRY(alloc_ws_into(g, &j->ws));
  GG_TRY(dalloc(g, j->ctr, 1024));
  GG_TRY(dalloc(g, j->stage, 4ull * g->n));
  GG_CUDA(cudaMallocHost(&j->hc, sizeof(SsspCounters)));
  GG_CUDA(cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking));
  GG_CUDA(cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming));
  return GRAPH_OK;
}

graph_status sssp_job_create(graph* g, SsspJob** out) {
  SsspJob* j = new SsspJob();
  const graph_status s = job_alloc(g, j);
  if (s != GRAPH_OK) {
    sssp_job_destroy(g, j);
    return s;
  }
  *out = j;
  return GRAPH_OK;
}

graph_status sssp_job_start(graph* g, SsspJob* j, uint32_t source, uint32_t* dst,
                            int dst_mem, uint32_t delta) {
  j->delta = delta;
  j->tau = delta ? delta : kInf;
  j->dst = dst;
  j->dst_mem = dst_mem;
  j->cur = 0;
  j->rounds = 0;
  j->overflow = false;
  SsspCounters* dc = (SsspCounters*)j->ctr.p;
  GG_TRY(launch_start(g, &j->ws, dc, source, j->st));
  GG_CUDA(cudaMemcpyAsync(j->hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, j->st));
  GG_CUDA(cudaEventRecord(j->ev, j->st));
  j->phase = 1;
  return GRAPH_OK;
}

static int job_fail(SsspJob* j, graph_status s) {
  j->phase = 0;
  return s;
}

int sssp_job_poll(graph* g, SsspJob* j, int* rounds) {
  if (j->phase == 0) return 0;
  const cudaError_t q = cudaEventQuery(j->ev);
  if (q == cudaErrorNotReady) return 0;
  if (q != cudaSuccess) return job_fail(j, cuda_fail(q, "sssp job event", __FILE__, __LINE__));
  if (rounds) *rounds = (int)j->rounds;
  SsspCounters* dc = (SsspCounters*)j->ctr.p;
  if (j->phase == 2) {
    j->phase = 0;
    if (j->overflow && j->hc->clamped) {
      set_error("a shortest distance reached 2^32 - 1");
      return GRAPH_ERANGE;
    }
    return 1;
  }
  const SsspCounters c = *j->hc;
  j->overflow |= c.overflow != 0;
  if (active_count(c) == 0 && c.far != 0) {
    // near-far: raise the threshold and queue the waiting vertices below it
    int64_t launches = 0;
    j->tau = next_threshold(c, j->delta);
    graph_status s = launch_refilter(g, &j->ws, dc, j->cur, j->tau, j->st, &launches);
    if (s != GRAPH_OK) return job_fail(j, s);
    cudaError_t e = cudaMemcpyAsync(j->hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
    if (e != cudaSuccess) return job_fail(j, cuda_fail(e, "sssp job refilter", __FILE__, __LINE__));
    return 0;
  }
  if (active_count(c) == 0) {
    uint32_t* out = j->dst_mem == GRAPH_MEM_DEVICE ? j->dst : (uint32_t*)j->stage.p;
    graph_status s = launch_collect(g, &j->ws, dc, j->cur, out, j->st);
    if (s != GRAPH_OK) return job_fail(j, s);
    cudaError_t e = cudaSuccess;
    if (j->dst_mem != GRAPH_MEM_DEVICE)
      e = cudaMemcpyAsync(j->dst, out, 4ull * g->n, cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(j->hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, j->st);
    if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
    if (e != cudaSuccess) return job_fail(j, cuda_fail(e, "sssp job collect", __FILE__, __LINE__));
    j->phase = 2;
    return 0;
  }
  if (j->rounds >= (int64_t)g->n + 1) {
    set_error("sssp job reached the superstep cap");
    return job_fail(j, GRAPH_ETIMEOUT);
  }
  int64_t launches = 0;
  graph_status s = launch_round(g, &j->ws, dc, c, j->cur, j->st, nullptr, &launches, false,
                                j->tau);
  if (s != GRAPH_OK) return job_fail(j, s);
  cudaError_t e = cudaMemcpyAsync(j->hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, j->st);
  if (e == cudaSuccess) e = cudaEventRecord(j->ev, j->st);
  if (e != cudaSuccess) return job_fail(j, cuda_fail(e, "sssp job round", __FILE__, __LINE__));
  j->cur = 1 - j->cur;
  j->rounds++;
  return 0;
}

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
  SsspCounters* dc = (SsspCounters*)g->counters.p;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  GG_TRY(launch_start(g, w, dc, source, st));
  SsspCounters* hc = (SsspCounters*)g->host_counters;
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  int64_t inspected = 0, messages = 0, launches = 1;
  bool overflow = false;
  int64_t rounds = 0;
  int cur = 0;
  uint32_t tau = at.delta ? at.delta : kInf;  // the source has distance 0 < delta
  for (;; ++rounds) {
    SsspCounters c = *hc;
    while (active_count(c) == 0 && c.far != 0) {
      // near-far: nothing below the threshold; move it up to the waiting vertices
      tau = next_threshold(c, at.delta);
      GG_TRY(launch_refilter(g, w, dc, cur, tau, st, &launches));
      GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      c = *hc;
    }
    if (active_count(c) == 0) break;
    if (rounds >= cap) {
      set_error("sssp reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    GG_TRY(launch_round(g, w, dc, c, cur, st, &timer, &launches, false, tau));
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    overflow |= hc->overflow != 0;
    cur = 1 - cur;
  }
  void* dd = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, dist, at.out_mem, 4ull * g->n + 64, 0, &dd, &staged));
  GG_TRY(launch_collect(g, w, dc, cur, (uint32_t*)dd, st));
  launches += 2;
  if (staged) GG_TRY(deliver(g, dist, dd, 4ull * g->n, GRAPH_MEM_HOST));
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

extern "C" graph_status connected_components(graph_t* g, uint32_t* labels,
                                             const cc_attr* attr, graph_stats* stats) {
  if (!g || !labels) {
    set_error("graph or labels is NULL");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before connected_components");
    return GRAPH_ESTATE;
  }
  cc_attr at;
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
  SsspCounters* dc = (SsspCounters*)g->counters.p;
  SsspCounters* hc = (SsspCounters*)g->host_counters;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_CUDA(cudaMemsetAsync(w->touched[p].p, 0, 4 * w->words[p], st));
    GG_CUDA(cudaMemsetAsync(w->omsg[p].p, 0xFF, 4ull * P.nout, st));
    GG_CUDA(cudaMemsetAsync(w->odirty[p].p, 0, 4 * w->owords[p], st));
  }
  GG_CUDA(cudaMemsetAsync(dc, 0, sizeof(SsspCounters), st));
  {
    const SsspArgs A = make_args(g, w, dc, 0);
    k_cc_init<<<grid_for(g->n, 256), 256, 0, st>>>(
        A, g->part[0].nv, g->n, (uint32_t*)w->queue[0][0].p, (uint32_t*)w->queue[1][0].p,
        (uint32_t*)w->hubq[0][0].p, (uint32_t*)w->hubq[1][0].p);
    k_cc_tails<<<1, 32, 0, st>>>(A);
    GG_CUDA(cudaGetLastError());
  }
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  timer.mark(2);
  int64_t inspected = 0, messages = 0, launches = 2, rounds = 0;
  int cur = 0;
  for (;; ++rounds) {
    const SsspCounters c = *hc;
    if (active_count(c) == 0) break;
    if (rounds >= cap) {
      set_error("connected_components reached the superstep cap (%lld)", (long long)cap);
      timer.finish(nullptr);
      return GRAPH_ETIMEOUT;
    }
    GG_TRY(launch_round(g, w, dc, c, cur, st, &timer, &launches, true));
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    messages += (int64_t)hc->messages;
    cur = 1 - cur;
  }
  void* out = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, labels, at.out_mem, 4ull * g->n + 64, 0, &out, &staged));
  GG_TRY(launch_collect(g, w, dc, cur, (uint32_t*)out, st));
  launches += 2;
  if (staged) GG_TRY(deliver(g, labels, out, 4ull * g->n, GRAPH_MEM_HOST));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)rounds;
    stats->edges_traversed = g->m;
    stats->edges_inspected = inspected;
    stats->messages = messages;
    stats->launches = launches;
  }
  timer.finish(stats);
  return s;
}

// ---------------------------------------------------------------------------------------
// sssp_hybrid: partition 0 on host threads, partition 1 on the GPU (Section 4.1, Figure 6;
// Section 7.3). Both sides run the same Bellman-Ford round (Figure 20) on their own active
// vertices; only outbox minima cross, as (target, distance) lists of the slots lowered in
// the round. Plain rounds (no near-far order).
// ---------------------------------------------------------------------------------------
namespace gg {
namespace {

graph_status ensure_hsssp(graph* g, SsspWs* w) {
  if (w->hyb) return GRAPH_OK;
  const Part& P0 = g->part[0];
  const Part& P1 = g->part[1];
  cudaStream_t st = g->stream;
  HsspHost* h = new HsspHost();
  w->hyb = h;
  h->off0.resize((size_t)P0.nv + 1);
  h->E0.resize((size_t)P0.ne);
  h->W0.resize((size_t)P0.ne);
  h->outbox0.resize(P0.nout);
  h->snap.resize(P0.nv);
  h->dist.reset(new std::atomic<uint32_t>[P0.nv + 1]);
  h->touched.reset(new std::atomic<uint8_t>[P0.nv + 1]);
  h->omsg.reset(new std::atomic<uint32_t>[P0.nout + 1]);
  h->odirty.reset(new std::atomic<uint8_t>[P0.nout + 1]);
  GG_CUDA(cudaMemcpyAsync(h->off0.data(), P0.off.p, 8ull * (P0.nv + 1), cudaMemcpyDeviceToHost, st));
  if (P0.ne) {
    GG_CUDA(cudaMemcpyAsync(h->E0.data(), P0.E.p, 4ull * P0.ne, cudaMemcpyDefault, st));
    GG_CUDA(cudaMemcpyAsync(h->W0.data(), P0.W.p, 4ull * P0.ne, cudaMemcpyDefault, st));
  }
  if (P0.nout)
    GG_CUDA(cudaMemcpyAsync(h->outbox0.data(), P0.outbox.p, 4ull * P0.nout, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  for (cudaEvent_t& e : h->ev) GG_CUDA(cudaEventCreate(&e));
  const size_t b0 = 8ull * std::max<uint32_t>(P0.nout, 1);
  const size_t b1 = 8ull * std::max<uint32_t>(P1.nout, 1) + 16;
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

extern "C" graph_status sssp_hybrid(graph_t* g, uint32_t source, uint32_t* dist,
                                    const sssp_attr* attr, int cpu_threads, graph_stats* stats,
                                    pagerank_hybrid_info* info) {
  using Clock = std::chrono::steady_clock;
  if (!g || !dist) {
    set_error("graph or dist is NULL");
    return GRAPH_EINVAL;
  }
  if (source >= g->n) {
    set_error("source %u >= n %u", source, g->n);
    return GRAPH_EINVAL;
  }
  if (!g->weighted) {
    set_error("sssp_hybrid needs edge weights (load the graph with weights)");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before sssp_hybrid");
    return GRAPH_ESTATE;
  }
  sssp_attr at;
  memset(&at, 0, sizeof(at));
  if (attr) at = *attr;
  if ((at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) || at.delta != 0 ||
      cpu_threads > GRAPH_HYBRID_MAX_THREADS) {
    set_error("bad sssp_hybrid attributes (plain rounds only: delta = 0; out_mem; cpu_threads)");
    return GRAPH_EINVAL;
  }
  const int nt = hybrid_threads(cpu_threads);
  const int64_t cap = at.max_supersteps > 0 ? at.max_supersteps : (int64_t)g->n + 1;
  GG_TRY(ensure_ws(g));
  SsspWs* w = g->sssp;
  {
    graph_status s = GRAPH_OK;
    try {
      s = ensure_hsssp(g, w);
    } catch (const std::bad_alloc&) {
      set_error("host allocation for the host partition failed");
      s = GRAPH_ENOMEM;
    }
    if (s != GRAPH_OK) {
      free_hsssp(g, w);
      return s;
    }
  }
  HsspHost* h = w->hyb;
  cudaStream_t st = g->stream;
  const Part& P0 = g->part[0];
  const uint32_t nv0 = P0.nv, nout0 = P0.nout;
  const auto t_start = Clock::now();
  SsspCounters* dc = (SsspCounters*)g->counters.p;
  SsspCounters* hc = (SsspCounters*)g->host_counters;
  GG_TRY(launch_start(g, w, dc, source, st));   // resets both sides; seeds a partition-1 source
  for (uint32_t v = 0; v < nv0; ++v) {
    h->dist[v].store(kInf, std::memory_order_relaxed);
    h->touched[v].store(0, std::memory_order_relaxed);
    h->snap[v] = kInf;
  }
  for (uint32_t i = 0; i < nout0; ++i) {
    h->omsg[i].store(kInf, std::memory_order_relaxed);
    h->odirty[i].store(0, std::memory_order_relaxed);
  }
  uint32_t gl = 0;
  GG_CUDA(cudaMemcpyAsync(&gl, (const uint32_t*)g->g2l.p + source, 4, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  std::vector<uint32_t> A0;   // partition 0's active vertices
  if (!(gl & kRemote)) {
    h->dist[gl].store(0, std::memory_order_relaxed);
    A0.push_back(gl);
    for (int b = 0; b < kNBucket; ++b) hc->tail[0][b] = 0;
  }
  int64_t inspected = 0, messages = 0, launches = 1, rounds = 0;
  bool overflow = false;
  double ms_cpu = 0, ms_gpu = 0, ms_xchg = 0;
  std::vector<std::vector<uint32_t>> ttouch(nt), tdirty(nt);
  std::vector<int64_t> tin(nt);
  std::vector<uint8_t> tovf(nt);
  int cur = 0;
  const uint32_t owords1 = (uint32_t)((g->part[1].nout + 31) / 32);
  const uint32_t words1 = (uint32_t)w->words[1];
  for (;; ++rounds) {
    SsspCounters c = *hc;
    uint64_t dev_active = 0;
    for (int b = 0; b < kNBucket; ++b) dev_active += c.tail[1][b];
    if (dev_active == 0 && A0.empty()) break;
    if (rounds >= cap) {
      set_error("sssp_hybrid reached the superstep cap (%lld)", (long long)cap);
      return GRAPH_ETIMEOUT;
    }
    // GPU: partition 1's round, then its lowered outbox slots as messages.
    GG_CUDA(cudaMemsetAsync(dc, 0, sizeof(SsspCounters), st));
    GG_CUDA(cudaMemsetAsync(h->dmsg.p, 0, 16, st));
    SsspArgs A = make_args(g, w, dc, cur);
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
        k_sssp_relax<false><<<pl.nblocks, kThreads, 0, st>>>(pl, A);
        launches++;
      }
    }
    GG_CUDA(cudaEventRecord(h->ev[1], st));
    if (owords1) {
      k_hsssp_out<<<grid_for(owords1, 256), 256, 0, st>>>(A, (uint32_t*)h->dmsg.p);
      launches++;
    }
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(h->pin_in, h->dmsg.p, 16, cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaEventRecord(h->ev[2], st));
    // Host: partition 0's round (Figure 20) while the GPU works.
    const auto tc0 = Clock::now();
    for (int k = 0; k < nt; ++k) {
      ttouch[k].clear();
      tdirty[k].clear();
      tin[k] = 0;
      tovf[k] = 0;
    }
    host_dynamic(nt, A0.size(), 1, [&](int k, uint64_t a, uint64_t b) {
      for (uint64_t i = a; i < b; ++i) {
        const uint32_t u = A0[i];
        const uint64_t du = h->dist[u].load(std::memory_order_relaxed);
        h->snap[u] = (uint32_t)du;
        const int64_t e1 = h->off0[u + 1];
        for (int64_t e = h->off0[u]; e < e1; ++e) {
          uint64_t s = du + h->W0[e];
          if (s >= kInf) {
            tovf[k] = 1;
            s = kInf - 1;
          }
          const uint32_t x = h->E0[e];
          if (!(x & kRemote)) {
            if (host_min(&h->dist[x], (uint32_t)s) && !h->touched[x].exchange(1))
              ttouch[k].push_back(x);
          } else {
            const uint32_t idx = x & kIdMask;
            if (host_min(&h->omsg[idx], (uint32_t)s) && !h->odirty[idx].exchange(1))
              tdirty[k].push_back(idx);
          }
        }
        tin[k] += e1 - h->off0[u];
      }
    });
    ms_cpu += std::chrono::duration<double, std::milli>(Clock::now() - tc0).count();
    // Exchange: the GPU's lowered slots come up and lower partition 0 ...
    GG_CUDA(cudaEventSynchronize(h->ev[2]));
    float gms = 0;
    GG_CUDA(cudaEventElapsedTime(&gms, h->ev[0], h->ev[1]));
    ms_gpu += gms;
    const auto tx0 = Clock::now();
    const uint32_t n1 = h->pin_in[0];
    if (n1) {
      GG_CUDA(cudaMemcpyAsync(h->pin_in + 4, (const uint32_t*)h->dmsg.p + 4, 8ull * n1,
                              cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
    }
    std::vector<uint32_t> in_touch;
    for (uint32_t i = 0; i < n1; ++i) {
      const uint32_t u = h->pin_in[4 + 2 * i], val = h->pin_in[4 + 2 * i + 1];
      if (host_min(&h->dist[u], val) && !h->touched[u].exchange(1)) in_touch.push_back(u);
    }
    // ... and the host's lowered slots go down and lower partition 1.
    uint32_t n0 = 0;
    for (int k = 0; k < nt; ++k)
      for (uint32_t idx : tdirty[k]) {
        h->odirty[idx].store(0, std::memory_order_relaxed);
        h->pin_out[2 * n0] = h->outbox0[idx];
        h->pin_out[2 * n0 + 1] = h->omsg[idx].load(std::memory_order_relaxed);
        ++n0;
      }
    if (n0) {
      GG_CUDA(cudaMemcpyAsync(h->dmsg.p, h->pin_out, 8ull * n0, cudaMemcpyHostToDevice, st));
      k_hsssp_in<<<std::min(grid_for(n0, 256), 152u * 8), 256, 0, st>>>(
          A, (const uint32_t*)h->dmsg.p, n0);
      launches++;
    }
    // Filter: partition 1 on the device (its words only), partition 0 on the host.
    {
      SsspArgs F = A;
      k_sssp_filter<<<grid_for(words1, kThreads), kThreads, 0, st>>>(F, 0u, words1, kInf, 0);
      launches++;
    }
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
    A0.clear();
    auto filter = [&](uint32_t x) {
      h->touched[x].store(0, std::memory_order_relaxed);
      if (h->dist[x].load(std::memory_order_relaxed) < h->snap[x]) A0.push_back(x);
    };
    for (int k = 0; k < nt; ++k) {
      for (uint32_t x : ttouch[k]) filter(x);
      inspected += tin[k];
      overflow |= tovf[k] != 0;
    }
    for (uint32_t x : in_touch) filter(x);
    GG_CUDA(cudaStreamSynchronize(st));
    inspected += (int64_t)hc->inspected;
    overflow |= hc->overflow != 0;
    messages += (int64_t)n1 + n0;
    ms_xchg += std::chrono::duration<double, std::milli>(Clock::now() - tx0).count();
    cur = 1 - cur;
  }
  // Collect: the host partition's distances join the device's.
  if (nv0) {
    std::vector<uint32_t> d0(nv0);
    for (uint32_t v = 0; v < nv0; ++v) d0[v] = h->dist[v].load(std::memory_order_relaxed);
    GG_CUDA(cudaMemcpyAsync(w->dist[0].p, d0.data(), 4ull * nv0, cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaStreamSynchronize(st));
  }
  void* dd = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, dist, at.out_mem, 4ull * g->n + 64, 0, &dd, &staged));
  GG_TRY(launch_collect(g, w, dc, cur, (uint32_t*)dd, st));
  launches += 2;
  if (staged) GG_TRY(deliver(g, dist, dd, 4ull * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaMemcpyAsync(hc, dc, sizeof(SsspCounters), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  graph_status s = check_device_error(g);
  if (!hc->clamped) overflow = false;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = (int)rounds;
    stats->edges_traversed = (int64_t)hc->reached_degree;
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
  if (s == GRAPH_OK && overflow) {
    set_error("a shortest distance reached 2^32 - 1");
    return GRAPH_ERANGE;
  }
  return s;
}
