// Pull PageRank on the partitioned graph (Section 7.1, Figure 14).
//
// One BSP superstep per iteration:
//  - communication (pull, Section 4.3.2): each partition publishes the contribution x of
//    its inbox vertices into the other partition's ghost slots (the outbox message array;
//    only messages move, the vertex-id arrays are symmetric).
//  - compute: every vertex sums the contributions of its neighbours (local ones from x,
//    boundary ones from the ghost slots) and sets r' = (1-d)/n + d (sum + D/n), then its
//    own contribution x' = r'/deg. Hub vertices (degree >= 2048) are split into chunks of
//    4096 edges, one CTA each; the chunk's edge ids are staged into shared memory by a bulk
//    (TMA engine) copy, the CTA sums its gathers, and the last CTA of a vertex adds the
//    chunk sums in chunk order and updates the vertex. Other vertices use one warp, four
//    lanes or one lane each, by degree class.
//  - reduction: FP64 block partials of the L1 residual and of the rank on degree-zero
//    vertices are summed in a fixed order by one CTA, which also forms the next
//    iteration's constant term.
// Precision variants: FP32 contributions and sums; FP64 throughout; FP16 contributions
// scaled by n (x = n r/deg keeps them away from FP16's subnormal range) with FP32 sums.
#include <string.h>

#include "common.cuh"

namespace gg {

struct PrWs {
  int prec = -1;
  size_t esize = 0;  // bytes per stored contribution
  size_t rsize = 0;  // bytes per stored rank
  DevBuf r[2], x[2][2], ghost[2], hubsum[2], ticket[2];
  DevBuf partials, scal, resid;
  uint32_t nblocks = 0;
  int max_iter = 0;
};

void free_pr(graph* g) {
  if (!g->pr) return;
  PrWs* w = g->pr;
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->r[p], &w->x[p][0], &w->x[p][1], &w->ghost[p], &w->hubsum[p],
                     &w->ticket[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  dfree(g, w->partials);
  dfree(g, w->scal);
  dfree(g, w->resid);
  delete w;
  g->pr = nullptr;
}

namespace {

// Scalars on the device: [0] constant term (1-d)/n + d D/n, [1] D, [2] last residual.
struct PrSide {
  PartView P;
  void* r;
  const void* x;      // contributions of this iteration
  void* xn;           // contributions of the next iteration
  void* ghost;        // contributions of the outbox targets
  void* hubsum;       // per hub chunk partial sum (accumulator type)
  uint32_t* ticket;   // per hub vertex chunk counter
  const uint32_t* chunk_vertex;
  const int64_t* chunk_first;
  const uint32_t* hub_chunk0;
};

struct PrArgs {
  PrSide side[2];
  double* scal;
  double2* partials;  // per block: (residual, dangling)
  double damping;
  double n;
  int* err;
};

template <class XT> struct XConv;
template <> struct XConv<float> {
  __device__ static float load(const float* p) { return *p; }
  __device__ static void store(float* p, float v) { *p = v; }
};
template <> struct XConv<double> {
  __device__ static double load(const double* p) { return *p; }
  __device__ static void store(double* p, double v) { *p = v; }
};
template <> struct XConv<__half> {
  __device__ static float load(const __half* p) { return __half2float(*p); }
  __device__ static void store(__half* p, float v) { *p = __float2half_rn(v); }
};

// Precision policy: XT stored contribution, AT accumulation, RT stored rank; SCALED means
// x holds n * r / deg.
template <class XT_, class AT_, class RT_, bool SCALED_>
struct Prec {
  using XT = XT_;
  using AT = AT_;
  using RT = RT_;
  static constexpr bool SCALED = SCALED_;
};
using PrecF32 = Prec<float, float, float, false>;
using PrecF64 = Prec<double, double, double, false>;
using PrecF16 = Prec<__half, float, float, true>;

template <class PR>
__device__ __forceinline__ typename PR::AT gather(const PrSide& S, uint32_t x) {
  const typename PR::XT* base =
      (x & kRemote) ? (const typename PR::XT*)S.ghost : (const typename PR::XT*)S.x;
  return (typename PR::AT)XConv<typename PR::XT>::load(base + (x & kIdMask));
}

// Vertex update from its neighbour sum; returns (|r' - r|, dangling share) in FP64.
template <class PR>
__device__ __forceinline__ double2 update_vertex(const PrSide& S, const PrArgs& A, uint32_t v,
                                                 typename PR::AT sum, int64_t deg) {
  using AT = typename PR::AT;
  using RT = typename PR::RT;
  const AT base = (AT)A.scal[0];
  const AT d = (AT)A.damping;
  AT rn;
  if (PR::SCALED) rn = base + (d / (AT)A.n) * sum;
  else rn = base + d * sum;
  RT* r = (RT*)S.r;
  const AT ro = (AT)r[v];
  r[v] = (RT)rn;
  typename PR::XT* xn = (typename PR::XT*)S.xn;
  if (deg > 0) {
    if (PR::SCALED) XConv<typename PR::XT>::store(xn + v, (rn * (AT)A.n) / (AT)deg);
    else XConv<typename PR::XT>::store(xn + v, rn / (AT)deg);
  } else {
    XConv<typename PR::XT>::store(xn + v, (AT)0);
  }
  const AT diff = rn > ro ? rn - ro : ro - rn;
  return make_double2((double)diff, deg == 0 ? (double)rn : 0.0);
}

__device__ void block_partial(double2 acc, double2* out) {
  __shared__ double sr[kThreads / 32], sd[kThreads / 32];
  acc.x = warp_sum(acc.x);
  acc.y = warp_sum(acc.y);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) {
    sr[w] = acc.x;
    sd[w] = acc.y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < kThreads / 32; ++i) {
      a += sr[i];
      b += sd[i];
    }
    out[blockIdx.x] = make_double2(a, b);
  }
}

template <class PR>
__global__ void __launch_bounds__(kThreads)
k_pr_compute(const __grid_constant__ Plan plan, const __grid_constant__ PrArgs A) {
  using AT = typename PR::AT;
  const Seg& G = plan.seg[find_seg(plan)];
  const PrSide& S = A.side[G.part];
  const uint32_t rel = blockIdx.x - G.blk0;
  double2 acc = make_double2(0.0, 0.0);
  if (G.gshift >= 8) {
    // One hub chunk per CTA.
    __shared__ alignas(16) uint32_t sE[kHubChunk + 8];
    __shared__ uint64_t bar;
    __shared__ AT wsum[kThreads / 32];
    __shared__ int last;
    const uint32_t k = G.v0 + rel;  // chunk index
    const uint32_t v = S.chunk_vertex[k];
    const int64_t e0 = S.chunk_first[k];
    const int64_t vend = S.P.off[v + 1];
    const int64_t e1 = min(e0 + (int64_t)kHubChunk, vend);
    const int64_t a0 = e0 & ~(int64_t)3, a1 = (e1 + 3) & ~(int64_t)3;
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t bytes = (uint32_t)((a1 - a0) * 4);
      mbar_expect_tx(&bar, bytes);
      bulk_g2s(sE, S.P.E + a0, bytes, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, A.err);
    AT s = 0;
    if (ok) {
      const uint32_t* src = sE + (e0 - a0);
      const int cnt = (int)(e1 - e0);
      #pragma unroll 4
      for (int i = threadIdx.x; i < cnt; i += kThreads) s += gather<PR>(S, src[i]);
    }
    s = warp_sum(s);
    if (lane_id() == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      AT t = 0;
      for (int i = 0; i < kThreads / 32; ++i) t += wsum[i];
      ((AT*)S.hubsum)[k] = t;
      __threadfence();
      const int64_t deg = vend - S.P.off[v];
      const uint32_t nch = (uint32_t)((deg + kHubChunk - 1) / kHubChunk);
      const uint32_t tk = atomicAdd(&S.ticket[v], 1u);
      last = (tk == nch - 1);
      if (last) {
        __threadfence();
        const uint32_t c0 = S.hub_chunk0[v];
        AT sum = 0;
        for (uint32_t c = 0; c < nch; ++c) sum += __ldcg((const AT*)S.hubsum + c0 + c);
        acc = update_vertex<PR>(S, A, v, sum, deg);
        S.ticket[v] = 0;
      }
    }
    block_partial(acc, A.partials);
    return;
  }
  const int gs = G.gshift;
  const int gsz = 1 << gs;
  const uint32_t gi = rel * (kThreads >> gs) + (threadIdx.x >> gs);
  const int gl = threadIdx.x & (gsz - 1);
  AT s = 0;
  int64_t deg = 0;
  uint32_t v = 0;
  const bool valid = gi < G.count;
  if (valid) {
    v = G.v0 + gi;
    const int64_t b = S.P.off[v], t = S.P.off[v + 1];
    deg = t - b;
    #pragma unroll 4
    for (int64_t e = b + gl; e < t; e += gsz) s += gather<PR>(S, S.P.E[e]);
  }
  s = group_sum(s, gs);
  if (valid && gl == 0) acc = update_vertex<PR>(S, A, v, s, deg);
  block_partial(acc, A.partials);
}

// Communication phase: ghost_p[i] = x_q[outbox_p[i]].
template <class XT>
__global__ void k_pr_publish(const __grid_constant__ PrArgs A) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n0 = A.side[0].P.nout;
  const int p = i < n0 ? 0 : 1;
  const uint32_t j = p == 0 ? i : i - n0;
  const PrSide& S = A.side[p];
  if (j >= S.P.nout) return;
  const PrSide& Q = A.side[1 - p];
  ((XT*)S.ghost)[j] = ((const XT*)Q.x)[S.P.outbox[j]];
}

// Fixed-order FP64 sum of the block partials; sets the next constant term.
__global__ void __launch_bounds__(1024) k_pr_finalize(double2* partials, uint32_t nblocks,
                                                      double* scal, double* resid_hist,
                                                      int iter, double damping, double n,
                                                      int dangling) {
  __shared__ double sr[32], sd[32];
  double a = 0, b = 0;
  for (uint32_t i = threadIdx.x; i < nblocks; i += blockDim.x) {
    a += partials[i].x;
    b += partials[i].y;
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane_id() == 0) {
    sr[threadIdx.x >> 5] = a;
    sd[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ra = 0, da = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      ra += sr[i];
      da += sd[i];
    }
    const double D = dangling ? da : 0.0;
    scal[1] = D;
    scal[0] = (1.0 - damping) / n + damping * D / n;
    scal[2] = ra;
    resid_hist[iter] = ra;
  }
}

template <class PR>
__global__ void k_pr_init(const __grid_constant__ PrArgs A, uint32_t nv0, uint32_t ntot) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const int p = i < nv0 ? 0 : 1;
  const uint32_t v = p == 0 ? i : i - nv0;
  const PrSide& S = A.side[p];
  using AT = typename PR::AT;
  const AT r0 = (AT)(1.0 / A.n);
  ((typename PR::RT*)S.r)[v] = (typename PR::RT)r0;
  const int64_t deg = S.P.off[v + 1] - S.P.off[v];
  typename PR::XT* x = (typename PR::XT*)S.x;
  if (deg > 0) {
    if (PR::SCALED) XConv<typename PR::XT>::store(x + v, (AT)1 / (AT)deg);
    else XConv<typename PR::XT>::store(x + v, r0 / (AT)deg);
  } else {
    XConv<typename PR::XT>::store(x + v, (AT)0);
  }
}

template <class RT>
__global__ void k_pr_collect(const __grid_constant__ PrArgs A, uint32_t nv0, uint32_t n,
                             double* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = i < nv0 ? 0 : 1;
  const uint32_t v = p == 0 ? i : i - nv0;
  const PrSide& S = A.side[p];
  out[S.P.l2g[v]] = (double)((const RT*)S.r)[v];
}

Plan make_plan(graph* g) {
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    const PartView V = P.view();
    plan_add(pl, nullptr, 0, P.nchunk, p, 8, 0);
    plan_add(pl, nullptr, V.bstart[1], V.bstart[2] - V.bstart[1], p, 5, 1);
    plan_add(pl, nullptr, V.bstart[2], V.bstart[3] - V.bstart[2], p, kSubShift, 2);
    plan_add(pl, nullptr, V.bstart[3], P.nv - V.bstart[3], p, 0, 3);  // incl. degree zero
  }
  return pl;
}

graph_status ensure_ws(graph* g, int prec, int max_iter, uint32_t nblocks) {
  const size_t es = prec == GRAPH_PR_FP64 ? 8 : (prec == GRAPH_PR_FP16 ? 2 : 4);
  const size_t rs = prec == GRAPH_PR_FP64 ? 8 : 4;
  const size_t as = prec == GRAPH_PR_FP64 ? 8 : 4;
  if (g->pr && (g->pr->prec != prec || g->pr->max_iter < max_iter)) free_pr(g);
  if (g->pr) return GRAPH_OK;
  PrWs* w = new PrWs();
  g->pr = w;
  w->prec = prec;
  w->esize = es;
  w->rsize = rs;
  w->max_iter = max_iter;
  w->nblocks = nblocks;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_TRY(dalloc(g, w->r[p], rs * P.nv));
    GG_TRY(dalloc(g, w->x[p][0], es * P.nv));
    GG_TRY(dalloc(g, w->x[p][1], es * P.nv));
    GG_TRY(dalloc(g, w->ghost[p], es * P.nout));
    GG_TRY(dalloc(g, w->hubsum[p], as * P.nchunk));
    GG_TRY(dalloc(g, w->ticket[p], 4ull * P.nhub));
    GG_CUDA(cudaMemsetAsync(w->ticket[p].p, 0, 4ull * P.nhub, g->stream));
  }
  GG_TRY(dalloc(g, w->partials, sizeof(double2) * (size_t)(nblocks + 1)));
  GG_TRY(dalloc(g, w->scal, 8 * sizeof(double)));
  GG_TRY(dalloc(g, w->resid, sizeof(double) * (size_t)(max_iter + 1)));
  return GRAPH_OK;
}

PrArgs make_args(graph* g, int cur, double damping) {
  PrWs* w = g->pr;
  PrArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    PrSide& S = A.side[p];
    S.P = P.view();
    S.r = w->r[p].p;
    S.x = w->x[p][cur].p;
    S.xn = w->x[p][1 - cur].p;
    S.ghost = w->ghost[p].p;
    S.hubsum = w->hubsum[p].p;
    S.ticket = (uint32_t*)w->ticket[p].p;
    S.chunk_vertex = (const uint32_t*)P.chunk_vertex.p;
    S.chunk_first = (const int64_t*)P.chunk_first.p;
    S.hub_chunk0 = (const uint32_t*)P.hub_chunk0.p;
  }
  A.scal = (double*)w->scal.p;
  A.partials = (double2*)w->partials.p;
  A.damping = damping;
  A.n = (double)g->n;
  A.err = (int*)g->err.p;
  return A;
}

template <class PR>
graph_status run(graph* g, const pagerank_attr& at, double* ranks, graph_stats* stats) {
  cudaStream_t st = g->stream;
  Plan pl = make_plan(g);
  GG_TRY(ensure_ws(g, at.precision, at.max_iter, pl.nblocks));
  PrWs* w = g->pr;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  const uint32_t nv0 = g->part[0].nv;
  int cur = 0;
  {
    PrArgs A = make_args(g, cur, at.damping);
    k_pr_init<PR><<<grid_for(g->n, 256), 256, 0, st>>>(A, nv0, g->n);
    GG_CUDA(cudaGetLastError());
    // D_0 = (number of degree-zero vertices) / n
    uint64_t zero = 0;
    for (int p = 0; p < 2; ++p) zero += g->part[p].nv - g->part[p].cls_end[1];
    double h[3];
    const double D0 = at.dangling ? (double)zero / (double)g->n : 0.0;
    h[0] = (1.0 - at.damping) / (double)g->n + at.damping * D0 / (double)g->n;
    h[1] = D0;
    h[2] = 0;
    GG_CUDA(cudaMemcpyAsync(w->scal.p, h, sizeof(h), cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaStreamSynchronize(st));
  }
  const uint32_t nout = g->part[0].nout + g->part[1].nout;
  int it = 0;
  int64_t launches = 1;
  double last_res = 0;
  for (; it < at.max_iter;) {
    PrArgs A = make_args(g, cur, at.damping);
    timer.mark(2);
    if (nout) k_pr_publish<typename PR::XT><<<grid_for(nout, 256), 256, 0, st>>>(A);
    timer.mark(1);
    if (pl.nblocks) k_pr_compute<PR><<<pl.nblocks, kThreads, 0, st>>>(pl, A);
    timer.mark(0);
    k_pr_finalize<<<1, 1024, 0, st>>>(A.partials, pl.nblocks, A.scal, (double*)w->resid.p, it,
                                      at.damping, (double)g->n, at.dangling);
    timer.mark(2);
    launches += 1 + (nout ? 1 : 0) + (pl.nblocks ? 1 : 0);
    GG_CUDA(cudaGetLastError());
    cur = 1 - cur;
    ++it;
    if (at.tol > 0) {
      GG_CUDA(cudaMemcpyAsync(&last_res, (double*)w->scal.p + 2, 8, cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      if (last_res < at.tol) break;
    }
  }
  double* out = ranks;
  if (at.out_mem == GRAPH_MEM_HOST) {
    GG_TRY(ensure_stage(g, 8ull * g->n));
    out = (double*)g->stage.p;
  }
  {
    PrArgs A = make_args(g, cur, at.damping);
    k_pr_collect<typename PR::RT><<<grid_for(g->n, 256), 256, 0, st>>>(A, nv0, g->n, out);
    launches++;
    GG_CUDA(cudaGetLastError());
  }
  if (at.out_mem == GRAPH_MEM_HOST) GG_TRY(deliver(g, ranks, out, 8ull * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaMemcpyAsync(&last_res, (double*)w->scal.p + 2, 8, cudaMemcpyDeviceToHost, st));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = it;
    stats->edges_traversed = g->m * (int64_t)it;
    stats->edges_inspected = g->m * (int64_t)it;
    stats->messages = (int64_t)nout * it;
    stats->residual = last_res;
    stats->launches = launches;
  }
  timer.finish(stats);
  return s;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" graph_status pagerank(graph_t* g, const pagerank_attr* attr, double* ranks,
                                 graph_stats* stats) {
  if (!g || !attr || !ranks) {
    set_error("graph, attr or ranks is NULL");
    return GRAPH_EINVAL;
  }
  const pagerank_attr at = *attr;
  if (!(at.damping >= 0.0 && at.damping <= 1.0) || at.max_iter < 1 ||
      (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) ||
      (at.dangling != 0 && at.dangling != 1)) {
    set_error("bad pagerank attributes");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before pagerank");
    return GRAPH_ESTATE;
  }
  switch (at.precision) {
    case GRAPH_PR_FP32: return run<PrecF32>(g, at, ranks, stats);
    case GRAPH_PR_FP64: return run<PrecF64>(g, at, ranks, stats);
    case GRAPH_PR_FP16: return run<PrecF16>(g, at, ranks, stats);
    default:
      set_error("bad precision %d", at.precision);
      return GRAPH_EINVAL;
  }
}
