// Pull PageRank on the partitioned graph (Section 7.1, Figure 14).
//
// One BSP superstep per iteration:
//  - communication (pull, Section 4.3.2): each partition publishes the contribution x of
//    its inbox vertices into the other partition's ghost slots (the outbox message array;
//    only messages move, the vertex-id arrays are symmetric).
//  - compute: every vertex sums the contributions of its neighbours (local ones from x,
//    boundary ones from the ghost slots) and sets r' = (1-d)/n + d (sum + D/n), then its
//    own contribution x' = r'/deg.
//  - reduction: each warp adds its partial sum of the L1 residual to one of kSlots FP64
//    slots (a reduction nobody waits for, so a block frees its SM slot as soon as its
//    vertices are written); a one-block kernel then sums the slots, forms the next
//    iteration's constant term and clears them. The FP64 additions happen in arrival
//    order, so the residual's last bits can differ between runs; the ranks cannot.
//
// Work items (one CTA each): hub chunks (kHubChunk edges of a vertex of degree >= 2048;
// each warp's partial sum of the chunk goes to hubsum[item][warp], and k_pr_hubs then adds
// each hub's partials in chunk and warp order and updates the hub), class tiles (at most
// kPrTileV vertices of degree class c, so at most kTileE edges) and tiles of degree-zero
// vertices. Items are resolved once per workspace into a table of 32-byte records (edge
// range, vertex range, kind), read with an L2 keep-resident hint, so a CTA issues its bulk
// copies after one L2 hit. A CTA stages its item's edge ids, offsets and previous ranks
// into shared memory with bulk copies (TMA engine) completing on an mbarrier. In a class
// tile the 2^(c-3) threads of a vertex gather its edges at that stride (at most 8 each,
// all issued before any is used) and add them in registers. Nothing in a CTA waits for
// another CTA: short-lived CTAs keep 8 per SM resident (the freed shared memory goes to
// L1), and the number of gathers in flight per SM is what sets the speed (the kernel is
// bound by gather latency and the load pipes, not by DRAM bandwidth).
//
// Degree-zero vertices: their neighbour sum is empty, so each of them holds exactly the
// iteration's constant term. Their share of the dangling mass D and of the residual is
// therefore (count x constant) and (count x |change of the constant|), formed in FP64 by
// the finalize kernel; no per-vertex FP64 work is done (this GPU's FP64 rate is far below
// its FP32 rate).
//
// Precision variants: FP32 contributions and sums; FP64 throughout; FP16 contributions
// scaled by n (x = n r/deg keeps them away from FP16's subnormal range) with FP32 sums.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "common.cuh"
#include "pr_seg.cuh"

namespace gg {

// State of pagerank_multi: the component layout it last validated, per-vertex component
// ids, the per-iteration constant table and the captured iteration graph.
struct MultiWs {
  std::vector<uint32_t> vbase;      // validated component boundaries (global ids)
  std::vector<uint32_t> nzero;      // degree-zero vertices per component
  DevBuf dvbase, dnzero, gix[2], base, dn, nf, res;
  size_t base_bytes = 0;
  cudaStream_t capture = nullptr;   // private stream used only to capture
  cudaGraphExec_t exec = nullptr;   // iterations [0, iters) of the last capture
  int iters = 0;
  double damping = -1;              // kernel parameters baked into the capture
  int dangling = -1;
};

struct HybWs;
void free_hyb(struct PrWs* w);

struct PrWs {
  int prec = -1;
  size_t esize = 0;  // bytes per stored contribution
  size_t rsize = 0;  // bytes per stored rank
  DevBuf r[2], x[2][2], ghost[2];
  DevBuf slots, scal, resid;
  DevBuf items, hubsum;      // resolved work items and hub-chunk partial sums
  uint32_t items_n = 0;      // items resolved for the current partition (0: not yet)
  int items_parts = 0;       // partitions (bit p) the resolved items cover
  int max_iter = 0;
  MultiWs* multi = nullptr;
  HybWs* hyb = nullptr;      // host side of pagerank_hybrid
};

void free_multi(graph* g, PrWs* w) {
  MultiWs* m = w->multi;
  if (!m) return;
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->capture) cudaStreamDestroy(m->capture);
  DevBuf* all[] = {&m->dvbase, &m->dnzero, &m->gix[0], &m->gix[1], &m->base, &m->dn, &m->nf,
                   &m->res};
  for (DevBuf* b : all) dfree(g, *b);
  delete m;
  w->multi = nullptr;
}

void free_pr(graph* g) {
  if (!g->pr) return;
  PrWs* w = g->pr;
  free_multi(g, w);
  free_hyb(w);
  for (int p = 0; p < 2; ++p) {
    DevBuf* all[] = {&w->r[p], &w->x[p][0], &w->x[p][1], &w->ghost[p]};
    for (DevBuf* b : all) dfree(g, *b);
  }
  dfree(g, w->slots);
  dfree(g, w->items);
  dfree(g, w->hubsum);
  dfree(g, w->scal);
  dfree(g, w->resid);
  delete w;
  g->pr = nullptr;
}

namespace {

constexpr int kPerThread = kTileE / kThreads;  // gathers a thread issues per tile

struct PrSide {
  PartView P;
  void* r;
  const void* x;      // contributions of this iteration
  void* xn;           // contributions of the next iteration
  void* ghost;        // contributions of the outbox targets
};

// Device scalars (doubles): [0] constant term of this iteration, (1-d)/n + d D/n;
// [1] D; [2] last residual; [3] rank of degree-zero vertices before this iteration;
// [4] the constant term rounded to FP32 (stored as a float in the first half).
constexpr uint32_t kSlots = 1024;  // FP64 residual slots (block b adds to slot b % kSlots);
                                   // slot kSlots holds the residual of a partition that the
                                   // host's cores update (pagerank_hybrid), else zero
constexpr int kHubParts = kThreads / 32;  // partial sums per hub chunk (one per warp)

struct PrItem;

struct PrArgs {
  PrSide side[2];
  const PrItem* items;  // [nitems] resolved work items
  void* hubsum;         // [nitems] partial sum of each hub-chunk item (accumulation type)
  double* scal;
  double* slots;      // [kSlots + 1] residual partial sums, zero between iterations
  double* resid;      // residual history
  double damping, n;
  float damping_f, n_f, d_over_n_f;
  double nzero;       // number of degree-zero vertices
  int* err;
  int e_host[2];      // partition p's edge ids live in host memory: no bulk copy of them
};

// Many independent graphs in one launch (pagerank_multi): vertex v of partition p belongs
// to component gix[p][v]; component g uses the constant term base[iter * G + g] (its own
// (1-d)/n_g + d D_g/n_g, a scalar recurrence computed on the host), dn[g] = d/n_g and
// nf[g] = n_g (FP16 scaling). On the last iteration each vertex adds |r' - r| to res[g].
struct MultiArgs {
  const uint32_t* gix[2];
  const void* base;   // [iters][G] in the accumulation type
  const void* dn;     // [G]
  const void* nf;     // [G]
  double* res;        // [G]
  uint32_t G;
  int last;           // this launch is the last iteration
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

template <class AT> struct Consts;
template <> struct Consts<float> {
  __device__ static float base(const PrArgs& A) { return ((const float*)(A.scal + 4))[0]; }
  __device__ static float d(const PrArgs& A) { return A.damping_f; }
  __device__ static float n(const PrArgs& A) { return A.n_f; }
  __device__ static float d_over_n(const PrArgs& A) { return A.d_over_n_f; }
};
template <> struct Consts<double> {
  __device__ static double base(const PrArgs& A) { return A.scal[0]; }
  __device__ static double d(const PrArgs& A) { return A.damping; }
  __device__ static double n(const PrArgs& A) { return A.n; }
  __device__ static double d_over_n(const PrArgs& A) { return A.damping / A.n; }
};

// Update of a vertex with degree deg > 0 from its neighbour sum and its previous rank ro;
// returns |r' - r| (MULTI: adds it to its component's residual on the last iteration and
// returns 0).
template <class PR, bool MULTI>
__device__ __forceinline__ typename PR::AT update_vertex(const PrSide& S, const PrArgs& A,
                                                         const MultiArgs& M, int p, int iter,
                                                         uint32_t v, typename PR::AT sum,
                                                         int deg, typename PR::AT ro) {
  using AT = typename PR::AT;
  using RT = typename PR::RT;
  using C = Consts<AT>;
  if (MULTI) {
    const uint32_t g = M.gix[p][v];
    const AT base = ((const AT*)M.base)[(size_t)iter * M.G + g];
    const AT rn = PR::SCALED ? base + ((const AT*)M.dn)[g] * sum : base + C::d(A) * sum;
    ((RT*)S.r)[v] = (RT)rn;
    typename PR::XT* xn = (typename PR::XT*)S.xn;
    if (PR::SCALED) XConv<typename PR::XT>::store(xn + v, (rn * ((const AT*)M.nf)[g]) / (AT)deg);
    else XConv<typename PR::XT>::store(xn + v, rn / (AT)deg);
    if (M.last) atomicAdd(M.res + g, (double)(rn > ro ? rn - ro : ro - rn));
    return (AT)0;
  }
  const AT rn = PR::SCALED ? C::base(A) + C::d_over_n(A) * sum : C::base(A) + C::d(A) * sum;
  ((RT*)S.r)[v] = (RT)rn;
  typename PR::XT* xn = (typename PR::XT*)S.xn;
  if (PR::SCALED) XConv<typename PR::XT>::store(xn + v, (rn * C::n(A)) / (AT)deg);
  else XConv<typename PR::XT>::store(xn + v, rn / (AT)deg);
  return rn > ro ? rn - ro : ro - rn;
}

// ---------------------------------------------------------------------------------------
// Work items of one iteration (see the file comment).
// ---------------------------------------------------------------------------------------
constexpr int kMaxRange = 28;
enum { kItemHub = 0, kItemLeaf = 1, kItemZero = 2 };

struct PrRange {
  uint32_t item0;  // first item index of the range
  uint32_t first;  // first vertex
  uint32_t end;    // end vertex
  uint32_t per;    // vertices per tile (leaf, zero)
  uint8_t kind, part, gshift, pad;
};

struct PrPlan {
  PrRange r[kMaxRange];
  int nr;
  uint32_t nitems;
  uint32_t hub_item0[2];  // first hub-chunk item of each partition
};

struct Desc {
  int64_t e0, e1;     // edge range (hub, leaf)
  uint32_t v0, v1;    // vertex range (one vertex for a hub)
  uint32_t eshift;    // e0 - start of the staged granule
  uint32_t oshift;    // v0 - start of the staged offsets
  uint32_t rshift;    // v0 - start of the staged ranks
  uint8_t kind, part, gshift, pad;
};

// Range holding `item` (item0 increases strictly along the ranges): a binary search, so
// the CTA's first bulk copy is not held up by a scan of the parameter table.
__device__ __forceinline__ int find_range(const PrPlan& P, uint32_t item) {
  int lo = 0, hi = P.nr;  // P.r[lo].item0 <= item, and item < P.r[hi].item0 when hi < nr
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.r[mid].item0 <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One work item, resolved once per workspace by k_pr_items so that a CTA starts its bulk
// copies after a single (L2-resident) 32-byte load instead of a search of the range table
// and two dependent offset loads from DRAM.
struct PrItem {
  int64_t e0, e1;     // edge range (a hub chunk's edges, a class tile's adjacencies)
  uint32_t v0, v1;    // vertex range (hub chunk: its vertex, v1 = v0 + 1)
  uint8_t kind, part, gshift, pad;
  uint32_t pad2;
};
static_assert(sizeof(PrItem) == 32, "PrItem is two 16-byte loads");

__global__ void k_pr_items(const __grid_constant__ PrPlan P, const __grid_constant__ PrArgs A,
                           PrItem* items) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.nitems) return;
  const PrRange& R = P.r[find_range(P, k)];
  const PartView& V = A.side[R.part].P;
  const uint32_t j = k - R.item0;
  PrItem it;
  it.kind = R.kind;
  it.part = R.part;
  it.gshift = R.gshift;
  it.pad = 0;
  it.pad2 = 0;
  if (R.kind == kItemHub) {  // hub chunk j of the partition
    it.v0 = V.chunk_vertex[j];
    it.v1 = it.v0 + 1;
    it.e0 = V.chunk_first[j];
    it.e1 = min(it.e0 + (int64_t)kHubChunk, V.off[it.v0 + 1]);
  } else {
    it.v0 = R.first + j * R.per;
    it.v1 = min(it.v0 + R.per, R.end);
    it.e0 = R.kind == kItemLeaf ? V.off[it.v0] : 0;
    it.e1 = R.kind == kItemLeaf ? V.off[it.v1] : 0;
  }
  items[k] = it;
}

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ PrItem load_item(const PrItem* p) {
  const uint64_t pol = l2_evict_last_policy();
  uint64_t a, b, c, d;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(a), "=l"(b) : "l"(p), "l"(pol));
  asm volatile("ld.global.nc.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(c), "=l"(d) : "l"(reinterpret_cast<const char*>(p) + 16), "l"(pol));
  PrItem it;
  it.e0 = (int64_t)a;
  it.e1 = (int64_t)b;
  it.v0 = (uint32_t)c;
  it.v1 = (uint32_t)(c >> 32);
  it.kind = (uint8_t)d;
  it.part = (uint8_t)(d >> 8);
  it.gshift = (uint8_t)(d >> 16);
  it.pad = 0;
  it.pad2 = 0;
  return it;
}

// Thread 0: describe item k and start the bulk copies of its edge ids (and, for class
// tiles, offsets and previous ranks) into shared memory; `bar` completes when the bytes
// have landed.
template <class RT>
__device__ void issue_item(const PrArgs& A, uint32_t k, Desc& d, uint32_t* sE, int64_t* sOff,
                           RT* sR, uint64_t* bar) {
  const PrItem it = load_item(A.items + k);
  const PrSide& S = A.side[it.part];
  d.kind = it.kind;
  d.part = it.part;
  d.gshift = it.gshift;
  d.pad = 0;
  d.eshift = d.oshift = d.rshift = 0;
  d.v0 = it.v0;
  d.v1 = it.v1;
  d.e0 = it.e0;
  d.e1 = it.e1;
  uint32_t ebytes = 0, obytes = 0, rbytes = 0, o0 = 0, q0 = 0;
  int64_t a0 = 0;
  if (it.kind != kItemZero) {
    a0 = d.e0 & ~(int64_t)3;
    const int64_t a1 = (d.e1 + 3) & ~(int64_t)3;
    d.eshift = (uint32_t)(d.e0 - a0);
    ebytes = (uint32_t)((a1 - a0) * 4);
  }
  if (it.kind == kItemLeaf) {
    o0 = d.v0 & ~1u;
    const uint32_t o1 = (d.v1 + 2) & ~1u;
    d.oshift = d.v0 - o0;
    obytes = (o1 - o0) * 8;
    // previous ranks of the tile's vertices, in whole 16-byte granules
    constexpr uint32_t g = 16 / sizeof(RT);
    q0 = d.v0 & ~(g - 1);
    const uint32_t q1 = (d.v1 + g - 1) & ~(g - 1);
    d.rshift = d.v0 - q0;
    rbytes = (q1 - q0) * (uint32_t)sizeof(RT);
  }
  // Edge ids in host memory are read by the CTA's threads after the wait instead.
  if (A.e_host[it.part]) ebytes = 0;
  mbar_expect_tx(bar, ebytes + obytes + rbytes);
  const uint64_t pol = l2_evict_first_policy();
  if (ebytes) bulk_g2s_stream(sE, S.P.E + a0, ebytes, bar, pol);
  if (obytes) bulk_g2s_stream(sOff, S.P.off + o0, obytes, bar, pol);
  if (rbytes) bulk_g2s_stream(sR, (const RT*)S.r + q0, rbytes, bar, pol);
}

template <class PR>
__device__ __forceinline__ typename PR::AT gather(const PrSide& S, uint32_t e) {
  using XT = typename PR::XT;
  const XT* base = (e & kRemote) ? (const XT*)S.ghost : (const XT*)S.x;
  return (typename PR::AT)XConv<XT>::load(base + (e & kIdMask));
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  if (lane_id() == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = 0;
  #pragma unroll
  for (int i = 0; i < kThreads / 32; ++i) t += red[i];
  __syncthreads();
  return t;
}

// Shared memory of a CTA: the item's edge ids (at most kTileE), and for a class tile
// (at most kPrTileV vertices: one round of the CTA's threads) its offsets and previous
// ranks, each staged in whole 16-byte granules.
constexpr int kPrTileV = kThreads;
template <class PR>
__host__ __device__ constexpr size_t ranks_offset() {
  return 4 * (kTileE + 8) + 8 * (kPrTileV + 4);
}
template <class PR>
__host__ __device__ constexpr size_t smem_bytes() {
  return ranks_offset<PR>() + sizeof(typename PR::RT) * (kPrTileV + 8);
}

template <class PR, bool MULTI>
__global__ void __launch_bounds__(kThreads)
k_pr_compute(const __grid_constant__ PrPlan plan, const __grid_constant__ PrArgs A, int iter,
             int dangling, const __grid_constant__ MultiArgs M) {
  using AT = typename PR::AT;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* sE = reinterpret_cast<uint32_t*>(smem);
  int64_t* sOff = reinterpret_cast<int64_t*>(smem + 4 * (kTileE + 8));
  using RT = typename PR::RT;
  RT* sR = reinterpret_cast<RT*>(smem + ranks_offset<PR>());
  __shared__ uint64_t bar;
  __shared__ Desc dsh;
  __shared__ AT red[kThreads / 32];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    issue_item<RT>(A, blockIdx.x, dsh, sE, sOff, sR, &bar);
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, A.err);
  AT res = 0;
  bool leaf = false;  // the CTA's item is a class tile (uniform over the CTA)
  if (__syncthreads_and(ok)) {
    const Desc d = dsh;
    const PrSide& S = A.side[d.part];
    if (A.e_host[d.part] && d.kind != kItemZero) {
      // host-resident edge ids: the same granules, loaded over the host link by the threads
      const int64_t a0 = d.e0 - (int64_t)d.eshift;
      const int64_t cnt = ((d.e1 + 3) & ~(int64_t)3) - a0;
      for (int64_t i = threadIdx.x; i < cnt; i += kThreads) sE[i] = S.P.E[a0 + i];
      __syncthreads();
    }
    if (d.kind == kItemHub) {
      // One chunk (at most kHubChunk edges) of a hub's adjacency: each warp's partial sum
      // goes to hubsum[item][warp]; k_pr_hubs adds a hub's partials in order and updates
      // the vertex.
      const int cnt = (int)(d.e1 - d.e0);
      const uint32_t* src = sE + d.eshift;
      uint32_t e[kPerThread];
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u) {
        const int i = threadIdx.x + u * kThreads;
        e[u] = i < cnt ? src[i] : 0u;
      }
      AT v[kPerThread];
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u)
        v[u] = (threadIdx.x + u * kThreads < cnt) ? gather<PR>(S, e[u]) : (AT)0;
      AT sum = 0;
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u) sum += v[u];
      sum = warp_sum(sum);  // one partial per warp: no CTA-wide barrier
      if (lane_id() == 0)
        ((AT*)A.hubsum)[(size_t)blockIdx.x * kHubParts + (threadIdx.x >> 5)] = sum;
    } else if (d.kind == kItemLeaf) {
      leaf = true;
      // Vertex j of the tile belongs to the 2^gs threads j << gs ...; they gather its edges
      // at stride 2^gs (at most kPerThread each, since a class-c degree is below 2^c and
      // 2^gs = 2^(c-3)) and add them in registers, so values never round-trip through
      // shared memory.
      const int gs = d.gshift;
      const int nvt = (int)(d.v1 - d.v0);
      const int64_t* so = sOff + d.oshift;
      const uint32_t* src = sE + d.eshift;
      const int j = (int)(threadIdx.x >> gs);  // one round: nvt <= kThreads >> gs
      const int gl = (int)(threadIdx.x & ((1u << gs) - 1));
      int es = 0, ee = 0;
      if (j < nvt) {
        es = (int)(so[j] - d.e0);
        ee = (int)(so[j + 1] - d.e0);
      }
      uint32_t e[kPerThread];
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u) {
        const int i = es + gl + (u << gs);
        e[u] = i < ee ? src[i] : 0u;
      }
      AT v[kPerThread];
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u)
        v[u] = (es + gl + (u << gs) < ee) ? gather<PR>(S, e[u]) : (AT)0;
      AT sm = 0;
      #pragma unroll
      for (int u = 0; u < kPerThread; ++u) sm += v[u];
      if (gs <= 5) {
        sm = group_sum(sm, gs);
        if (j < nvt && gl == 0)
          res += update_vertex<PR, MULTI>(S, A, M, d.part, iter, d.v0 + j, sm, ee - es,
                                          (AT)sR[d.rshift + j]);
      } else {
        // Several warps per vertex (tiles of at most four vertices): warp sums meet in
        // shared memory and the group's first thread updates the vertex.
        sm = warp_sum(sm);
        if (lane_id() == 0) red[threadIdx.x >> 5] = sm;
        __syncthreads();
        if (j < nvt && gl == 0) {
          AT t = 0;
          for (int k = 0; k < (1 << (gs - 5)); ++k) t += red[(threadIdx.x >> 5) + k];
          res += update_vertex<PR, MULTI>(S, A, M, d.part, iter, d.v0 + j, t, ee - es,
                                          (AT)sR[d.rshift + j]);
        }
        __syncthreads();  // red is reused by the residual sum
      }
    } else {
      // Degree-zero vertices: the rank is the constant term, the contribution zero.
      const typename PR::RT b = (typename PR::RT)Consts<AT>::base(A);
      for (uint32_t v = d.v0 + threadIdx.x; v < d.v1; v += kThreads) {
        ((typename PR::RT*)S.r)[v] =
            MULTI ? (typename PR::RT)((const AT*)M.base)[(size_t)iter * M.G + M.gix[d.part][v]]
                  : b;
        XConv<typename PR::XT>::store((typename PR::XT*)S.xn + v, (AT)0);
      }
    }
  }
  // Components keep no global scalars: their constants come from the host's table. Only
  // class tiles update vertices here (hub chunks and degree-zero tiles leave no residual).
  if (MULTI || !leaf) return;
  res = warp_sum(res);
  if (lane_id() == 0 && res != (AT)0)
    atomicAdd(A.slots + ((blockIdx.x * kHubParts + (threadIdx.x >> 5)) % kSlots), (double)res);
}

// Hub vertices (degree >= kHubChunk), one warp each: the sum of the vertex's chunk partial
// sums in chunk order, then the vertex update. Runs after k_pr_compute in every iteration.
template <class PR, bool MULTI>
__global__ void __launch_bounds__(kThreads)
k_pr_hubs(const __grid_constant__ PrPlan plan, const __grid_constant__ PrArgs A, int iter,
          const __grid_constant__ MultiArgs M) {
  using AT = typename PR::AT;
  using RT = typename PR::RT;
  __shared__ AT red[kThreads / 32];
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nh0 = A.side[0].P.bstart[1], nh1 = A.side[1].P.bstart[1];
  AT res = 0;
  if (w < nh0 + nh1) {
    const int p = w < nh0 ? 0 : 1;
    const uint32_t v = p ? w - nh0 : w;
    const PrSide& S = A.side[p];
    const int64_t deg = S.P.off[v + 1] - S.P.off[v];
    const uint32_t nch = (uint32_t)((deg + kHubChunk - 1) / kHubChunk);
    const AT* hs = (const AT*)A.hubsum +
                   (size_t)(plan.hub_item0[p] + S.P.hub_chunk0[v]) * kHubParts;
    AT sum = 0;
    for (uint32_t c = lane_id(); c < nch * kHubParts; c += 32) sum += hs[c];
    sum = warp_sum(sum);
    if (lane_id() == 0)
      res = update_vertex<PR, MULTI>(S, A, M, p, iter, v, sum, (int)deg,
                                     (AT)((const RT*)S.r)[v]);
  }
  if (MULTI) return;
  res = block_sum<AT>(res, red);
  if (threadIdx.x == 0) atomicAdd(A.slots + (blockIdx.x % kSlots), (double)res);
}

// End of an iteration (one block): the residual is the sum of the slots plus the
// degree-zero vertices' closed-form share; the next constant term follows from the
// dangling mass D, which degree-zero vertices hold as count x constant.
__global__ void __launch_bounds__(kThreads) k_pr_finalize(const __grid_constant__ PrArgs A,
                                                          int iter, int dangling) {
  __shared__ double rd[kThreads / 32];
  double a = 0;
  for (uint32_t i = threadIdx.x; i < kSlots; i += kThreads) {
    a += A.slots[i];
    A.slots[i] = 0.0;
  }
  a = block_sum<double>(a, rd);
  if (threadIdx.x == 0) {
    a += A.slots[kSlots];
    A.slots[kSlots] = 0.0;
    const double zr = A.scal[0];  // rank every degree-zero vertex now holds
    a += A.nzero * fabs(zr - A.scal[3]);
    const double D = dangling ? A.nzero * zr : 0.0;
    const double base = (1.0 - A.damping) / A.n + A.damping * D / A.n;
    A.scal[1] = D;
    A.scal[2] = a;
    A.scal[3] = zr;
    A.scal[0] = base;
    ((float*)(A.scal + 4))[0] = (float)base;
    A.resid[iter] = a;
  }
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

template <class PR, bool MULTI>
__global__ void k_pr_init(const __grid_constant__ PrArgs A, uint32_t nv0, uint32_t ntot,
                          const __grid_constant__ MultiArgs M) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntot) return;
  const int p = i < nv0 ? 0 : 1;
  const uint32_t v = p == 0 ? i : i - nv0;
  const PrSide& S = A.side[p];
  using AT = typename PR::AT;
  // r_0 = 1/n (MULTI: 1/n_g of the vertex's component)
  const AT r0 = MULTI ? (AT)(1.0 / (double)((const AT*)M.nf)[M.gix[p][v]]) : (AT)(1.0 / A.n);
  ((typename PR::RT*)S.r)[v] = (typename PR::RT)r0;
  const int deg = (int)(S.P.off[v + 1] - S.P.off[v]);
  typename PR::XT* x = (typename PR::XT*)S.x;
  if (deg > 0) {
    if (PR::SCALED) XConv<typename PR::XT>::store(x + v, (AT)1 / (AT)deg);
    else XConv<typename PR::XT>::store(x + v, r0 / (AT)deg);
  } else {
    XConv<typename PR::XT>::store(x + v, (AT)0);
  }
}

// Ranks in global order: thread i reads vertex i's local rank through g2l, so the writes
// (possibly over the host link) are coalesced.
template <class RT>
__global__ void k_pr_collect(const __grid_constant__ PrArgs A, uint32_t n, const uint32_t* g2l,
                             double* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t gl = g2l[i];
  out[i] = (double)((const RT*)A.side[gl >> 31].r)[gl & kIdMask];
}

// Threads per vertex (log2) of a class-c tile: kLeafEdges >> (c-1) vertices share the
// CTA's kThreads threads, so every vertex gets 2^(c-3) of them (one round, 4 to 8 edges
// per thread); classes 1-3 take one thread per vertex.
inline int leaf_gshift(int c) { return std::max(0, c - 3); }

// Work items of the partitions in `parts` (bit p: partition p).
PrPlan make_plan(graph* g, int parts = 3) {
  PrPlan pl;
  memset(&pl, 0, sizeof(pl));
  auto add = [&](uint32_t count_items, uint32_t first, uint32_t end, uint32_t per, int kind,
                 int part, int gshift) {
    if (count_items == 0) return;
    PrRange& R = pl.r[pl.nr++];
    R.item0 = pl.nitems;
    R.first = first;
    R.end = end;
    R.per = per;
    R.kind = (uint8_t)kind;
    R.part = (uint8_t)part;
    R.gshift = (uint8_t)gshift;
    pl.nitems += count_items;
  };
  for (int p = 0; p < 2; ++p) {
    if (!(parts & (1 << p))) continue;
    const Part& P = g->part[p];
    pl.hub_item0[p] = pl.nitems;
    add(P.nchunk, 0, P.nchunk, 1, kItemHub, p, 8);
    for (int c = kClassHub - 1; c >= 1; --c) {
      const uint32_t v0 = P.cls_end[c + 1], v1 = P.cls_end[c];
      // one round of the CTA's threads: at most kThreads >> gshift vertices
      const uint32_t per = std::min<uint32_t>(std::max<uint32_t>(1u, (uint32_t)kLeafEdges >> (c - 1)),
                                              (uint32_t)kPrTileV >> leaf_gshift(c));
      add((v1 - v0 + per - 1) / per, v0, v1, per, kItemLeaf, p, leaf_gshift(c));
    }
    const uint32_t z0 = P.cls_end[1], z1 = P.nv;
    add((z1 - z0 + kTileV - 1) / kTileV, z0, z1, kTileV, kItemZero, p, 0);
  }
  return pl;
}

// The kernel's 8 resident CTAs per SM need only part of the SM's 228 KB of shared
// memory; the carveout hint leaves the rest to the L1 cache, which keeps the most-gathered
// contributions (those of the highest-degree vertices) close to the SM.
template <class PR, bool MULTI>
graph_status prepare_kernel() {
  static bool done = false;
  if (!done) {
    auto fn = k_pr_compute<PR, MULTI>;
    const int smem = (int)smem_bytes<PR>();
    GG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int pct = (int)((100.0 * 8 * (smem + 1024) + 228.0 * 1024 - 1) / (228.0 * 1024));
    GG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 std::min(100, pct)));
    done = true;
  }
  return GRAPH_OK;
}

graph_status alloc_ws(graph* g, int prec, int max_iter) {
  const size_t es = prec == GRAPH_PR_FP64 ? 8 : (prec == GRAPH_PR_FP16 ? 2 : 4);
  const size_t rs = prec == GRAPH_PR_FP64 ? 8 : 4;
  if (g->pr && (g->pr->prec != prec || g->pr->max_iter < max_iter)) free_pr(g);
  if (g->pr) return GRAPH_OK;
  PrWs* w = new PrWs();
  g->pr = w;
  w->prec = prec;
  w->esize = es;
  w->rsize = rs;
  w->max_iter = max_iter;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    GG_TRY(dalloc(g, w->r[p], rs * ((size_t)P.nv + 8)));  // bulk copies read 16-B granules
    GG_TRY(dalloc(g, w->x[p][0], es * P.nv));
    GG_TRY(dalloc(g, w->x[p][1], es * P.nv));
    GG_TRY(dalloc(g, w->ghost[p], es * P.nout));
  }
  GG_TRY(dalloc(g, w->slots, sizeof(double) * (kSlots + 1)));
  GG_TRY(dalloc(g, w->scal, 8 * sizeof(double)));
  GG_TRY(dalloc(g, w->resid, sizeof(double) * (size_t)(max_iter + 1)));
  return GRAPH_OK;
}

// A failed allocation leaves no half-built workspace behind for the next call.
graph_status ensure_ws(graph* g, int prec, int max_iter) {
  const graph_status s = alloc_ws(g, prec, max_iter);
  if (s != GRAPH_OK) free_pr(g);
  return s;
}

PrArgs make_args(graph* g, int cur, double damping);

// Resolves the plan's work items once per workspace (the partition and the plan do not
// change while the workspace lives).
template <class PR>
graph_status prepare_items(graph* g, PrWs* w, const PrPlan& pl, int parts = 3) {
  if ((w->items_n == pl.nitems && w->items_parts == parts) || pl.nitems == 0) return GRAPH_OK;
  dfree(g, w->items);
  dfree(g, w->hubsum);
  w->items_n = 0;
  w->items_parts = parts;
  GG_TRY(dalloc(g, w->items, sizeof(PrItem) * (size_t)pl.nitems));
  GG_TRY(dalloc(g, w->hubsum, sizeof(typename PR::AT) * kHubParts * (size_t)pl.nitems));
  k_pr_items<<<grid_for(pl.nitems, 256), 256, 0, g->stream>>>(pl, make_args(g, 0, 0.85),
                                                              (PrItem*)w->items.p);
  GG_CUDA(cudaGetLastError());
  w->items_n = pl.nitems;
  return GRAPH_OK;
}

PrArgs make_args(graph* g, int cur, double damping) {
  PrWs* w = g->pr;
  PrArgs A;
  memset(&A, 0, sizeof(A));
  uint64_t zero = 0;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    PrSide& S = A.side[p];
    S.P = P.view();
    S.r = w->r[p].p;
    S.x = w->x[p][cur].p;
    S.xn = w->x[p][1 - cur].p;
    S.ghost = w->ghost[p].p;
    zero += P.nv - P.cls_end[1];
  }
  A.scal = (double*)w->scal.p;
  A.slots = (double*)w->slots.p;
  A.items = (const PrItem*)w->items.p;
  A.hubsum = w->hubsum.p;
  A.resid = (double*)w->resid.p;
  A.damping = damping;
  A.n = (double)g->n;
  A.damping_f = (float)damping;
  A.n_f = (float)g->n;
  A.d_over_n_f = (float)(damping / (double)g->n);
  A.nzero = (double)zero;
  A.err = (int*)g->err.p;
  for (int p = 0; p < 2; ++p) A.e_host[p] = g->part[p].E.host != nullptr;
  return A;
}

template <class PR>
graph_status run(graph* g, const pagerank_attr& at, double* ranks, graph_stats* stats) {
  cudaStream_t st = g->stream;
  // Segmented neighbour sums (pr_seg.cu) when asked for (FP32 and FP16); the per-edge
  // gather kernel otherwise (GRAPH_PR_AUTO: it is the faster of the two on this GPU).
  constexpr bool kSegCapable = sizeof(typename PR::AT) == 4;
  bool seg = false;
  if (at.method == GRAPH_PR_SEGMENTED && !kSegCapable) {
    set_error("the segmented method needs FP32 or FP16 precision");
    return GRAPH_EINVAL;
  }
  if (kSegCapable && at.method == GRAPH_PR_SEGMENTED) {
    const SegParams prm{at.seg_log2, at.seg_chunk, at.seg_bin};
    GG_TRY(seg_prepare(g, prm, &seg));
    if (!seg && at.method == GRAPH_PR_SEGMENTED) {
      set_error("the graph exceeds a limit of the segmented layout");
      return GRAPH_EINVAL;
    }
  }
  const PrPlan pl = make_plan(g);
  if (!seg) GG_TRY((prepare_kernel<PR, false>()));
  GG_TRY(ensure_ws(g, at.precision, at.max_iter));
  PrWs* w = g->pr;
  if (!seg) GG_TRY(prepare_items<PR>(g, w, pl));
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  const uint32_t nv0 = g->part[0].nv;
  int cur = 0;
  GG_CUDA(cudaMemsetAsync(w->slots.p, 0, sizeof(double) * (kSlots + 1), st));
  {
    PrArgs A = make_args(g, cur, at.damping);
    k_pr_init<PR, false><<<grid_for(g->n, 256), 256, 0, st>>>(A, nv0, g->n, MultiArgs{});
    GG_CUDA(cudaGetLastError());
    // D_0 = (number of degree-zero vertices) / n; degree-zero vertices start at 1/n.
    const double D0 = at.dangling ? A.nzero / (double)g->n : 0.0;
    const double base = (1.0 - at.damping) / (double)g->n + at.damping * D0 / (double)g->n;
    double h[5] = {base, D0, 0.0, 1.0 / (double)g->n, 0.0};
    const float bf = (float)base;
    memcpy(&h[4], &bf, sizeof(float));
    GG_CUDA(cudaMemcpyAsync(w->scal.p, h, sizeof(h), cudaMemcpyHostToDevice, st));
    GG_CUDA(cudaStreamSynchronize(st));
  }
  const uint32_t nout = g->part[0].nout + g->part[1].nout;
  const uint32_t nhubs = g->part[0].nhub + g->part[1].nhub;
  const size_t smem = smem_bytes<PR>();
  const int seg_launches = seg ? seg_launches_per_iter(g) : 0;
  int it = 0;
  int64_t launches = 1;
  double last_res = 0;
  for (; it < at.max_iter;) {
    PrArgs A = make_args(g, cur, at.damping);
    timer.mark(2);
    if (nout) k_pr_publish<typename PR::XT><<<grid_for(nout, 256), 256, 0, st>>>(A);
    timer.mark(1);
    if (seg) {
      SegIter si;
      for (int p = 0; p < 2; ++p) {
        si.x[p] = A.side[p].x;
        si.ghost[p] = A.side[p].ghost;
        si.xn[p] = A.side[p].xn;
        si.r[p] = A.side[p].r;
      }
      si.scal = A.scal;
      si.slots = A.slots;
      si.nslots = kSlots;
      si.d = A.damping_f;
      si.d_over_n = A.d_over_n_f;
      si.n = A.n_f;
      si.fp16 = PR::SCALED;
      GG_TRY(seg_launch(g, si));
      k_pr_finalize<<<1, kThreads, 0, st>>>(A, it, at.dangling);
      launches += (nout ? 1 : 0) + seg_launches + 1;
    } else {
      if (pl.nitems) {
        k_pr_compute<PR, false><<<pl.nitems, kThreads, smem, st>>>(pl, A, it, at.dangling,
                                                                   MultiArgs{});
        if (nhubs)
          k_pr_hubs<PR, false><<<grid_for(nhubs, kThreads / 32), kThreads, 0, st>>>(pl, A, it,
                                                                                     MultiArgs{});
        k_pr_finalize<<<1, kThreads, 0, st>>>(A, it, at.dangling);
      }
      launches += (nout ? 1 : 0) + (pl.nitems ? 2 : 0) + (pl.nitems && nhubs ? 1 : 0);
    }
    timer.mark(0);
    GG_CUDA(cudaGetLastError());
    cur = 1 - cur;
    ++it;
    if (at.tol > 0) {
      GG_CUDA(cudaMemcpyAsync(&last_res, (double*)w->scal.p + 2, 8, cudaMemcpyDeviceToHost, st));
      GG_CUDA(cudaStreamSynchronize(st));
      if (last_res < at.tol) break;
    }
  }
  void* out = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, ranks, at.out_mem, 8ull * g->n, 0, &out, &staged));
  {
    PrArgs A = make_args(g, cur, at.damping);
    k_pr_collect<typename PR::RT><<<grid_for(g->n, 256), 256, 0, st>>>(
        A, g->n, (const uint32_t*)g->g2l.p, (double*)out);
    GG_CUDA(cudaGetLastError());
    launches++;
  }
  if (staged) GG_TRY(deliver(g, ranks, out, 8ull * g->n, GRAPH_MEM_HOST));
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

// ---------------------------------------------------------------------------------------
// pagerank_multi: components given as global-id ranges [vbase[c], vbase[c+1]).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t component_of(const uint32_t* vbase, uint32_t G, uint32_t v) {
  uint32_t lo = 0, hi = G;  // vbase[lo] <= v < vbase[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (vbase[mid] <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One warp per vertex u (grid stride): every neighbour must lie in u's component; counts
// the degree-zero vertices of each component. bad != 0 if an edge crosses components.
__global__ void k_multi_validate(const int64_t* off, const uint32_t* col, uint32_t n,
                                 const uint32_t* vbase, uint32_t G, uint32_t* nzero, int* bad) {
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t u = w0; u < n; u += nw) {
    const uint32_t c = component_of(vbase, G, u);
    const uint32_t lo = vbase[c], hi = vbase[c + 1];
    const int64_t e0 = off[u], e1 = off[u + 1];
    if (e0 == e1) {
      if (lane_id() == 0) atomicAdd(nzero + c, 1u);
      continue;
    }
    bool out = false;
    for (int64_t e = e0 + lane_id(); e < e1; e += 32) {
      const uint32_t x = col[e];
      out |= x < lo || x >= hi;
    }
    if (__any_sync(kFull, out) && lane_id() == 0) atomicOr(bad, 1);
  }
}

__global__ void k_multi_gix(const uint32_t* l2g, uint32_t nv, const uint32_t* vbase, uint32_t G,
                            uint32_t* gix) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) gix[v] = component_of(vbase, G, l2g[v]);
}

// Validates the component layout (once per layout and workspace) and builds the
// per-vertex component ids.
graph_status prepare_multi(graph* g, PrWs* w, uint32_t G, const uint32_t* vbase) {
  if (!w->multi) w->multi = new MultiWs();
  MultiWs* m = w->multi;
  if (m->vbase.size() == (size_t)G + 1 && memcmp(m->vbase.data(), vbase, 4ull * (G + 1)) == 0)
    return GRAPH_OK;
  cudaStream_t st = g->stream;
  m->vbase.clear();
  m->nzero.assign(G, 0);
  if (m->exec) {
    cudaGraphExecDestroy(m->exec);
    m->exec = nullptr;
    m->iters = 0;
  }
  DevBuf* old[] = {&m->dvbase, &m->dnzero, &m->gix[0], &m->gix[1], &m->dn, &m->nf, &m->res};
  for (DevBuf* b : old) dfree(g, *b);
  GG_TRY(dalloc(g, m->dvbase, 4ull * (G + 1)));
  GG_TRY(dalloc(g, m->dnzero, 4ull * G));
  GG_TRY(dalloc(g, m->dn, 8ull * G));
  GG_TRY(dalloc(g, m->nf, 8ull * G));
  GG_TRY(dalloc(g, m->res, 8ull * G));
  for (int p = 0; p < 2; ++p) GG_TRY(dalloc(g, m->gix[p], 4ull * g->part[p].nv));
  GG_CUDA(cudaMemcpyAsync(m->dvbase.p, vbase, 4ull * (G + 1), cudaMemcpyHostToDevice, st));
  GG_CUDA(cudaMemsetAsync(m->dnzero.p, 0, 4ull * G, st));
  GG_CUDA(cudaMemsetAsync(g->err.p, 0, sizeof(int), st));
  int* bad = (int*)g->err.p;
  k_multi_validate<<<152 * 8, 256, 0, st>>>((const int64_t*)g->off.p, (const uint32_t*)g->col.p,
                                            g->n, (const uint32_t*)m->dvbase.p, G,
                                            (uint32_t*)m->dnzero.p, bad);
  GG_CUDA(cudaGetLastError());
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    if (P.nv == 0) continue;
    k_multi_gix<<<grid_for(P.nv, 256), 256, 0, st>>>((const uint32_t*)P.l2g.p, P.nv,
                                                     (const uint32_t*)m->dvbase.p, G,
                                                     (uint32_t*)m->gix[p].p);
    GG_CUDA(cudaGetLastError());
  }
  int hbad = 0;
  GG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaMemcpyAsync(m->nzero.data(), m->dnzero.p, 4ull * G, cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  if (hbad) {
    GG_CUDA(cudaMemsetAsync(g->err.p, 0, sizeof(int), st));
    GG_CUDA(cudaStreamSynchronize(st));
    set_error("an edge joins two components of vbase");
    return GRAPH_EINVAL;
  }
  m->vbase.assign(vbase, vbase + G + 1);
  return GRAPH_OK;
}

template <class PR>
graph_status run_multi(graph* g, uint32_t G, const uint32_t* vbase, const pagerank_attr& at,
                       double* ranks, double* residuals, graph_stats* stats) {
  using AT = typename PR::AT;
  cudaStream_t st = g->stream;
  const PrPlan pl = make_plan(g);
  GG_TRY((prepare_kernel<PR, true>()));
  GG_TRY(ensure_ws(g, at.precision, at.max_iter));
  PrWs* w = g->pr;
  GG_TRY(prepare_items<PR>(g, w, pl));
  {
    const graph_status s = prepare_multi(g, w, G, vbase);
    if (s != GRAPH_OK) {
      free_multi(g, w);
      return s;
    }
  }
  MultiWs* m = w->multi;
  const int K = at.max_iter;
  // Per-component constants, FP64 on the host. A degree-zero vertex has an empty neighbour
  // sum, so it holds the constant term base_t itself; the dangling mass is therefore
  // D_{t+1} = nzero_c base_t and base_{t+1} = (1-d)/n_c + d D_{t+1}/n_c, from D_0 =
  // nzero_c / n_c (ranks start at 1/n_c).
  const double d = at.damping;
  std::vector<AT> hbase((size_t)K * G), hdn(G), hnf(G);
  std::vector<double> zres(G, 0.0);
  for (uint32_t c = 0; c < G; ++c) {
    const double nc = (double)(vbase[c + 1] - vbase[c]);
    hdn[c] = (AT)(nc > 0 ? d / nc : 0.0);
    hnf[c] = (AT)nc;
    if (nc == 0) continue;
    double D = at.dangling ? m->nzero[c] / nc : 0.0, prev = 1.0 / nc, base = 0;
    for (int t = 0; t < K; ++t) {
      base = (1.0 - d) / nc + d * D / nc;
      hbase[(size_t)t * G + c] = (AT)base;
      if (t == K - 1) zres[c] = m->nzero[c] * fabs(base - prev);
      prev = base;
      D = at.dangling ? m->nzero[c] * base : 0.0;
    }
  }
  const size_t bb = sizeof(AT) * (size_t)K * G;
  if (m->base_bytes < bb) {
    dfree(g, m->base);
    GG_TRY(dalloc(g, m->base, bb));
    m->base_bytes = bb;
    if (m->exec) {
      cudaGraphExecDestroy(m->exec);
      m->exec = nullptr;
      m->iters = 0;
    }
  }
  GG_CUDA(cudaMemcpyAsync(m->base.p, hbase.data(), bb, cudaMemcpyHostToDevice, st));
  GG_CUDA(cudaMemcpyAsync(m->dn.p, hdn.data(), sizeof(AT) * G, cudaMemcpyHostToDevice, st));
  GG_CUDA(cudaMemcpyAsync(m->nf.p, hnf.data(), sizeof(AT) * G, cudaMemcpyHostToDevice, st));
  GG_CUDA(cudaMemsetAsync(m->res.p, 0, 8ull * G, st));
  MultiArgs M;
  memset(&M, 0, sizeof(M));
  for (int p = 0; p < 2; ++p) M.gix[p] = (const uint32_t*)m->gix[p].p;
  M.base = m->base.p;
  M.dn = m->dn.p;
  M.nf = m->nf.p;
  M.res = (double*)m->res.p;
  M.G = G;
  PhaseTimer timer;
  timer.start(at.timing != 0 && stats != nullptr, st);
  timer.mark(2);
  const uint32_t nv0 = g->part[0].nv;
  k_pr_init<PR, true><<<grid_for(g->n, 256), 256, 0, st>>>(make_args(g, 0, d), nv0, g->n, M);
  GG_CUDA(cudaGetLastError());
  timer.mark(2);
  // The K supersteps (publish + compute) as one CUDA graph, captured on a private stream
  // and replayed while the layout, the workspace, K and the damping stay the same.
  const uint32_t nhubs = g->part[0].nhub + g->part[1].nhub;
  const uint32_t nout = g->part[0].nout + g->part[1].nout;
  const size_t smem = smem_bytes<PR>();
  if (!m->exec || m->iters != K || m->damping != d || m->dangling != at.dangling) {
    if (m->exec) cudaGraphExecDestroy(m->exec);
    m->exec = nullptr;
    if (!m->capture) GG_CUDA(cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking));
    GG_CUDA(cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeThreadLocal));
    int cur = 0;
    for (int it = 0; it < K; ++it) {
      const PrArgs A = make_args(g, cur, d);
      M.last = it == K - 1;
      if (nout) k_pr_publish<typename PR::XT><<<grid_for(nout, 256), 256, 0, m->capture>>>(A);
      if (pl.nitems)
        k_pr_compute<PR, true><<<pl.nitems, kThreads, smem, m->capture>>>(pl, A, it,
                                                                          at.dangling, M);
      if (pl.nitems && nhubs)
        k_pr_hubs<PR, true><<<grid_for(nhubs, kThreads / 32), kThreads, 0, m->capture>>>(
            pl, A, it, M);
      cur = 1 - cur;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(m->capture, &graph);
    if (ce != cudaSuccess) return cuda_fail(ce, "capture of the iterations", __FILE__, __LINE__);
    const cudaError_t ie = cudaGraphInstantiate(&m->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      m->exec = nullptr;
      return cuda_fail(ie, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    m->iters = K;
    m->damping = d;
    m->dangling = at.dangling;
  }
  GG_CUDA(cudaGraphLaunch(m->exec, st));
  timer.mark(0);
  void* out = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, ranks, at.out_mem, 8ull * g->n, 0, &out, &staged));
  k_pr_collect<typename PR::RT><<<grid_for(g->n, 256), 256, 0, st>>>(
      make_args(g, K & 1, d), g->n, (const uint32_t*)g->g2l.p, (double*)out);
  GG_CUDA(cudaGetLastError());
  if (staged) GG_TRY(deliver(g, ranks, out, 8ull * g->n, GRAPH_MEM_HOST));
  std::vector<double> hres(G);
  GG_CUDA(cudaMemcpyAsync(hres.data(), m->res.p, 8ull * G, cudaMemcpyDeviceToHost, st));
  timer.mark(2);
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  double total = 0;
  for (uint32_t c = 0; c < G; ++c) {
    hres[c] += zres[c];
    total += hres[c];
  }
  if (residuals) memcpy(residuals, hres.data(), 8ull * G);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = K;
    stats->edges_traversed = g->m * (int64_t)K;
    stats->edges_inspected = g->m * (int64_t)K;
    stats->messages = (int64_t)nout * K;
    stats->residual = total;
    stats->launches =
        2 + (int64_t)K * ((nout ? 1 : 0) + (pl.nitems ? 1 : 0) + (pl.nitems && nhubs ? 1 : 0));
  }
  timer.finish(stats);
  return s;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// pagerank_hybrid: the paper's hybrid placement (Section 4.1, Figure 6; Section 6.2, HIGH).
// Partition 0 (the high-degree vertices) is updated by host threads from host copies of
// its arrays while the GPU updates partition 1 with the kernels above. Every superstep
// moves only the message arrays across the host/device boundary (Section 4.3.2):
// partition 0's ghost slots come down from the device, partition 1's go up.
// ---------------------------------------------------------------------------------------
struct HybWs {
  std::vector<int64_t> off0;      // partition 0: offsets and edge ids (host copies)
  std::vector<uint32_t> E0;
  std::vector<uint32_t> outbox1;  // partition 1's outbox: partition-0 local ids it pulls
  std::vector<uint32_t> cut;      // host threads' vertex ranges, balanced by edge count
  size_t vsize = 0;               // bytes of one rank / contribution
  std::vector<unsigned char> r0, x0[2];
  void* ghost0 = nullptr;         // pinned [nout0]: partition 0's ghost slots
  void* ghost1 = nullptr;         // pinned [nout1]: partition 1's ghost slots
  double* io = nullptr;           // pinned [2]: host residual out, device residual in
  cudaEvent_t ev[5] = {};         // ghost0 landed, compute start / end, exchange start / end
};

void free_hyb(PrWs* w) {
  HybWs* h = w->hyb;
  if (!h) return;
  if (h->ghost0) cudaFreeHost(h->ghost0);
  if (h->ghost1) cudaFreeHost(h->ghost1);
  if (h->io) cudaFreeHost(h->io);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
  w->hyb = nullptr;
}

namespace {

// Runs f(k, begin, end) on nt host threads over [0, n) split evenly, or over the ranges
// [cut[k], cut[k+1]) when cut is given. A thread that cannot be started runs its range on
// the calling thread, so no exception leaves while other threads are running.
template <class F>
void host_parallel(int nt, uint32_t n, const std::vector<uint32_t>* cut, F&& f) {
  if (n == 0 || nt < 1) return;
  auto lo = [&](int k) {
    return cut ? (*cut)[k] : (uint32_t)((uint64_t)n * (uint64_t)k / (uint64_t)nt);
  };
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int k = 1; k < nt; ++k) {
    try {
      th.emplace_back(f, k, lo(k), lo(k + 1));
    } catch (...) {
      f(k, lo(k), lo(k + 1));
    }
  }
  f(0, lo(0), lo(1));
  for (auto& t : th) t.join();
}

// Host copies of partition 0's CSR and of partition 1's outbox (once per partition), the
// per-precision host arrays and pinned message buffers, and the threads' vertex ranges.
template <class T>
graph_status ensure_hyb(graph* g, PrWs* w, int nt) {
  const Part& P0 = g->part[0];
  const Part& P1 = g->part[1];
  cudaStream_t st = g->stream;
  if (!w->hyb) {
    HybWs* h = new HybWs();
    w->hyb = h;
    h->off0.resize((size_t)P0.nv + 1);
    h->E0.resize((size_t)P0.ne);
    h->outbox1.resize(P1.nout);
    GG_CUDA(cudaMemcpyAsync(h->off0.data(), P0.off.p, 8ull * (P0.nv + 1),
                            cudaMemcpyDeviceToHost, st));
    if (P0.ne)
      GG_CUDA(cudaMemcpyAsync(h->E0.data(), P0.E.p, 4ull * P0.ne, cudaMemcpyDefault, st));
    if (P1.nout)
      GG_CUDA(cudaMemcpyAsync(h->outbox1.data(), P1.outbox.p, 4ull * P1.nout,
                              cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    for (cudaEvent_t& e : h->ev) GG_CUDA(cudaEventCreate(&e));
    if (cudaHostAlloc((void**)&h->io, 2 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
      h->io = nullptr;
      set_error("pinned host allocation failed");
      return GRAPH_ENOMEM;
    }
  }
  HybWs* h = w->hyb;
  if (h->vsize != sizeof(T)) {
    if (h->ghost0) cudaFreeHost(h->ghost0);
    if (h->ghost1) cudaFreeHost(h->ghost1);
    h->ghost0 = h->ghost1 = nullptr;
    h->vsize = 0;
    const size_t b0 = sizeof(T) * std::max<size_t>(1, P0.nout);
    const size_t b1 = sizeof(T) * std::max<size_t>(1, P1.nout);
    if (cudaHostAlloc(&h->ghost0, b0, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&h->ghost1, b1, cudaHostAllocDefault) != cudaSuccess) {
      set_error("pinned host allocation of the message arrays failed");
      return GRAPH_ENOMEM;
    }
    h->r0.assign(sizeof(T) * (size_t)P0.nv, 0);
    for (auto& x : h->x0) x.assign(sizeof(T) * (size_t)P0.nv, 0);
    h->vsize = sizeof(T);
  }
  if ((int)h->cut.size() != nt + 1) {
    // Thread k takes the vertices whose first edge lies in [k ne / nt, (k+1) ne / nt).
    h->cut.assign(nt + 1, P0.nv);
    h->cut[0] = 0;
    for (int k = 1; k < nt; ++k) {
      const int64_t e = P0.ne * (int64_t)k / nt;
      h->cut[k] = (uint32_t)(std::lower_bound(h->off0.begin(), h->off0.begin() + P0.nv, e) -
                             h->off0.begin());
    }
    for (int k = 1; k <= nt; ++k) h->cut[k] = std::max(h->cut[k], h->cut[k - 1]);
  }
  return GRAPH_OK;
}

// One superstep of partition 0 on the host: the vertex update of update_vertex in the
// same precision (T = float: FP32 constant term, damping and sums; T = double: FP64).
// The neighbour sum is pairwise over blocks of kHostBlock edges in CSR order: a block is
// summed as four interleaved partial sums (four independent chains of loads), and the
// block sums are merged like a binary counter, so a hub with many edges sees a rounding
// chain of about log2(blocks) additions, not one per edge. (A sequential FP32 sum over
// 20,000 edges is off by ~1e-6 relative in each iteration, as the GPU's chunked tree is
// not.) Degree-zero vertices take the constant term (their residual is the closed form
// k_pr_finalize adds). Returns sum |r' - r| over the vertices with edges.
constexpr int kHostBlock = 32;

template <class T>
double host_update(const HybWs& h, uint32_t v0, uint32_t v1, const T* x, const T* ghost,
                   T* r, T* xn, T base, T d) {
  auto val = [&](uint32_t id) { return (id & kRemote) ? ghost[id & kIdMask] : x[id]; };
  const uint32_t* E = h.E0.data();
  auto chunk_sum = [&](int64_t e, int64_t e1) {
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (; e + 4 <= e1; e += 4) {
      s0 += val(E[e]);
      s1 += val(E[e + 1]);
      s2 += val(E[e + 2]);
      s3 += val(E[e + 3]);
    }
    if (e < e1) s0 += val(E[e]);
    if (e + 1 < e1) s1 += val(E[e + 1]);
    if (e + 2 < e1) s2 += val(E[e + 2]);
    return (s0 + s1) + (s2 + s3);
  };
  double res = 0;
  for (uint32_t v = v0; v < v1; ++v) {
    const int64_t e0 = h.off0[v], e1 = h.off0[v + 1];
    if (e0 == e1) {
      r[v] = base;
      xn[v] = (T)0;
      continue;
    }
    T sum;
    if (e1 - e0 <= kHostBlock) {
      sum = chunk_sum(e0, e1);
    } else {
      T level[48];  // level[k]: sum of 2^k consecutive blocks still waiting for a partner
      uint64_t nb = 0;
      for (int64_t b = e0; b < e1; b += kHostBlock) {
        T t = chunk_sum(b, std::min(b + kHostBlock, e1));
        int k = 0;
        for (uint64_t c = nb; c & 1; c >>= 1, ++k) t = level[k] + t;
        level[k] = t;
        ++nb;
      }
      sum = 0;
      for (int k = 0; (nb >> k) != 0; ++k)
        if ((nb >> k) & 1) sum = level[k] + sum;
    }
    const T rn = base + d * sum;
    const T ro = r[v];
    r[v] = rn;
    xn[v] = rn / (T)(e1 - e0);
    res += (double)(rn > ro ? rn - ro : ro - rn);
  }
  return res;
}

template <class PR>
graph_status run_hybrid(graph* g, const pagerank_attr& at, int nt, double* ranks,
                        graph_stats* stats, pagerank_hybrid_info* info) {
  using T = typename PR::AT;
  using Clock = std::chrono::steady_clock;
  auto ms_since = [](Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
  };
  const auto t_start = Clock::now();
  cudaStream_t st = g->stream;
  const PrPlan pl = make_plan(g, 2);  // the GPU's share: partition 1
  GG_TRY((prepare_kernel<PR, false>()));
  GG_TRY(ensure_ws(g, at.precision, at.max_iter));
  PrWs* w = g->pr;
  GG_TRY(prepare_items<PR>(g, w, pl, 2));
  {
    graph_status s = GRAPH_OK;
    try {
      s = ensure_hyb<T>(g, w, nt);
    } catch (const std::bad_alloc&) {
      set_error("host allocation for the host partition failed");
      s = GRAPH_ENOMEM;
    }
    if (s != GRAPH_OK) {
      free_hyb(w);
      return s;
    }
  }
  HybWs* h = w->hyb;
  const uint32_t nv0 = g->part[0].nv, nout0 = g->part[0].nout, nout1 = g->part[1].nout;
  const uint32_t nhubs1 = g->part[1].nhub;
  const size_t vs = sizeof(T), smem = smem_bytes<PR>();
  const double n = (double)g->n, d = at.damping;
  int cur = 0;
  int64_t launches = 1;
  GG_CUDA(cudaMemsetAsync(w->slots.p, 0, sizeof(double) * (kSlots + 1), st));
  PrArgs A = make_args(g, cur, at.damping);
  k_pr_init<PR, false><<<grid_for(g->n, 256), 256, 0, st>>>(A, nv0, g->n, MultiArgs{});
  GG_CUDA(cudaGetLastError());
  // The constant term follows the scalar recurrence k_pr_finalize evaluates (D_0 =
  // nzero / n; after an iteration with constant c, D = nzero c), so the host keeps its own
  // bit-identical copy instead of reading it back.
  double D = at.dangling ? A.nzero / n : 0.0;
  double base = (1.0 - d) / n + d * D / n;
  {
    double hs[5] = {base, D, 0.0, 1.0 / n, 0.0};
    const float bf = (float)base;
    memcpy(&hs[4], &bf, sizeof(float));
    GG_CUDA(cudaMemcpyAsync(w->scal.p, hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  }
  T* r0 = (T*)h->r0.data();
  {
    const T rinit = (T)(1.0 / n);
    T* x = (T*)h->x0[cur].data();
    host_parallel(nt, nv0, nullptr, [&](int, uint32_t a, uint32_t b) {
      for (uint32_t v = a; v < b; ++v) {
        const int64_t deg = h->off0[v + 1] - h->off0[v];
        r0[v] = rinit;
        x[v] = deg > 0 ? rinit / (T)deg : (T)0;
      }
    });
  }
  GG_CUDA(cudaStreamSynchronize(st));
  double ms_cpu = 0, ms_gpu = 0, ms_xchg = 0, ms_comp = 0, last_res = 0;
  std::vector<double> part(nt);
  int it = 0;
  while (it < at.max_iter) {
    A = make_args(g, cur, at.damping);
    A.side[0].P.bstart[1] = 0;   // partition 0's hubs are updated on the host
    PrArgs Apub = A;
    Apub.side[1].P.nout = 0;     // the device fills only partition 0's ghost slots
    const T* xh = (const T*)h->x0[cur].data();
    T* xhn = (T*)h->x0[1 - cur].data();
    // Communication phase: partition 0's ghost slots down, partition 1's up.
    GG_CUDA(cudaEventRecord(h->ev[3], st));
    if (nout0) {
      k_pr_publish<T><<<grid_for(nout0, 256), 256, 0, st>>>(Apub);
      GG_CUDA(cudaMemcpyAsync(h->ghost0, w->ghost[0].p, vs * nout0, cudaMemcpyDeviceToHost,
                              st));
      ++launches;
    }
    GG_CUDA(cudaEventRecord(h->ev[0], st));
    if (nout1) {
      T* g1 = (T*)h->ghost1;
      host_parallel(nt, nout1, nullptr, [&](int, uint32_t a, uint32_t b) {
        for (uint32_t j = a; j < b; ++j) g1[j] = xh[h->outbox1[j]];
      });
      GG_CUDA(cudaMemcpyAsync(w->ghost[1].p, g1, vs * nout1, cudaMemcpyHostToDevice, st));
    }
    GG_CUDA(cudaEventRecord(h->ev[4], st));
    // Compute phase: the GPU's partition is queued, then the host updates its own.
    GG_CUDA(cudaEventRecord(h->ev[1], st));
    if (pl.nitems) {
      k_pr_compute<PR, false><<<pl.nitems, kThreads, smem, st>>>(pl, A, it, at.dangling,
                                                                 MultiArgs{});
      ++launches;
      if (nhubs1) {
        k_pr_hubs<PR, false><<<grid_for(nhubs1, kThreads / 32), kThreads, 0, st>>>(
            pl, A, it, MultiArgs{});
        ++launches;
      }
    }
    GG_CUDA(cudaEventRecord(h->ev[2], st));
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaEventSynchronize(h->ev[0]));
    const auto tc0 = Clock::now();
    const T* g0 = (const T*)h->ghost0;
    const T bT = (T)base, dT = (T)d;
    host_parallel(nt, nv0, &h->cut, [&](int k, uint32_t a, uint32_t b) {
      part[k] = host_update<T>(*h, a, b, xh, g0, r0, xhn, bT, dT);
    });
    double cres = 0;
    for (int k = 0; k < nt; ++k) cres += part[k];
    const auto tc1 = Clock::now();
    h->io[0] = cres;
    GG_CUDA(cudaMemcpyAsync((double*)w->slots.p + kSlots, h->io, sizeof(double),
                            cudaMemcpyHostToDevice, st));
    k_pr_finalize<<<1, kThreads, 0, st>>>(A, it, at.dangling);
    ++launches;
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(h->io + 1, (double*)w->scal.p + 2, sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaStreamSynchronize(st));
    last_res = h->io[1];
    float gms = 0, xms = 0;
    GG_CUDA(cudaEventElapsedTime(&gms, h->ev[1], h->ev[2]));
    GG_CUDA(cudaEventElapsedTime(&xms, h->ev[3], h->ev[4]));
    const double cms = ms_since(tc0, tc1);
    ms_cpu += cms;
    ms_gpu += gms;
    ms_xchg += xms;
    ms_comp += std::max(cms, (double)gms);
    D = at.dangling ? A.nzero * base : 0.0;
    base = (1.0 - d) / n + d * D / n;
    cur = 1 - cur;
    ++it;
    if (at.tol > 0 && last_res < at.tol) break;
  }
  // Collect: the host partition's ranks join the device's, then the usual local -> global
  // write.
  if (nv0)
    GG_CUDA(cudaMemcpyAsync(w->r[0].p, r0, vs * nv0, cudaMemcpyHostToDevice, st));
  void* out = nullptr;
  bool staged = false;
  GG_TRY(out_target(g, ranks, at.out_mem, 8ull * g->n, 0, &out, &staged));
  A = make_args(g, cur, at.damping);
  k_pr_collect<T><<<grid_for(g->n, 256), 256, 0, st>>>(A, g->n, (const uint32_t*)g->g2l.p,
                                                       (double*)out);
  GG_CUDA(cudaGetLastError());
  launches++;
  if (staged) GG_TRY(deliver(g, ranks, out, 8ull * g->n, GRAPH_MEM_HOST));
  GG_CUDA(cudaStreamSynchronize(st));
  const graph_status s = check_device_error(g);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->supersteps = it;
    stats->edges_traversed = g->m * (int64_t)it;
    stats->edges_inspected = g->m * (int64_t)it;
    stats->messages = (int64_t)(nout0 + nout1) * it;
    stats->residual = last_res;
    stats->launches = launches;
    if (at.timing) {
      stats->ms_total = ms_since(t_start, Clock::now());
      stats->ms_compute = ms_comp;
      stats->ms_exchange = ms_xchg;
    }
  }
  if (info) {
    info->cpu_threads = nt;
    info->cpu_vertices = nv0;
    info->gpu_vertices = g->part[1].nv;
    info->cpu_edges = g->part[0].ne;
    info->gpu_edges = g->part[1].ne;
    info->ms_cpu_compute = ms_cpu;
    info->ms_gpu_compute = ms_gpu;
    info->ms_exchange = ms_xchg;
  }
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
      (at.dangling != 0 && at.dangling != 1) || at.method < GRAPH_PR_AUTO ||
      at.method > GRAPH_PR_SEGMENTED) {
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

extern "C" graph_status pagerank_hybrid(graph_t* g, const pagerank_attr* attr, int cpu_threads,
                                        double* ranks, graph_stats* stats,
                                        pagerank_hybrid_info* info) {
  if (!g || !attr || !ranks) {
    set_error("graph, attr or ranks is NULL");
    return GRAPH_EINVAL;
  }
  const pagerank_attr at = *attr;
  if (!(at.damping >= 0.0 && at.damping <= 1.0) || at.max_iter < 1 ||
      (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) ||
      (at.dangling != 0 && at.dangling != 1) || cpu_threads > GRAPH_HYBRID_MAX_THREADS) {
    set_error("bad pagerank_hybrid attributes");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before pagerank_hybrid");
    return GRAPH_ESTATE;
  }
  int nt = cpu_threads;
  if (nt <= 0) nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()),
                                            (unsigned)GRAPH_HYBRID_MAX_THREADS);
  switch (at.precision) {
    case GRAPH_PR_FP32: return run_hybrid<PrecF32>(g, at, nt, ranks, stats, info);
    case GRAPH_PR_FP64: return run_hybrid<PrecF64>(g, at, nt, ranks, stats, info);
    default:
      set_error("pagerank_hybrid runs FP32 or FP64 (precision %d)", at.precision);
      return GRAPH_EINVAL;
  }
}

extern "C" graph_status pagerank_multi(graph_t* g, uint32_t ngraphs, const uint32_t* vbase,
                                       const pagerank_attr* attr, double* ranks,
                                       double* residuals, graph_stats* stats) {
  if (!g || !attr || !ranks || !vbase || ngraphs == 0) {
    set_error("graph, vbase, attr or ranks is NULL, or ngraphs is 0");
    return GRAPH_EINVAL;
  }
  if (vbase[0] != 0 || vbase[ngraphs] != g->n) {
    set_error("vbase must start at 0 and end at n = %u", g->n);
    return GRAPH_EINVAL;
  }
  for (uint32_t c = 0; c < ngraphs; ++c)
    if (vbase[c + 1] < vbase[c]) {
      set_error("vbase decreases at %u", c);
      return GRAPH_EINVAL;
    }
  const pagerank_attr at = *attr;
  if (!(at.damping >= 0.0 && at.damping <= 1.0) || at.max_iter < 1 || at.tol != 0.0 ||
      (at.out_mem != GRAPH_MEM_HOST && at.out_mem != GRAPH_MEM_DEVICE) ||
      (at.dangling != 0 && at.dangling != 1)) {
    set_error("bad pagerank_multi attributes (tol must be 0: fixed iteration count)");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph_partition must run before pagerank_multi");
    return GRAPH_ESTATE;
  }
  switch (at.precision) {
    case GRAPH_PR_FP32: return run_multi<PrecF32>(g, ngraphs, vbase, at, ranks, residuals, stats);
    case GRAPH_PR_FP64: return run_multi<PrecF64>(g, ngraphs, vbase, at, ranks, residuals, stats);
    case GRAPH_PR_FP16: return run_multi<PrecF16>(g, ngraphs, vbase, at, ranks, residuals, stats);
    default:
      set_error("bad precision %d", at.precision);
      return GRAPH_EINVAL;
  }
}
