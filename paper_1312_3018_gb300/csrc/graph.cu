// Graph load (device CSR, Section 4.3.1) and the two-way partition with per-partition CSR,
// local-first neighbour order, boundary edges as outbox indices, and outbox/inbox lists
// (Section 4.3.1-4.3.2, Figure 6), assigned by degree (Section 6.2-6.3.1).
#include <stdarg.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace gg {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

graph_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) return GRAPH_ENOMEM;
  return GRAPH_ECUDA;
}

graph_status dalloc(graph* g, DevBuf& b, size_t bytes) {
  b.p = nullptr;
  b.bytes = bytes;
  if (bytes == 0) bytes = 16;
  // Round up so that bulk copies may read whole 16-byte granules at the tail.
  bytes = (bytes + 255) & ~(size_t)255;
  b.bytes = bytes;
  if (g->rt.alloc) {
    b.p = g->rt.alloc(bytes, g->rt.ctx);
    if (!b.p) {
      set_error("caller allocator returned NULL for %zu bytes", bytes);
      return GRAPH_ENOMEM;
    }
    if (((uintptr_t)b.p & 255) != 0) {
      g->rt.free(b.p, bytes, g->rt.ctx);
      b.p = nullptr;
      set_error("caller allocator returned memory not aligned to 256 bytes");
      return GRAPH_EINVAL;
    }
    return GRAPH_OK;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return GRAPH_ENOMEM;
  }
  return GRAPH_OK;
}

void dfree(graph* g, DevBuf& b) {
  if (b.host) {
    cudaFreeHost(b.host);
    b = DevBuf();
    return;
  }
  if (!b.p) return;
  if (g->rt.free) g->rt.free(b.p, b.bytes, g->rt.ctx);
  else if (!g->rt.alloc) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

graph_status ensure_host_counters(graph* g, size_t bytes) {
  if (g->host_counters_bytes >= bytes) return GRAPH_OK;
  if (g->host_counters) cudaFreeHost(g->host_counters);
  g->host_counters = nullptr;
  g->host_counters_bytes = 0;
  GG_CUDA(cudaMallocHost(&g->host_counters, bytes));
  g->host_counters_bytes = bytes;
  return GRAPH_OK;
}

graph_status ensure_stage(graph* g, size_t bytes) {
  if (g->stage.bytes >= bytes && g->stage.p) return GRAPH_OK;
  dfree(g, g->stage);
  return dalloc(g, g->stage, bytes);
}

graph_status check_device_error(graph* g) {
  int flag = 0;
  GG_CUDA(cudaMemcpyAsync(&flag, g->err.p, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  GG_CUDA(cudaStreamSynchronize(g->stream));
  if (flag) {
    cudaMemsetAsync(g->err.p, 0, sizeof(int), g->stream);
    set_error("a bounded device wait expired (device error flag %d)", flag);
    return GRAPH_ETIMEOUT;
  }
  return GRAPH_OK;
}

graph_status deliver(graph* g, void* dst, const void* dev_src, size_t bytes, int out_mem) {
  if (bytes == 0) return GRAPH_OK;
  if (out_mem == GRAPH_MEM_DEVICE) {
    if (dst != dev_src)
      GG_CUDA(cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToDevice, g->stream));
  } else {
    GG_CUDA(cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToHost, g->stream));
  }
  return GRAPH_OK;
}

graph_status out_target(graph* g, void* dst, int out_mem, size_t stage_bytes, size_t stage_off,
                        void** target, bool* staged) {
  *staged = false;
  *target = dst;
  if (out_mem == GRAPH_MEM_DEVICE) return GRAPH_OK;
  cudaPointerAttributes a;
  memset(&a, 0, sizeof(a));
  if (cudaPointerGetAttributes(&a, dst) == cudaSuccess && a.type == cudaMemoryTypeHost &&
      a.devicePointer) {
    *target = a.devicePointer;
    return GRAPH_OK;
  }
  cudaGetLastError();  // an unregistered pointer is not an error here
  GG_TRY(ensure_stage(g, stage_bytes));
  *target = (char*)g->stage.p + stage_off;
  *staged = true;
  return GRAPH_OK;
}

unsigned plan_grid(uint32_t plan_blocks) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
  }
  const uint32_t cap = (uint32_t)sms * 8u;
  return plan_blocks < cap ? plan_blocks : cap;
}

PartView Part::view() const {
  PartView v;
  v.nv = nv;
  v.nout = nout;
  v.ne = ne;
  v.off = (const int64_t*)off.p;
  v.E = (const uint32_t*)E.p;
  v.W = (const uint32_t*)W.p;
  v.l2g = (const uint32_t*)l2g.p;
  v.outbox = (const uint32_t*)outbox.p;
  v.chunk_vertex = (const uint32_t*)chunk_vertex.p;
  v.chunk_first = (const int64_t*)chunk_first.p;
  v.hub_chunk0 = (const uint32_t*)hub_chunk0.p;
  v.nchunk = nchunk;
  v.bstart[0] = 0;
  v.bstart[1] = cls_end[kClassHub];
  v.bstart[2] = cls_end[kClassWarp];
  v.bstart[3] = cls_end[kClassSub];
  v.bstart[4] = cls_end[1];
  return v;
}

namespace {

// ---------------------------------------------------------------------------- load
// Validation flags: 1 offsets[0] != 0, 2 offsets decrease, 4 offsets[n] != m,
// 8 column id >= n, 16 weight == 0.
__global__ void k_validate_offsets(const int64_t* off, uint32_t n, int64_t m, int* flags) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    if (off[0] != 0) atomicOr(flags, 1);
    if (off[n] != m) atomicOr(flags, 4);
  }
  if (i < n && off[i] > off[i + 1]) atomicOr(flags, 2);
}

__global__ void k_validate_cols(const uint32_t* col, const uint32_t* w, int64_t m, uint32_t n,
                                int* flags) {
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (col[e] >= n) bad |= 8;
    if (w && w[e] == 0) bad |= 16;
  }
  bad = __reduce_or_sync(kFull, bad);
  if (bad && lane_id() == 0) atomicOr(flags, bad);
}

// ---------------------------------------------------------------------------- partition
__device__ __forceinline__ int degree_class(int64_t d) {
  return d <= 0 ? 0 : 64 - __clzll((unsigned long long)d);
}

// Partition id per vertex. mode 0: all 1 (NONE); 1: deg >= T -> 0 (DEGREE); 2: explicit.
__global__ void k_assign(const int64_t* off, uint32_t n, int mode, uint32_t T,
                         const uint8_t* explicit_part, uint8_t* part, int* flags) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint8_t p;
  if (mode == 0) {
    p = 1;
  } else if (mode == 1) {
    p = (off[v + 1] - off[v]) >= (int64_t)T ? 0 : 1;
  } else {
    p = explicit_part[v];
    if (p > 1) {
      atomicOr(flags, 32);
      p = 1;
    }
  }
  part[v] = p;
}

__global__ void k_max_degree(const int64_t* off, uint32_t n, unsigned long long* out) {
  unsigned long long mx = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    mx = max(mx, (unsigned long long)(off[v + 1] - off[v]));
  #pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane_id() == 0) atomicMax(out, mx);
}

__global__ void k_sum_degree_ge(const int64_t* off, uint32_t n, int64_t T,
                                unsigned long long* out) {
  unsigned long long s = 0;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int64_t d = off[v + 1] - off[v];
    if (d >= T) s += (unsigned long long)d;
  }
  s = warp_sum(s);
  if (lane_id() == 0 && s) atomicAdd(out, s);
}

constexpr int kKeys = 2 * kNClass;  // key = part * 34 + (33 - class): partition-major,
                                    // class descending
constexpr int kSortTile = 1024;     // vertices per warp tile

__device__ __forceinline__ int sort_key(const int64_t* off, const uint8_t* part, uint32_t v) {
  return (int)part[v] * kNClass + (kNClass - 1 - degree_class(off[v + 1] - off[v]));
}

// hist[key * ntiles + tile] = vertices of `tile` with `key`.
__global__ void __launch_bounds__(kThreads) k_key_hist(const int64_t* off, const uint8_t* part,
                                                       uint32_t n, uint32_t ntiles,
                                                       uint32_t* hist) {
  __shared__ uint32_t cnt[kThreads / 32][kKeys];
  const int w = threadIdx.x >> 5;
  for (int k = lane_id(); k < kKeys; k += 32) cnt[w][k] = 0;
  __syncwarp();
  const uint32_t tile = blockIdx.x * (kThreads / 32) + w;
  if (tile < ntiles) {
    for (int i = lane_id(); i < kSortTile; i += 32) {
      uint64_t v = (uint64_t)tile * kSortTile + i;
      if (v < n) atomicAdd(&cnt[w][sort_key(off, part, (uint32_t)v)], 1u);
    }
    __syncwarp();
    for (int k = lane_id(); k < kKeys; k += 32) hist[(uint64_t)k * ntiles + tile] = cnt[w][k];
  }
}

// Stable scatter: order[base[key, tile] + rank within tile] = v.
__global__ void __launch_bounds__(kThreads) k_key_scatter(const int64_t* off, const uint8_t* part,
                                                          uint32_t n, uint32_t ntiles,
                                                          const uint32_t* base,
                                                          uint32_t* order) {
  __shared__ uint32_t run[kThreads / 32][kKeys];
  const int w = threadIdx.x >> 5;
  const uint32_t tile = blockIdx.x * (kThreads / 32) + w;
  if (tile >= ntiles) return;
  for (int k = lane_id(); k < kKeys; k += 32) run[w][k] = base[(uint64_t)k * ntiles + tile];
  __syncwarp();
  for (int g0 = 0; g0 < kSortTile; g0 += 32) {
    uint64_t v = (uint64_t)tile * kSortTile + g0 + lane_id();
    const bool valid = v < n;
    const int key = valid ? sort_key(off, part, (uint32_t)v) : kKeys;  // sentinel
    const unsigned peers = __match_any_sync(kFull, key);
    const uint32_t rank = __popc(peers & lanemask_lt());
    if (valid) order[run[w][key] + rank] = (uint32_t)v;
    __syncwarp();
    if (valid && rank == 0) run[w][key] += __popc(peers);
    __syncwarp();
  }
}

// Key starts: start[k] = base[k * ntiles] (start[kKeys] = n).
__global__ void k_key_starts(const uint32_t* base, uint32_t ntiles, uint32_t n,
                             uint32_t* start) {
  int k = threadIdx.x;
  if (k < kKeys) start[k] = base[(uint64_t)k * ntiles];
  if (k == kKeys) start[k] = n;
}

__global__ void k_local_ids(const uint32_t* order, uint32_t n, uint32_t nv0, uint32_t* l2g0,
                            uint32_t* l2g1, uint32_t* g2l, const int64_t* off,
                            int64_t* deg0, int64_t* deg1) {
  uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n) return;
  uint32_t v = order[pos];
  int64_t d = off[v + 1] - off[v];
  if (pos < nv0) {
    l2g0[pos] = v;
    g2l[v] = pos;
    deg0[pos] = d;
  } else {
    uint32_t lid = pos - nv0;
    l2g1[lid] = v;
    g2l[v] = kRemote | lid;
    deg1[lid] = d;
  }
}

// Per-vertex edge work over one partition in bucket segments. Mode 0: count local
// neighbours into nloc and mark remote targets (mark[local id in the other partition] =
// 1). Mode 1: write the partition's E (and W) in local-first order.
struct BuildArgs {
  const int64_t* goff;   // original CSR
  const uint32_t* gcol;
  const uint32_t* gw;
  const uint32_t* g2l;
  const uint32_t* l2g;   // this partition
  const int64_t* poff;   // this partition's new offsets (mode 1)
  uint32_t* nloc;        // [nv]
  uint8_t* mark;         // other partition's marks (mode 0)
  const uint32_t* oidx;  // other partition's outbox index per local id (mode 1)
  uint32_t* E;
  uint32_t* W;
  uint32_t p;
};

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_build(const __grid_constant__ Plan plan, BuildArgs a) {
  __shared__ uint32_t wl[kThreads / 32], wr[kThreads / 32];
  __shared__ uint32_t red[kThreads / 32];
  const Seg& S = plan.seg[find_seg(plan)];
  const uint32_t rel = blockIdx.x - S.blk0;
  const int gshift = S.gshift;
  if (gshift >= 8) {
    // whole CTA on one vertex, chunks of kThreads edges
    const uint32_t lid = S.v0 + rel;
    const uint32_t v = a.l2g[lid];
    const int64_t s = a.goff[v], t = a.goff[v + 1];
    const int w = threadIdx.x >> 5;
    if (MODE == 0) {
      uint32_t cnt = 0;
      for (int64_t e = s + threadIdx.x; e < t; e += kThreads) {
        const uint32_t gu = a.g2l[a.gcol[e]];
        if ((gu >> 31) == a.p) cnt++;
        else a.mark[gu & kIdMask] = 1;
      }
      cnt = warp_sum(cnt);
      if (lane_id() == 0) red[w] = cnt;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int i = 0; i < kThreads / 32; ++i) tot += red[i];
        a.nloc[lid] = tot;
      }
    } else {
      int64_t curl = a.poff[lid], curr = curl + a.nloc[lid];
      for (int64_t c0 = s; c0 < t; c0 += kThreads) {
        const int64_t e = c0 + threadIdx.x;
        const bool valid = e < t;
        uint32_t gu = 0, wt = 0;
        if (valid) {
          gu = a.g2l[a.gcol[e]];
          if (a.W) wt = a.gw[e];
        }
        const bool loc = valid && (gu >> 31) == a.p;
        const bool rem = valid && !loc;
        const unsigned bl = __ballot_sync(kFull, loc), br = __ballot_sync(kFull, rem);
        if (lane_id() == 0) {
          wl[w] = __popc(bl);
          wr[w] = __popc(br);
        }
        __syncthreads();
        uint32_t pl = 0, pr = 0, tl = 0, tr = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
          if (i < w) {
            pl += wl[i];
            pr += wr[i];
          }
          tl += wl[i];
          tr += wr[i];
        }
        if (loc) {
          const int64_t pos = curl + pl + __popc(bl & lanemask_lt());
          a.E[pos] = gu & kIdMask;
          if (a.W) a.W[pos] = wt;
        } else if (rem) {
          const int64_t pos = curr + pr + __popc(br & lanemask_lt());
          a.E[pos] = kRemote | a.oidx[gu & kIdMask];
          if (a.W) a.W[pos] = wt;
        }
        curl += tl;
        curr += tr;
        __syncthreads();
      }
    }
    return;
  }
  // groups of 2^gshift lanes, one vertex each
  const int gl = threadIdx.x & ((1 << gshift) - 1);
  const uint32_t gi = rel * (kThreads >> gshift) + (threadIdx.x >> gshift);
  const bool vvalid = gi < S.count;
  const uint32_t lid = S.v0 + (vvalid ? gi : 0);
  int64_t s = 0, t = 0;
  uint32_t v = 0;
  if (vvalid) {
    v = a.l2g[lid];
    s = a.goff[v];
    t = a.goff[v + 1];
  }
  const int gsz = 1 << gshift;
  const unsigned gmask = (gsz == 32) ? kFull : (((1u << gsz) - 1) << (lane_id() & ~(gsz - 1)));
  if (MODE == 0) {
    uint32_t cnt = 0;
    for (int64_t e = s + gl; e < t; e += gsz) {
      const uint32_t gu = a.g2l[a.gcol[e]];
      if ((gu >> 31) == a.p) cnt++;
      else a.mark[gu & kIdMask] = 1;
    }
    cnt = group_sum(cnt, gshift);
    if (vvalid && gl == 0) a.nloc[lid] = cnt;
  } else {
    int64_t curl = 0, curr = 0;
    if (vvalid) {
      curl = a.poff[lid];
      curr = curl + a.nloc[lid];
    }
    for (int64_t c0 = s; __any_sync(kFull, c0 < t); c0 += gsz) {
      const int64_t e = c0 + gl;
      const bool valid = e < t;
      uint32_t gu = 0, wt = 0;
      if (valid) {
        gu = a.g2l[a.gcol[e]];
        if (a.W) wt = a.gw[e];
      }
      const bool loc = valid && (gu >> 31) == a.p;
      const bool rem = valid && !loc;
      const unsigned bl = __ballot_sync(kFull, loc) & gmask;
      const unsigned br = __ballot_sync(kFull, rem) & gmask;
      if (loc) {
        const int64_t pos = curl + __popc(bl & lanemask_lt());
        a.E[pos] = gu & kIdMask;
        if (a.W) a.W[pos] = wt;
      } else if (rem) {
        const int64_t pos = curr + __popc(br & lanemask_lt());
        a.E[pos] = kRemote | a.oidx[gu & kIdMask];
        if (a.W) a.W[pos] = wt;
      }
      curl += __popc(bl);
      curr += __popc(br);
    }
  }
}

__global__ void k_outbox_fill(const uint8_t* mark, const uint32_t* idx, uint32_t nq,
                              uint32_t* outbox) {
  uint32_t ql = blockIdx.x * blockDim.x + threadIdx.x;
  if (ql < nq && mark[ql]) outbox[idx[ql]] = ql;
}

__global__ void k_hub_chunks(const int64_t* poff, uint32_t nhub, int64_t* nch) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nhub) nch[v] = (poff[v + 1] - poff[v] + kHubChunk - 1) / kHubChunk;
}

__global__ void k_hub_chunk_table(const int64_t* poff, const int64_t* chunk0, uint32_t nhub,
                                  uint32_t* hub_chunk0, uint32_t* chunk_vertex,
                                  int64_t* chunk_first) {
  uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nhub) return;
  const int64_t c0 = chunk0[v];
  hub_chunk0[v] = (uint32_t)c0;
  const int64_t s = poff[v], t = poff[v + 1];
  int64_t k = c0;
  for (int64_t e = s; e < t; e += kHubChunk, ++k) {
    chunk_vertex[k] = v;
    chunk_first[k] = e;
  }
}

void free_part(graph* g, Part& P) {
  dfree(g, P.off);
  dfree(g, P.E);
  dfree(g, P.W);
  dfree(g, P.l2g);
  dfree(g, P.outbox);
  dfree(g, P.chunk_vertex);
  dfree(g, P.chunk_first);
  dfree(g, P.hub_chunk0);
  P = Part();
}

Plan dense_plan(const Part& P, int part) {
  Plan pl;
  memset(&pl, 0, sizeof(pl));
  PartView v = P.view();
  const int gsh[kNBucket] = {8, 5, kSubShift, 0};
  for (int b = 0; b < kNBucket; ++b)
    plan_add(pl, nullptr, v.bstart[b], v.bstart[b + 1] - v.bstart[b], part, gsh[b], b);
  return pl;
}

graph_status build_partition(graph* g, int mode, uint32_t T, const uint8_t* explicit_host) {
  const uint32_t n = g->n;
  graph_status st = GRAPH_OK;
  DevBuf partb, flags, expl, hist, order, starts, deg[2], nloc[2], mark[2], oidx[2];
  auto cleanup = [&]() {
    DevBuf* all[] = {&partb, &flags, &expl, &hist, &order, &starts, &deg[0], &deg[1],
                     &nloc[0], &nloc[1], &mark[0], &mark[1], &oidx[0], &oidx[1]};
    cudaStreamSynchronize(g->stream);
    for (DevBuf* b : all) dfree(g, *b);
  };
#define STEP(x)                \
  do {                         \
    st = (x);                  \
    if (st != GRAPH_OK) {      \
      cleanup();               \
      return st;               \
    }                          \
  } while (0)
#define CSTEP(x) STEP(((x) == cudaSuccess) ? GRAPH_OK : cuda_fail(cudaGetLastError(), #x, __FILE__, __LINE__))

  STEP(dalloc(g, partb, n));
  STEP(dalloc(g, flags, sizeof(int)));
  CSTEP(cudaMemsetAsync(flags.p, 0, sizeof(int), g->stream));
  if (mode == 2) {
    STEP(dalloc(g, expl, n));
    CSTEP(cudaMemcpyAsync(expl.p, explicit_host, n, cudaMemcpyHostToDevice, g->stream));
  }
  k_assign<<<grid_for(n, 256), 256, 0, g->stream>>>((const int64_t*)g->off.p, n, mode, T,
                                                    (const uint8_t*)expl.p,
                                                    (uint8_t*)partb.p, (int*)flags.p);
  CSTEP(cudaGetLastError());
  int hflags = 0;
  CSTEP(cudaMemcpyAsync(&hflags, flags.p, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CSTEP(cudaStreamSynchronize(g->stream));
  if (hflags) {
    set_error("explicit assignment holds a partition id other than 0 or 1");
    cleanup();
    return GRAPH_EINVAL;
  }

  // Stable counting sort of vertices by (partition, class descending).
  const uint32_t ntiles = (n + kSortTile - 1) / kSortTile;
  STEP(dalloc(g, hist, sizeof(uint32_t) * (size_t)kKeys * ntiles));
  STEP(dalloc(g, order, sizeof(uint32_t) * (size_t)n));
  STEP(dalloc(g, starts, sizeof(uint32_t) * (kKeys + 1)));
  const unsigned sort_blocks = (ntiles + kThreads / 32 - 1) / (kThreads / 32);
  k_key_hist<<<sort_blocks, kThreads, 0, g->stream>>>((const int64_t*)g->off.p,
                                                      (const uint8_t*)partb.p, n, ntiles,
                                                      (uint32_t*)hist.p);
  CSTEP(cudaGetLastError());
  STEP(exclusive_scan_u32(g, (const uint32_t*)hist.p, (uint32_t*)hist.p,
                          (uint64_t)kKeys * ntiles, nullptr));
  k_key_scatter<<<sort_blocks, kThreads, 0, g->stream>>>((const int64_t*)g->off.p,
                                                         (const uint8_t*)partb.p, n, ntiles,
                                                         (const uint32_t*)hist.p,
                                                         (uint32_t*)order.p);
  k_key_starts<<<1, 128, 0, g->stream>>>((const uint32_t*)hist.p, ntiles, n,
                                          (uint32_t*)starts.p);
  CSTEP(cudaGetLastError());
  uint32_t hstart[kKeys + 1];
  CSTEP(cudaMemcpyAsync(hstart, starts.p, sizeof(hstart), cudaMemcpyDeviceToHost, g->stream));
  CSTEP(cudaStreamSynchronize(g->stream));

  Part NP[2];
  for (int p = 0; p < 2; ++p) {
    const uint32_t first = hstart[p * kNClass];
    const uint32_t last = hstart[(p + 1) * kNClass];
    NP[p].nv = last - first;
    // cls_end[c] = number of local vertices with class >= c
    for (int c = 0; c < kNClass; ++c) {
      // key of class c: p*34 + 33 - c; vertices with class >= c have keys <= that key
      const int key = p * kNClass + (kNClass - 1 - c);
      NP[p].cls_end[c] = hstart[key + 1] - first;
    }
    NP[p].cls_end[kNClass - 1] = 0;
  }
  const uint32_t nv0 = NP[0].nv;
  auto fail_parts = [&](graph_status s) {
    cleanup();
    free_part(g, NP[0]);
    free_part(g, NP[1]);
    return s;
  };
#undef STEP
#define STEP(x)                          \
  do {                                   \
    st = (x);                            \
    if (st != GRAPH_OK) return fail_parts(st); \
  } while (0)

  for (int p = 0; p < 2; ++p) {
    STEP(dalloc(g, NP[p].l2g, sizeof(uint32_t) * (size_t)NP[p].nv));
    STEP(dalloc(g, deg[p], sizeof(int64_t) * ((size_t)NP[p].nv + 1)));
    // +2 entries: bulk copies of offset slices read whole 16-byte granules
    STEP(dalloc(g, NP[p].off, sizeof(int64_t) * ((size_t)NP[p].nv + 3)));
    STEP(dalloc(g, nloc[p], sizeof(uint32_t) * (size_t)NP[p].nv));
    STEP(dalloc(g, mark[p], (size_t)NP[p].nv + 1));
    STEP(dalloc(g, oidx[p], sizeof(uint32_t) * ((size_t)NP[p].nv + 1)));
    CSTEP(cudaMemsetAsync(mark[p].p, 0, (size_t)NP[p].nv + 1, g->stream));
  }
  k_local_ids<<<grid_for(n, 256), 256, 0, g->stream>>>(
      (const uint32_t*)order.p, n, nv0, (uint32_t*)NP[0].l2g.p, (uint32_t*)NP[1].l2g.p,
      (uint32_t*)g->g2l.p, (const int64_t*)g->off.p, (int64_t*)deg[0].p, (int64_t*)deg[1].p);
  CSTEP(cudaGetLastError());
  for (int p = 0; p < 2; ++p) {
    int64_t tot = 0;
    STEP(exclusive_scan_i64(g, (const int64_t*)deg[p].p, (int64_t*)NP[p].off.p, NP[p].nv,
                            &tot));
    NP[p].ne = tot;
    CSTEP(cudaMemcpyAsync((int64_t*)NP[p].off.p + NP[p].nv, &NP[p].ne, sizeof(int64_t),
                          cudaMemcpyHostToDevice, g->stream));
    CSTEP(cudaStreamSynchronize(g->stream));
  }
  // Pass 0: local counts and remote marks.
  for (int p = 0; p < 2; ++p) {
    if (NP[p].nv == 0) continue;
    BuildArgs a;
    memset(&a, 0, sizeof(a));
    a.goff = (const int64_t*)g->off.p;
    a.gcol = (const uint32_t*)g->col.p;
    a.gw = (const uint32_t*)g->w.p;
    a.g2l = (const uint32_t*)g->g2l.p;
    a.l2g = (const uint32_t*)NP[p].l2g.p;
    a.nloc = (uint32_t*)nloc[p].p;
    a.mark = (uint8_t*)mark[1 - p].p;
    a.p = (uint32_t)p;
    Plan pl = dense_plan(NP[p], p);
    if (pl.nblocks) k_build<0><<<pl.nblocks, kThreads, 0, g->stream>>>(pl, a);
    CSTEP(cudaGetLastError());
  }
  // Outbox of p = marked vertices of q, ascending local id.
  for (int p = 0; p < 2; ++p) {
    const int q = 1 - p;
    uint32_t tot = 0;
    STEP(exclusive_scan_u8_to_u32(g, (const uint8_t*)mark[q].p, (uint32_t*)oidx[q].p,
                                  NP[q].nv, &tot));
    NP[p].nout = tot;
    STEP(dalloc(g, NP[p].outbox, sizeof(uint32_t) * (size_t)tot));
    if (NP[q].nv)
      k_outbox_fill<<<grid_for(NP[q].nv, 256), 256, 0, g->stream>>>(
          (const uint8_t*)mark[q].p, (const uint32_t*)oidx[q].p, NP[q].nv,
          (uint32_t*)NP[p].outbox.p);
    CSTEP(cudaGetLastError());
  }
  // Pass 1: edges in local-first order.
  for (int p = 0; p < 2; ++p) {
    // +16 entries of padding: bulk copies read whole 16-byte granules
    STEP(dalloc(g, NP[p].E, sizeof(uint32_t) * ((size_t)NP[p].ne + 16)));
    CSTEP(cudaMemsetAsync(NP[p].E.p, 0, NP[p].E.bytes, g->stream));
    if (g->weighted) {
      STEP(dalloc(g, NP[p].W, sizeof(uint32_t) * ((size_t)NP[p].ne + 16)));
      CSTEP(cudaMemsetAsync(NP[p].W.p, 0, NP[p].W.bytes, g->stream));
    }
    if (NP[p].nv == 0) continue;
    BuildArgs a;
    memset(&a, 0, sizeof(a));
    a.goff = (const int64_t*)g->off.p;
    a.gcol = (const uint32_t*)g->col.p;
    a.gw = (const uint32_t*)g->w.p;
    a.g2l = (const uint32_t*)g->g2l.p;
    a.l2g = (const uint32_t*)NP[p].l2g.p;
    a.poff = (const int64_t*)NP[p].off.p;
    a.nloc = (uint32_t*)nloc[p].p;
    a.oidx = (const uint32_t*)oidx[1 - p].p;
    a.E = (uint32_t*)NP[p].E.p;
    a.W = (uint32_t*)NP[p].W.p;
    a.p = (uint32_t)p;
    Plan pl = dense_plan(NP[p], p);
    if (pl.nblocks) k_build<1><<<pl.nblocks, kThreads, 0, g->stream>>>(pl, a);
    CSTEP(cudaGetLastError());
  }
  // Hub chunk tables for dense (PageRank) hub work.
  for (int p = 0; p < 2; ++p) {
    Part& P = NP[p];
    P.nhub = P.cls_end[kClassHub];
    STEP(dalloc(g, P.hub_chunk0, sizeof(uint32_t) * ((size_t)P.nhub + 1)));
    if (P.nhub == 0) {
      P.nchunk = 0;
      continue;
    }
    DevBuf nch;
    STEP(dalloc(g, nch, sizeof(int64_t) * ((size_t)P.nhub + 1)));
    k_hub_chunks<<<grid_for(P.nhub, 256), 256, 0, g->stream>>>((const int64_t*)P.off.p,
                                                               P.nhub, (int64_t*)nch.p);
    int64_t tot = 0;
    st = exclusive_scan_i64(g, (const int64_t*)nch.p, (int64_t*)nch.p, P.nhub, &tot);
    if (st != GRAPH_OK) {
      dfree(g, nch);
      return fail_parts(st);
    }
    P.nchunk = (uint32_t)tot;
    st = dalloc(g, P.chunk_vertex, sizeof(uint32_t) * (size_t)tot);
    if (st == GRAPH_OK) st = dalloc(g, P.chunk_first, sizeof(int64_t) * (size_t)tot);
    if (st != GRAPH_OK) {
      dfree(g, nch);
      return fail_parts(st);
    }
    k_hub_chunk_table<<<grid_for(P.nhub, 256), 256, 0, g->stream>>>(
        (const int64_t*)P.off.p, (const int64_t*)nch.p, P.nhub, (uint32_t*)P.hub_chunk0.p,
        (uint32_t*)P.chunk_vertex.p, (int64_t*)P.chunk_first.p);
    cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(g->stream);
    dfree(g, nch);
    if (e != cudaSuccess) return fail_parts(cuda_fail(e, "hub chunk table", __FILE__, __LINE__));
  }
  CSTEP(cudaStreamSynchronize(g->stream));
  cleanup();
  free_bfs(g);
  free_sssp(g);
  free_pr(g);
  free_msbfs(g);
  free_bc(g);
  free_ssspb(g);
  free_seg(g);
  free_part(g, g->part[0]);
  free_part(g, g->part[1]);
  g->part[0] = NP[0];
  g->part[1] = NP[1];
  g->partitioned = true;
  return GRAPH_OK;
#undef STEP
#undef CSTEP
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" {

const char* graph_strerror(graph_status s) {
  switch (s) {
    case GRAPH_OK: return "success";
    case GRAPH_EINVAL: return "invalid argument";
    case GRAPH_ENOMEM: return "out of memory";
    case GRAPH_ECUDA: return "CUDA error";
    case GRAPH_ETIMEOUT: return "bounded wait or superstep cap expired";
    case GRAPH_ERANGE: return "result out of range";
    case GRAPH_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* graph_last_error(void) { return g_last_error.c_str(); }

graph_status graph_load_csr(uint32_t n, int64_t m, const int64_t* offsets,
                            const uint32_t* cols, const uint32_t* weights, int mem,
                            const graph_runtime* rt, graph_t** out) {
  g_last_error.clear();
  if (!out) {
    set_error("out is NULL");
    return GRAPH_EINVAL;
  }
  *out = nullptr;
  if (n == 0 || n >= 0x80000000u || m < 0 || !offsets || (m > 0 && !cols) ||
      (mem != GRAPH_MEM_HOST && mem != GRAPH_MEM_DEVICE)) {
    set_error("invalid sizes or pointers (n=%u m=%lld mem=%d)", n, (long long)m, mem);
    return GRAPH_EINVAL;
  }
  if (mem == GRAPH_MEM_HOST && offsets[n] != m) {
    set_error("offsets[n]=%lld differs from m=%lld", (long long)offsets[n], (long long)m);
    return GRAPH_EINVAL;
  }
  if (rt && ((rt->alloc == nullptr) != (rt->free == nullptr))) {
    set_error("allocator hooks must be given together");
    return GRAPH_EINVAL;
  }
  graph* g = new graph();
  if (rt) g->rt = *rt;
  g->stream = (cudaStream_t)g->rt.stream;
  cudaGetDevice(&g->device);
  g->n = n;
  g->m = m;
  g->weighted = weights != nullptr;
  graph_status st = GRAPH_OK;
  auto fail = [&](graph_status s) {
    graph_free(g);
    return s;
  };
  if ((st = dalloc(g, g->err, sizeof(int))) != GRAPH_OK) return fail(st);
  if ((st = dalloc(g, g->off, sizeof(int64_t) * ((size_t)n + 1))) != GRAPH_OK) return fail(st);
  if ((st = dalloc(g, g->col, sizeof(uint32_t) * ((size_t)m + 16))) != GRAPH_OK) return fail(st);
  if (weights && (st = dalloc(g, g->w, sizeof(uint32_t) * ((size_t)m + 16))) != GRAPH_OK)
    return fail(st);
  if ((st = dalloc(g, g->g2l, sizeof(uint32_t) * (size_t)n)) != GRAPH_OK) return fail(st);
  const cudaMemcpyKind kind =
      mem == GRAPH_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaMemsetAsync(g->err.p, 0, sizeof(int), g->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->off.p, offsets, sizeof(int64_t) * ((size_t)n + 1), kind, g->stream);
  if (e == cudaSuccess && m > 0)
    e = cudaMemcpyAsync(g->col.p, cols, sizeof(uint32_t) * (size_t)m, kind, g->stream);
  if (e == cudaSuccess && weights && m > 0)
    e = cudaMemcpyAsync(g->w.p, weights, sizeof(uint32_t) * (size_t)m, kind, g->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "graph copy", __FILE__, __LINE__));
  k_validate_offsets<<<grid_for((uint64_t)n + 1, 256), 256, 0, g->stream>>>(
      (const int64_t*)g->off.p, n, m, (int*)g->err.p);
  if (m > 0)
    k_validate_cols<<<std::min<unsigned>(grid_for(m, 256), 152 * 16), 256, 0, g->stream>>>(
        (const uint32_t*)g->col.p, (const uint32_t*)g->w.p, m, n, (int*)g->err.p);
  int flags = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flags, g->err.p, sizeof(int), cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return fail(cuda_fail(e, "graph validation", __FILE__, __LINE__));
  if (flags) {
    set_error("invalid CSR (flags 0x%x: 1 offsets[0]!=0, 2 decreasing offsets, 4 "
              "offsets[n]!=m, 8 column id >= n, 16 zero weight)", flags);
    graph_free(g);
    return GRAPH_EINVAL;
  }
  cudaMemsetAsync(g->err.p, 0, sizeof(int), g->stream);
  *out = g;
  return GRAPH_OK;
}

graph_status graph_partition(graph_t* g, const graph_partition_attr* attr) {
  g_last_error.clear();
  if (!g || !attr) {
    set_error("graph or attr is NULL");
    return GRAPH_EINVAL;
  }
  int mode;
  uint32_t T = 0;
  if (attr->strategy == GRAPH_PART_NONE) {
    mode = 0;
  } else if (attr->strategy == GRAPH_PART_DEGREE) {
    mode = 1;
    if (attr->edge_share > 0) {
      if (attr->edge_share > 1.0) {
        set_error("edge_share must be in (0, 1]");
        return GRAPH_EINVAL;
      }
      // Largest t with sum_{deg >= t} deg >= share * m (binary search on the device sums).
      DevBuf acc;
      GG_TRY(dalloc(g, acc, sizeof(unsigned long long)));
      unsigned long long maxdeg = 0, s = 0;
      cudaMemsetAsync(acc.p, 0, 8, g->stream);
      k_max_degree<<<152 * 8, 256, 0, g->stream>>>((const int64_t*)g->off.p, g->n,
                                                   (unsigned long long*)acc.p);
      cudaMemcpyAsync(&maxdeg, acc.p, 8, cudaMemcpyDeviceToHost, g->stream);
      cudaError_t e = cudaStreamSynchronize(g->stream);
      const double need = attr->edge_share * (double)g->m;
      int64_t lo = 0, hi = (int64_t)maxdeg + 1;  // S(lo) >= need (share <= 1), S(hi) = 0
      while (e == cudaSuccess && hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        cudaMemsetAsync(acc.p, 0, 8, g->stream);
        k_sum_degree_ge<<<152 * 8, 256, 0, g->stream>>>((const int64_t*)g->off.p, g->n, mid,
                                                        (unsigned long long*)acc.p);
        cudaMemcpyAsync(&s, acc.p, 8, cudaMemcpyDeviceToHost, g->stream);
        e = cudaStreamSynchronize(g->stream);
        if ((double)s >= need) lo = mid;
        else hi = mid;
      }
      dfree(g, acc);
      if (e != cudaSuccess) return cuda_fail(e, "edge-share threshold", __FILE__, __LINE__);
      T = (uint32_t)std::min<int64_t>(lo, 0xFFFFFFFFll);
    } else {
      T = attr->degree_threshold;
    }
  } else if (attr->strategy == GRAPH_PART_EXPLICIT) {
    mode = 2;
    if (!attr->assignment) {
      set_error("EXPLICIT strategy needs an assignment array");
      return GRAPH_EINVAL;
    }
  } else {
    set_error("unknown partition strategy %d", attr->strategy);
    return GRAPH_EINVAL;
  }
  graph_status st = build_partition(g, mode, T, attr->assignment);
  if (st == GRAPH_OK) {
    g->strategy = attr->strategy;
    g->threshold = mode == 1 ? T : 0;
  }
  return st;
}

graph_status graph_get_partition_info(const graph_t* g, graph_partition_info* info) {
  if (!g || !info) {
    set_error("graph or info is NULL");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph is not partitioned");
    return GRAPH_ESTATE;
  }
  memset(info, 0, sizeof(*info));
  info->n = g->n;
  info->m = g->m;
  info->threshold = g->threshold;
  int64_t bytes = 0;
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    info->nv[p] = P.nv;
    info->ne[p] = P.ne;
    info->nout[p] = P.nout;
    for (int c = 0; c < kNClass; ++c) info->cls_end[p][c] = P.cls_end[c];
    // eid |V_p| + vid |E_p| + w |E_p| + vid (|V_i| + |V_o|); the message arrays belong to
    // each algorithm's workspace.
    bytes += 8 * ((int64_t)P.nv + 1) + 4 * P.ne + (g->weighted ? 4 * P.ne : 0) +
             4 * ((int64_t)P.nout + (int64_t)g->part[1 - p].nout);
  }
  info->bytes_graph = bytes;
  return GRAPH_OK;
}

graph_status graph_export_partition(const graph_t* g, int p, uint32_t* l2g, int64_t* off,
                                    uint32_t* E, uint32_t* W, uint32_t* outbox,
                                    uint32_t* g2l) {
  if (!g || p < 0 || p > 1) {
    set_error("bad graph or partition index");
    return GRAPH_EINVAL;
  }
  if (!g->partitioned) {
    set_error("graph is not partitioned");
    return GRAPH_ESTATE;
  }
  if (W && !g->weighted) {
    set_error("graph has no weights");
    return GRAPH_EINVAL;
  }
  const Part& P = g->part[p];
  cudaStream_t s = g->stream;
  if (l2g && P.nv) GG_CUDA(cudaMemcpyAsync(l2g, P.l2g.p, 4ull * P.nv, cudaMemcpyDeviceToHost, s));
  if (off) GG_CUDA(cudaMemcpyAsync(off, P.off.p, 8ull * (P.nv + 1), cudaMemcpyDeviceToHost, s));
  // (the edge arrays may be host-resident: let the runtime infer the direction)
  if (E && P.ne) GG_CUDA(cudaMemcpyAsync(E, P.E.p, 4ull * P.ne, cudaMemcpyDefault, s));
  if (W && P.ne) GG_CUDA(cudaMemcpyAsync(W, P.W.p, 4ull * P.ne, cudaMemcpyDefault, s));
  if (outbox && P.nout)
    GG_CUDA(cudaMemcpyAsync(outbox, P.outbox.p, 4ull * P.nout, cudaMemcpyDeviceToHost, s));
  if (g2l) GG_CUDA(cudaMemcpyAsync(g2l, g->g2l.p, 4ull * g->n, cudaMemcpyDeviceToHost, s));
  GG_CUDA(cudaStreamSynchronize(s));
  return GRAPH_OK;
}

namespace gg {
namespace {

// Moves a buffer into page-locked host memory mapped into the device (p becomes the
// device alias of the host allocation), or back into device memory.
graph_status move_to_host(graph* g, DevBuf& b) {
  if (b.host || !b.p) return GRAPH_OK;
  void* h = nullptr;
  if (cudaHostAlloc(&h, b.bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot allocate %zu bytes of page-locked host memory", b.bytes);
    return GRAPH_ENOMEM;
  }
  void* d = nullptr;
  cudaError_t e = cudaMemcpyAsync(h, b.p, b.bytes, cudaMemcpyDeviceToHost, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&d, h, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(h);
    return cuda_fail(e, "moving an edge array to host memory", __FILE__, __LINE__);
  }
  const size_t bytes = b.bytes;
  dfree(g, b);
  b.p = d;
  b.bytes = bytes;
  b.host = h;
  return GRAPH_OK;
}

graph_status move_to_device(graph* g, DevBuf& b) {
  if (!b.host) return GRAPH_OK;
  DevBuf nb;
  GG_TRY(dalloc(g, nb, b.bytes));
  cudaError_t e = cudaMemcpyAsync(nb.p, b.host, b.bytes, cudaMemcpyHostToDevice, g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    dfree(g, nb);
    return cuda_fail(e, "moving an edge array to device memory", __FILE__, __LINE__);
  }
  cudaFreeHost(b.host);
  b = nb;
  return GRAPH_OK;
}

}  // namespace
}  // namespace gg

extern "C" graph_status graph_set_edge_memory(graph_t* g, int which, int mem) {
  if (!g || which <= 0 || which > 7 || (mem != GRAPH_MEM_HOST && mem != GRAPH_MEM_DEVICE)) {
    set_error("bad graph, edge-array mask or memory kind");
    return GRAPH_EINVAL;
  }
  if ((which & 3) && !g->partitioned) {
    set_error("graph_partition must run before a partition's edges can move");
    return GRAPH_ESTATE;
  }
  GG_CUDA(cudaStreamSynchronize(g->stream));
  // Workspaces and captured supersteps hold edge-array addresses: they are rebuilt on
  // their next use.
  free_bfs(g);
  free_sssp(g);
  free_pr(g);
  free_msbfs(g);
  free_bc(g);
  free_ssspb(g);
  free_seg(g);
  DevBuf* bufs[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (which & 1) { bufs[0] = &g->part[0].E; bufs[1] = &g->part[0].W; }
  if (which & 2) { bufs[2] = &g->part[1].E; bufs[3] = &g->part[1].W; }
  if (which & 4) { bufs[4] = &g->col; bufs[5] = &g->w; }
  for (DevBuf* b : bufs) {
    if (!b) continue;
    GG_TRY(mem == GRAPH_MEM_HOST ? move_to_host(g, *b) : move_to_device(g, *b));
  }
  return GRAPH_OK;
}

extern "C" graph_status graph_get_edge_memory(const graph_t* g, int* placement) {
  if (!g || !placement) {
    set_error("graph or placement is NULL");
    return GRAPH_EINVAL;
  }
  int m = 0;
  if (g->part[0].E.host) m |= 1;
  if (g->part[1].E.host) m |= 2;
  if (g->col.host) m |= 4;
  *placement = m;
  return GRAPH_OK;
}

void graph_free(graph_t* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  free_bfs(g);
  free_sssp(g);
  free_pr(g);
  free_msbfs(g);
  free_bc(g);
  free_ssspb(g);
  free_seg(g);
  free_part(g, g->part[0]);
  free_part(g, g->part[1]);
  dfree(g, g->off);
  dfree(g, g->col);
  dfree(g, g->w);
  dfree(g, g->g2l);
  dfree(g, g->err);
  dfree(g, g->counters);
  dfree(g, g->stage);
  if (g->host_counters) cudaFreeHost(g->host_counters);
  delete g;
}

}  // extern "C"
