// Segmented pull PageRank (Section 7.1, Figure 14) for FP32 and FP16-stored contributions.
//
// The neighbour sum of Figure 14 gathers one contribution x[u] per edge entry. Done as a
// scattered 4-byte global load per entry, those gathers run at about one element per SM
// clock on this GPU, far below the HBM rate. This file reorganises each partition's edges
// once (the plan, built on the device by the first pagerank() call after a partition) so
// that every gather reads shared memory instead (CSR segmenting, Zhang et al., "Making
// Caches Work for Graph Analytics", IEEE BigData 2017):
//  - a partition's source space (its own vertices, then its ghost slots) is cut into
//    segments of 2^log2 consecutive ids, small enough that one segment's contributions fit
//    in a CTA's shared memory;
//  - the partition's edge entries are stably sorted by the segment of their source; inside
//    a segment the entries of one destination vertex form a row (rows follow destination
//    order). An entry is 2 bytes: a 15-bit source offset within the segment and a
//    row-start bit;
//  - phase 1 (k_pr_seg): one persistent CTA per SM walks a contiguous range of chunks of
//    rows. It holds the current segment's contributions in shared memory (one bulk copy
//    per segment change), stages each chunk's entries by bulk copy while the previous chunk
//    is summed, and writes one partial sum per row;
//  - phase 2 (k_pr_merge): destination vertices are grouped into bins of about `bin`
//    partial sums. A CTA bulk-copies its bin's partial sums (one contiguous run per
//    segment) into a shared-memory window and adds each vertex's partials in segment order,
//    reading a 15-bit window position per partial, then applies Figure 14's update.
// Each destination therefore reads 2 bytes per edge entry plus about 10 bytes per partial
// sum, and gathers nothing from global memory. On RMAT graphs most entries point at the
// few high-degree vertices, so a destination's entries fall into few segments: about 0.12
// partial sums per entry at scale 22, which is what makes the layout pay.
//
// Both phases add with one deterministic segmented sum (fixed per-thread runs and a fixed
// scan over the CTA's threads), so ranks repeat bit for bit from run to run. The summation
// order differs from a sequential neighbour sum; the FP32 result stays within the same
// bound against FP64.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "pr_seg.cuh"

namespace gg {

namespace {

constexpr int kChunkEntriesMax = 8176;                 // entries per phase-1 chunk
constexpr uint32_t kMini = 256;                        // entries per phase-1 warp piece
constexpr uint32_t kMiniPerChunk = 32;                 // mini-chunks per chunk frame
constexpr uint32_t kWinMax = 16384;                    // window slots (fit 15-bit positions)
constexpr uint32_t kMergeVerts = 2048;                 // destination vertices per bin (max)
constexpr uint32_t kMaxPartials = 2047;                // partial sums of one destination
constexpr uint16_t kRowStart = 0x8000;
constexpr uint16_t kOffMask = 0x7FFF;
constexpr int kSortTile = 16384;                       // entries per warp in the stable sort
constexpr int kDefLog2 = 15, kDefChunk = 8176, kDefBin = 12288;
constexpr int kMaxBin = (int)(kWinMax - kMaxPartials - 1);   // 14336

struct SegChunk {   // 32 bytes
  uint32_t e0;      // first entry in the partition's packed entry array (multiple of 8)
  uint32_t nent;    // entries (<= kChunkEntriesMax)
  uint32_t row0;    // first row (index into the partition's partial sums)
  uint32_t src0;    // first source id of the segment (in its space)
  uint32_t srclen;  // sources in the segment
  uint32_t key;     // segment id over both partitions (changes when the slice must reload)
  uint32_t cl;      // chunk index within its partition (its mini-chunk row offsets)
  uint8_t part, ghost;
  uint16_t pad;
};
static_assert(sizeof(SegChunk) == 32, "SegChunk is 32 bytes");

struct SegBin {     // 32 bytes
  uint32_t v0, v1;      // destination vertices [v0, v1) of partition `part`
  uint32_t run0, run1;  // runs of partial sums (window copies)
  uint32_t pos0, npos;  // positions [pos0, pos0 + npos) in the partition's position list
  uint32_t wgran;       // window size in 16-byte granules
  uint32_t part;
};
static_assert(sizeof(SegBin) == 32, "SegBin is 32 bytes");

struct SegPart {
  uint32_t S = 0, L = 0, nz = 0, nbin = 0, nchunk = 0;
  uint32_t P = 0;     // rows (partial sums)
  uint64_t nruns = 0;
  DevBuf ent, part, plist, runs, deg, mrow;
};

// Arguments of both phases (one struct, passed by value).
struct SegArgs {
  const void* x[2];
  const void* ghost[2];
  void* xn[2];
  void* r[2];
  const uint32_t* deg[2];  // degree of each vertex (plan copy, 32-bit)
  const uint16_t* ent[2];
  const uint16_t* mrow[2];  // [chunk][32] first row of each mini-chunk, relative to row0
  float* part[2];
  const uint16_t* plist[2];
  const uint2* runs[2];
  const SegChunk* chunks;
  const SegBin* bins;
  const uint32_t* cta0;   // first chunk of each phase-1 CTA, [grid + 1]
  uint32_t nz[2], nv[2];
  const double* scal;
  double* slots;
  uint32_t nslots;
  float d, d_over_n, n;
  int* err;
};

}  // namespace

struct SegWs {
  int log2 = 0, chunk = 0, bin = 0;
  bool usable = false;
  double build_ms = 0;
  SegPart pp[2];
  DevBuf chunks, bins, cta0;
  uint32_t nchunk = 0, nbin = 0, grid1 = 0;
};

void free_seg(graph* g) {
  SegWs* w = g->seg;
  if (!w) return;
  for (int p = 0; p < 2; ++p) {
    SegPart& P = w->pp[p];
    DevBuf* all[] = {&P.ent, &P.part, &P.plist, &P.runs, &P.deg, &P.mrow};
    for (DevBuf* b : all) dfree(g, *b);
  }
  dfree(g, w->chunks);
  dfree(g, w->bins);
  dfree(g, w->cta0);
  delete w;
  g->seg = nullptr;
}

namespace {

// ---------------------------------------------------------------------------------------
// Plan construction (device kernels; one partition at a time)
// ---------------------------------------------------------------------------------------

// Segment of an edge entry: local sources in segments [0, L), ghost slots in [L, S).
__device__ __forceinline__ uint32_t seg_of(uint32_t e, int log2, uint32_t L) {
  return (e & kRemote) ? L + ((e & kIdMask) >> log2) : (e >> log2);
}

// vrow[e] = the local vertex owning entry e (one warp per vertex, grid stride).
__global__ void k_sg_vrow(const int64_t* off, uint32_t nv, uint32_t* vrow) {
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = w0; v < nv; v += nw)
    for (int64_t e = off[v] + lane_id(); e < off[v + 1]; e += 32) vrow[e] = v;
}

// hist[key * ntiles + tile] += entries of `tile` in segment key (one warp per tile).
__global__ void k_sg_hist(const uint32_t* E, int64_t ne, int log2, uint32_t L, uint32_t ntiles,
                          uint32_t* hist) {
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t tile = w0; tile < ntiles; tile += nw) {
    const int64_t a = (int64_t)tile * kSortTile;
    const int64_t b = min(a + (int64_t)kSortTile, ne);
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane_id();
      const bool valid = e < b;
      const uint32_t key = valid ? seg_of(E[e], log2, L) : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(kFull, key);
      if (valid && (lanemask_lt() & peers) == 0)
        atomicAdd(&hist[(uint64_t)key * ntiles + tile], (uint32_t)__popc(peers));
    }
  }
}

// Stable scatter by segment: sorted position = base[key, tile] + rank within the tile.
__global__ void k_sg_scatter(const uint32_t* E, const uint32_t* vrow, int64_t ne, int log2,
                             uint32_t L, uint32_t ntiles, uint32_t* base, uint32_t* sv,
                             uint16_t* sidx) {
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t mask = (1u << log2) - 1;
  for (uint32_t tile = w0; tile < ntiles; tile += nw) {
    const int64_t a = (int64_t)tile * kSortTile;
    const int64_t b = min(a + (int64_t)kSortTile, ne);
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane_id();
      const bool valid = e < b;
      const uint32_t x = valid ? E[e] : 0u;
      const uint32_t key = valid ? seg_of(x, log2, L) : 0xFFFFFFFFu;
      const unsigned peers = __match_any_sync(kFull, key);
      const uint32_t rank = __popc(peers & lanemask_lt());
      uint32_t* slot = valid ? &base[(uint64_t)key * ntiles + tile] : nullptr;
      const uint32_t at = valid ? *slot : 0u;
      if (valid) {
        sv[at + rank] = vrow[e];
        sidx[at + rank] = (uint16_t)((x & kIdMask) & mask);
      }
      __syncwarp();
      if (valid && rank == 0) *slot = at + (uint32_t)__popc(peers);
      __syncwarp();
    }
  }
}

__global__ void k_sg_segstart(const uint32_t* base, uint32_t S, uint32_t ntiles, uint32_t ne,
                              uint32_t* segstart) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) segstart[s] = base[(uint64_t)s * ntiles];
  if (s == S) segstart[s] = ne;
}

// Row starts: a new destination, or the first entry of a chunk.
__global__ void k_sg_flags(const uint32_t* sv, uint32_t ne, uint8_t* f) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ne) f[j] = (j == 0 || sv[j] != sv[j - 1]) ? 1 : 0;
}
// Rows also start at the first entry of every chunk.
__global__ void k_sg_chunkflag(const uint32_t* ce0, uint32_t nchunk, uint8_t* f) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nchunk) f[ce0[c]] = 1;
}

// mrow[c][w]: rows of chunk c that start before mini-chunk w, the 256-entry piece of the
// chunk that warp w of phase 1 sums (all the chunk's rows if w is past its end).
__global__ void k_sg_mrow(const uint32_t* ce0, const uint32_t* cn, const uint32_t* rowid,
                          uint32_t nchunk, uint32_t ne, uint32_t P, uint16_t* mrow) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunk) return;
  const uint32_t e0 = ce0[c], e1 = e0 + cn[c], a0 = e0;
  const uint32_t r0 = rowid[e0];
  const uint32_t rend = e1 < ne ? rowid[e1] : P;
  for (uint32_t w = 0; w < kMiniPerChunk; ++w) {
    const uint32_t pos = a0 + w * kMini;
    mrow[(size_t)c * kMiniPerChunk + w] =
        (uint16_t)(w == 0 ? 0u : (pos < e1 ? rowid[pos] - r0 : rend - r0));
  }
}

// The destination of every row.
__global__ void k_sg_rowv(const uint32_t* sv, const uint8_t* f, const uint32_t* rowid,
                          uint32_t ne, uint32_t* rowv) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ne && f[j]) rowv[rowid[j]] = sv[j];
}

// Entry words of chunk c at its 16-byte-aligned place pe0[c] (one warp per chunk).
__global__ void k_sg_entpack(const uint16_t* sidx, const uint8_t* f, const uint32_t* ce0,
                             const uint32_t* cn, const uint32_t* pe0, uint32_t nchunk,
                             uint16_t* ent) {
  const uint32_t c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= nchunk) return;
  const uint32_t e0 = ce0[c], n = cn[c], o = pe0[c];
  for (uint32_t i = lane_id(); i < n; i += 32)
    ent[o + i] = (uint16_t)(sidx[e0 + i] | (f[e0 + i] ? kRowStart : 0));
}

__global__ void k_sg_chunkrow(const uint32_t* ce0, const uint32_t* rowid, uint32_t nchunk,
                              uint32_t* crow) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nchunk) crow[c] = rowid[ce0[c]];
}

// rowseg[r] = segment of row r (one thread per chunk: its rows are consecutive).
__global__ void k_sg_rowseg(const uint32_t* crow, const uint32_t* cseg, uint32_t nchunk,
                            uint32_t P, uint32_t* rowseg) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunk) return;
  const uint32_t r1 = c + 1 < nchunk ? crow[c + 1] : P;
  for (uint32_t r = crow[c]; r < r1; ++r) rowseg[r] = cseg[c];
}

__global__ void k_sg_pcount(const uint32_t* rowv, uint32_t P, uint32_t* pcount) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < P) atomicAdd(&pcount[rowv[r]], 1u);
}

__global__ void k_sg_maxp(const uint32_t* pcount, uint32_t nv, uint32_t* out) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t c = v < nv ? pcount[v] : 0u;
  c = __reduce_max_sync(kFull, c);
  if (lane_id() == 0 && c) atomicMax(out, c);
}

// Bin of a destination: a new bin starts every `wb` partial sums and every kMergeVerts
// vertices (both terms never decrease along v).
__device__ __forceinline__ uint32_t bin_key(const uint32_t* pstart, uint32_t v, uint32_t wb) {
  return pstart[v] / wb + v / kMergeVerts;
}

__global__ void k_sg_binv0(const uint32_t* pstart, uint32_t nz, uint32_t wb, uint32_t* binv0) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nz) return;
  const uint32_t k = bin_key(pstart, v, wb);
  const uint32_t kp = v ? bin_key(pstart, v - 1, wb) + 1 : 0u;
  for (uint32_t b = kp; b <= k; ++b) binv0[b] = v;  // bins skipped over start (empty) here
}

__global__ void k_sg_mc(const uint32_t* rowv, const uint32_t* rowseg, const uint32_t* pstart,
                        uint32_t P, uint32_t S, uint32_t wb, uint32_t* mc) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < P) atomicAdd(&mc[(uint64_t)bin_key(pstart, rowv[r], wb) * S + rowseg[r]], 1u);
}

// rs[k][s]: first row of segment s that falls in bin k (one thread per segment).
__global__ void k_sg_rs(const uint32_t* mc, const uint32_t* segrow0, uint32_t S, uint32_t nbin,
                        uint32_t* rs) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  uint32_t acc = segrow0[s];
  for (uint32_t k = 0; k < nbin; ++k) {
    rs[(uint64_t)k * S + s] = acc;
    acc += mc[(uint64_t)k * S + s];
  }
}

// Window placement of bin k (one thread per bin): the runs of its segments, in segment
// order, each copied as whole 16-byte granules to the next free granule of the window.
// woff[k][s] = window slot of row rs[k][s]. Pass 0 counts runs and granules; pass 1 writes
// the run records (source granule, window granule | granules << 16).
__global__ void k_sg_window(const uint32_t* mc, const uint32_t* rs, uint32_t S, uint32_t nbin,
                            int pass, uint32_t* woff, uint32_t* nruns, uint32_t* wgran,
                            const uint32_t* runoff, uint2* runs) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbin) return;
  uint32_t cur = 0, nr = 0;
  for (uint32_t s = 0; s < S; ++s) {
    const uint64_t i = (uint64_t)k * S + s;
    const uint32_t c = mc[i];
    if (!c) continue;
    const uint32_t r0 = rs[i];
    const uint32_t g0 = r0 >> 2, g1 = (r0 + c + 3) >> 2;
    if (pass == 0) woff[i] = 4 * cur + (r0 & 3);
    else runs[runoff[k] + nr] = make_uint2(g0, cur | ((g1 - g0) << 16));
    cur += g1 - g0;
    ++nr;
  }
  if (pass == 0) {
    nruns[k] = nr;
    wgran[k] = cur;
  }
}

// Window position of every row, collected per destination (unordered).
__global__ void k_sg_pos(const uint32_t* rowv, const uint32_t* rowseg, const uint32_t* pstart,
                         const uint32_t* woff, const uint32_t* rs, uint32_t P, uint32_t S,
                         uint32_t wb, uint32_t* cur, uint16_t* tmp) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P) return;
  const uint32_t v = rowv[r];
  const uint64_t i = (uint64_t)bin_key(pstart, v, wb) * S + rowseg[r];
  const uint32_t w = woff[i] + (r - rs[i]);
  tmp[pstart[v] + atomicAdd(&cur[v], 1u)] = (uint16_t)w;
}

// Each destination's positions in ascending order (= segment order), the first marked
// (one warp per vertex; rank by counting, positions of one vertex are distinct).
// Position lists are stored bin by bin, each bin's list starting at a multiple of 8
// entries: destination v's list goes to pstart[v] + shift[bin of v].
__global__ void k_sg_plist(const uint32_t* pstart, uint32_t nz, uint32_t wb, const uint16_t* tmp,
                           const uint32_t* shift, uint16_t* plist) {
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t v = w0; v < nz; v += nw) {
    const uint32_t a = pstart[v], L = pstart[v + 1] - a;
    const uint32_t o = a + shift[bin_key(pstart, v, wb)];
    for (uint32_t i = lane_id(); i < L; i += 32) {
      const uint16_t wi = tmp[a + i];
      uint32_t rank = 0;
      for (uint32_t j = 0; j < L; ++j) rank += tmp[a + j] < wi;
      plist[o + rank] = (uint16_t)(wi | (rank == 0 ? kRowStart : 0));
    }
  }
}

__global__ void k_sg_deg(const int64_t* off, uint32_t nv, uint32_t* deg) {
  const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) deg[v] = (uint32_t)(off[v + 1] - off[v]);
}

__global__ void k_sg_gather_u32(const uint32_t* src, const uint32_t* idx, uint32_t n,
                                uint32_t* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = src[idx[i]];
}

// Scoped device buffers of the plan build: freed on every exit.
struct Temps {
  graph* g;
  std::vector<DevBuf> bufs;
  explicit Temps(graph* gg_) : g(gg_) {}
  ~Temps() {
    for (DevBuf& b : bufs) dfree(g, b);
  }
  graph_status get(size_t bytes, void** p) {
    bufs.emplace_back();
    const graph_status s = dalloc(g, bufs.back(), bytes ? bytes : 16);
    *p = bufs.back().p;
    return s;
  }
};

template <class T>
graph_status to_host(graph* g, std::vector<T>& h, const void* d, size_t n) {
  h.resize(n);
  if (n) GG_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, g->stream));
  GG_CUDA(cudaStreamSynchronize(g->stream));
  return GRAPH_OK;
}

template <class T>
graph_status to_dev(graph* g, void* d, const std::vector<T>& h) {
  if (!h.empty())
    GG_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, g->stream));
  GG_CUDA(cudaStreamSynchronize(g->stream));
  return GRAPH_OK;
}

// Host records of one partition's plan, merged into the unified tables afterwards.
struct PartHost {
  std::vector<SegChunk> chunks;
  std::vector<SegBin> bins;
};

// Builds partition p's plan. *fits = false (and nothing kept) when a limit of the layout is
// exceeded.
graph_status build_part(graph* g, int p, int log2, uint32_t ce, uint32_t wb, SegPart& SP,
                        PartHost& H, uint32_t key0, bool* fits) {
  *fits = false;
  const Part& P = g->part[p];
  cudaStream_t st = g->stream;
  const uint32_t nv = P.nv, nout = P.nout;
  const uint32_t seg = 1u << log2;
  if (P.ne >= (int64_t)0x7FFFFFF0) return GRAPH_OK;     // 32-bit entry and row indices
  const uint32_t ne = (uint32_t)P.ne;
  SP.L = (nv + seg - 1) / seg;
  SP.S = SP.L + (nout + seg - 1) / seg;
  SP.nz = P.cls_end[1];
  const uint32_t S = SP.S;
  // A bin's window holds fewer than wb + kMaxPartials partial sums plus at most 6 slots of
  // granule padding per run (one run per segment): keep it within the 15-bit positions.
  if ((uint64_t)kMaxPartials + 6ull * S + 64 >= kWinMax) return GRAPH_OK;
  wb = std::min<uint32_t>(wb, kWinMax - kMaxPartials - 6 * S - 1);
  GG_TRY(dalloc(g, SP.deg, 4ull * nv + 64));
  if (nv) {
    k_sg_deg<<<grid_for(nv, 256), 256, 0, st>>>((const int64_t*)P.off.p, nv, (uint32_t*)SP.deg.p);
    GG_CUDA(cudaGetLastError());
  }
  if (ne == 0) {
    *fits = true;
    GG_TRY(dalloc(g, SP.mrow, 64));
    GG_TRY(dalloc(g, SP.ent, 64));
    GG_TRY(dalloc(g, SP.part, 64));
    GG_TRY(dalloc(g, SP.plist, 64));
    GG_TRY(dalloc(g, SP.runs, 64));
    return GRAPH_OK;
  }
  const uint32_t ntiles = (ne + kSortTile - 1) / kSortTile;
  if ((uint64_t)S * ntiles >= (1ull << 28)) return GRAPH_OK;
  Temps T(g);
  uint32_t *vrow, *hist, *sv, *rowid, *segstart;
  uint16_t* sidx;
  uint8_t* f;
  GG_TRY(T.get(4ull * ne, (void**)&vrow));
  GG_TRY(T.get(4ull * S * ntiles, (void**)&hist));
  GG_TRY(T.get(4ull * ne, (void**)&sv));
  GG_TRY(T.get(2ull * ne, (void**)&sidx));
  GG_TRY(T.get(4ull * (S + 1), (void**)&segstart));
  const uint32_t* E = (const uint32_t*)P.E.p;
  const int64_t* off = (const int64_t*)P.off.p;
  const unsigned gridw = 152 * 8;
  k_sg_vrow<<<gridw, 256, 0, st>>>(off, nv, vrow);
  GG_CUDA(cudaMemsetAsync(hist, 0, 4ull * S * ntiles, st));
  k_sg_hist<<<gridw, 256, 0, st>>>(E, ne, log2, SP.L, ntiles, hist);
  GG_CUDA(cudaGetLastError());
  GG_TRY(exclusive_scan_u32(g, hist, hist, (uint64_t)S * ntiles, nullptr));
  k_sg_segstart<<<grid_for(S + 1, 256), 256, 0, st>>>(hist, S, ntiles, ne, segstart);
  k_sg_scatter<<<gridw, 256, 0, st>>>(E, vrow, ne, log2, SP.L, ntiles, hist, sv, sidx);
  GG_CUDA(cudaGetLastError());
  std::vector<uint32_t> hseg;
  GG_TRY(to_host(g, hseg, segstart, S + 1));

  // Chunks: consecutive entries of one segment, at most ce each.
  std::vector<uint32_t> ce0, cseg;
  for (uint32_t s = 0; s < S; ++s)
    for (uint32_t a = hseg[s]; a < hseg[s + 1]; a += ce) {
      ce0.push_back(a);
      cseg.push_back(s);
    }
  const uint32_t nchunk = (uint32_t)ce0.size();
  std::vector<uint32_t> cn(nchunk);
  for (uint32_t c = 0; c < nchunk; ++c) cn[c] = std::min(ce, hseg[cseg[c] + 1] - ce0[c]);
  uint32_t *dce0, *dcseg, *dcrow, *dcn;
  GG_TRY(T.get(4ull * nchunk, (void**)&dce0));
  GG_TRY(T.get(4ull * nchunk, (void**)&dcseg));
  GG_TRY(T.get(4ull * nchunk, (void**)&dcrow));
  GG_TRY(T.get(4ull * nchunk, (void**)&dcn));
  GG_TRY(to_dev(g, dce0, ce0));
  GG_TRY(to_dev(g, dcseg, cseg));
  GG_TRY(to_dev(g, dcn, cn));

  GG_TRY(T.get(ne, (void**)&f));
  GG_TRY(T.get(4ull * ne, (void**)&rowid));
  k_sg_flags<<<grid_for(ne, 256), 256, 0, st>>>(sv, ne, f);
  k_sg_chunkflag<<<grid_for(nchunk, 256), 256, 0, st>>>(dce0, nchunk, f);
  GG_CUDA(cudaGetLastError());
  uint32_t nrow = 0;
  GG_TRY(exclusive_scan_u8_to_u32(g, f, rowid, ne, &nrow));
  if (nrow >= 0x7FFFFFF0u) return GRAPH_OK;
  SP.P = nrow;
  // chunks start at 16-byte-aligned entry positions (the frame of phase 1 begins exactly at
  // a chunk's first entry)
  std::vector<uint32_t> pe0(nchunk);
  uint64_t packed = 0;
  for (uint32_t c = 0; c < nchunk; ++c) {
    pe0[c] = (uint32_t)packed;
    packed += (cn[c] + 7) & ~7u;
  }
  if (packed >= 0xFFFFFFF0ull) return GRAPH_OK;
  uint32_t* dpe0;
  GG_TRY(T.get(4ull * nchunk, (void**)&dpe0));
  GG_TRY(to_dev(g, dpe0, pe0));
  GG_TRY(dalloc(g, SP.ent, 2ull * packed + 64));
  GG_CUDA(cudaMemsetAsync(SP.ent.p, 0, 2ull * packed + 64, st));
  uint32_t *rowv, *rowseg;
  GG_TRY(T.get(4ull * nrow, (void**)&rowv));
  GG_TRY(T.get(4ull * nrow, (void**)&rowseg));
  k_sg_rowv<<<grid_for(ne, 256), 256, 0, st>>>(sv, f, rowid, ne, rowv);
  k_sg_entpack<<<grid_for(32ull * nchunk, 256), 256, 0, st>>>(sidx, f, dce0, dcn, dpe0, nchunk,
                                                              (uint16_t*)SP.ent.p);
  GG_CUDA(cudaGetLastError());
  k_sg_chunkrow<<<grid_for(nchunk, 256), 256, 0, st>>>(dce0, rowid, nchunk, dcrow);
  GG_TRY(dalloc(g, SP.mrow, 2ull * kMiniPerChunk * nchunk + 64));
  k_sg_mrow<<<grid_for(nchunk, 128), 128, 0, st>>>(dce0, dcn, rowid, nchunk, ne, nrow,
                                                   (uint16_t*)SP.mrow.p);
  k_sg_rowseg<<<grid_for(nchunk, 128), 128, 0, st>>>(dcrow, dcseg, nchunk, nrow, rowseg);
  GG_CUDA(cudaGetLastError());
  std::vector<uint32_t> crow;
  GG_TRY(to_host(g, crow, dcrow, nchunk));

  // Partial sums per destination and the bins of phase 2.
  uint32_t *pcount, *pstart, *dmax;
  GG_TRY(T.get(4ull * (nv + 1), (void**)&pcount));
  GG_TRY(T.get(4ull * (nv + 1), (void**)&pstart));
  GG_TRY(T.get(4, (void**)&dmax));
  GG_CUDA(cudaMemsetAsync(pcount, 0, 4ull * (nv + 1), st));
  GG_CUDA(cudaMemsetAsync(dmax, 0, 4, st));
  k_sg_pcount<<<grid_for(nrow, 256), 256, 0, st>>>(rowv, nrow, pcount);
  k_sg_maxp<<<grid_for(nv, 256), 256, 0, st>>>(pcount, nv, dmax);
  GG_CUDA(cudaGetLastError());
  uint32_t total = 0;
  GG_TRY(exclusive_scan_u32(g, pcount, pstart, nv + 1, &total));
  std::vector<uint32_t> hmax;
  GG_TRY(to_host(g, hmax, dmax, 1));
  if (hmax[0] > kMaxPartials || total != nrow) return GRAPH_OK;
  const uint32_t nz = SP.nz;
  std::vector<uint32_t> hlast;
  GG_TRY(to_host(g, hlast, pstart + (nz ? nz - 1 : 0), 1));
  const uint32_t nbin = nz ? hlast[0] / wb + (nz - 1) / kMergeVerts + 1 : 0;
  if ((uint64_t)nbin * S >= (1ull << 28)) return GRAPH_OK;
  SP.nbin = nbin;
  uint32_t *binv0, *mc, *rs, *woff, *nruns, *wgran, *runoff, *segrow0;
  GG_TRY(T.get(4ull * (nbin + 1), (void**)&binv0));
  GG_TRY(T.get(4ull * nbin * S, (void**)&mc));
  GG_TRY(T.get(4ull * nbin * S, (void**)&rs));
  GG_TRY(T.get(4ull * nbin * S, (void**)&woff));
  GG_TRY(T.get(4ull * (nbin + 1), (void**)&nruns));
  GG_TRY(T.get(4ull * (nbin + 1), (void**)&wgran));
  GG_TRY(T.get(4ull * (nbin + 1), (void**)&runoff));
  GG_TRY(T.get(4ull * S, (void**)&segrow0));
  k_sg_binv0<<<grid_for(nz, 256), 256, 0, st>>>(pstart, nz, wb, binv0);
  GG_CUDA(cudaMemcpyAsync(binv0 + nbin, &nz, 4, cudaMemcpyHostToDevice, st));
  GG_CUDA(cudaMemsetAsync(mc, 0, 4ull * nbin * S, st));
  k_sg_mc<<<grid_for(nrow, 256), 256, 0, st>>>(rowv, rowseg, pstart, nrow, S, wb, mc);
  GG_CUDA(cudaGetLastError());
  // first row of every segment (segments without entries: never read)
  std::vector<uint32_t> hsegrow0(S, 0);
  for (uint32_t c = 0; c < nchunk; ++c)
    if (c == 0 || cseg[c] != cseg[c - 1]) hsegrow0[cseg[c]] = crow[c];
  GG_TRY(to_dev(g, segrow0, hsegrow0));
  k_sg_rs<<<grid_for(S, 128), 128, 0, st>>>(mc, segrow0, S, nbin, rs);
  k_sg_window<<<grid_for(nbin, 128), 128, 0, st>>>(mc, rs, S, nbin, 0, woff, nruns, wgran,
                                                   nullptr, nullptr);
  GG_CUDA(cudaGetLastError());
  uint32_t R = 0;
  GG_TRY(exclusive_scan_u32(g, nruns, runoff, nbin, &R));
  GG_CUDA(cudaMemcpyAsync(runoff + nbin, &R, 4, cudaMemcpyHostToDevice, st));
  SP.nruns = R;
  GG_TRY(dalloc(g, SP.runs, 8ull * R + 16));
  k_sg_window<<<grid_for(nbin, 128), 128, 0, st>>>(mc, rs, S, nbin, 1, woff, nruns, wgran,
                                                   runoff, (uint2*)SP.runs.p);
  GG_CUDA(cudaGetLastError());
  std::vector<uint32_t> hbinv0, hwgran, hrunoff, hbinpos;
  GG_TRY(to_host(g, hbinv0, binv0, nbin + 1));
  GG_TRY(to_host(g, hwgran, wgran, nbin));
  GG_TRY(to_host(g, hrunoff, runoff, nbin + 1));
  for (uint32_t k = 0; k < nbin; ++k)
    if (4ull * hwgran[k] > kWinMax) return GRAPH_OK;
  {
    uint32_t* bpos;
    GG_TRY(T.get(4ull * (nbin + 1), (void**)&bpos));
    k_sg_gather_u32<<<grid_for(nbin + 1, 256), 256, 0, st>>>(pstart, binv0, nbin + 1, bpos);
    GG_CUDA(cudaGetLastError());
    GG_TRY(to_host(g, hbinpos, bpos, nbin + 1));
  }

  // Position lists, each bin's starting at a multiple of 8 entries.
  std::vector<uint32_t> hppos(nbin + 1), hshift(nbin + 1, 0);
  {
    uint64_t acc = 0;
    for (uint32_t k = 0; k < nbin; ++k) {
      hppos[k] = (uint32_t)acc;
      hshift[k] = hppos[k] - hbinpos[k];   // modulo 2^32
      acc += ((uint64_t)(hbinpos[k + 1] - hbinpos[k]) + 7) & ~7ull;
    }
    if (acc >= 0xFFFFFFF0ull) return GRAPH_OK;
    hppos[nbin] = (uint32_t)acc;
  }
  uint32_t *cur, *dshift;
  uint16_t* tmp;
  GG_TRY(T.get(4ull * nv, (void**)&cur));
  GG_TRY(T.get(2ull * nrow, (void**)&tmp));
  GG_TRY(T.get(4ull * (nbin + 1), (void**)&dshift));
  GG_TRY(to_dev(g, dshift, hshift));
  GG_TRY(dalloc(g, SP.plist, 2ull * hppos[nbin] + 64));
  GG_CUDA(cudaMemsetAsync(SP.plist.p, 0, 2ull * hppos[nbin] + 64, st));
  GG_CUDA(cudaMemsetAsync(cur, 0, 4ull * nv, st));
  k_sg_pos<<<grid_for(nrow, 256), 256, 0, st>>>(rowv, rowseg, pstart, woff, rs, nrow, S, wb,
                                                cur, tmp);
  k_sg_plist<<<gridw, 256, 0, st>>>(pstart, nz, wb, tmp, dshift, (uint16_t*)SP.plist.p);
  GG_CUDA(cudaGetLastError());
  GG_TRY(dalloc(g, SP.part, 4ull * nrow + 64));
  GG_CUDA(cudaMemsetAsync(SP.part.p, 0, 4ull * nrow + 64, st));

  // Host records.
  H.chunks.resize(nchunk);
  for (uint32_t c = 0; c < nchunk; ++c) {
    SegChunk& C = H.chunks[c];
    const uint32_t s = cseg[c];
    C.e0 = pe0[c];
    C.nent = cn[c];
    C.row0 = crow[c];
    C.cl = c;
    C.ghost = s >= SP.L;
    C.src0 = (s >= SP.L ? s - SP.L : s) << log2;
    const uint32_t lim = C.ghost ? nout : nv;
    C.srclen = std::min(seg, lim - C.src0);
    C.key = key0 + s;
    C.part = (uint8_t)p;
    C.pad = 0;
  }
  H.bins.resize(nbin);
  for (uint32_t k = 0; k < nbin; ++k) {
    SegBin& B = H.bins[k];
    B.v0 = hbinv0[k];
    B.v1 = hbinv0[k + 1];
    B.run0 = hrunoff[k];
    B.run1 = hrunoff[k + 1];
    B.pos0 = hppos[k];
    B.npos = hbinpos[k + 1] - hbinpos[k];
    B.wgran = hwgran[k];
    B.part = (uint32_t)p;
  }
  SP.nchunk = nchunk;
  GG_CUDA(cudaStreamSynchronize(st));
  *fits = true;
  return GRAPH_OK;
}

void free_seg_part(graph* g, SegPart& SP) {
  DevBuf* all[] = {&SP.ent, &SP.part, &SP.plist, &SP.runs, &SP.deg, &SP.mrow};
  for (DevBuf* b : all) dfree(g, *b);
  SP = SegPart();
}

int sm_count(graph* g) {
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

// ---------------------------------------------------------------------------------------
// The deterministic segmented sum used by both phases.
// ---------------------------------------------------------------------------------------
// Staged 2-byte entries (table offset | row-start bit) are split into mini-chunks of kMini
// entries, one per warp, 8 consecutive entries per lane. A row-start bit begins a new row.
// A warp sums its mini-chunk on its own: warp-uniform fast paths when the mini-chunk has no
// row start (one sum) or a row start at every entry (the rows are the gathered values);
// otherwise each lane summarises its entries as (sum since its last row start, or of all of
// them; number of row starts), an exclusive warp scan of these summaries gives each lane
// the running value of the row open at its first entry, and a walk closes rows at row
// starts. Completed rows go to a shared-memory row buffer at index pad_row(row) (one
// skipped slot every 16 rows, so that lanes closing rows 8 or 16 apart write different
// banks); the entries before a mini-chunk's first row start (its head) continue a row of an
// earlier mini-chunk and are added to it afterwards, in mini-chunk order. Every row's value
// therefore has one fixed summation order, whatever the timing.
__device__ __forceinline__ int pad_row(int r) { return r + (r >> 4); }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// ---------------------------------------------------------------------------------------
// Phase 1: partial sum of every (segment, destination) row.
// ---------------------------------------------------------------------------------------
// A chunk's entries are staged as a frame of kMiniPerChunk mini-chunks of kMini entries
// (16-byte aligned); warp w sums mini-chunk w on its own: a warp-level version of the
// segmented sum above, with the rows that start in its mini-chunk in a private shared-memory
// buffer. A row that runs past the end of a mini-chunk continues in the next ones: each
// warp also leaves the head of its mini-chunk (the entries before its first row start, or
// all of them) and whether it has a row start. After one CTA barrier every warp writes its
// rows to the partial sums (coalesced, at the mini-chunk's staged row offset), adding to its
// last row the heads of the following mini-chunks in order up to the next row start, so
// every row keeps one fixed summation order. A second barrier frees the frame and, at a
// segment change, the slice.
constexpr int kSegThreads = 1024;                      // phase-1 CTA (one per SM)
constexpr int kSegK = 8;                               // entries per lane of a mini-chunk
constexpr int kFrame = kMiniPerChunk * kMini;          // 8192 staged entries
constexpr int kSegStages = 3;                          // chunks staged ahead
constexpr int kFrameBytes = 2 * kFrame + 2 * kMiniPerChunk;   // entries, then row offsets
constexpr int kWarpRows = kMini + kMini / 16 + 16;     // padded rows of one mini-chunk
static_assert(kMini == 32 * kSegK && kSegThreads / 32 == (int)kMiniPerChunk, "warp per mini-chunk");

template <class XT>
__host__ __device__ constexpr size_t seg_slice_bytes(int log2) {
  return ((sizeof(XT) << log2) + 127) & ~(size_t)127;
}
template <class XT>
__host__ __device__ constexpr size_t seg_smem_bytes(int log2) {
  return seg_slice_bytes<XT>(log2) + kSegStages * (size_t)kFrameBytes +
         4 * (size_t)kWarpRows * (kSegThreads / 32);
}

// Thread 0: bulk copies of chunk c's entries (whole 16-byte granules from the granule
// holding its first entry) and of its mini-chunk row offsets into `frame`.
__device__ __forceinline__ void seg_issue_chunk(const SegArgs& A, const SegChunk& C,
                                                unsigned char* frame, uint64_t* bar) {
  const uint32_t a0 = C.e0 & ~7u;
  const uint32_t bytes = (((C.e0 - a0) + C.nent) * 2 + 15) & ~15u;
  mbar_expect_tx(bar, bytes + 2 * kMiniPerChunk);
  const uint64_t pol = l2_evict_first_policy();
  bulk_g2s_stream(frame, A.ent[C.part] + a0, bytes, bar, pol);
  bulk_g2s_stream(frame + 2 * kFrame, A.mrow[C.part] + (size_t)C.cl * kMiniPerChunk,
                  2 * kMiniPerChunk, bar, pol);
}

template <class XT>
__global__ void __launch_bounds__(kSegThreads, 1)
k_pr_seg(const __grid_constant__ SegArgs A, int log2) {
  extern __shared__ __align__(128) unsigned char smem[];
  XT* slice = reinterpret_cast<XT*>(smem);
  unsigned char* frames = smem + seg_slice_bytes<XT>(log2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* rows = reinterpret_cast<float*>(frames + kSegStages * (size_t)kFrameBytes) +
                warp * kWarpRows;
  __shared__ uint64_t bar_slice, bar_chunk[kSegStages];
  __shared__ float head_sh[kMiniPerChunk];    // head of each mini-chunk (see above)
  __shared__ int starts_sh[kMiniPerChunk];    // the mini-chunk has a row start
  const uint32_t c0 = A.cta0[blockIdx.x], c1 = A.cta0[blockIdx.x + 1];
  if (c0 >= c1) return;
  uint32_t phases = 0;       // bit s: parity of bar_chunk[s]; bit 4: bar_slice
  uint32_t outstanding = 0;  // (thread 0) bit s: a copy on bar_chunk[s] not yet waited for;
                             // bit 4: the slice copy
  if (threadIdx.x == 0) {
    mbar_init(&bar_slice, 1);
    for (int s = 0; s < kSegStages; ++s) mbar_init(&bar_chunk[s], 1);
    fence_mbar_init();
    for (uint32_t k = 0; k < kSegStages - 1 && c0 + k < c1; ++k) {
      seg_issue_chunk(A, A.chunks[c0 + k], frames + k * kFrameBytes, &bar_chunk[k]);
      outstanding |= 1u << k;
    }
  }
  __syncthreads();
  uint32_t key = 0xFFFFFFFFu;
  bool ok = true;
  int stage = 0;
  for (uint32_t c = c0; c < c1; ++c, stage = stage + 1 == kSegStages ? 0 : stage + 1) {
    const SegChunk C = A.chunks[c];
    if (C.key != key) {
      // every thread finished the previous chunk (barrier at the end of the loop body)
      if (threadIdx.x == 0) {
        const XT* src = reinterpret_cast<const XT*>(C.ghost ? A.ghost[C.part] : A.x[C.part]) + C.src0;
        const uint32_t bytes = (uint32_t)((C.srclen * sizeof(XT) + 15) & ~(size_t)15);
        mbar_expect_tx(&bar_slice, bytes);
        bulk_g2s(slice, src, bytes, &bar_slice);
        outstanding |= 16u;
      }
      ok = mbar_wait_bounded(&bar_slice, (phases >> 4) & 1u, A.err);
      if (ok) {
        phases ^= 16u;
        outstanding &= ~16u;
      }
      key = C.key;
      if (!__syncthreads_and(ok)) break;
    }
    if (threadIdx.x == 0 && c + kSegStages - 1 < c1) {
      const int s2 = (stage + kSegStages - 1) % kSegStages;   // freed by chunk c - 1
      seg_issue_chunk(A, A.chunks[c + kSegStages - 1], frames + s2 * kFrameBytes,
                      &bar_chunk[s2]);
      outstanding |= 1u << s2;
    }
    ok = mbar_wait_bounded(&bar_chunk[stage], (phases >> stage) & 1u, A.err);
    if (ok) {
      phases ^= 1u << stage;
      outstanding &= ~(1u << stage);
    }
    if (!__syncthreads_and(ok)) break;
    const uint16_t* frame = reinterpret_cast<const uint16_t*>(frames + stage * kFrameBytes);
    const int lo = (int)(C.e0 & 7u), hi = lo + (int)C.nent;
    const int m0 = warp * (int)kMini;
    int nrows = 0;
    if (m0 < hi) {  // warp-uniform: this warp's mini-chunk has entries
      const int j0 = m0 + lane * kSegK;
      const uint4 q = *reinterpret_cast<const uint4*>(frame + j0);
      const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
      const bool full = m0 + (int)kMini <= hi;
      const uint32_t fl_or = (q.x | q.y | q.z | q.w) & 0x80008000u;
      const uint32_t fl_and = q.x & q.y & q.z & q.w & 0x80008000u;
      if (full && !__any_sync(kFull, fl_or != 0)) {
        // no row start (long rows): the whole mini-chunk continues the open row
        float sum = 0.f;
        #pragma unroll
        for (int k = 0; k < kSegK; ++k)
          sum += to_f(slice[(k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu)]);
        sum = warp_sum(sum);
        if (lane == 0) {
          head_sh[warp] = sum;
          starts_sh[warp] = 0;
        }
        goto written;
      }
      if (full && __all_sync(kFull, fl_and == 0x80008000u)) {
        // every entry starts a row of its own: the rows are the gathered values
        #pragma unroll
        for (int k = 0; k < kSegK; ++k) {
          const uint32_t e = (k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu);
          rows[pad_row(lane * kSegK + k)] = to_f(slice[e & kOffMask]);
        }
        nrows = (int)kMini;
        if (lane == 0) {
          head_sh[warp] = 0.f;
          starts_sh[warp] = 1;
        }
        goto written;
      }
      float val[kSegK];
      uint32_t fm = 0;
      #pragma unroll
      for (int k = 0; k < kSegK; ++k) {
        const bool in = j0 + k >= lo && j0 + k < hi;
        const uint32_t e = in ? ((k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu)) : 0u;
        fm |= (e >> 15) << k;
        val[k] = in ? to_f(slice[e & kOffMask]) : 0.f;
      }
      // warp-level segmented scan: (sum since the lane's last row start, row starts)
      float v = 0.f;
      #pragma unroll
      for (int k = 0; k < kSegK; ++k) v = ((fm >> k) & 1u) ? val[k] : v + val[k];
      int n = __popc(fm);
      #pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float yv = __shfl_up_sync(kFull, v, o);
        const int yn = __shfl_up_sync(kFull, n, o);
        if (lane >= o) {
          v = n > 0 ? v : yv + v;
          n += yn;
        }
      }
      nrows = __shfl_sync(kFull, n, 31);
      float ev = __shfl_up_sync(kFull, v, 1);
      int en = __shfl_up_sync(kFull, n, 1);
      if (lane == 0) {
        ev = 0.f;
        en = 0;
      }
      // walk: close the open row at each row start; row -1 is the head (a row of an
      // earlier mini-chunk)
      int row = en - 1;
      float acc = ev;
      #pragma unroll
      for (int k = 0; k < kSegK; ++k) {
        if ((fm >> k) & 1u) {
          if (row >= 0) rows[pad_row(row)] = acc;
          else head_sh[warp] = acc;
          ++row;
          acc = 0.f;
        }
        acc += val[k];
      }
      const int last = min(hi, m0 + (int)kMini) - 1;   // the mini-chunk's last entry
      if (j0 <= last && last < j0 + kSegK) {
        if (row >= 0) rows[pad_row(row)] = acc;
        else head_sh[warp] = acc;                      // no row start at all
      }
      if (lane == 0) starts_sh[warp] = nrows > 0;
    } else if (lane == 0) {
      starts_sh[warp] = 1;   // past the chunk's end: ends every carry
      head_sh[warp] = 0.f;
    }
  written:
    __syncthreads();
    if (nrows > 0) {
      const uint16_t* mrow = reinterpret_cast<const uint16_t*>(frames + stage * kFrameBytes +
                                                               2 * kFrame);
      float* part = A.part[C.part] + C.row0 + mrow[warp];
      for (int j = lane; j < nrows; j += 32) {
        float x = rows[pad_row(j)];
        if (j == nrows - 1)   // the row open at the end continues in the next mini-chunks
          for (int w2 = warp + 1; w2 < (int)kMiniPerChunk; ++w2) {
            x += head_sh[w2];
            if (starts_sh[w2]) break;
          }
        part[j] = x;
      }
    }
    __syncthreads();  // the frame, the row buffers and the slice are free again
  }
  if (!ok && threadIdx.x == 0) {
    // copies may still be in flight into shared memory: wait for them (bounded) first
    if (outstanding & 16u) mbar_wait_bounded(&bar_slice, (phases >> 4) & 1u, A.err);
    for (int s = 0; s < kSegStages; ++s)
      if (outstanding & (1u << s)) mbar_wait_bounded(&bar_chunk[s], (phases >> s) & 1u, A.err);
  }
}

// ---------------------------------------------------------------------------------------
// Phase 2: per bin, add each destination's partial sums and update the vertex.
// ---------------------------------------------------------------------------------------
constexpr int kMergeThreads = 512;                     // phase-2 CTA (two per SM)
constexpr int kMergeK = 8;
constexpr int kMergeFrame = kMergeThreads * kMergeK;   // 4096 staged positions per pass
constexpr int kMergePass = kMergeFrame;                // positions per pass (bins start aligned)
constexpr int kRowBuf2 = kMergeVerts + kMergeVerts / 16 + 32;
constexpr size_t kMWin = 4ull * kWinMax;
constexpr size_t kMPos = 2ull * kMergeFrame;                 // one position frame
constexpr size_t kMDeg = 4ull * (kMergeVerts + 8);
constexpr size_t kMRank = 4ull * (kMergeVerts + 8);
constexpr size_t kMergeSmem = kMWin + 2 * kMPos + kMDeg + kMRank + 4ull * kRowBuf2;

__device__ __forceinline__ void merge_issue_pos(const uint16_t* plist, uint32_t start,
                                                uint32_t cnt, uint16_t* frame, uint64_t* bar) {
  const uint32_t a0 = start & ~7u;
  const uint32_t bytes = (((start - a0) + cnt) * 2 + 15) & ~15u;
  mbar_expect_tx(bar, bytes);
  bulk_g2s_stream(frame, plist + a0, bytes, bar, l2_evict_first_policy());
}

// One pass of a bin: kMergeFrame positions, one mini-chunk of kMini per warp, summed like
// phase 1 (warp-uniform fast paths, else a warp-level segmented sum); rows are the bin's
// vertices. A row that runs past its mini-chunk (or pass) is finished by thread 0, which
// adds the following mini-chunks' heads to it in order after the pass.
template <class XT, bool SCALED>
__global__ void __launch_bounds__(kMergeThreads, 2) k_pr_merge(const __grid_constant__ SegArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* win = reinterpret_cast<float*>(smem);
  uint16_t* pframe = reinterpret_cast<uint16_t*>(smem + kMWin);
  uint32_t* sdeg = reinterpret_cast<uint32_t*>(smem + kMWin + 2 * kMPos);
  float* sr = reinterpret_cast<float*>(smem + kMWin + 2 * kMPos + kMDeg);
  float* rowbuf = reinterpret_cast<float*>(smem + kMWin + 2 * kMPos + kMDeg + kMRank);
  constexpr int NW = kMergeThreads / 32;
  __shared__ uint64_t bar_w, bar_p[2];
  __shared__ int cnt_sh[NW], starts_sh[NW], last_sh[NW];
  __shared__ float head_sh[NW];
  __shared__ int rows_sh, pending_sh;
  __shared__ float red[NW];
  const SegBin B = A.bins[blockIdx.x];
  if (B.v0 >= B.v1) return;
  const int p = (int)B.part;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t q0 = B.v0 & ~3u;
  const uint32_t npass = (B.npos + kMergePass - 1) / kMergePass;
  if (threadIdx.x == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_p[0], 1);
    mbar_init(&bar_p[1], 1);
    fence_mbar_init();
    const uint32_t vbytes = ((B.v1 - q0) * 4 + 15) & ~15u;
    mbar_expect_tx(&bar_w, 16u * B.wgran + 2 * vbytes);
    const uint64_t pol = l2_evict_first_policy();
    bulk_g2s_stream(sdeg, A.deg[p] + q0, vbytes, &bar_w, pol);
    bulk_g2s_stream(sr, reinterpret_cast<const float*>(A.r[p]) + q0, vbytes, &bar_w, pol);
    merge_issue_pos(A.plist[p], B.pos0, min(B.npos, (uint32_t)kMergePass), pframe, &bar_p[0]);
    rows_sh = 0;
    pending_sh = -1;
  }
  __syncthreads();
  {
    const uint2* runs = A.runs[p];
    const float* part = A.part[p];
    const uint64_t pol = l2_evict_first_policy();
    for (uint32_t i = B.run0 + threadIdx.x; i < B.run1; i += kMergeThreads) {
      const uint2 R = runs[i];
      bulk_g2s_stream(win + 4 * (R.y & 0xFFFF), part + 4ull * R.x, 16u * (R.y >> 16), &bar_w, pol);
    }
  }
  const bool okw = mbar_wait_bounded(&bar_w, 0, A.err);
  bool ok = okw;
  uint32_t ph = 0;                 // bit b: parity of bar_p[b]
  uint32_t out_p = 1;              // (thread 0) bit b: a copy on bar_p[b] not yet waited for
  for (uint32_t q = 0; q < npass; ++q) {
    const int b = q & 1;
    const uint32_t start = B.pos0 + q * kMergePass;
    const uint32_t cnt = min(B.npos - q * kMergePass, (uint32_t)kMergePass);
    if (threadIdx.x == 0 && q + 1 < npass) {
      merge_issue_pos(A.plist[p], start + cnt,
                      min(B.npos - (q + 1) * kMergePass, (uint32_t)kMergePass),
                      pframe + (1 - b) * kMergeFrame, &bar_p[1 - b]);
      out_p |= 2u >> b;
    }
    const bool okp = ok && mbar_wait_bounded(&bar_p[b], (ph >> b) & 1u, A.err);
    if (okp) {
      ph ^= 1u << b;
      out_p &= ~(1u << b);
    }
    ok = okp;
    if (!__syncthreads_and(ok)) break;
    const uint16_t* frame = pframe + b * kMergeFrame;
    const int hi = (int)cnt;             // frames start at multiples of 8 entries
    const int m0 = warp * (int)kMini;
    const int j0 = m0 + lane * kMergeK;
    uint4 qv = make_uint4(0, 0, 0, 0);
    if (m0 < hi) qv = *reinterpret_cast<const uint4*>(frame + j0);
    const uint32_t wd[4] = {qv.x, qv.y, qv.z, qv.w};
    uint32_t fm = 0;
    #pragma unroll
    for (int k = 0; k < kMergeK; ++k) {
      const uint32_t e = (k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu);
      if (j0 + k < hi) fm |= (e >> 15) << k;
    }
    const int nflag = __reduce_add_sync(kFull, __popc(fm));
    if (lane == 0) cnt_sh[warp] = nflag;
    __syncthreads();
    int rb = rows_sh;   // rows of the bin that start before this warp's mini-chunk
    for (int w2 = 0; w2 < warp; ++w2) rb += cnt_sh[w2];
    if (m0 < hi) {
      const bool full = m0 + (int)kMini <= hi;
      if (full && nflag == 0) {
        float sum = 0.f;
        #pragma unroll
        for (int k = 0; k < kMergeK; ++k)
          sum += win[(k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu)];
        sum = warp_sum(sum);
        if (lane == 0) head_sh[warp] = sum;
      } else if (full && nflag == (int)kMini) {
        #pragma unroll
        for (int k = 0; k < kMergeK; ++k) {
          const uint32_t e = (k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu);
          rowbuf[pad_row(rb + lane * kMergeK + k)] = win[e & kOffMask];
        }
        if (lane == 0) head_sh[warp] = 0.f;
      } else {
        float val[kMergeK];
        #pragma unroll
        for (int k = 0; k < kMergeK; ++k) {
          const uint32_t e = (k & 1) ? (wd[k >> 1] >> 16) : (wd[k >> 1] & 0xFFFFu);
          val[k] = j0 + k < hi ? win[e & kOffMask] : 0.f;
        }
        float v = 0.f;
        #pragma unroll
        for (int k = 0; k < kMergeK; ++k) v = ((fm >> k) & 1u) ? val[k] : v + val[k];
        int n = __popc(fm);
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float yv = __shfl_up_sync(kFull, v, o);
          const int yn = __shfl_up_sync(kFull, n, o);
          if (lane >= o) {
            v = n > 0 ? v : yv + v;
            n += yn;
          }
        }
        float ev = __shfl_up_sync(kFull, v, 1);
        int en = __shfl_up_sync(kFull, n, 1);
        if (lane == 0) {
          ev = 0.f;
          en = 0;
        }
        int row = en - 1;   // local row; -1: the head
        float acc = ev;
        #pragma unroll
        for (int k = 0; k < kMergeK; ++k) {
          if ((fm >> k) & 1u) {
            if (row >= 0) rowbuf[pad_row(rb + row)] = acc;
            else head_sh[warp] = acc;
            ++row;
            acc = 0.f;
          }
          acc += val[k];
        }
        const int last = min(hi, m0 + (int)kMini) - 1;
        if (j0 <= last && last < j0 + kMergeK) {
          if (row >= 0) rowbuf[pad_row(rb + row)] = acc;
          else head_sh[warp] = acc;
        }
      }
      if (lane == 0) {
        starts_sh[warp] = nflag > 0;
        last_sh[warp] = rb + nflag - 1;
      }
    } else if (lane == 0) {   // past the pass's end: contributes nothing
      head_sh[warp] = 0.f;
      starts_sh[warp] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // heads continue the row open before their mini-chunk, in order
      int pending = pending_sh, total = 0;
      for (int w2 = 0; w2 < NW; ++w2) {
        if (pending >= 0) rowbuf[pad_row(pending)] += head_sh[w2];
        if (starts_sh[w2]) pending = last_sh[w2];
        total += cnt_sh[w2];
      }
      pending_sh = pending;
      rows_sh += total;
    }
    // the next pass reads rows_sh / pending_sh after its first barrier
  }
  if (!ok) {
    // copies may still be in flight into shared memory: wait for them (bounded) first
    if (threadIdx.x == 0) {
      if (!okw) mbar_wait_bounded(&bar_w, 0, A.err);
      for (int b = 0; b < 2; ++b)
        if (out_p & (1u << b)) mbar_wait_bounded(&bar_p[b], (ph >> b) & 1u, A.err);
    }
    return;
  }
  __syncthreads();
  // Vertex updates (Figure 14), one thread per vertex of the bin.
  const float base = reinterpret_cast<const float*>(A.scal + 4)[0];
  float res = 0.f;
  float* rg = reinterpret_cast<float*>(A.r[p]);
  for (uint32_t i = threadIdx.x; i < B.v1 - B.v0; i += kMergeThreads) {
    const uint32_t v = B.v0 + i;
    const float sum = rowbuf[pad_row((int)i)];
    const float deg = (float)sdeg[v - q0];
    const float ro = sr[v - q0];
    const float rn = SCALED ? base + A.d_over_n * sum : base + A.d * sum;
    rg[v] = rn;
    if (SCALED) reinterpret_cast<__half*>(A.xn[p])[v] = __float2half_rn((rn * A.n) / deg);
    else reinterpret_cast<float*>(A.xn[p])[v] = rn / deg;
    res += fabsf(rn - ro);
  }
  res = warp_sum(res);
  if (lane == 0) red[warp] = res;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < NW ? red[threadIdx.x] : 0.f;
    t = warp_sum(t);
    if (threadIdx.x == 0 && t != 0.f)
      atomicAdd(A.slots + (blockIdx.x % A.nslots), (double)t);
  }
}

// Degree-zero vertices: the rank is the constant term, the contribution zero.
template <class XT>
__global__ void k_pr_seg_zero(const __grid_constant__ SegArgs A) {
  const float base = reinterpret_cast<const float*>(A.scal + 4)[0];
  const uint32_t z0 = A.nv[0] - A.nz[0];
  const uint32_t total = z0 + (A.nv[1] - A.nz[1]);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += gridDim.x * blockDim.x) {
    const int p = i < z0 ? 0 : 1;
    const uint32_t v = A.nz[p] + (p ? i - z0 : i);
    reinterpret_cast<float*>(A.r[p])[v] = base;
    reinterpret_cast<XT*>(A.xn[p])[v] = XT(0.f);
  }
}

template <class F>
graph_status set_smem(F fn, size_t bytes) {
  GG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return GRAPH_OK;
}

}  // namespace

graph_status seg_prepare(graph* g, const SegParams& prm, bool* usable) {
  *usable = false;
  const int log2 = prm.log2 ? prm.log2 : kDefLog2;
  const int ce = prm.chunk ? prm.chunk : kDefChunk;
  const int wb = prm.bin ? prm.bin : kDefBin;
  if (log2 < 6 || log2 > 15 || ce < 64 || ce > kChunkEntriesMax || wb < 64 || wb > kMaxBin) {
    set_error("segmented PageRank parameters out of range (log2 %d, chunk %d, bin %d)", log2,
              ce, wb);
    return GRAPH_EINVAL;
  }
  if (g->seg && g->seg->log2 == log2 && g->seg->chunk == ce && g->seg->bin == wb) {
    *usable = g->seg->usable;
    return GRAPH_OK;
  }
  free_seg(g);
  const auto t0 = std::chrono::steady_clock::now();
  SegWs* w = new SegWs();
  g->seg = w;
  w->log2 = log2;
  w->chunk = ce;
  w->bin = wb;
  PartHost H[2];
  bool fits[2] = {false, false};
  for (int p = 0; p < 2 && (p == 0 || fits[0]); ++p) {
    const graph_status s = build_part(g, p, log2, (uint32_t)ce, (uint32_t)wb, w->pp[p], H[p],
                                      p ? w->pp[0].S : 0u, &fits[p]);
    if (s != GRAPH_OK) {
      free_seg(g);
      return s;
    }
  }
  if (!fits[0] || !fits[1]) {  // keep the decision, drop the partial plan
    for (int p = 0; p < 2; ++p) free_seg_part(g, w->pp[p]);
    w->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GRAPH_OK;
  }
  std::vector<SegChunk> chunks(H[0].chunks);
  chunks.insert(chunks.end(), H[1].chunks.begin(), H[1].chunks.end());
  std::vector<SegBin> bins(H[0].bins);
  bins.insert(bins.end(), H[1].bins.begin(), H[1].bins.end());
  w->nchunk = (uint32_t)chunks.size();
  w->nbin = (uint32_t)bins.size();
  // Phase-1 CTAs: one per SM, each a contiguous run of chunks of about equal work
  // (entries plus a fixed cost per chunk).
  const uint32_t grid = (uint32_t)std::max(1, std::min<int>(sm_count(g), (int)std::max<uint32_t>(w->nchunk, 1)));
  std::vector<uint32_t> cta0(grid + 1, w->nchunk);
  {
    double tot = 0;
    for (const SegChunk& C : chunks) tot += C.nent + 512.0;
    double acc = 0;
    uint32_t b = 0;
    cta0[0] = 0;
    for (uint32_t c = 0; c < w->nchunk && b + 1 < grid; ++c) {
      acc += chunks[c].nent + 512.0;
      while (b + 1 < grid && acc >= tot * (b + 1) / grid) cta0[++b] = c + 1;
    }
    while (b + 1 <= grid) cta0[++b] = w->nchunk;
  }
  w->grid1 = grid;
  graph_status s = dalloc(g, w->chunks, sizeof(SegChunk) * std::max<size_t>(chunks.size(), 1));
  if (s == GRAPH_OK) s = dalloc(g, w->bins, sizeof(SegBin) * std::max<size_t>(bins.size(), 1));
  if (s == GRAPH_OK) s = dalloc(g, w->cta0, 4 * cta0.size());
  if (s == GRAPH_OK) s = to_dev(g, w->chunks.p, chunks);
  if (s == GRAPH_OK) s = to_dev(g, w->bins.p, bins);
  if (s == GRAPH_OK) s = to_dev(g, w->cta0.p, cta0);
  if (s == GRAPH_OK) s = set_smem(k_pr_seg<float>, seg_smem_bytes<float>(log2));
  if (s == GRAPH_OK) s = set_smem(k_pr_seg<__half>, seg_smem_bytes<__half>(log2));
  if (s == GRAPH_OK) s = set_smem(k_pr_merge<float, false>, kMergeSmem);
  if (s == GRAPH_OK) s = set_smem(k_pr_merge<__half, true>, kMergeSmem);
  if (s != GRAPH_OK) {
    free_seg(g);
    return s;
  }
  w->usable = true;
  *usable = true;
  w->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return GRAPH_OK;
}

graph_status seg_launch(graph* g, const SegIter& it) {
  SegWs* w = g->seg;
  SegArgs A;
  memset(&A, 0, sizeof(A));
  for (int p = 0; p < 2; ++p) {
    const Part& P = g->part[p];
    A.x[p] = it.x[p];
    A.ghost[p] = it.ghost[p];
    A.xn[p] = it.xn[p];
    A.r[p] = it.r[p];
    A.deg[p] = (const uint32_t*)w->pp[p].deg.p;
    A.ent[p] = (const uint16_t*)w->pp[p].ent.p;
    A.mrow[p] = (const uint16_t*)w->pp[p].mrow.p;
    A.part[p] = (float*)w->pp[p].part.p;
    A.plist[p] = (const uint16_t*)w->pp[p].plist.p;
    A.runs[p] = (const uint2*)w->pp[p].runs.p;
    A.nz[p] = P.cls_end[1];
    A.nv[p] = P.nv;
  }
  A.chunks = (const SegChunk*)w->chunks.p;
  A.bins = (const SegBin*)w->bins.p;
  A.cta0 = (const uint32_t*)w->cta0.p;
  A.scal = it.scal;
  A.slots = it.slots;
  A.nslots = it.nslots;
  A.d = it.d;
  A.d_over_n = it.d_over_n;
  A.n = it.n;
  A.err = (int*)g->err.p;
  cudaStream_t st = g->stream;
  if (w->nchunk) {
    if (it.fp16)
      k_pr_seg<__half><<<w->grid1, kSegThreads, seg_smem_bytes<__half>(w->log2), st>>>(A, w->log2);
    else
      k_pr_seg<float><<<w->grid1, kSegThreads, seg_smem_bytes<float>(w->log2), st>>>(A, w->log2);
    GG_CUDA(cudaGetLastError());
  }
  if (w->nbin) {
    if (it.fp16) k_pr_merge<__half, true><<<w->nbin, kMergeThreads, kMergeSmem, st>>>(A);
    else k_pr_merge<float, false><<<w->nbin, kMergeThreads, kMergeSmem, st>>>(A);
    GG_CUDA(cudaGetLastError());
  }
  const uint32_t zeros = (A.nv[0] - A.nz[0]) + (A.nv[1] - A.nz[1]);
  if (zeros) {
    if (it.fp16) k_pr_seg_zero<__half><<<std::min(grid_for(zeros, 256), 152u * 8), 256, 0, st>>>(A);
    else k_pr_seg_zero<float><<<std::min(grid_for(zeros, 256), 152u * 8), 256, 0, st>>>(A);
    GG_CUDA(cudaGetLastError());
  }
  return GRAPH_OK;
}

int seg_launches_per_iter(const graph* g) {
  const SegWs* w = g->seg;
  if (!w) return 0;
  const uint32_t zeros = (g->part[0].nv - g->part[0].cls_end[1]) + (g->part[1].nv - g->part[1].cls_end[1]);
  return (w->nchunk ? 1 : 0) + (w->nbin ? 1 : 0) + (zeros ? 1 : 0);
}

}  // namespace gg

using namespace gg;

extern "C" graph_status pagerank_plan_get(const graph_t* g, pagerank_plan_info* info) {
  if (!g || !info) {
    set_error("graph or info is NULL");
    return GRAPH_EINVAL;
  }
  memset(info, 0, sizeof(*info));
  const SegWs* w = g->seg;
  if (!w) return GRAPH_OK;
  info->built = 1;
  info->usable = w->usable ? 1 : 0;
  info->seg_log2 = w->log2;
  info->seg_chunk = w->chunk;
  info->seg_bin = w->bin;
  info->partials = (uint64_t)w->pp[0].P + w->pp[1].P;
  info->chunks = w->nchunk;
  info->bins = w->nbin;
  info->build_ms = w->build_ms;
  return GRAPH_OK;
}
