// Device-wide exclusive prefix sums (three passes: tile reduce, scan of tile sums, tile
// scan with carry-in). Used by the partition builder for offsets, outbox indices and the
// stable counting sort of vertices into (partition, degree class) order.
#include "common.cuh"

namespace gg {
namespace {

constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

template <class T>
__device__ T block_exclusive_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  T x = v;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T t = lane < nwarps ? warp_tot[lane] : T(0);
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nwarps) warp_tot[lane] = t;
  }
  __syncthreads();
  T excl = (warp > 0 ? warp_tot[warp - 1] : T(0)) + x - v;
  *total = warp_tot[nwarps - 1];
  __syncthreads();
  return excl;
}

template <class In, class Acc>
__global__ void __launch_bounds__(kThreads) k_tile_reduce(const In* in, uint64_t n, Acc* part) {
  __shared__ Acc wt[32];
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  Acc s = 0;
  #pragma unroll
  for (int k = 0; k < kItems; ++k) {
    uint64_t i = base + (uint64_t)k * kThreads + threadIdx.x;
    if (i < n) s += (Acc)in[i];
  }
  Acc tot;
  block_exclusive_scan<Acc>(s, wt, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single CTA: exclusive scan of `n` values in place; total to *total.
template <class Acc>
__global__ void __launch_bounds__(1024) k_scan_single(Acc* a, uint64_t n, Acc* total) {
  __shared__ Acc wt[32];
  Acc carry = 0;
  for (uint64_t base = 0; base < n; base += blockDim.x) {
    uint64_t i = base + threadIdx.x;
    Acc v = i < n ? a[i] : Acc(0);
    Acc tot;
    Acc e = block_exclusive_scan<Acc>(v, wt, &tot);
    if (i < n) a[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = carry;
}

template <class In, class Acc>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const In* in, Acc* out, uint64_t n,
                                                        const Acc* part) {
  __shared__ Acc wt[32];
  const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)threadIdx.x * kItems;
  Acc v[kItems];
  Acc s = 0;
  #pragma unroll
  for (int k = 0; k < kItems; ++k) {
    uint64_t i = base + k;
    v[k] = i < n ? (Acc)in[i] : Acc(0);
    s += v[k];
  }
  Acc tot;
  Acc run = block_exclusive_scan<Acc>(s, wt, &tot) + part[blockIdx.x];
  #pragma unroll
  for (int k = 0; k < kItems; ++k) {
    uint64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

template <class In, class Acc>
graph_status scan_impl(graph* g, const In* in, Acc* out, uint64_t n, Acc* total_host) {
  const uint64_t tiles = (n + kTile - 1) / kTile;
  DevBuf part;
  GG_TRY(dalloc(g, part, sizeof(Acc) * (tiles + 1)));
  Acc* d_part = (Acc*)part.p;
  if (n > 0) {
    k_tile_reduce<In, Acc><<<(unsigned)tiles, kThreads, 0, g->stream>>>(in, n, d_part);
    k_scan_single<Acc><<<1, 1024, 0, g->stream>>>(d_part, tiles, d_part + tiles);
    k_tile_scan<In, Acc><<<(unsigned)tiles, kThreads, 0, g->stream>>>(in, out, n, d_part);
  } else {
    cudaMemsetAsync(d_part, 0, sizeof(Acc), g->stream);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    dfree(g, part);
    return cuda_fail(e, "scan launch", __FILE__, __LINE__);
  }
  if (total_host) {
    e = cudaMemcpyAsync(total_host, d_part + tiles, sizeof(Acc), cudaMemcpyDeviceToHost,
                        g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  } else {
    e = cudaStreamSynchronize(g->stream);  // `part` is freed below
  }
  dfree(g, part);
  if (e != cudaSuccess) return cuda_fail(e, "scan total", __FILE__, __LINE__);
  return GRAPH_OK;
}

}  // namespace

graph_status exclusive_scan_u32(graph* g, const uint32_t* in, uint32_t* out, uint64_t n,
                                uint32_t* total_host) {
  return scan_impl<uint32_t, uint32_t>(g, in, out, n, total_host);
}
graph_status exclusive_scan_u8_to_u32(graph* g, const uint8_t* in, uint32_t* out, uint64_t n,
                                      uint32_t* total_host) {
  return scan_impl<uint8_t, uint32_t>(g, in, out, n, total_host);
}
graph_status exclusive_scan_i64(graph* g, const int64_t* in, int64_t* out, uint64_t n,
                                int64_t* total_host) {
  return scan_impl<int64_t, int64_t>(g, in, out, n, total_host);
}

}  // namespace gg
