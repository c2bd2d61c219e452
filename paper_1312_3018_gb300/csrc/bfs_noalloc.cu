// Allocation-free BFS entry point.
//
// Some callers cannot allocate device memory at the point where they need a search: code
// running inside a host callback or a driver-level hook where cudaMalloc is forbidden or
// would deadlock, allocators that must not grow after start-up, or embedded services with a
// fixed device-memory budget. bfs_csr_noalloc serves them: it runs a level-synchronous
// top-down BFS straight on the caller's device CSR and writes the caller's device output
// arrays, keeping every scratch structure (visited bitmap, two frontier queues, counters) in
// one fixed array in this file. It never calls cudaMalloc, cudaFree or any allocating
// library routine.
//
// The scratch array is a file-scope __device__ array: every GPU that loads this library
// holds it ((2^21/32 + 2 * 2^21 + 64) words = 17,039,616 bytes: 17.0 MB, 16.25 MiB) until
// the process exits. Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress while that
// device is current and caches it; that first call should therefore come before any stream
// capture. All calls share the one array, which keeps the last call's contents: each call
// clears what must start at zero, and calls that overlap on the GPU (two streams, two
// threads) race on it. The call blocks the host: it synchronises its stream after the CSR
// check and after every level (the level loop reads the next frontier's size).
#include <mutex>

#include "common.cuh"

namespace gg {
namespace {

constexpr uint32_t kNoAllocMaxVertices = GRAPH_NOALLOC_MAX_VERTICES;
constexpr uint32_t kBitmapWords = kNoAllocMaxVertices / 32;
constexpr size_t kScratchWords = (size_t)kBitmapWords + 2ull * kNoAllocMaxVertices + 64;

// visited bitmap | frontier queue A | frontier queue B | counters (tail, validation flags)
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint32_t* g_scratch_ptr[kMaxDevices] = {nullptr};

struct Scratch {
  uint32_t* visited;
  uint32_t* queue[2];
  uint32_t* tail;   // next-queue length
  uint32_t* flags;  // CSR validation result
};

Scratch layout(uint32_t* base) {
  Scratch s;
  s.visited = base;
  s.queue[0] = base + kBitmapWords;
  s.queue[1] = s.queue[0] + kNoAllocMaxVertices;
  s.tail = s.queue[1] + kNoAllocMaxVertices;
  s.flags = s.tail + 1;
  return s;
}

// CSR checks before any traversal: 1 offsets[0] != 0, 2 decreasing offsets,
// 4 offsets[n] != m, 8 a column id >= n.
__global__ void k_na_validate(const int64_t* off, const uint32_t* cols, uint32_t n, int64_t m,
                              uint32_t* flags) {
  uint32_t bad = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) {
    if (off[0] != 0) bad |= 1;
    if (off[n] != m) bad |= 4;
  }
  for (uint64_t i = t0; i < n; i += stride)
    if (off[i] > off[i + 1]) bad |= 2;
  for (uint64_t e = t0; e < (uint64_t)m; e += stride)
    if (cols[e] >= n) bad |= 8;
  bad = __reduce_or_sync(kFull, bad);
  if (bad && lane_id() == 0) atomicOr(flags, bad);
}

__global__ void k_na_clear(uint32_t n, uint32_t* levels, uint32_t* parents, uint32_t* visited,
                           uint32_t words, uint32_t* tail) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    levels[i] = kInf;
    if (parents) parents[i] = kInf;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) visited[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) *tail = 0;
}

__global__ void k_na_seed(uint32_t source, uint32_t* levels, uint32_t* parents, uint32_t* visited,
                          uint32_t* queue) {
  levels[source] = 0;
  if (parents) parents[source] = source;
  visited[source >> 5] |= 1u << (source & 31u);
  queue[0] = source;
}

// One warp per frontier vertex: claim unvisited neighbours, record level and parent, and
// append the new vertices to the next frontier.
__global__ void __launch_bounds__(256) k_na_expand(const int64_t* off, const uint32_t* cols,
                                                   const uint32_t* frontier, uint32_t count,
                                                   uint32_t level, uint32_t* levels,
                                                   uint32_t* parents, uint32_t* visited,
                                                   uint32_t* next, uint32_t* tail) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= count) return;  // warp-uniform
  const uint32_t v = frontier[w];
  const int64_t s = off[v], t = off[v + 1];
  for (int64_t e = s + lane_id(); __any_sync(kFull, e < t); e += 32) {
    bool won = false;
    uint32_t u = 0;
    if (e < t) {
      u = cols[e];
      if (bitmap_claim(visited, u)) {
        won = true;
        levels[u] = level + 1;
        if (parents) parents[u] = v;
      }
    }
    warp_append(won, u, tail, next);
  }
}

graph_status scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  GG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index %d out of the supported range", dev);
    return GRAPH_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    GG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = (uint32_t*)p;
  }
  *out = g_scratch_ptr[dev];
  return GRAPH_OK;
}

}  // namespace
}  // namespace gg

using namespace gg;

extern "C" graph_status bfs_csr_noalloc(uint32_t n, int64_t m, const int64_t* offsets,
                                        const uint32_t* cols, uint32_t source, uint32_t* levels,
                                        uint32_t* parents, void* stream) {
  if (n == 0 || m < 0 || !offsets || (m > 0 && !cols) || !levels) {
    set_error("invalid sizes or pointers (n=%u m=%lld)", n, (long long)m);
    return GRAPH_EINVAL;
  }
  if (n > kNoAllocMaxVertices) {
    set_error("n=%u exceeds the allocation-free limit of %u vertices", n, kNoAllocMaxVertices);
    return GRAPH_EINVAL;
  }
  if (source >= n) {
    set_error("source %u >= n %u", source, n);
    return GRAPH_EINVAL;
  }
  uint32_t* base = nullptr;
  GG_TRY(scratch_for_current_device(&base));
  const Scratch S = layout(base);
  cudaStream_t st = (cudaStream_t)stream;
  const uint32_t words = (n + 31) / 32;
  uint32_t flags = 0;
  GG_CUDA(cudaMemsetAsync(S.flags, 0, sizeof(uint32_t), st));
  k_na_validate<<<152 * 8, 256, 0, st>>>(offsets, cols, n, m, S.flags);
  GG_CUDA(cudaGetLastError());
  GG_CUDA(cudaMemcpyAsync(&flags, S.flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  GG_CUDA(cudaStreamSynchronize(st));
  if (flags) {
    set_error("invalid CSR (flags 0x%x: 1 offsets[0]!=0, 2 decreasing offsets, 4 "
              "offsets[n]!=m, 8 column id >= n)", flags);
    return GRAPH_EINVAL;
  }
  k_na_clear<<<152 * 4, 256, 0, st>>>(n, levels, parents, S.visited, words, S.tail);
  k_na_seed<<<1, 1, 0, st>>>(source, levels, parents, S.visited, S.queue[0]);
  GG_CUDA(cudaGetLastError());
  uint32_t count = 1;
  int cur = 0;
  for (uint32_t level = 0; count > 0; ++level) {
    if (level > n) {
      set_error("bfs_csr_noalloc exceeded n levels");
      return GRAPH_ETIMEOUT;
    }
    const uint64_t threads = (uint64_t)count * 32;
    k_na_expand<<<grid_for(threads, 256), 256, 0, st>>>(offsets, cols, S.queue[cur], count, level,
                                                        levels, parents, S.visited,
                                                        S.queue[1 - cur], S.tail);
    GG_CUDA(cudaGetLastError());
    GG_CUDA(cudaMemcpyAsync(&count, S.tail, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GG_CUDA(cudaMemsetAsync(S.tail, 0, sizeof(uint32_t), st));
    GG_CUDA(cudaStreamSynchronize(st));
    cur = 1 - cur;
  }
  return GRAPH_OK;
}
