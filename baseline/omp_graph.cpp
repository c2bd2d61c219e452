// Timed CPU baseline: the paper's CPU kernels on all host cores with OpenMP.
//
// This is NOT part of the library and NOT the oracle. It is a separate, straightforward
// multi-core implementation of the three CPU kernels the paper runs on the host side of
// its hybrid system (Section 4.2: OpenMP over the partition's vertices), used only by
// bench.py to time the benchmark step on the host's cores and by tests that check it
// against the oracle:
//  - top-down level-synchronous BFS with a visited bitmap (Section 6.3.2, Figure 11): every
//    vertex of the current frontier claims its unvisited neighbours with an atomic
//    test-and-set on the bitmap and gives them the next level;
//  - pull PageRank (Section 7.1, Figure 14): every vertex sums its neighbours'
//    contributions r/deg (FP32 contributions and sums, FP64 dangling mass), the same
//    reading of the update as the library's FP32 path;
//  - Bellman-Ford SSSP (Section 7.3, Figure 20): every active vertex relaxes its edges
//    with an atomic minimum on the target's distance; a vertex whose distance dropped is
//    active in the next round (same-round reads of newer distances are allowed).
// Frontiers are vertex lists built from per-thread buffers. Distances are uint32 with a
// saturating add, as in the library.
#include <omp.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <vector>

namespace {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr size_t kBuf = 4096;

// Appends to a shared list through a per-thread buffer (one atomic per kBuf items).
struct Appender {
  uint32_t* list;
  std::atomic<uint64_t>* tail;
  uint32_t buf[kBuf];
  size_t k = 0;
  void push(uint32_t v) {
    buf[k++] = v;
    if (k == kBuf) flush();
  }
  void flush() {
    if (!k) return;
    const uint64_t at = tail->fetch_add(k);
    memcpy(list + at, buf, 4 * k);
    k = 0;
  }
};

}  // namespace

extern "C" {

int omp_threads(void) { return omp_get_max_threads(); }

// Levels (kInf unreached) from src; returns the number of levels.
int omp_bfs(uint32_t n, const int64_t* off, const uint32_t* col, uint32_t src, uint32_t* level) {
  std::vector<std::atomic<uint64_t>> vis((n + 63) / 64);
  std::vector<uint32_t> cur(n), nxt(n);
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; ++i) level[i] = kInf;
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)vis.size(); ++i) vis[i].store(0, std::memory_order_relaxed);
  level[src] = 0;
  vis[src >> 6].store(1ull << (src & 63));
  cur[0] = src;
  uint64_t ncur = 1;
  int levels = 0;
  while (ncur) {
    std::atomic<uint64_t> tail(0);
    const uint32_t next_level = (uint32_t)levels + 1;
    #pragma omp parallel
    {
      Appender out{nxt.data(), &tail};
      #pragma omp for schedule(dynamic, 64)
      for (int64_t i = 0; i < (int64_t)ncur; ++i) {
        const uint32_t u = cur[i];
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
          const uint32_t v = col[e];
          const uint64_t bit = 1ull << (v & 63);
          if (vis[v >> 6].load(std::memory_order_relaxed) & bit) continue;
          if (vis[v >> 6].fetch_or(bit) & bit) continue;
          level[v] = next_level;
          out.push(v);
        }
      }
      out.flush();
    }
    ncur = tail.load();
    cur.swap(nxt);
    ++levels;
  }
  return levels;
}

// Bellman-Ford distances (kInf unreachable) from src; returns the number of rounds, or -1
// if a distance would reach kInf (the library reports that as an overflow too).
int omp_sssp(uint32_t n, const int64_t* off, const uint32_t* col, const uint32_t* w,
             uint32_t src, uint32_t* dist) {
  std::vector<std::atomic<uint32_t>> d(n);
  std::vector<std::atomic<uint8_t>> queued(n);
  std::vector<uint32_t> cur(n), nxt(n);
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; ++i) {
    d[i].store(kInf, std::memory_order_relaxed);
    queued[i].store(0, std::memory_order_relaxed);
  }
  d[src].store(0);
  cur[0] = src;
  uint64_t ncur = 1;
  int rounds = 0;
  std::atomic<int> overflow(0);
  while (ncur) {
    std::atomic<uint64_t> tail(0);
    #pragma omp parallel
    {
      Appender out{nxt.data(), &tail};
      #pragma omp for schedule(dynamic, 64)
      for (int64_t i = 0; i < (int64_t)ncur; ++i) {
        const uint32_t u = cur[i];
        // Clear the queued mark before reading the distance, in one total order with the
        // lowering threads' minimum and mark (sequentially consistent): a lowering that this
        // read misses sees the cleared mark and queues u again. With relaxed order the two
        // could be reordered (weakly ordered hosts) and the improvement lost.
        queued[u].store(0, std::memory_order_seq_cst);
        const uint64_t du = d[u].load(std::memory_order_seq_cst);
        for (int64_t e = off[u]; e < off[u + 1]; ++e) {
          const uint32_t v = col[e];
          const uint64_t s = du + w[e];
          if (s >= kInf) {
            overflow.store(1, std::memory_order_relaxed);
            continue;
          }
          const uint32_t nd = (uint32_t)s;
          uint32_t old = d[v].load(std::memory_order_relaxed);
          while (nd < old && !d[v].compare_exchange_weak(old, nd, std::memory_order_seq_cst,
                                                          std::memory_order_relaxed)) {
          }
          if (nd < old && !queued[v].exchange(1, std::memory_order_seq_cst)) out.push(v);
        }
      }
      out.flush();
    }
    ncur = tail.load();
    cur.swap(nxt);
    ++rounds;
    if (rounds > (int)n + 1) break;
  }
  #pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)n; ++i) dist[i] = d[i].load(std::memory_order_relaxed);
  return overflow.load() ? -1 : rounds;
}

// iters iterations of pull PageRank from r = 1/n (FP32 contributions and sums, degree-zero
// rank spread uniformly when dangling != 0); ranks out in double. Returns the last L1
// change.
double omp_pagerank(uint32_t n, const int64_t* off, const uint32_t* col, double damping,
                    int iters, int dangling, double* ranks) {
  std::vector<float> r(n, (float)(1.0 / n)), x(n);
  double res = 0;
  for (int it = 0; it < iters; ++it) {
    double D = 0;
    #pragma omp parallel for schedule(static) reduction(+ : D)
    for (int64_t u = 0; u < (int64_t)n; ++u) {
      const int64_t deg = off[u + 1] - off[u];
      if (deg > 0) x[u] = r[u] / (float)deg;
      else {
        x[u] = 0.f;
        D += r[u];
      }
    }
    const float base = (float)((1.0 - damping) / n + (dangling ? damping * D / n : 0.0));
    const float dd = (float)damping;
    res = 0;
    #pragma omp parallel for schedule(dynamic, 1024) reduction(+ : res)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
      float s = 0.f;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) s += x[col[e]];
      const float rn = base + dd * s;
      res += rn > r[v] ? rn - r[v] : r[v] - rn;
      r[v] = rn;  // x holds this iteration's contributions, so r can change in place
    }
  }
  #pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < (int64_t)n; ++v) ranks[v] = r[v];
  return res;
}

}  // extern "C"
