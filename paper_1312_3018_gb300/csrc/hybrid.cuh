// Host-thread helpers of the hybrid entry points (bfs_hybrid, sssp_hybrid): partition 0 is
// processed by host threads while the GPU processes partition 1 (Section 4.1, Figure 6).
#pragma once

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"

namespace gg {

// Runs f(worker, begin, end) on nt host threads over [0, n) in dynamic blocks of `grain`
// items. A thread that cannot be started leaves its share to the others (the caller always
// works), so every block is processed exactly once.
template <class F>
void host_dynamic(int nt, uint64_t n, uint64_t grain, F&& f) {
  if (n == 0) return;
  std::atomic<uint64_t> next(0);
  auto body = [&](int k) {
    for (;;) {
      const uint64_t a = next.fetch_add(grain);
      if (a >= n) break;
      f(k, a, std::min(n, a + grain));
    }
  };
  std::vector<std::thread> th;
  th.reserve(nt > 1 ? nt - 1 : 0);
  for (int k = 1; k < nt; ++k) {
    try {
      th.emplace_back(body, k);
    } catch (...) {
      break;
    }
  }
  body(0);
  for (auto& t : th) t.join();
}

// Host threads for a hybrid call: `requested` in 1 ... GRAPH_HYBRID_MAX_THREADS, or the
// host's hardware threads (capped) when requested <= 0.
inline int hybrid_threads(int requested) {
  if (requested > 0) return std::min(requested, (int)GRAPH_HYBRID_MAX_THREADS);
  const unsigned hw = std::thread::hardware_concurrency();
  return std::max(1, std::min((int)(hw ? hw : 1), (int)GRAPH_HYBRID_MAX_THREADS));
}

// Atomic test-and-set of bit i in a host bitmap of 64-bit words; true if this call set it.
inline bool host_claim(std::atomic<uint64_t>* bm, uint32_t i) {
  const uint64_t bit = 1ull << (i & 63u);
  if (bm[i >> 6].load(std::memory_order_relaxed) & bit) return false;
  return !(bm[i >> 6].fetch_or(bit, std::memory_order_relaxed) & bit);
}

// Atomic minimum on a host word; true if v lowered it.
inline bool host_min(std::atomic<uint32_t>* p, uint32_t v) {
  uint32_t old = p->load(std::memory_order_relaxed);
  while (v < old) {
    if (p->compare_exchange_weak(old, v, std::memory_order_relaxed)) return true;
  }
  return false;
}

}  // namespace gg
