// Seeded synthetic inputs: RMAT graphs as symmetric CSR, edge weights, BFS/SSSP sources
// and random vertex assignments.
//
// This module is shared by the CPU oracle and the GPU path as their common source of
// inputs. It contains no graph-algorithm arithmetic (no traversal, relaxation or ranking).
//
// Recursive-matrix (RMAT) edge generation follows the workload description of Table 2:
// quadrant probabilities (A,B,C) = (0.57, 0.19, 0.19), D = 1-A-B-C, average degree 16.
// The paper's graphs are directed (Section 5, footnote 4); the workloads built here are
// symmetrised, self-loop free and deduplicated, with a seeded random vertex relabelling
// so that hubs are not clustered at id 0.
//
// Random numbers: every draw is the splitmix64 output at a fixed counter position
// (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
//   state_j = key + (j+1) * 0x9E3779B97F4A7C15,  out_j = mix64(state_j)
// with mix64 the splitmix64 finaliser. Counters are derived from (edge index, level), so
// the output does not depend on the thread count.
//
// Build: g++ -O3 -std=c++17 -fPIC -shared -pthread rmat.cpp -o librmat.so

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace {

const uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// splitmix64 output number j of the stream keyed by `key`.
inline uint64_t sm64_at(uint64_t key, uint64_t j) { return mix64(key + (j + 1) * kGamma); }

// Stream key of a user seed; distinct purposes use distinct salts.
inline uint64_t stream_key(uint64_t seed, uint64_t salt) {
  return mix64(seed * kGamma + salt);
}

// Lemire's multiply-shift reduction of a 32-bit draw to [0, range).
inline uint32_t bounded(uint32_t r, uint32_t range) {
  return (uint32_t)(((uint64_t)r * (uint64_t)range) >> 32);
}

int pick_threads(int threads) {
  if (threads > 0) return threads;
  unsigned hc = std::thread::hardware_concurrency();
  return hc ? (int)hc : 1;
}

template <class F>
void parallel_for(int64_t count, int threads, F&& f) {
  // f(begin, end, thread_index) over contiguous chunks.
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, count));
  if (threads == 1) {
    f((int64_t)0, count, 0);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(threads);
  for (int t = 0; t < threads; ++t) {
    int64_t b = count * t / threads, e = count * (t + 1) / threads;
    pool.emplace_back([&f, b, e, t]() { f(b, e, t); });
  }
  for (auto& th : pool) th.join();
}

// Dynamic scheduling over `count` items (used for uneven per-bucket work).
template <class F>
void parallel_dynamic(int64_t count, int threads, F&& f) {
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, count));
  std::atomic<int64_t> next(0);
  auto worker = [&]() {
    for (;;) {
      int64_t i = next.fetch_add(1);
      if (i >= count) break;
      f(i);
    }
  };
  if (threads == 1) {
    worker();
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < threads; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
}

struct RmatParams {
  int scale;
  uint32_t ta, tab, tabc;  // cumulative quadrant thresholds on a 32-bit draw
  uint64_t key;
};

// Edge number i of the RMAT stream, before relabelling: bits chosen from the most
// significant downward, one quadrant draw per level, two levels per 64-bit output.
inline void rmat_edge(const RmatParams& p, uint64_t i, uint32_t* u, uint32_t* v) {
  uint32_t a = 0, b = 0;
  uint64_t h = 0;
  for (int l = 0; l < p.scale; ++l) {
    uint32_t r;
    if ((l & 1) == 0) {
      h = sm64_at(p.key, i * 16 + (uint64_t)(l >> 1));
      r = (uint32_t)h;
    } else {
      r = (uint32_t)(h >> 32);
    }
    uint32_t bu, bv;
    if (r < p.ta) { bu = 0; bv = 0; }
    else if (r < p.tab) { bu = 0; bv = 1; }
    else if (r < p.tabc) { bu = 1; bv = 0; }
    else { bu = 1; bv = 1; }
    a = (a << 1) | bu;
    b = (b << 1) | bv;
  }
  *u = a;
  *v = b;
}

inline uint32_t prob_threshold(double x) {
  if (x <= 0) return 0;
  if (x >= 1) return 0xFFFFFFFFu;
  return (uint32_t)(x * 4294967296.0);
}

struct Csr {
  uint32_t n = 0;
  int64_t m = 0;
  int64_t* offsets = nullptr;
  uint32_t* cols = nullptr;
};

}  // namespace

extern "C" {

// Seeded random permutation of [0, n) (Fisher-Yates with splitmix64 draws).
void synth_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  for (uint32_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t key = stream_key(seed, 0x7065726dULL);
  for (uint32_t i = n; i > 1; --i) {
    uint32_t j = bounded((uint32_t)sm64_at(key, i), i);
    std::swap(perm[i - 1], perm[j]);
  }
}

// Builds a symmetric, deduplicated, self-loop-free CSR from edge_factor * 2^scale RMAT
// edges. Returns an opaque handle (NULL on failure); n and m are written to *n_out and
// *m_out; synth_csr_offsets / synth_csr_cols expose the arrays; synth_csr_free releases.
void* synth_rmat_csr(int scale, int edge_factor, double a, double b, double c,
                     uint64_t seed, int permute, uint64_t perm_seed, int threads,
                     uint32_t* n_out, int64_t* m_out) {
  if (scale < 1 || scale > 31 || edge_factor < 1) return nullptr;
  threads = pick_threads(threads);
  const uint32_t n = 1u << scale;
  const int64_t M = (int64_t)edge_factor << scale;

  RmatParams p;
  p.scale = scale;
  p.ta = prob_threshold(a);
  p.tab = prob_threshold(a + b);
  p.tabc = prob_threshold(a + b + c);
  p.key = stream_key(seed, 0x726d6174ULL);

  std::vector<uint32_t> perm;
  if (permute) {
    perm.resize(n);
    synth_permutation(n, perm_seed, perm.data());
  }
  auto edge = [&](int64_t i, uint32_t* u, uint32_t* v) {
    rmat_edge(p, (uint64_t)i, u, v);
    if (permute) {
      *u = perm[*u];
      *v = perm[*v];
    }
  };

  // Bucket directed entries (u -> v) by the high bits of u.
  const int bucket_shift = scale > 14 ? 14 : scale;  // 16K vertices per bucket
  const int64_t nbuckets = (int64_t)n >> bucket_shift;
  std::vector<int64_t> counts((size_t)threads * nbuckets, 0);
  parallel_for(M, threads, [&](int64_t beg, int64_t end, int t) {
    int64_t* cnt = &counts[(size_t)t * nbuckets];
    for (int64_t i = beg; i < end; ++i) {
      uint32_t u, v;
      edge(i, &u, &v);
      if (u == v) continue;
      cnt[u >> bucket_shift]++;
      cnt[v >> bucket_shift]++;
    }
  });
  // Exclusive prefix in (bucket, thread) order.
  std::vector<int64_t> bstart(nbuckets + 1, 0);
  std::vector<int64_t> pos((size_t)threads * nbuckets, 0);
  int64_t run = 0;
  for (int64_t bk = 0; bk < nbuckets; ++bk) {
    bstart[bk] = run;
    for (int t = 0; t < threads; ++t) {
      pos[(size_t)t * nbuckets + bk] = run;
      run += counts[(size_t)t * nbuckets + bk];
    }
  }
  bstart[nbuckets] = run;
  const int64_t total = run;
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)std::max<int64_t>(total, 1));
  if (!keys) return nullptr;
  parallel_for(M, threads, [&](int64_t beg, int64_t end, int t) {
    int64_t* ps = &pos[(size_t)t * nbuckets];
    for (int64_t i = beg; i < end; ++i) {
      uint32_t u, v;
      edge(i, &u, &v);
      if (u == v) continue;
      keys[ps[u >> bucket_shift]++] = ((uint64_t)u << 32) | v;
      keys[ps[v >> bucket_shift]++] = ((uint64_t)v << 32) | u;
    }
  });
  // Sort and deduplicate each bucket; count degrees.
  std::vector<int64_t> bunique(nbuckets, 0);
  int64_t* offsets = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!offsets) {
    free(keys);
    return nullptr;
  }
  memset(offsets, 0, sizeof(int64_t) * ((size_t)n + 1));
  parallel_dynamic(nbuckets, threads, [&](int64_t bk) {
    uint64_t* kb = keys + bstart[bk];
    int64_t len = bstart[bk + 1] - bstart[bk];
    std::sort(kb, kb + len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i) {
      if (w == 0 || kb[i] != kb[w - 1]) kb[w++] = kb[i];
    }
    bunique[bk] = w;
    for (int64_t i = 0; i < w; ++i) offsets[(kb[i] >> 32) + 1]++;
  });
  for (uint32_t v = 0; v < n; ++v) offsets[v + 1] += offsets[v];
  const int64_t m = offsets[n];
  uint32_t* cols = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)std::max<int64_t>(m, 1));
  if (!cols) {
    free(keys);
    free(offsets);
    return nullptr;
  }
  parallel_dynamic(nbuckets, threads, [&](int64_t bk) {
    const uint64_t* kb = keys + bstart[bk];
    int64_t w = bunique[bk];
    if (w == 0) return;
    int64_t dst = offsets[kb[0] >> 32];
    for (int64_t i = 0; i < w; ++i) cols[dst + i] = (uint32_t)kb[i];
  });
  free(keys);
  Csr* csr = new Csr;
  csr->n = n;
  csr->m = m;
  csr->offsets = offsets;
  csr->cols = cols;
  *n_out = n;
  *m_out = m;
  return csr;
}

const int64_t* synth_csr_offsets(void* h) { return ((Csr*)h)->offsets; }
const uint32_t* synth_csr_cols(void* h) { return ((Csr*)h)->cols; }

void synth_csr_free(void* h) {
  if (!h) return;
  Csr* c = (Csr*)h;
  free(c->offsets);
  free(c->cols);
  delete c;
}

// Symmetric edge weights in [1, wmax]: w(u,v) = w(v,u) = 1 + (draw(min, max) mod wmax),
// with draw the splitmix64 output at counter position (min << 32 | max).
void synth_weights(uint32_t n, const int64_t* offsets, const uint32_t* cols,
                   uint64_t seed, uint32_t wmax, int threads, uint32_t* w) {
  threads = pick_threads(threads);
  uint64_t key = stream_key(seed, 0x77656967ULL);
  parallel_for((int64_t)n, threads, [&](int64_t beg, int64_t end, int) {
    for (int64_t u = beg; u < end; ++u) {
      for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
        uint32_t v = cols[e];
        uint64_t lo = (uint64_t)std::min<uint32_t>((uint32_t)u, v);
        uint64_t hi = (uint64_t)std::max<uint32_t>((uint32_t)u, v);
        uint64_t h = sm64_at(key, (lo << 32) | hi);
        w[e] = 1u + (uint32_t)(h % wmax);
      }
    }
  });
}

// `count` distinct vertices with degree > 0, drawn in order from the seeded stream.
// Returns the number written (less than count only if the graph has fewer such vertices).
int64_t synth_sources(uint32_t n, const int64_t* offsets, int64_t count, uint64_t seed,
                      uint32_t* out) {
  uint64_t key = stream_key(seed, 0x73726373ULL);
  int64_t nonisolated = 0;
  for (uint32_t v = 0; v < n; ++v) nonisolated += offsets[v + 1] > offsets[v];
  if (count > nonisolated) count = nonisolated;
  std::vector<uint8_t> taken(n, 0);
  int64_t got = 0;
  for (uint64_t j = 0; got < count; ++j) {
    uint32_t v = bounded((uint32_t)sm64_at(key, j), n);
    if (offsets[v + 1] == offsets[v] || taken[v]) continue;
    taken[v] = 1;
    out[got++] = v;
  }
  return got;
}

// Per-vertex partition ids for a random split: vertex v goes to partition 0 with
// probability share0 (a seeded coin per vertex), else partition 1.
void synth_random_assignment(uint32_t n, double share0, uint64_t seed, uint8_t* part) {
  uint64_t key = stream_key(seed, 0x72616e64ULL);
  uint32_t thr = prob_threshold(share0);
  for (uint32_t v = 0; v < n; ++v) part[v] = ((uint32_t)sm64_at(key, v) < thr) ? 0 : 1;
}

}  // extern "C"
