/*
 * CPU oracle for the BSP graph hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded, deliberately unoptimised C. Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library; the product path
 * never calls it. It shares no code, header or table with the CUDA library.
 *
 * What each function computes, and where the paper defines it (Gharaibeh et al.,
 * "Efficient Large-Scale Graph Processing on Hybrid CPU and GPU Systems"):
 *
 *   orc_bfs            BFS level of every vertex (hop distance from the source) and one
 *                      BFS tree. Definition of level-synchronous BFS, Section 6.3.2,
 *                      Figure 11 and the Appendix (levels start at 0 for the source,
 *                      unreached vertices keep INF). A FIFO queue visits vertices in
 *                      non-decreasing level order, which yields the same unique levels.
 *   orc_sssp           Single-source shortest-path distances, Section 7.3. The paper's
 *                      Bellman-Ford kernel (Figure 20) converges to the unique shortest
 *                      distances; the oracle computes them by the textbook definition,
 *                      Dijkstra with an indexed binary heap, in 64-bit sums.
 *   orc_pagerank       Pull PageRank, Section 7.1, Figure 14, in FP64, following the
 *                      algorithm's steps in order, with these readings of the figure:
 *                      a neighbour contributes rank/out-degree (standard PageRank, the
 *                      paper's reference [Page et al. 1999]); the rank of degree-zero
 *                      vertices is either spread uniformly (mode 1) or dropped, which is
 *                      the figure taken literally (mode 0); ranks start at 1/n; the loop
 *                      runs a fixed number of iterations or stops once the L1 change
 *                      falls below tol.
 *   orc_partition      Two-way vertex partition with per-partition CSR, local ids,
 *                      boundary edges encoded as outbox indices (partition id in the high
 *                      bit), local-first neighbour order and outbox/inbox vertex lists,
 *                      Section 4.3.1-4.3.2 and Figure 6; degree-based assignment,
 *                      Section 6.2 and 6.3.1 (HIGH: the high-degree vertices form one
 *                      partition).
 *   orc_check_bfs      Validator for BFS levels and parents (the invariants a BFS tree
 *                      must satisfy; parents are not unique, so they are validated).
 *   orc_check_sssp     Optimality certificate for shortest-path distances.
 *   orc_traversed      TEPS numerator of Section 5: sum of the degrees of the vertices
 *                      that were reached.
 *   orc_bc             Betweenness centrality summed over a list of sources, Section 7.2
 *                      and Figure 18 (Brandes' algorithm, the paper's reference [Brandes
 *                      2001]): a BFS counts the shortest paths sigma from the source, then
 *                      vertices in reverse BFS order accumulate the dependency
 *                      delta(v) = sum over successors w (neighbours one level further) of
 *                      sigma(v) / sigma(w) * (1 + delta(w)), and every vertex other than the
 *                      source adds delta(v) to its score. FP64 throughout.
 *   orc_cc             Connected components (Section 9.4): every vertex labelled with the
 *                      smallest vertex id of its component, found by a BFS from each
 *                      still unlabelled vertex in increasing id order.
 *
 * Graph format: CSR with int64 offsets[n+1] and uint32 cols[m]; optional uint32 weights.
 * INF is 0xFFFFFFFF for levels, parents and distances.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_INF 0xFFFFFFFFu
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ERANGE (-5)

/* ------------------------------------------------------------------------------------ */
/* BFS                                                                                   */
/* ------------------------------------------------------------------------------------ */

int orc_bfs(uint32_t n, const int64_t* off, const uint32_t* col, uint32_t source,
            uint32_t* level, uint32_t* parent) {
  if (source >= n) return ORC_EINVAL;
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!queue) return ORC_ENOMEM;
  for (uint32_t v = 0; v < n; ++v) {
    level[v] = ORC_INF;
    if (parent) parent[v] = ORC_INF;
  }
  size_t head = 0, tail = 0;
  level[source] = 0;
  if (parent) parent[source] = source;
  queue[tail++] = source;
  while (head < tail) {
    uint32_t v = queue[head++];
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      uint32_t u = col[e];
      if (level[u] == ORC_INF) {
        level[u] = level[v] + 1;
        if (parent) parent[u] = v;
        queue[tail++] = u;
      }
    }
  }
  free(queue);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* SSSP: Dijkstra, indexed binary min-heap keyed by 64-bit tentative distance             */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  uint32_t* heap; /* vertex ids */
  uint32_t* pos;  /* position of a vertex in heap, ORC_INF if absent */
  uint64_t* key;  /* tentative distance */
  uint32_t size;
} orc_heap;

static void heap_swap(orc_heap* h, uint32_t i, uint32_t j) {
  uint32_t a = h->heap[i], b = h->heap[j];
  h->heap[i] = b;
  h->heap[j] = a;
  h->pos[b] = i;
  h->pos[a] = j;
}

static void heap_up(orc_heap* h, uint32_t i) {
  while (i > 0) {
    uint32_t p = (i - 1) / 2;
    if (h->key[h->heap[p]] <= h->key[h->heap[i]]) break;
    heap_swap(h, i, p);
    i = p;
  }
}

static void heap_down(orc_heap* h, uint32_t i) {
  for (;;) {
    uint32_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < h->size && h->key[h->heap[l]] < h->key[h->heap[s]]) s = l;
    if (r < h->size && h->key[h->heap[r]] < h->key[h->heap[s]]) s = r;
    if (s == i) break;
    heap_swap(h, i, s);
    i = s;
  }
}

/* dist[v] = min over paths of the sum of weights; ORC_INF if unreachable.
 * Returns ORC_ERANGE if a finite distance does not fit below 0xFFFFFFFF. */
int orc_sssp(uint32_t n, const int64_t* off, const uint32_t* col, const uint32_t* w,
             uint32_t source, uint32_t* dist) {
  if (source >= n) return ORC_EINVAL;
  orc_heap h;
  h.heap = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  h.pos = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  h.key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  uint8_t* done = (uint8_t*)calloc((size_t)n, 1);
  if (!h.heap || !h.pos || !h.key || !done) {
    free(h.heap); free(h.pos); free(h.key); free(done);
    return ORC_ENOMEM;
  }
  const uint64_t UNSEEN = UINT64_MAX;
  for (uint32_t v = 0; v < n; ++v) {
    h.pos[v] = ORC_INF;
    h.key[v] = UNSEEN;
  }
  h.size = 0;
  h.key[source] = 0;
  h.heap[0] = source;
  h.pos[source] = 0;
  h.size = 1;
  while (h.size > 0) {
    uint32_t v = h.heap[0];
    h.size--;
    if (h.size > 0) {
      h.heap[0] = h.heap[h.size];
      h.pos[h.heap[0]] = 0;
      heap_down(&h, 0);
    }
    h.pos[v] = ORC_INF;
    done[v] = 1;
    uint64_t dv = h.key[v];
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      uint32_t u = col[e];
      if (done[u]) continue;
      uint64_t nd = dv + (uint64_t)w[e];
      if (nd < h.key[u]) {
        h.key[u] = nd;
        if (h.pos[u] == ORC_INF) {
          h.heap[h.size] = u;
          h.pos[u] = h.size;
          h.size++;
        }
        heap_up(&h, h.pos[u]);
      }
    }
  }
  int rc = ORC_OK;
  for (uint32_t v = 0; v < n; ++v) {
    if (h.key[v] == UNSEEN) {
      dist[v] = ORC_INF;
    } else if (h.key[v] >= (uint64_t)ORC_INF) {
      dist[v] = ORC_INF - 1;
      rc = ORC_ERANGE;
    } else {
      dist[v] = (uint32_t)h.key[v];
    }
  }
  free(h.heap); free(h.pos); free(h.key); free(done);
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* PageRank (pull), FP64                                                                  */
/* ------------------------------------------------------------------------------------ */

/* Runs up to max_iter iterations of
 *     x[u]  = r[u] / deg(u)                       (deg(u) > 0)
 *     D     = sum of r[u] over deg(u) == 0        (mode 1; D = 0 in mode 0)
 *     r'[v] = (1 - d)/n + d * (sum_{u in N(v)} x[u] + D/n)
 *     res   = sum_v |r'[v] - r[v]|
 * from r = 1/n, stopping after the first iteration whose res < tol. The symmetric CSR
 * gives each vertex's in-neighbours (N_in = N_out). Neighbours are summed in CSR order.
 * resid[k] receives the residual of iteration k+1 (may be NULL); *iters the count run. */
int orc_pagerank(uint32_t n, const int64_t* off, const uint32_t* col, double d,
                 int max_iter, double tol, int dangling_mode, double* r, double* resid,
                 int* iters) {
  if (n == 0) {
    if (iters) *iters = 0;
    return ORC_OK;
  }
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* rn = (double*)malloc(sizeof(double) * (size_t)n);
  if (!x || !rn) {
    free(x); free(rn);
    return ORC_ENOMEM;
  }
  for (uint32_t v = 0; v < n; ++v) r[v] = 1.0 / (double)n;
  int it = 0;
  while (it < max_iter) {
    double D = 0.0;
    for (uint32_t u = 0; u < n; ++u) {
      int64_t deg = off[u + 1] - off[u];
      if (deg > 0) {
        x[u] = r[u] / (double)deg;
      } else {
        x[u] = 0.0;
        if (dangling_mode == 1) D += r[u];
      }
    }
    double res = 0.0;
    for (uint32_t v = 0; v < n; ++v) {
      double s = 0.0;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) s += x[col[e]];
      rn[v] = (1.0 - d) / (double)n + d * (s + D / (double)n);
      res += fabs(rn[v] - r[v]);
    }
    memcpy(r, rn, sizeof(double) * (size_t)n);
    if (resid) resid[it] = res;
    ++it;
    if (res < tol) break;
  }
  if (iters) *iters = it;
  free(x);
  free(rn);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Two-way partition (Section 4.3, Figure 6; degree assignment Section 6.2-6.3.1)        */
/* ------------------------------------------------------------------------------------ */

/* Degree class: number of significant bits of the degree (0 for an isolated vertex).
 * Vertices of one partition are ordered by class, largest first, then by global id. */
static int degree_class(int64_t deg) {
  int c = 0;
  while (deg > 0) {
    c++;
    deg >>= 1;
  }
  return c;
}

#define ORC_NCLASS 34
#define ORC_REMOTE 0x80000000u

/* assign[v] in {0,1} names the partition of global vertex v.
 * Outputs per partition p (arrays sized by the caller, upper bounds: nv_p, ne_p, nv_q):
 *   l2g[p][lid]      global id of local vertex lid
 *   poff[p][lid]     CSR offsets (nv_p + 1 entries)
 *   pE[p][e]         local id of a local neighbour, or ORC_REMOTE | outbox index
 *   pW[p][e]         weights in the same order (if w != NULL)
 *   outbox[p][i]     local id (in the other partition) of remote target i, ascending
 *   cls_end[p][c]    number of local vertices with class >= c (c = 0..33); vertices of
 *                    class c occupy [cls_end[c+1], cls_end[c])
 *   g2l[v]           (p << 31) | lid
 *   nv[p], ne[p], nout[p] counts. */
int orc_partition(uint32_t n, const int64_t* off, const uint32_t* col, const uint32_t* w,
                  const uint8_t* assign, uint32_t** l2g, int64_t** poff, uint32_t** pE,
                  uint32_t** pW, uint32_t** outbox, uint32_t** cls_end, uint32_t* g2l,
                  uint32_t* nv, int64_t* ne, uint32_t* nout) {
  uint32_t p, v;
  int c;
  uint32_t count[2][ORC_NCLASS];
  memset(count, 0, sizeof(count));
  for (v = 0; v < n; ++v) {
    if (assign[v] > 1) return ORC_EINVAL;
    count[assign[v]][degree_class(off[v + 1] - off[v])]++;
  }
  /* Stable counting sort by class, descending: next free slot per (partition, class). */
  uint32_t next[2][ORC_NCLASS];
  for (p = 0; p < 2; ++p) {
    uint32_t run = 0;
    cls_end[p][ORC_NCLASS - 1] = 0;
    for (c = ORC_NCLASS - 2; c >= 0; --c) {
      next[p][c] = run;
      run += count[p][c];
      cls_end[p][c] = run;
    }
    nv[p] = run;
  }
  for (v = 0; v < n; ++v) {
    p = assign[v];
    c = degree_class(off[v + 1] - off[v]);
    uint32_t lid = next[p][c]++;
    l2g[p][lid] = v;
    g2l[v] = (p << 31) | lid;
  }
  /* Outbox of p: the distinct remote targets, in ascending local id of their owner. */
  for (p = 0; p < 2; ++p) {
    uint32_t q = 1 - p;
    uint8_t* mark = (uint8_t*)calloc((size_t)nv[q] + 1, 1);
    uint32_t* index = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)nv[q] + 1));
    if (!mark || !index) {
      free(mark); free(index);
      return ORC_ENOMEM;
    }
    for (uint32_t lid = 0; lid < nv[p]; ++lid) {
      uint32_t g = l2g[p][lid];
      for (int64_t e = off[g]; e < off[g + 1]; ++e) {
        uint32_t u = col[e];
        if (assign[u] != p) mark[g2l[u] & 0x7FFFFFFFu] = 1;
      }
    }
    uint32_t k = 0;
    for (uint32_t ql = 0; ql < nv[q]; ++ql) {
      if (mark[ql]) {
        index[ql] = k;
        outbox[p][k] = ql;
        k++;
      }
    }
    nout[p] = k;
    /* CSR of p, local neighbours first, then remote ones, original order within each. */
    int64_t pos = 0;
    poff[p][0] = 0;
    for (uint32_t lid = 0; lid < nv[p]; ++lid) {
      uint32_t g = l2g[p][lid];
      for (int64_t e = off[g]; e < off[g + 1]; ++e) {
        uint32_t u = col[e];
        if (assign[u] == p) {
          pE[p][pos] = g2l[u] & 0x7FFFFFFFu;
          if (w) pW[p][pos] = w[e];
          pos++;
        }
      }
      for (int64_t e = off[g]; e < off[g + 1]; ++e) {
        uint32_t u = col[e];
        if (assign[u] != p) {
          pE[p][pos] = ORC_REMOTE | index[g2l[u] & 0x7FFFFFFFu];
          if (w) pW[p][pos] = w[e];
          pos++;
        }
      }
      poff[p][lid + 1] = pos;
    }
    ne[p] = pos;
    free(mark);
    free(index);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Validators and the TEPS numerator                                                     */
/* ------------------------------------------------------------------------------------ */

static int has_edge(const int64_t* off, const uint32_t* col, uint32_t a, uint32_t b) {
  for (int64_t e = off[a]; e < off[a + 1]; ++e)
    if (col[e] == b) return 1;
  return 0;
}

/* Returns 0 if (level, parent) is a valid BFS result from source on a symmetric graph:
 *  1 source level/parent wrong; 2 an edge joins a reached and an unreached vertex;
 *  3 an edge spans more than one level; 4 parent of a reached vertex invalid (not a
 *  neighbour, or not exactly one level up); 5 unreached vertex with a parent. */
int orc_check_bfs(uint32_t n, const int64_t* off, const uint32_t* col, uint32_t source,
                  const uint32_t* level, const uint32_t* parent) {
  if (source >= n) return ORC_EINVAL;
  if (level[source] != 0) return 1;
  if (parent && parent[source] != source) return 1;
  for (uint32_t u = 0; u < n; ++u) {
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      int ru = level[u] != ORC_INF, rv = level[v] != ORC_INF;
      if (ru != rv) return 2;
      if (ru) {
        int64_t diff = (int64_t)level[u] - (int64_t)level[v];
        if (diff > 1 || diff < -1) return 3;
      }
    }
  }
  if (parent) {
    for (uint32_t v = 0; v < n; ++v) {
      if (v == source) continue;
      if (level[v] == ORC_INF) {
        if (parent[v] != ORC_INF) return 5;
        continue;
      }
      uint32_t p = parent[v];
      if (p >= n || level[p] == ORC_INF || level[p] + 1 != level[v]) return 4;
      if (!has_edge(off, col, v, p)) return 4;
    }
  }
  return 0;
}

/* Returns 0 if dist are the shortest-path distances from source on a symmetric graph
 * with symmetric positive weights: 1 dist[source] != 0; 2 some edge (u,v) has
 * dist[v] > dist[u] + w; 3 a reached vertex other than the source has no neighbour u
 * with dist[u] + w == dist[v]. (2) bounds every distance from above by the true one; (3)
 * gives each reached vertex a strictly shorter predecessor, so following predecessors
 * ends at the source and bounds it from below. */
int orc_check_sssp(uint32_t n, const int64_t* off, const uint32_t* col, const uint32_t* w,
                   uint32_t source, const uint32_t* dist) {
  if (source >= n) return ORC_EINVAL;
  if (dist[source] != 0) return 1;
  for (uint32_t u = 0; u < n; ++u) {
    if (dist[u] == ORC_INF) continue;
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      uint32_t v = col[e];
      uint64_t via = (uint64_t)dist[u] + (uint64_t)w[e];
      if (dist[v] == ORC_INF || (uint64_t)dist[v] > via) return 2;
    }
  }
  for (uint32_t v = 0; v < n; ++v) {
    if (v == source || dist[v] == ORC_INF) continue;
    int tight = 0;
    for (int64_t e = off[v]; e < off[v + 1] && !tight; ++e) {
      uint32_t u = col[e];
      if (dist[u] != ORC_INF && (uint64_t)dist[u] + (uint64_t)w[e] == (uint64_t)dist[v])
        tight = 1;
    }
    if (!tight) return 3;
  }
  return 0;
}

/* Sum of degrees of the vertices whose value is not INF (levels or distances). */
int64_t orc_traversed(uint32_t n, const int64_t* off, const uint32_t* value) {
  int64_t s = 0;
  for (uint32_t v = 0; v < n; ++v)
    if (value[v] != ORC_INF) s += off[v + 1] - off[v];
  return s;
}

/* ------------------------------------------------------------------------------------ */
/* Betweenness centrality (Brandes)                                                      */
/* ------------------------------------------------------------------------------------ */

/* bc[v] += sum over the sources s of delta_s(v) for v != s; traversed (optional) receives
 * twice the degree sum of the vertices each source reaches (Section 5: forward and
 * backward phases), summed over the sources. */
int orc_bc(uint32_t n, const int64_t* off, const uint32_t* col, uint32_t nsrc,
           const uint32_t* sources, double* bc, int64_t* traversed) {
  uint32_t* dist = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  double* sigma = (double*)malloc(sizeof(double) * (n ? n : 1));
  double* delta = (double*)malloc(sizeof(double) * (n ? n : 1));
  if (!dist || !order || !sigma || !delta) {
    free(dist); free(order); free(sigma); free(delta);
    return ORC_ENOMEM;
  }
  for (uint32_t v = 0; v < n; ++v) bc[v] = 0.0;
  int64_t trav = 0;
  for (uint32_t k = 0; k < nsrc; ++k) {
    const uint32_t s = sources[k];
    if (s >= n) {
      free(dist); free(order); free(sigma); free(delta);
      return ORC_EINVAL;
    }
    for (uint32_t v = 0; v < n; ++v) {
      dist[v] = ORC_INF;
      sigma[v] = 0.0;
      delta[v] = 0.0;
    }
    /* forward: BFS in FIFO order, counting shortest paths */
    uint32_t head = 0, tail = 0;
    dist[s] = 0;
    sigma[s] = 1.0;
    order[tail++] = s;
    while (head < tail) {
      const uint32_t v = order[head++];
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        const uint32_t w = col[e];
        if (dist[w] == ORC_INF) {
          dist[w] = dist[v] + 1;
          order[tail++] = w;
        }
        if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];
      }
    }
    /* backward: reverse BFS order, so every successor's dependency is final */
    for (uint32_t i = tail; i-- > 0;) {
      const uint32_t v = order[i];
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        const uint32_t w = col[e];
        if (dist[w] == dist[v] + 1) delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w]);
      }
      if (v != s) bc[v] += delta[v];
      trav += 2 * (off[v + 1] - off[v]);
    }
  }
  if (traversed) *traversed = trav;
  free(dist); free(order); free(sigma); free(delta);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Connected components                                                                  */
/* ------------------------------------------------------------------------------------ */

int orc_cc(uint32_t n, const int64_t* off, const uint32_t* col, uint32_t* label) {
  uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  if (!queue) return ORC_ENOMEM;
  for (uint32_t v = 0; v < n; ++v) label[v] = ORC_INF;
  for (uint32_t r = 0; r < n; ++r) {
    if (label[r] != ORC_INF) continue;
    uint32_t head = 0, tail = 0;
    label[r] = r;
    queue[tail++] = r;
    while (head < tail) {
      const uint32_t v = queue[head++];
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        const uint32_t w = col[e];
        if (label[w] == ORC_INF) {
          label[w] = r;
          queue[tail++] = w;
        }
      }
    }
  }
  free(queue);
  return ORC_OK;
}
