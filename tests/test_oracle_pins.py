"""Pins for the CPU oracle: closed forms, brute force, library routines and invariants.

Each check is independent of the oracle's own code, and chosen so that a plausible slip
in the oracle (a dropped term, a wrong index, an off-by-one level, a missing division by
the degree, in-place updates) fails at least one of them. No GPU is used.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
import synth

INF = oracle.INF
D = 0.85


# ---------------------------------------------------------------- independent helpers

def floyd_warshall(g, weighted):
    """All-pairs shortest paths by the textbook triple loop (vectorised over one index)."""
    n = g.n
    dist = np.full((n, n), np.inf)
    np.fill_diagonal(dist, 0.0)
    for u in range(n):
        for e in range(g.offsets[u], g.offsets[u + 1]):
            v = int(g.cols[e])
            w = float(g.weights[e]) if weighted else 1.0
            dist[u, v] = min(dist[u, v], w)
    for k in range(n):
        dist = np.minimum(dist, dist[:, k:k + 1] + dist[k:k + 1, :])
    return dist


def as_u32(row):
    out = np.full(row.shape, INF, dtype=np.uint64)
    fin = np.isfinite(row)
    out[fin] = row[fin].astype(np.uint64)
    return out.astype(np.uint32)


def transition(g):
    """Dense column-stochastic-ish matrix M[v, u] = 1/deg(u) for each edge u -> v."""
    n = g.n
    M = np.zeros((n, n))
    deg = g.degrees()
    for u in range(n):
        for e in range(g.offsets[u], g.offsets[u + 1]):
            M[int(g.cols[e]), u] += 1.0 / deg[u]
    return M


def dense_pr_iterate(g, iters, dangling):
    """Power iteration in matrix form: r <- (1-d)/n + d (M r + [dangling] (delta.r)/n)."""
    n = g.n
    M = transition(g)
    delta = (g.degrees() == 0).astype(float)
    r = np.full(n, 1.0 / n)
    for _ in range(iters):
        r = (1 - D) / n + D * (M @ r + (delta @ r) / n * dangling)
    return r


def er_with_isolated(n, p, seed, n_isolated=6):
    """Random graph on n vertices plus n_isolated degree-zero vertices spread among them."""
    base = synth.erdos_renyi(n, p, seed)
    total = n + n_isolated
    rng = np.random.default_rng(seed + 1000)
    ids = np.sort(rng.choice(total, n, replace=False))   # new id of each base vertex
    edges = [(ids[u], ids[int(v)]) for u in range(n)
             for v in base.cols[base.offsets[u]:base.offsets[u + 1]]]
    return synth.from_edges(total, edges)


def dense_pr_solve(g, dangling):
    """Fixed point by a dense linear solve (the limit of the iteration)."""
    n = g.n
    M = transition(g)
    delta = (g.degrees() == 0).astype(float)
    A = np.eye(n) - D * M - (D / n) * np.outer(np.ones(n), delta) * dangling
    return np.linalg.solve(A, np.full(n, (1 - D) / n))


# ---------------------------------------------------------------- BFS pins

@pytest.mark.parametrize("n,s", [(1, 0), (2, 1), (17, 0), (17, 8), (33, 32)])
def test_bfs_path_levels_are_distance_along_path(n, s):
    g = synth.path(n)
    lv, pa = oracle.bfs(g.n, g.offsets, g.cols, s)
    idx = np.arange(n)
    assert np.array_equal(lv, np.abs(idx - s).astype(np.uint32))
    exp_parent = np.where(idx < s, idx + 1, np.where(idx > s, idx - 1, s))
    assert np.array_equal(pa, exp_parent.astype(np.uint32))


@pytest.mark.parametrize("w,h,s", [(7, 5, 0), (7, 5, 17), (1, 9, 4), (12, 12, 143)])
def test_bfs_grid_levels_are_manhattan(w, h, s):
    g = synth.grid(w, h)
    lv, pa = oracle.bfs(g.n, g.offsets, g.cols, s)
    x, y = np.arange(w * h) % w, np.arange(w * h) // w
    man = np.abs(x - s % w) + np.abs(y - s // w)
    assert np.array_equal(lv, man.astype(np.uint32))
    assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0


def test_bfs_star_from_centre_and_leaf():
    g = synth.star(9)
    lv, _ = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert lv[0] == 0 and np.all(lv[1:] == 1)
    lv, pa = oracle.bfs(g.n, g.offsets, g.cols, 4)
    exp = np.full(10, 2, np.uint32)
    exp[0], exp[4] = 1, 0
    assert np.array_equal(lv, exp)
    assert pa[0] == 4 and all(pa[i] == 0 for i in range(1, 10) if i != 4)


def test_bfs_disconnected_part_stays_inf():
    g = synth.from_edges(8, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 7)])
    lv, pa = oracle.bfs(g.n, g.offsets, g.cols, 5)
    assert list(lv) == [INF, INF, INF, INF, 1, 0, 1, 2]
    assert pa[0] == INF and pa[3] == INF and pa[5] == 5


@pytest.mark.parametrize("seed", range(6))
def test_bfs_brute_force_floyd_warshall(seed):
    g = synth.erdos_renyi(40 + seed * 4, 0.06, seed)
    fw = floyd_warshall(g, weighted=False)
    for s in (0, g.n // 2, g.n - 1):
        lv, pa = oracle.bfs(g.n, g.offsets, g.cols, s)
        assert np.array_equal(lv, as_u32(fw[s]))
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0


def test_bfs_matches_scipy_on_rmat():
    g = synth.rmat(11, seed=7)
    A = sp.csr_matrix((np.ones(g.m), g.cols.astype(np.int64), g.offsets), shape=(g.n, g.n))
    for s in synth.sources(g, 3, seed=2):
        lv, pa = oracle.bfs(g.n, g.offsets, g.cols, s)
        ref = csg.shortest_path(A, unweighted=True, indices=int(s))
        assert np.array_equal(lv, as_u32(ref))
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0


def test_bfs_validator_rejects_planted_mistakes():
    g = synth.grid(6, 6)
    lv, pa = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, lv, pa) == 0
    bad = lv.copy(); bad[20] += 2
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, bad, pa) != 0
    bad = pa.copy(); bad[20] = 0           # not a neighbour of 20
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, lv, bad) == 4
    bad = pa.copy(); bad[7] = 8            # neighbour on the same level
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, lv, bad) == 4
    bad = lv.copy(); bad[35] = INF         # reached neighbour left unreached
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, bad, None) == 2
    bad = lv.copy(); bad[0] = 1
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, bad, pa) == 1
    # a parent one level up that is not a neighbour: only the edge rule rejects it
    # (vertex 8 = (2,1) at level 3; vertex 12 = (0,2) at level 2 is not adjacent to it)
    bad = pa.copy(); bad[8] = 12
    assert lv[12] + 1 == lv[8]
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, lv, bad) == 4


def test_bfs_validator_rejects_level_jump_on_a_non_tree_edge():
    """Triangle 0-1-2: true levels from 0 are [0,1,1]. Levels [0,1,2] with parents [0,0,1]
    form a consistent tree, and only the non-tree edge 0-2, which spans two levels, shows
    them wrong."""
    g = synth.from_edges(3, [(0, 1), (1, 2), (0, 2)])
    lv = np.array([0, 1, 2], np.uint32)
    pa = np.array([0, 0, 1], np.uint32)
    assert oracle.check_bfs(g.n, g.offsets, g.cols, 0, lv, pa) == 3
    ref, _ = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert list(ref) == [0, 1, 1]


def test_traversed_edges_is_degree_sum_of_reached():
    g = synth.from_edges(7, [(0, 1), (0, 2), (2, 3), (4, 5), (5, 6), (4, 6)])
    lv, _ = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert oracle.traversed(g.n, g.offsets, lv) == 2 + 1 + 2 + 1
    lv, _ = oracle.bfs(g.n, g.offsets, g.cols, 5)
    assert oracle.traversed(g.n, g.offsets, lv) == 6


# ---------------------------------------------------------------- SSSP pins

def test_sssp_weighted_path_is_prefix_sum():
    n = 25
    rng = np.random.default_rng(0)
    w = rng.integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    for s in (0, 12, n - 1):
        dist = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
        pref = np.concatenate([[0], np.cumsum(w)])
        assert np.array_equal(dist, np.abs(pref - pref[s]).astype(np.uint32))


@pytest.mark.parametrize("wconst", [1, 7, 255])
def test_sssp_uniform_weight_is_weight_times_hops(wconst):
    g = synth.grid(9, 7)
    w = np.full(g.m, wconst, np.uint32)
    s = 31
    dist = oracle.sssp(g.n, g.offsets, g.cols, w, s)
    x, y = np.arange(g.n) % 9, np.arange(g.n) // 9
    man = np.abs(x - s % 9) + np.abs(y - s // 9)
    assert np.array_equal(dist, (wconst * man).astype(np.uint32))


@pytest.mark.parametrize("seed", range(6))
def test_sssp_brute_force_floyd_warshall(seed):
    g = synth.erdos_renyi(36 + seed * 5, 0.08, 100 + seed)
    synth.weights(g, 64, seed=seed)
    fw = floyd_warshall(g, weighted=True)
    for s in (0, 7, g.n - 1):
        dist = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
        assert np.array_equal(dist, as_u32(fw[s]))
        assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, dist) == 0


def test_sssp_matches_scipy_dijkstra_on_rmat():
    g = synth.rmat(11, seed=9)
    synth.weights(g, 255, seed=4)
    A = sp.csr_matrix((g.weights.astype(np.float64), g.cols.astype(np.int64), g.offsets),
                      shape=(g.n, g.n))
    for s in synth.sources(g, 3, seed=5):
        dist = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
        ref = csg.dijkstra(A, indices=int(s))
        assert np.array_equal(dist, as_u32(ref))


def test_sssp_certificate_rejects_planted_mistakes():
    g = synth.rmat(9, seed=3)
    synth.weights(g, 64, seed=1)
    s = int(synth.sources(g, 1, seed=1)[0])
    dist = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
    assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, dist) == 0
    reached = np.flatnonzero((dist != INF) & (np.arange(g.n) != s))
    v = int(reached[len(reached) // 2])
    bad = dist.copy(); bad[v] += 1          # too long: some edge certifies a shorter path
    assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, bad) != 0
    bad = dist.copy(); bad[v] -= 1          # too short: no tight predecessor
    assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, bad) != 0
    bad = dist.copy(); bad[s] = 1
    assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, bad) == 1


def test_sssp_overflow_is_reported():
    g = synth.from_edges(4, [(0, 1), (1, 2), (2, 3)], w=[2**31, 2**31, 5])
    with pytest.raises(oracle.OracleError):
        oracle.sssp(g.n, g.offsets, g.cols, g.weights, 0)


# ---------------------------------------------------------------- PageRank pins

@pytest.mark.parametrize("n", [3, 10, 101])
def test_pagerank_cycle_is_uniform_every_iteration(n):
    g = synth.cycle(n)
    for k in (1, 2, 7):
        r, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=k)
        assert it == k
        assert np.allclose(r, 1.0 / n, rtol=0, atol=1e-15)
        assert np.all(res < 1e-15)


def test_pagerank_complete_graph_is_uniform():
    g = synth.complete(12)
    r, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=30)
    assert np.allclose(r, 1 / 12, rtol=0, atol=1e-15)


@pytest.mark.parametrize("k", [1, 3, 40])
def test_pagerank_star_closed_form(k):
    g = synth.star(k)
    n = k + 1
    r, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=400)
    rc = (1 + D * k) / (n * (1 + D))
    rl = (1 - D) / n + D * rc / k
    assert abs(r[0] - rc) < 1e-13
    assert np.allclose(r[1:], rl, rtol=0, atol=1e-13)
    assert abs(r.sum() - 1) < 1e-13


@pytest.mark.parametrize("seed,dangling", [(0, 1), (1, 1), (2, 0), (3, 0), (4, 1)])
def test_pagerank_iterates_match_dense_matrix_iteration(seed, dangling):
    g = er_with_isolated(44, 0.05, seed)
    assert (g.degrees() == 0).any()
    for iters in (1, 2, 20):
        r, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=iters,
                                     dangling=dangling)
        ref = dense_pr_iterate(g, iters, dangling)
        assert np.max(np.abs(r - ref)) < 1e-15
        prev = dense_pr_iterate(g, iters - 1, dangling)
        assert abs(res[-1] - np.abs(ref - prev).sum()) < 1e-14


@pytest.mark.parametrize("seed,dangling", [(10, 1), (11, 0)])
def test_pagerank_converges_to_dense_solve(seed, dangling):
    g = er_with_isolated(56, 0.05, seed)
    r, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=1000, tol=1e-15,
                                 dangling=dangling)
    ref = dense_pr_solve(g, dangling)
    assert np.max(np.abs(r - ref)) < 1e-13
    if dangling:
        assert abs(r.sum() - 1) < 1e-12
    else:
        assert r.sum() < 1 - 1e-3            # mass leaks through dangling vertices


def test_pagerank_mass_is_conserved_with_dangling_redistribution():
    g = synth.rmat(12, seed=5)
    assert (g.degrees() == 0).any()
    r, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=25)
    assert abs(r.sum() - 1) < 1e-12
    assert np.all(r >= (1 - D) / g.n - 1e-18)


def test_pagerank_tolerance_stops_at_first_residual_below():
    g = synth.rmat(10, seed=2)
    _, res_all, _ = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=200)
    tol = 1e-9
    kstar = int(np.argmax(res_all < tol)) + 1
    _, res, it = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=1000, tol=tol)
    assert it == kstar and res[-1] < tol and np.all(res[:-1] >= tol)


def test_pagerank_path3_golden():
    """Fixed point on the 3-vertex path, hand-derived (tests/golden/path3_pagerank.txt)."""
    vals = {}
    for line in open(__file__.replace("test_oracle_pins.py", "golden/path3_pagerank.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    g = synth.path(3)
    r, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, D, max_iter=600, tol=0.0)
    assert abs(r[0] - vals["r0"]) < 1e-12 and abs(r[2] - vals["r2"]) < 1e-12
    assert abs(r[1] - vals["r1"]) < 1e-12


def test_small_graph_golden_bfs_sssp():
    """Hand-worked BFS levels and distances (tests/golden/small_weighted.txt)."""
    lines = [l.split("#")[0].strip() for l in
             open(__file__.replace("test_oracle_pins.py", "golden/small_weighted.txt"))]
    lines = [l for l in lines if l]
    n = int(lines[0].split()[1])
    edges, ws, exp = [], [], {}
    for l in lines[1:]:
        tok = l.split()
        if tok[0] == "edge":
            edges.append((int(tok[1]), int(tok[2])))
            ws.append(int(tok[3]))
        else:
            exp[tok[0]] = [INF if t == "INF" else int(t) for t in tok[1:]]
    g = synth.from_edges(n, edges, w=ws)
    lv, _ = oracle.bfs(g.n, g.offsets, g.cols, 0)
    assert list(lv) == exp["levels"]
    dist = oracle.sssp(g.n, g.offsets, g.cols, g.weights, 0)
    assert list(dist) == exp["dist"]


# ---------------------------------------------------------------- partition pins

def _rebuild_global(P, n):
    """Global adjacency lists from the partitioned structures (inverse of the partition)."""
    adj = [[] for _ in range(n)]
    for p in (0, 1):
        q = 1 - p
        part, other = P["parts"][p], P["parts"][q]
        for lid in range(part["nv"]):
            g = int(part["l2g"][lid])
            for e in range(part["off"][lid], part["off"][lid + 1]):
                x = int(part["E"][e])
                if x & oracle.REMOTE:
                    adj[g].append(int(other["l2g"][part["outbox"][x & 0x7FFFFFFF]]))
                else:
                    adj[g].append(int(part["l2g"][x]))
    return adj


def _degree_class(d):
    return int(d).bit_length()


@pytest.mark.parametrize("how", ["deg0", "deg4", "deg16", "deginf", "random"])
def test_partition_is_an_exact_relabelling(how):
    g = synth.rmat(10, seed=11)
    synth.weights(g, 64, seed=2)
    if how == "random":
        asg = synth.random_assignment(g.n, 0.3, seed=5)
    else:
        T = {"deg0": 0, "deg4": 4, "deg16": 16, "deginf": 1 << 40}[how]
        asg = oracle.degree_assignment(g.offsets, T)
    P = oracle.partition(g.n, g.offsets, g.cols, asg, g.weights)
    deg = g.degrees()
    # bijection, partition membership, g2l inverse of l2g
    seen = np.zeros(g.n, bool)
    for p in (0, 1):
        part = P["parts"][p]
        assert part["nv"] == int((asg == p).sum())
        l2g = part["l2g"].astype(np.int64)
        assert np.all(asg[l2g] == p)
        assert not seen[l2g].any()
        seen[l2g] = True
        assert np.array_equal(P["g2l"][l2g], (p << 31) | np.arange(part["nv"]))
        # order: degree class descending, then global id ascending
        keys = [(-_degree_class(deg[v]), int(v)) for v in l2g]
        assert keys == sorted(keys)
        # class boundaries
        ce = part["cls_end"].astype(np.int64)
        for c in range(oracle.NCLASS - 1):
            sel = np.flatnonzero([_degree_class(deg[v]) == c for v in l2g])
            if len(sel):
                assert sel[0] == ce[c + 1] and sel[-1] == ce[c] - 1
            else:
                assert ce[c + 1] == ce[c]
        # local-first order inside every adjacency
        for lid in range(part["nv"]):
            seg = part["E"][part["off"][lid]:part["off"][lid + 1]]
            rem = (seg & oracle.REMOTE) != 0
            assert not np.any(rem[:-1] & ~rem[1:])
        # outbox: sorted, unique, exactly the remote targets
        ob = part["outbox"]
        assert np.all(np.diff(ob.astype(np.int64)) > 0)
        other = P["parts"][1 - p]
        targets = set()
        for v in l2g:
            for u in g.cols[g.offsets[v]:g.offsets[v + 1]]:
                if asg[u] != p:
                    targets.add(int(P["g2l"][u]) & 0x7FFFFFFF)
        assert set(int(x) for x in ob) == targets
        assert all(x < other["nv"] for x in ob)
    assert seen.all()
    # the partitioned graph is the original graph, with the same neighbour multiset,
    # local neighbours in original order, then remote ones in original order
    adj = _rebuild_global(P, g.n)
    for v in range(g.n):
        orig = [int(u) for u in g.cols[g.offsets[v]:g.offsets[v + 1]]]
        loc = [u for u in orig if asg[u] == asg[v]]
        rem = [u for u in orig if asg[u] != asg[v]]
        assert adj[v] == loc + rem
    # weights travel with their edges
    for p in (0, 1):
        part, other = P["parts"][p], P["parts"][1 - p]
        for lid in range(0, part["nv"], 7):
            v = int(part["l2g"][lid])
            wmap = {int(u): int(w) for u, w in zip(g.cols[g.offsets[v]:g.offsets[v + 1]],
                                                   g.weights[g.offsets[v]:g.offsets[v + 1]])}
            for e in range(part["off"][lid], part["off"][lid + 1]):
                x = int(part["E"][e])
                if x & oracle.REMOTE:
                    u = int(other["l2g"][part["outbox"][x & 0x7FFFFFFF]])
                else:
                    u = int(part["l2g"][x])
                assert int(part["W"][e]) == wmap[u]


def test_edge_share_threshold_brute_force():
    g = synth.rmat(9, seed=4)
    deg = g.degrees()
    m = int(deg.sum())
    for share in (0.05, 0.25, 0.5, 0.8, 1.0):
        T = oracle.edge_share_threshold(g.offsets, share)
        best = max(t for t in range(0, int(deg.max()) + 2)
                   if deg[deg >= t].sum() >= share * m)
        assert T == best
    assert oracle.edge_share_threshold(g.offsets, 0.0) == int(deg.max()) + 1


# ---------------------------------------------------------------- betweenness centrality

def dense_adjacency(g):
    A = np.zeros((g.n, g.n), dtype=np.float64)
    for u in range(g.n):
        for e in range(g.offsets[u], g.offsets[u + 1]):
            A[u, int(g.cols[e])] = 1.0
    return A


def path_counts(g):
    """Distances and numbers of shortest paths for all pairs from powers of the adjacency
    matrix: d(s,t) is the first k with (A^k)[s,t] > 0, and every walk of that length is a
    shortest path, so sigma(s,t) = (A^d)[s,t]."""
    A = dense_adjacency(g)
    n = g.n
    d = np.full((n, n), np.inf)
    sig = np.zeros((n, n))
    np.fill_diagonal(d, 0)
    np.fill_diagonal(sig, 1)
    P = np.eye(n)
    for k in range(1, n):
        P = P @ A
        new = (P > 0) & ~np.isfinite(d)
        d[new] = k
        sig[new] = P[new]
    return d, sig


def bc_by_pair_dependencies(g, sources):
    """Definition of betweenness: BC(v) = sum over sources s and targets t (s, t, v
    distinct) of sigma(s,v) sigma(v,t) / sigma(s,t) when v lies on a shortest s-t path."""
    d, sig = path_counts(g)
    bc = np.zeros(g.n)
    for s in sources:
        for t in range(g.n):
            if t == s or not np.isfinite(d[s, t]):
                continue
            for v in range(g.n):
                if v in (s, t):
                    continue
                if d[s, v] + d[v, t] == d[s, t]:
                    bc[v] += sig[s, v] * sig[v, t] / sig[s, t]
    return bc


@pytest.mark.parametrize("n", [2, 6, 31])
def test_bc_path_closed_form(n):
    g = synth.path(n)
    bc, trav = oracle.bc(g.n, g.offsets, g.cols, np.arange(n))
    i = np.arange(n)
    assert np.array_equal(bc, 2.0 * i * (n - 1 - i))
    assert trav == n * 2 * g.m


@pytest.mark.parametrize("k", [1, 2, 9])
def test_bc_star_closed_form(k):
    g = synth.star(k)
    bc, _ = oracle.bc(g.n, g.offsets, g.cols, np.arange(k + 1))
    assert bc[0] == k * (k - 1) and np.all(bc[1:] == 0)
    # from the centre alone nothing is between; from one leaf the centre carries k-1
    assert np.all(oracle.bc(g.n, g.offsets, g.cols, [0])[0] == 0)
    assert oracle.bc(g.n, g.offsets, g.cols, [1])[0][0] == k - 1


def test_bc_complete_graph_is_zero():
    g = synth.complete(7)
    assert np.all(oracle.bc(g.n, g.offsets, g.cols, np.arange(7))[0] == 0)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_bc_matches_pair_dependency_definition(seed):
    rng = np.random.default_rng(seed)
    n = 11
    g = synth.erdos_renyi(n, 0.28, seed=seed + 40)
    srcs = sorted(rng.choice(n, size=4, replace=False).tolist())
    for S in (srcs, list(range(n))):
        bc, _ = oracle.bc(g.n, g.offsets, g.cols, S)
        assert np.allclose(bc, bc_by_pair_dependencies(g, S), rtol=1e-12, atol=1e-12)


def test_bc_cycle_and_grid_pair_definition():
    for g in (synth.cycle(9), synth.cycle(10), synth.grid(4, 3)):
        bc, _ = oracle.bc(g.n, g.offsets, g.cols, np.arange(g.n))
        assert np.allclose(bc, bc_by_pair_dependencies(g, range(g.n)), rtol=1e-12)


def test_bc_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = synth.rmat(9, 8, seed=5)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for e in range(g.offsets[u], g.offsets[u + 1]):
            G.add_edge(u, int(g.cols[e]))
    ref = nx.betweenness_centrality(G, normalized=False)  # unordered pairs
    bc, _ = oracle.bc(g.n, g.offsets, g.cols, np.arange(g.n))
    assert np.allclose(bc, 2 * np.array([ref[v] for v in range(g.n)]), rtol=1e-9, atol=1e-9)


def test_bc_sum_is_total_interior_length():
    """Every connected ordered pair (s, t) spreads exactly d(s,t) - 1 over the interior
    vertices of its shortest paths."""
    g = synth.rmat(7, 6, seed=8)
    d = floyd_warshall(g, weighted=False)
    fin = np.isfinite(d) & (d > 0)
    bc, _ = oracle.bc(g.n, g.offsets, g.cols, np.arange(g.n))
    assert abs(bc.sum() - (d[fin] - 1).sum()) <= 1e-9 * max(1.0, bc.sum())


# ---------------------------------------------------------------- connected components

def test_cc_closed_forms():
    parts = [synth.path(5), synth.star(3), synth.from_edges(1, []), synth.cycle(4),
             synth.from_edges(2, [])]
    u, vb = synth.disjoint_union(parts)
    lab = oracle.cc(u.n, u.offsets, u.cols)
    expect = np.concatenate([np.full(p.n, vb[i]) if i != 4 else vb[i] + np.arange(p.n)
                             for i, p in enumerate(parts)]).astype(np.uint32)
    assert np.array_equal(lab, expect)


@pytest.mark.parametrize("scale,ef", [(12, 2), (10, 1), (13, 16)])
def test_cc_matches_scipy(scale, ef):
    g = synth.rmat(scale, ef, seed=scale)
    A = sp.csr_matrix((np.ones(g.m), np.asarray(g.cols), np.asarray(g.offsets)),
                      shape=(g.n, g.n))
    k, comp = csg.connected_components(A, directed=False)
    mins = np.full(k, g.n, np.int64)
    np.minimum.at(mins, comp, np.arange(g.n))
    lab = oracle.cc(g.n, g.offsets, g.cols)
    assert np.array_equal(lab, mins[comp].astype(np.uint32))
