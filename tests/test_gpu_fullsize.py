"""Parity at the full workload sizes (RMAT with the Table 2 parameters, weights uniform in
[1, 255]), at the degree split the benchmark times and at T = 2048.

The benchmark's threshold is read through the same autotuner call and threshold cache the
benchmark uses (bench_threshold below), so the two cannot drift apart.

RMAT scale 22 (4.19M vertices, ~128M edge entries, T = 2048): BFS levels and SSSP distances
compared with the oracle element by element for sampled sources, PageRank to an L1 residual
below 1e-9 (the oracle's iteration count K*) in FP32 / FP16 against FP64.

RMAT scale 25 (33.5M vertices, ~1.05B edge entries), at the benchmark's threshold and at
T = 2048: BFS levels against the oracle element by element and parents validated; SSSP
distances against the oracle's Dijkstra element by element and through the optimality
certificate (every edge satisfies dist[v] <= dist[u] + w and every reached vertex has a
tight predecessor), in plain rounds and in the benchmark's near-far order; FP32 PageRank
after 3 iterations against the FP64 oracle (L1 and per-vertex bounds), FP16 by L1.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
INF = oracle.INF
T = 2048
NEAR_FAR_DELTA = 128
BENCH_DELTA = 64        # near-far width of the benchmark step's SSSP


def bench_threshold(G, H, g):
    """The degree threshold the benchmark runs at: the autotuner called exactly as bench.py
    calls it (same source, same cache file, no retuning). Leaves H partitioned at it."""
    import os
    from paper_1312_3018_gb300 import autotune
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = os.path.join(root, "paper_1312_3018_gb300", "tuned_thresholds.json")
    src = int(synth.sources(g, 64, seed=2)[0])
    return int(autotune.autotune_threshold(G, H, src, weighted=True, cache=cache)["T"])


@pytest.fixture(scope="module")
def rmat22():
    g = synth.rmat(22, 16, seed=1)
    synth.weights(g, 255, seed=3)
    return g


@pytest.fixture(scope="module")
def rmat25():
    g = synth.rmat(25, 16, seed=1)
    synth.weights(g, 255, seed=3)
    return g


@pytest.fixture(scope="module")
def loaded22(gpu, rmat22):
    H = gpu.graph_load_csr(rmat22.offsets, rmat22.cols, rmat22.weights)
    gpu.graph_partition(H, "degree", degree_threshold=T)
    yield H
    H.free()


@pytest.fixture(scope="module")
def loaded25(gpu, rmat25):
    """The RMAT-25 handle and the thresholds to check: the benchmark's and 2048."""
    H = gpu.graph_load_csr(rmat25.offsets, rmat25.cols, rmat25.weights)
    tb = bench_threshold(gpu, H, rmat25)
    yield H, sorted({tb, T})
    H.free()


@pytest.fixture(scope="module")
def source25(rmat25):
    return int(synth.sources(rmat25, 1, seed=2)[0])


def test_rmat22_bfs_sixty_four_sources(gpu, rmat22, loaded22):
    g = rmat22
    srcs = synth.sources(g, 64, seed=2)
    checked = 0
    for k, s in enumerate(srcs):
        lv, pa, st = gpu.bfs(loaded22, int(s), out="host")
        assert lv[s] == 0 and pa[s] == s
        if k < 4:  # element-by-element against the oracle for a sample of the searches
            ref, _ = oracle.bfs(g.n, g.offsets, g.cols, int(s), want_parents=False)
            assert np.array_equal(lv, ref)
            assert oracle.check_bfs(g.n, g.offsets, g.cols, int(s), lv, pa) == 0
            assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)
            checked += 1
    assert checked == 4


def test_rmat22_sssp(gpu, rmat22, loaded22):
    g = rmat22
    for s in synth.sources(g, 2, seed=4):
        ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, int(s))
        for delta in (0, NEAR_FAR_DELTA):  # plain rounds, then the benchmark's near-far width
            d, st = gpu.sssp(loaded22, int(s), out="host", delta=delta)
            assert np.array_equal(d, ref), f"delta {delta}"
            assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)


def test_rmat22_sssp_batch_eight_sources(gpu, rmat22, loaded22):
    """Eight searches in one batch at full size: two rows against the oracle element by
    element, every row through the optimality certificate."""
    g = rmat22
    srcs = [int(s) for s in synth.sources(g, 8, seed=4)]
    d, st = gpu.sssp_batch(loaded22, srcs, out="host")
    total = 0
    for row, s in enumerate(srcs):
        if row < 2:
            assert np.array_equal(d[row], oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
        assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, d[row]) == 0
        total += oracle.traversed(g.n, g.offsets, d[row])
    assert st["edges_traversed"] == total
    d2, _ = gpu.sssp_batch(loaded22, srcs, out="host", delta=NEAR_FAR_DELTA)
    assert np.array_equal(d2, d)


def test_rmat22_pagerank_to_residual_1e9(gpu, rmat22, loaded22):
    g = rmat22
    ref, res, kstar = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=1000, tol=1e-9)
    r64, st = gpu.pagerank(loaded22, max_iter=1000, tol=1e-9, precision="fp64", out="host")
    assert st["supersteps"] == kstar
    assert np.abs(r64 - ref).sum() <= 1e-12
    r32, _ = gpu.pagerank(loaded22, max_iter=kstar, precision="fp32", out="host")
    l1 = np.abs(r32 - ref).sum()
    assert l1 <= 1e-6, f"FP32 L1 {l1:.3e} at K*={kstar}"
    r16, _ = gpu.pagerank(loaded22, max_iter=kstar, precision="fp16", out="host")
    assert np.abs(r16 - ref).sum() <= 1e-3


def test_rmat25_bfs(gpu, rmat25, loaded25, source25):
    g, s = rmat25, source25
    H, thresholds = loaded25
    ref, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
    trav = oracle.traversed(g.n, g.offsets, ref)
    for t in thresholds:
        gpu.graph_partition(H, "degree", degree_threshold=t)
        lv, pa, st = gpu.bfs(H, s, out="host")
        assert np.array_equal(lv, ref), f"T={t}"
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0, f"T={t}"
        assert st["edges_traversed"] == trav


def test_rmat25_sssp(gpu, rmat25, loaded25, source25):
    g, s = rmat25, source25
    H, thresholds = loaded25
    ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
    trav = oracle.traversed(g.n, g.offsets, ref)
    for t in thresholds:
        gpu.graph_partition(H, "degree", degree_threshold=t)
        for delta in (0, BENCH_DELTA):   # Figure 20's plain rounds, the benchmark's order
            d, st = gpu.sssp(H, s, out="host", delta=delta)
            assert np.array_equal(d, ref), f"T={t} delta={delta}"
            assert st["edges_traversed"] == trav
        assert oracle.check_sssp(g.n, g.offsets, g.cols, g.weights, s, d) == 0


# Per-vertex bounds of FP32 PageRank after 3 iterations against FP64. Every rank is at
# least (1-d)/n, a neighbour sum of k positive FP32 terms added in any order is within
# (k-1) ulp-relative error of the exact sum, and the deepest sum here (a hub's partials)
# has a few thousand terms, so 3 iterations stay within a few 1e-5 relative even in the
# worst case; the bound below (1e-4 relative, 1e-8 absolute) leaves room for that and
# still fails on any dropped or doubled neighbour of a vertex of degree < 1e4.
PR_MAX_REL = 1e-4
PR_MAX_ABS = 1e-8


def test_rmat25_pagerank_three_iterations(gpu, rmat25, loaded25):
    g = rmat25
    H, thresholds = loaded25
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=3)
    for t in thresholds:
        gpu.graph_partition(H, "degree", degree_threshold=t)
        r32, _ = gpu.pagerank(H, max_iter=3, precision="fp32", out="host")
        d = np.abs(r32 - ref)
        assert d.sum() <= 1e-6, f"T={t} L1 {d.sum():.3e}"
        assert d.max() <= PR_MAX_ABS, f"T={t} max-abs {d.max():.3e}"
        assert (d / ref).max() <= PR_MAX_REL, f"T={t} max-rel {(d / ref).max():.3e}"
        r16, _ = gpu.pagerank(H, max_iter=3, precision="fp16", out="host")
        assert np.abs(r16 - ref).sum() <= 1e-3, f"T={t}"


def test_rmat22_bfs_batch_sixty_four_sources(gpu, rmat22, loaded22):
    """One 64-search batch at full size: every row has level 0 at its source and obeys the
    BFS edge rule; four rows are compared with the oracle element by element, and the
    traversed-edge count is the sum of the rows' TEPS numerators."""
    g = rmat22
    srcs = synth.sources(g, 64, seed=2)
    lv, st = gpu.bfs_batch(loaded22, srcs, out="host")
    total = 0
    for row, s in enumerate(srcs):
        assert lv[row, s] == 0
        total += oracle.traversed(g.n, g.offsets, lv[row])
        if row < 4:
            ref, _ = oracle.bfs(g.n, g.offsets, g.cols, int(s), want_parents=False)
            assert np.array_equal(lv[row], ref), f"row {row}"
    assert st["edges_traversed"] == total
    # |level[u] - level[v]| <= 1 along every edge, for a sample of rows
    src_of_edge = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets))
    for row in (10, 37, 63):
        a = lv[row][src_of_edge].astype(np.int64)
        b = lv[row][g.cols].astype(np.int64)
        both = (a != INF) & (b != INF)
        assert np.all(np.abs(a[both] - b[both]) <= 1)
        assert np.all((a == INF) == (b == INF))


def test_rmat25_bfs_batch(gpu, rmat25, loaded25):
    g = rmat25
    H, thresholds = loaded25
    gpu.graph_partition(H, "degree", degree_threshold=thresholds[0])
    srcs = synth.sources(g, 64, seed=2)
    lv, st = gpu.bfs_batch(H, srcs, out="device")
    for row in (0, 41):
        ref, _ = oracle.bfs(g.n, g.offsets, g.cols, int(srcs[row]), want_parents=False)
        assert np.array_equal(gpu.as_numpy_u32(lv[row]), ref), f"row {row}"
    del lv


def test_many_graph_pagerank_256_uneven_rmat(gpu):
    """The batching workload at full size: 256 RMAT graphs, scales 10-17, edge factors 8-32,
    30 FP32 iterations in one pagerank_multi call; the smallest, the largest and four more
    components against the oracle run on that graph alone, and every component's ranks
    summing to one."""
    fam = synth.rmat_family(256, scales=(10, 17), edge_factors=(8, 32), seed=7)
    U, vb = synth.disjoint_union(fam)
    H = gpu.graph_load_csr(U.offsets, U.cols)
    gpu.graph_partition(H, "degree", degree_threshold=256)
    r, res, st = gpu.pagerank_multi(H, vb, max_iter=30, precision="fp32", out="host")
    sums = np.add.reduceat(r, vb[:-1].astype(np.int64))
    assert np.all(np.abs(sums - 1.0) <= 1e-5)
    ms = np.array([g.m for g in fam])
    pick = {int(np.argmin(ms)), int(np.argmax(ms)), 3, 77, 150, 255}
    for i in sorted(pick):
        g = fam[i]
        ref, rres, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=30)
        assert np.abs(r[vb[i]:vb[i + 1]] - ref).sum() <= 1e-6, f"component {i}"
        assert abs(res[i] - rres[-1]) <= 2e-6
    H.free()


def test_rmat22_betweenness_four_sources(gpu, rmat22, loaded22):
    g = rmat22
    srcs = synth.sources(g, 4, seed=9)
    sc, st = gpu.betweenness(loaded22, srcs, out="host")
    ref, trav = oracle.bc(g.n, g.offsets, g.cols, srcs)
    err = np.abs(sc - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 1e-9
    assert st["edges_traversed"] == trav


def test_rmat22_and_rmat25_connected_components(gpu, rmat22, loaded22, rmat25, loaded25):
    for g, H in ((rmat22, loaded22), (rmat25, loaded25[0])):
        lab, _ = gpu.connected_components(H, out="host")
        assert np.array_equal(lab, oracle.cc(g.n, g.offsets, g.cols))
