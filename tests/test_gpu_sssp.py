"""SSSP on the GPU: distances bit-exact against the oracle (Dijkstra), for every partition
(Section 7.3, Figure 20)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
INF = oracle.INF


def check_sssp(G, H, g, src, out="host"):
    d, st = G.sssp(H, src, out=out)
    d = G.as_numpy_u32(d) if out == "device" else d
    ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, src)
    assert np.array_equal(d, ref), f"distances differ (src {src})"
    assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)
    return st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_sssp_rmat14_four_sources(gpu, p):
    """Small-config workload: RMAT scale 14, weights uniform in [1, 64], 4 sources."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    apply_partition(gpu, H, g, p)
    for k, s in enumerate(synth.sources(g, 4, seed=2)):
        check_sssp(gpu, H, g, int(s), out=("host", "device")[k % 2])
    H.free()


def test_sssp_wide_weights(gpu):
    g = rmat_graph(13, seed=5, wmax=255, wseed=7)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", edge_share=0.4)
    for s in synth.sources(g, 3, seed=8):
        check_sssp(gpu, H, g, int(s))
    H.free()


def test_sssp_multi_chunk_hub(gpu):
    g = star_plus(20000, extra_seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        for s in (0, 5, 19999):
            check_sssp(gpu, H, g, s)
    H.free()


def test_sssp_weighted_path_prefix_sums(gpu):
    n = 2000
    rng = np.random.default_rng(1)
    w = rng.integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(n, 0.5, 3))
    d, st = gpu.sssp(H, 0, out="host")
    assert np.array_equal(d, np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    H.free()


def test_sssp_edge_cases(gpu):
    g = synth.from_edges(6, [(0, 1), (1, 2), (3, 4)], w=[5, 7, 1])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=2)
    d, st = gpu.sssp(H, 0, out="host")
    assert list(d) == [0, 5, 12, INF, INF, INF]
    d, st = gpu.sssp(H, 5, out="host")                # isolated source
    assert list(d) == [INF] * 5 + [0]
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.sssp(H, 6)
    H.free()
    # no weights
    g = synth.path(4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "none")
    with pytest.raises(gpu.GraphError, match="weights"):
        gpu.sssp(H, 0)
    H.free()


def test_sssp_overflow_reports_range_error(gpu):
    g = synth.from_edges(4, [(0, 1), (1, 2), (2, 3)], w=[2**31, 2**31, 5])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "none")
    with pytest.raises(gpu.GraphError, match="out of range"):
        gpu.sssp(H, 0)
    H.free()


# Near-far order (delta > 0): the same distances with fewer wasted relaxations. Widths from
# 1 (a bucket per distance value) to beyond every distance (one bucket: plain rounds).
DELTAS = [1, 7, 64, 300, 1 << 30]


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_sssp_near_far_rmat14(gpu, p):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    apply_partition(gpu, H, g, p)
    srcs = synth.sources(g, 2, seed=2)
    refs = [oracle.sssp(g.n, g.offsets, g.cols, g.weights, int(s)) for s in srcs]
    for delta in DELTAS:
        for s, ref in zip(srcs, refs):
            d, st = gpu.sssp(H, int(s), out="host", delta=delta)
            assert np.array_equal(d, ref), f"delta {delta} src {s}"
            assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)
    H.free()


def test_sssp_near_far_inspects_no_more_than_plain(gpu):
    """On a power-law graph with wide weights, a moderate bucket width relaxes fewer edges
    than plain rounds (and never a different distance)."""
    g = rmat_graph(15, seed=3, wmax=255, wseed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=256)
    s = int(synth.sources(g, 1, seed=9)[0])
    ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
    d0, st0 = gpu.sssp(H, s, out="host")
    d1, st1 = gpu.sssp(H, s, out="host", delta=64)
    assert np.array_equal(d0, ref) and np.array_equal(d1, ref)
    assert st1["edges_inspected"] < st0["edges_inspected"]
    H.free()


def test_sssp_near_far_multi_chunk_hub_and_path(gpu):
    g = star_plus(20000, extra_seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=3)
    for s in (0, 5):
        ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
        for delta in (1, 32):
            d, _ = gpu.sssp(H, s, out="host", delta=delta)
            assert np.array_equal(d, ref)
    H.free()
    n = 3000
    w = np.random.default_rng(2).integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(n, 0.5, 3))
    d, st = gpu.sssp(H, n - 1, out="host", delta=100)
    assert np.array_equal(d, np.concatenate([np.cumsum(w[::-1])[::-1], [0]]).astype(np.uint32))
    H.free()


@pytest.mark.parametrize("delta", [0, 100])
def test_sssp_long_path(gpu, delta):
    """A 2,500-vertex path: 2,499 rounds of one vertex each, with threshold moves in near-far
    order; distances are the prefix sums."""
    n = 2500
    w = np.random.default_rng(4).integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(n, 0.5, 9))
    d, st = gpu.sssp(H, 0, out="host", delta=delta)
    assert np.array_equal(d, np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    assert st["supersteps"] >= n - 1
    H.free()


@pytest.mark.parametrize("timing", [False, True])
@pytest.mark.parametrize("delta", [0, 2])
def test_sssp_cap_boundary(gpu, timing, delta):
    """The number of rounds a search needs is enough as a cap and one fewer is not, with and
    without phase timing."""
    g = synth.from_edges(12, [(i, i + 1) for i in range(11)], w=[1] * 11)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 5))
    for s in (0, 3, 6):
        ref = np.abs(np.arange(12) - s).astype(np.uint32)
        d, st = gpu.sssp(H, s, out="host", delta=delta, timing=timing)
        assert np.array_equal(d, ref)
        r = st["supersteps"]
        d, _ = gpu.sssp(H, s, out="host", delta=delta, timing=timing, max_supersteps=r)
        assert np.array_equal(d, ref)
        with pytest.raises(gpu.GraphError, match="cap"):
            gpu.sssp(H, s, delta=delta, timing=timing, max_supersteps=r - 1)
    H.free()
