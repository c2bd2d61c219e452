"""Batched SSSP on the GPU: every row of sssp_batch equals the oracle's Dijkstra distances
for its source (the distances of k separate Bellman-Ford searches, Section 7.3, Figure 20),
for every partition, every batch width 1..8, duplicate and isolated sources, hubs split
into chunks, host and device outputs; bad arguments are rejected."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
INF = oracle.INF


def check_batch(G, H, g, srcs, out="host"):
    d, st = G.sssp_batch(H, srcs, out=out)
    d = G.as_numpy_u32(d) if out == "device" else d
    assert d.shape == (len(srcs), g.n)
    total = 0
    for row, s in enumerate(srcs):
        ref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, int(s))
        assert np.array_equal(d[row], ref), f"row {row} (source {s})"
        total += oracle.traversed(g.n, g.offsets, ref)
    assert st["edges_traversed"] == total
    return d, st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_sssp_batch_rmat14_eight_sources(gpu, p):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    apply_partition(gpu, H, g, p)
    srcs = [int(s) for s in synth.sources(g, 8, seed=2)]
    check_batch(gpu, H, g, srcs, out="host")
    check_batch(gpu, H, g, srcs[:3], out="device")
    H.free()


def test_sssp_batch_widths_duplicates_and_isolated(gpu):
    g = rmat_graph(13, seed=5, wmax=255, wseed=7)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    srcs = [int(s) for s in synth.sources(g, 8, seed=8)]
    isolated = int(np.flatnonzero(np.diff(g.offsets) == 0)[0])
    for k in range(1, 9):
        check_batch(gpu, H, g, srcs[:k])
    check_batch(gpu, H, g, [srcs[0], srcs[0], isolated, srcs[1], srcs[0]])
    H.free()


@pytest.mark.parametrize("p", PARTITIONS[:5], ids=part_id)
def test_sssp_batch_near_far_rmat14(gpu, p):
    """Near-far order with one threshold for all lanes: every row still equals the
    oracle's, for widths from one distance value per bucket to beyond every distance."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    apply_partition(gpu, H, g, p)
    srcs = [int(s) for s in synth.sources(g, 8, seed=2)]
    refs = [oracle.sssp(g.n, g.offsets, g.cols, g.weights, s) for s in srcs]
    for delta in (1, 16, 64, 1 << 30):
        d, st = gpu.sssp_batch(H, srcs, out="host", delta=delta)
        for row in range(len(srcs)):
            assert np.array_equal(d[row], refs[row]), f"delta {delta} row {row}"
    H.free()


def test_sssp_batch_near_far_hub_path_and_duplicates(gpu):
    g = star_plus(20000, extra_seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=3)
    srcs = [0, 5, 5, 19999, 20016]
    d, _ = gpu.sssp_batch(H, srcs, out="host", delta=8)
    for row, s in enumerate(srcs):
        assert np.array_equal(d[row], oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
    H.free()
    n = 3000
    w = np.random.default_rng(2).integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(n, 0.5, 3))
    d, _ = gpu.sssp_batch(H, [0, n - 1, 1500], out="host", delta=100)
    assert np.array_equal(d[0], np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    assert np.array_equal(d[1], np.concatenate([np.cumsum(w[::-1])[::-1], [0]]).astype(np.uint32))
    H.free()


def test_sssp_batch_reads_each_edge_once_per_pass(gpu):
    """Eight copies of one source run the passes of one search: the edge entries read stay
    those of a single search (up to the timing-dependent same-round activations, which
    let a vertex relax with a distance lowered earlier in the same round), not eight
    times as many."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=256)
    s = int(synth.sources(g, 1, seed=3)[0])
    d1, st1 = gpu.sssp_batch(H, [s], out="host")
    d8, st8 = gpu.sssp_batch(H, [s] * 8, out="host")
    assert all(np.array_equal(d8[r], d1[0]) for r in range(8))
    assert abs(st8["edges_inspected"] - st1["edges_inspected"]) <= 0.1 * st1["edges_inspected"]
    assert abs(st8["supersteps"] - st1["supersteps"]) <= 2
    assert st8["edges_traversed"] == 8 * st1["edges_traversed"]
    H.free()


def test_sssp_batch_multi_chunk_hub_and_path(gpu):
    g = star_plus(20000, extra_seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        check_batch(gpu, H, g, [0, 5, 19999, 20016])
    H.free()
    n = 3000
    w = np.random.default_rng(2).integers(1, 256, n - 1)
    g = synth.from_edges(n, [(i, i + 1) for i in range(n - 1)], w=w)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(n, 0.5, 3))
    d, st = gpu.sssp_batch(H, [0, n - 1], out="host")
    assert np.array_equal(d[0], np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    assert np.array_equal(d[1], np.concatenate([np.cumsum(w[::-1])[::-1], [0]]).astype(np.uint32))
    assert st["supersteps"] >= n - 1
    H.free()


def test_sssp_batch_rejects_bad_arguments(gpu):
    g = synth.from_edges(6, [(0, 1), (1, 2), (3, 4)], w=[5, 7, 1])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=2)
    d, _ = gpu.sssp_batch(H, [0, 5, 3], out="host")
    assert list(d[0]) == [0, 5, 12, INF, INF, INF]
    assert list(d[1]) == [INF] * 5 + [0]
    assert list(d[2]) == [INF, INF, INF, 0, 1, INF]
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.sssp_batch(H, [])
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.sssp_batch(H, list(range(6)) + [0, 1, 2])  # nine searches
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.sssp_batch(H, [0, 6])
    H.free()
    g = synth.path(4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "none")
    with pytest.raises(gpu.GraphError, match="weights"):
        gpu.sssp_batch(H, [0])
    H.free()


def test_sssp_batch_overflow_reports_range_error(gpu):
    g = synth.from_edges(4, [(0, 1), (1, 2), (2, 3)], w=[2**31, 2**31, 5])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "none")
    with pytest.raises(gpu.GraphError, match="out of range"):
        gpu.sssp_batch(H, [0, 3])
    H.free()


@pytest.mark.parametrize("delta", [0, 1, 16, 300])
def test_sssp_batch_device_loop_matches_host_loop(gpu, delta):
    """Without timing the rounds run as one CUDA graph while loop (threshold moves, the
    termination vote and the cap on the device); with timing the host drives them. Same
    distances and TEPS numerator, plain rounds and near-far order, on two partitions (the
    graph is captured again after re-partitioning). Round and relaxation counts are
    compared loosely: a vertex relaxes with the newest distances of its row, which depend
    on the order in which the round's atomic minima land, so the counts vary slightly from
    call to call in either loop."""
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    srcs = [int(s) for s in synth.sources(g, 8, seed=4)]
    for T in (64, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        for k in (8, 3):
            a, sa = gpu.sssp_batch(H, srcs[:k], out="host", delta=delta)
            b, sb = gpu.sssp_batch(H, srcs[:k], out="host", delta=delta, timing=True)
            assert np.array_equal(a, b)
            assert sa["edges_traversed"] == sb["edges_traversed"]
            assert abs(sa["supersteps"] - sb["supersteps"]) <= 2
            assert abs(sa["edges_inspected"] - sb["edges_inspected"]) <= 0.1 * sb["edges_inspected"]
            for row, s in enumerate(srcs[:k]):
                assert np.array_equal(a[row], oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
    H.free()


@pytest.mark.parametrize("timing", [False, True])
@pytest.mark.parametrize("delta", [0, 2])
def test_sssp_batch_cap_boundary_both_loops(gpu, timing, delta):
    """The exact number of rounds a search needs is enough as a cap and one fewer is not,
    in both loops; odd and even round counts end the device loop in either half of its
    body."""
    g = synth.from_edges(12, [(i, i + 1) for i in range(11)], w=[1] * 11)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 5))
    for s in (0, 3, 6):
        ref = np.abs(np.arange(12) - s).astype(np.uint32)
        d, st = gpu.sssp_batch(H, [s], out="host", delta=delta, timing=timing)
        assert np.array_equal(d[0], ref)
        r = st["supersteps"]
        d, _ = gpu.sssp_batch(H, [s], out="host", delta=delta, timing=timing,
                              max_supersteps=r)
        assert np.array_equal(d[0], ref)
        with pytest.raises(gpu.GraphError, match="cap"):
            gpu.sssp_batch(H, [s], delta=delta, timing=timing, max_supersteps=r - 1)
    H.free()
