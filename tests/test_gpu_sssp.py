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
