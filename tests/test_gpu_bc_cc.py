"""Betweenness centrality and connected components on the GPU against the oracle.

Betweenness (Section 7.2, Figure 18): path counts are integers in FP64 and exact below
2^53 in any summation order; the dependencies sum quotients in another order than the
oracle, so scores are compared with a relative tolerance of 1e-9 (FP64 rounding of sums of
at most ~10^6 terms stays near 1e-12 relative). Graphs whose scores are integers (paths,
stars) are compared exactly. Connected components: labels are unique (the smallest id of
the component) and compared bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
RTOL = 1e-9


def check_bc(G, H, g, sources, out="host", exact=False):
    sc, st = G.betweenness(H, sources, out=out)
    sc = sc.cpu().numpy() if out == "device" else sc
    ref, trav = oracle.bc(g.n, g.offsets, g.cols, sources)
    if exact:
        assert np.array_equal(sc, ref)
    else:
        err = np.abs(sc - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() <= RTOL, f"max relative error {err.max():.3e}"
    assert st["edges_traversed"] == trav
    return sc, st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_bc_rmat12_eight_sources(gpu, p):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    check_bc(gpu, H, g, synth.sources(g, 8, seed=5), out=("host", "device")[len(p[1]) % 2])
    H.free()


def test_bc_closed_forms(gpu):
    for g, exact in ((synth.path(40), True), (synth.star(25), True), (synth.complete(9), True),
                     (synth.grid(7, 5), False), (synth.cycle(11), False)):
        H = gpu.graph_load_csr(g.offsets, g.cols)
        gpu.graph_partition(H, "degree", degree_threshold=3)
        check_bc(gpu, H, g, np.arange(g.n), exact=exact)
        H.free()


@pytest.mark.parametrize("T", [3, 2048, 1 << 30])
def test_bc_multi_chunk_hub(gpu, T):
    g = star_plus(20000, extra_seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=T)
    check_bc(gpu, H, g, [0, 1, 5, 19999, 20001])
    H.free()


def test_bc_long_path_exact(gpu):
    g = synth.path(1500)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 4))
    _, st = check_bc(gpu, H, g, [0, 749, 1499, 749], exact=True)
    H.free()


def test_bc_path_seventy_thousand_levels(gpu):
    """A 70,000-vertex path from one end: levels up to 69,999 (beyond any 16-bit level
    encoding), 70,000 forward and 69,999 backward supersteps over the level queues. Closed
    form: from source 0, vertex v >= 1 lies on the paths to the n - 1 - v vertices beyond
    it."""
    n = 70000
    g = synth.path(n)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 6))
    sc, st = gpu.betweenness(H, [0], out="host")
    want = (n - 1 - np.arange(n)).astype(np.float64)
    want[0] = 0.0
    assert np.array_equal(sc, want)
    assert st["edges_traversed"] == 2 * (2 * (n - 1))
    H.free()


def test_bc_edge_cases(gpu):
    g = synth.from_edges(9, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 7)])
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="out of order"):
        gpu.betweenness(H, [0])
    gpu.graph_partition(H, "degree", degree_threshold=2)
    check_bc(gpu, H, g, [5, 8, 0, 3], exact=True)     # 3 and 8 are isolated
    for bad in ([], [9]):
        with pytest.raises(gpu.GraphError, match="invalid argument"):
            gpu.betweenness(H, bad)
    H.free()


def check_cc(G, H, g, out="host"):
    lab, st = G.connected_components(H, out=out)
    lab = G.as_numpy_u32(lab) if out == "device" else lab
    assert np.array_equal(lab, oracle.cc(g.n, g.offsets, g.cols))
    return st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
@pytest.mark.parametrize("scale,ef", [(14, 2), (12, 16)])
def test_cc_rmat(gpu, p, scale, ef):
    g = synth.rmat(scale, ef, seed=scale + ef)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    check_cc(gpu, H, g, out=("host", "device")[ef % 2 == 0 and len(p[1]) % 2])
    H.free()


def test_cc_structured_and_hub(gpu):
    parts = [synth.path(300), star_plus(5000, extra_seed=3), synth.grid(20, 9),
             synth.from_edges(4, []), synth.cycle(17)]
    u, _ = synth.disjoint_union(parts)
    H = gpu.graph_load_csr(u.offsets, u.cols)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        check_cc(gpu, H, u)
    H.free()


def test_cc_long_path_and_cap(gpu):
    g = synth.path(3000)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 2))
    st = check_cc(gpu, H, g)
    assert st["supersteps"] >= 2999
    with pytest.raises(gpu.GraphError, match="cap"):
        gpu.connected_components(H, max_supersteps=3)
    H.free()
    H = gpu.graph_load_csr(np.zeros(2, np.int64), np.zeros(0, np.uint32))
    gpu.graph_partition(H, "none")
    lab, _ = gpu.connected_components(H, out="host")
    assert lab[0] == 0
    H.free()
