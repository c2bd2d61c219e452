"""BFS on the GPU: levels bit-exact against the oracle, parents valid, TEPS numerator equal
to the oracle's, for every partition and direction policy (Section 6.3.2, Figure 11)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
INF = oracle.INF


def check_bfs(G, H, g, src, direction="auto", out="host"):
    lv, pa, st = G.bfs(H, src, direction=direction, out=out)
    lv = G.as_numpy_u32(lv) if out == "device" else lv
    pa = G.as_numpy_u32(pa) if out == "device" else pa
    ref, _ = oracle.bfs(g.n, g.offsets, g.cols, src, want_parents=False)
    assert np.array_equal(lv, ref), f"levels differ (src {src}, {direction})"
    assert oracle.check_bfs(g.n, g.offsets, g.cols, src, lv, pa) == 0, "invalid parents"
    assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)
    assert st["supersteps"] == int(ref[ref != INF].max()) + 1
    return st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_bfs_rmat14_sixteen_sources(gpu, p):
    """Small-config workload: RMAT scale 14, 16 seeded non-isolated sources."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    for k, s in enumerate(synth.sources(g, 16, seed=2)):
        check_bfs(gpu, H, g, int(s), direction=("auto", "topdown", "bottomup")[k % 3],
                  out=("host", "device")[k % 2])
    H.free()


@pytest.mark.parametrize("direction", ["auto", "topdown", "bottomup"])
def test_bfs_multi_chunk_hub(gpu, direction):
    g = star_plus(20000, extra_seed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        for s in (0, 1, 17, 19999):
            check_bfs(gpu, H, g, s, direction)
    H.free()


def test_bfs_long_path_many_supersteps(gpu):
    g = synth.path(3000)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    asg = synth.random_assignment(g.n, 0.5, 9)
    gpu.graph_partition(H, "explicit", assignment=asg)
    st = check_bfs(gpu, H, g, 1234)
    assert st["supersteps"] == 1766
    H.free()


def test_bfs_grid_levels_manhattan(gpu):
    w, h = 61, 37
    g = synth.grid(w, h)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=4)   # interior vs border split
    s = 17 * w + 29
    lv, pa, _ = gpu.bfs(H, s, out="host")
    x, y = np.arange(g.n) % w, np.arange(g.n) // w
    assert np.array_equal(lv, (np.abs(x - s % w) + np.abs(y - s // w)).astype(np.uint32))
    H.free()


def test_bfs_edge_cases(gpu):
    # disconnected parts stay INF; isolated source reaches only itself
    g = synth.from_edges(9, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 7)])
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=2)
    check_bfs(gpu, H, g, 5)
    lv, pa, st = gpu.bfs(H, 8, out="host")          # vertex 8 isolated
    assert lv[8] == 0 and pa[8] == 8 and np.all(np.delete(lv, 8) == INF)
    assert st["edges_traversed"] == 0
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.bfs(H, 9)
    with pytest.raises(gpu.GraphError, match="cap"):
        gpu.bfs(H, 4, max_supersteps=2)
    H.free()
    # one vertex, no edges
    H = gpu.graph_load_csr(np.zeros(2, np.int64), np.zeros(0, np.uint32))
    gpu.graph_partition(H, "none")
    lv, pa, _ = gpu.bfs(H, 0, out="host")
    assert lv[0] == 0 and pa[0] == 0
    H.free()


def test_bfs_without_parents_and_repeat(gpu):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    s = int(synth.sources(g, 1, seed=11)[0])
    a, _, _ = gpu.bfs(H, s, want_parents=False, out="host")
    b, _, _ = gpu.bfs(H, s, want_parents=False, out="host")
    assert np.array_equal(a, b)
    assert np.array_equal(a, oracle.bfs(g.n, g.offsets, g.cols, s)[0])
    H.free()
