"""Batched BFS on the GPU: every row of the k-search batch bit-exact against the oracle's
single-source BFS from that source (Section 6.3.2, Figure 11: the batch only shares the
supersteps), for every partition, both forced directions and the automatic choice, odd and
duplicate source lists, multi-chunk hubs, long paths and degenerate graphs."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
INF = oracle.INF


def check_batch(G, H, g, sources, direction="auto", out="host"):
    lv, st = G.bfs_batch(H, sources, direction=direction, out=out)
    lv = G.as_numpy_u32(lv) if out == "device" else lv
    assert lv.shape == (len(sources), g.n)
    total, deepest = 0, 0
    cache = {}
    for row, s in enumerate(sources):
        s = int(s)
        if s not in cache:
            cache[s] = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)[0]
        ref = cache[s]
        assert np.array_equal(lv[row], ref), f"row {row} (source {s}, {direction}) differs"
        total += oracle.traversed(g.n, g.offsets, ref)
        deepest = max(deepest, int(ref[ref != INF].max()))
    assert st["edges_traversed"] == total
    assert st["supersteps"] == deepest + 1
    return st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_batch_rmat14_sixty_four_sources(gpu, p):
    """Small-config workload: RMAT scale 14, 64 seeded non-isolated sources in one batch."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    srcs = synth.sources(g, 64, seed=2)
    for k, d in enumerate(("auto", "topdown", "bottomup")):
        st = check_batch(gpu, H, g, srcs, direction=d, out=("host", "device")[k % 2])
        if d == "topdown":
            assert st["bottomup_steps"] == 0
        if d == "bottomup":
            assert st["topdown_steps"] == 1
    H.free()


@pytest.mark.parametrize("k", [1, 3, 37, 63])
def test_batch_sizes_and_duplicate_sources(gpu, k):
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    base = synth.sources(g, k, seed=7)
    srcs = base.copy()
    if k > 2:
        srcs[k // 2] = srcs[0]       # the same source twice in one batch
        srcs[-1] = srcs[1]
    check_batch(gpu, H, g, srcs, direction=("auto", "topdown", "bottomup")[k % 3])
    H.free()


@pytest.mark.parametrize("direction", ["auto", "topdown", "bottomup"])
def test_batch_multi_chunk_hub(gpu, direction):
    g = star_plus(20000, extra_seed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        check_batch(gpu, H, g, [0, 1, 17, 19999, 20003], direction)
    H.free()


def test_batch_long_path_many_supersteps(gpu):
    g = synth.path(3000)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 9))
    st = check_batch(gpu, H, g, [1234, 0, 2999, 1500, 1234])
    assert st["supersteps"] == 3000
    H.free()


def test_batch_grid_levels_manhattan(gpu):
    w, h = 61, 37
    g = synth.grid(w, h)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=4)
    srcs = [17 * w + 29, 0, w * h - 1]
    lv, _ = gpu.bfs_batch(H, srcs, out="host")
    x, y = np.arange(g.n) % w, np.arange(g.n) // w
    for row, s in enumerate(srcs):
        assert np.array_equal(lv[row], (np.abs(x - s % w) + np.abs(y - s // w)).astype(np.uint32))
    H.free()


def test_batch_edge_cases(gpu):
    # disconnected parts stay INF per search; an isolated source reaches only itself
    g = synth.from_edges(9, [(0, 1), (1, 2), (4, 5), (5, 6), (6, 7)])
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=2)
    check_batch(gpu, H, g, [5, 8, 0, 3, 8])
    lv, st = gpu.bfs_batch(H, [8], out="host")
    assert lv[0, 8] == 0 and np.all(np.delete(lv[0], 8) == INF)
    assert st["edges_traversed"] == 0 and st["supersteps"] == 1
    for bad in ([], list(range(65)), [9]):
        with pytest.raises(gpu.GraphError, match="invalid argument"):
            gpu.bfs_batch(H, bad)
    with pytest.raises(gpu.GraphError, match="cap"):
        gpu.bfs_batch(H, [4], max_supersteps=2)
    H.free()
    # not partitioned
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="out of order"):
        gpu.bfs_batch(H, [0])
    H.free()
    # one vertex, no edges, the whole batch on it
    H = gpu.graph_load_csr(np.zeros(2, np.int64), np.zeros(0, np.uint32))
    gpu.graph_partition(H, "none")
    lv, _ = gpu.bfs_batch(H, [0] * 64, out="host")
    assert np.all(lv == 0)
    H.free()


def test_batch_after_repartition_and_wider_batch(gpu):
    """The workspace follows re-partitioning and grows when a later call asks for more
    level lanes than an earlier one."""
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=2048)
    srcs = synth.sources(g, 64, seed=12)
    check_batch(gpu, H, g, srcs[:4])
    check_batch(gpu, H, g, srcs)
    gpu.graph_partition(H, "degree", degree_threshold=16)
    check_batch(gpu, H, g, srcs[:9])
    H.free()


STAT_KEYS = ("supersteps", "topdown_steps", "bottomup_steps", "edges_traversed",
             "edges_inspected", "messages")


@pytest.mark.parametrize("direction", ["auto", "topdown", "bottomup"])
def test_batch_device_loop_matches_host_loop(gpu, direction):
    """Without timing the supersteps run as one CUDA graph while loop (termination vote,
    cap and direction rule on the device); with timing the host drives them. Same levels,
    same step counts and statistics, for several alphas (the direction rule's switch
    point) and batch widths (each change re-captures the graph)."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    srcs = synth.sources(g, 64, seed=5)
    for k, alpha in ((40, 0.0), (3, 4.0), (64, 40.0), (40, 0.0)):
        a, sa = gpu.bfs_batch(H, srcs[:k], direction=direction, alpha=alpha, out="host")
        b, sb = gpu.bfs_batch(H, srcs[:k], direction=direction, alpha=alpha, out="host",
                              timing=True)
        assert np.array_equal(a, b)
        for key in STAT_KEYS:
            assert sa[key] == sb[key], key
        check_batch(gpu, H, g, srcs[:k], direction)
    H.free()


@pytest.mark.parametrize("timing", [False, True])
def test_batch_cap_boundary_both_loops(gpu, timing):
    """A 10-vertex path from vertex 0 takes 10 supersteps: a cap of 10 is enough, 9 is not;
    odd and even superstep counts end the device loop in either half of its body."""
    g = synth.path(10)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 3))
    lv, st = gpu.bfs_batch(H, [0], max_supersteps=10, out="host", timing=timing)
    assert np.array_equal(lv[0], np.arange(10, dtype=np.uint32)) and st["supersteps"] == 10
    with pytest.raises(gpu.GraphError, match="cap"):
        gpu.bfs_batch(H, [0], max_supersteps=9, timing=timing)
    for s, steps in ((1, 9), (2, 8), (5, 6)):
        lv, st = gpu.bfs_batch(H, [s], out="host", timing=timing)
        assert st["supersteps"] == steps
        assert np.array_equal(lv[0], np.abs(np.arange(10) - s).astype(np.uint32))
    H.free()
