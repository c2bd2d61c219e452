"""Hybrid BFS and SSSP (partition 0 on the host's cores, partition 1 on the GPU; the
paper's hybrid placement, Section 4.1, Figure 6; Sections 6.2-6.3 and 7.3) against the
oracle: BFS levels bit-exact and parents validated (Section 6.3.2, Figure 11), SSSP
distances bit-exact (Section 7.3, Figure 20). Every partition setting, 1 / 4 / 16 host
threads, sources on either side, host and device outputs, the degenerate placements
(everything on the GPU, everything on the host), interleaving with the GPU-only calls,
message counts, and the bad arguments."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_hybrid_bfs_and_sssp_rmat14(gpu, p):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    info, asg = apply_partition(gpu, H, g, p)
    deg = np.diff(g.offsets)
    for s in synth.sources(g, 4, seed=2):
        s = int(s)
        ref, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
        lv, pa, st = gpu.bfs_hybrid(H, s, cpu_threads=4, out="host")
        assert np.array_equal(lv, ref)
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0
        assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, ref)
        assert st["supersteps"] == int(ref[ref != oracle.INF].max()) + 1
        h = st["hybrid"]
        assert h["cpu_vertices"] == int((asg == 0).sum())
        assert h["cpu_edges"] == int(deg[asg == 0].sum())
        dref = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
        d, sst = gpu.sssp_hybrid(H, s, cpu_threads=4, out="host")
        assert np.array_equal(d, dref)
        assert sst["edges_traversed"] == oracle.traversed(g.n, g.offsets, dref)
    H.free()


@pytest.mark.parametrize("threads", [1, 4, 16])
def test_hybrid_thread_counts_sources_on_both_sides(gpu, threads):
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=32)
    deg = np.diff(g.offsets)
    hub = int(np.argmax(deg))                                  # partition 0 (host)
    leaf = int(np.flatnonzero((deg > 0) & (deg < 32))[0])     # partition 1 (GPU)
    for s in (hub, leaf):
        ref, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
        lv, pa, st = gpu.bfs_hybrid(H, s, cpu_threads=threads, out="device")
        lv, pa = gpu.as_numpy_u32(lv), gpu.as_numpy_u32(pa)
        assert np.array_equal(lv, ref) and pa[s] == s
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0
        assert st["hybrid"]["cpu_threads"] == threads
        d, _ = gpu.sssp_hybrid(H, s, cpu_threads=threads, out="device")
        assert np.array_equal(gpu.as_numpy_u32(d), oracle.sssp(g.n, g.offsets, g.cols,
                                                               g.weights, s))
    H.free()


def test_hybrid_degenerate_placements_hubs_and_interleaving(gpu):
    g = star_plus(20000, extra_seed=8)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    for T in (0, 3, 2048, 1 << 30):   # all on the host ... all on the GPU
        gpu.graph_partition(H, "degree", degree_threshold=T)
        for s in (0, 5, 17):
            ref, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
            lv, pa, _ = gpu.bfs_hybrid(H, s, cpu_threads=3, out="host")
            assert np.array_equal(lv, ref), f"T={T} s={s}"
            assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0
            d, _ = gpu.sssp_hybrid(H, s, cpu_threads=3, out="host")
            assert np.array_equal(d, oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
            # the GPU-only calls in between see their own state
            lv2, _, _ = gpu.bfs(H, s, out="host")
            assert np.array_equal(lv2, ref)
            d2, _ = gpu.sssp(H, s, out="host")
            assert np.array_equal(d2, d)
    H.free()


def test_hybrid_paths_and_disconnected_parts(gpu):
    g = synth.path(2000)
    synth.weights(g, 64, seed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 9))
    lv, pa, st = gpu.bfs_hybrid(H, 7, cpu_threads=2, out="host")
    assert np.array_equal(lv, np.abs(np.arange(2000) - 7).astype(np.uint32))
    assert st["supersteps"] == 1993
    d, _ = gpu.sssp_hybrid(H, 7, cpu_threads=2, out="host")
    assert np.array_equal(d, oracle.sssp(g.n, g.offsets, g.cols, g.weights, 7))
    H.free()
    g = synth.from_edges(10, [(0, 1), (1, 2), (5, 6)])
    synth.weights(g, 9, seed=1)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=2)
    lv, _, _ = gpu.bfs_hybrid(H, 0, out="host")
    assert lv.tolist() == [0, 1, 2] + [oracle.INF] * 7
    d, _ = gpu.sssp_hybrid(H, 0, out="host")
    assert np.array_equal(d, oracle.sssp(g.n, g.offsets, g.cols, g.weights, 0))
    H.free()


def test_hybrid_bad_arguments(gpu):
    from paper_1312_3018_gb300 import _lib
    g = rmat_graph(10)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    lv = np.zeros(g.n, np.uint32)
    L = _lib.load()
    assert L.bfs_hybrid(H.handle, 0, lv.ctypes.data, None, None, 2, None, None) == _lib.GRAPH_ESTATE
    gpu.graph_partition(H, "degree", degree_threshold=16)
    assert L.bfs_hybrid(None, 0, lv.ctypes.data, None, None, 2, None, None) == _lib.GRAPH_EINVAL
    assert L.bfs_hybrid(H.handle, g.n, lv.ctypes.data, None, None, 2, None, None) == _lib.GRAPH_EINVAL
    assert L.bfs_hybrid(H.handle, 0, lv.ctypes.data, None, None, 5000, None, None) == _lib.GRAPH_EINVAL
    bu = _lib.bfs_attr(_lib.GRAPH_MEM_HOST, 2, 0.0, 0.0, 0, 0)    # bottom-up: refused
    assert L.bfs_hybrid(H.handle, 0, lv.ctypes.data, None, bu, 2, None, None) == _lib.GRAPH_EINVAL
    nf = _lib.sssp_attr(_lib.GRAPH_MEM_HOST, 0, 0, 16)             # near-far: refused
    assert L.sssp_hybrid(H.handle, 0, lv.ctypes.data, nf, 2, None, None) == _lib.GRAPH_EINVAL
    H.free()
    u = rmat_graph(10)
    H = gpu.graph_load_csr(u.offsets, u.cols)       # no weights
    gpu.graph_partition(H, "degree", degree_threshold=16)
    assert L.sssp_hybrid(H.handle, 0, lv.ctypes.data, None, 2, None, None) == _lib.GRAPH_EINVAL
    H.free()
