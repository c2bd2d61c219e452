"""Edge arrays in page-locked host memory (Section 4.3.4 (iii), Section 8: the immutable,
sequentially read edge arrays of a partition kept in mapped host memory so that graphs
larger than the GPU's memory fit). With any placement every algorithm must give the
oracle's results: BFS levels and valid parents, SSSP distances, component labels, PageRank
(gather and segmented methods, three precisions), batched BFS and SSSP, betweenness, the
hybrid calls and the query server; moving the arrays back, and re-partitioning from a
host-resident input CSR, must leave the partition bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import rmat_graph

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3}


def check_all(G, H, g):
    srcs = [int(s) for s in synth.sources(g, 3, seed=11)]
    s = srcs[0]
    ref_l = oracle.bfs(g.n, g.offsets, g.cols, s)[0]
    ref_d = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
    for d in ("auto", "topdown", "bottomup"):
        lv, pa, _ = G.bfs(H, s, out="host", direction=d)
        assert np.array_equal(lv, ref_l), d
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, lv, pa) == 0
    for delta in (0, 16):
        dist, _ = G.sssp(H, s, out="host", delta=delta)
        assert np.array_equal(dist, ref_d), delta
    lab, _ = G.connected_components(H, out="host")
    assert np.array_equal(lab, oracle.cc(g.n, g.offsets, g.cols))
    ref_r, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=10)
    for prec in ("fp32", "fp16", "fp64"):
        r, _ = G.pagerank(H, max_iter=10, precision=prec, out="host")
        assert np.abs(r - ref_r).sum() <= TOL[prec], prec
    r, _ = G.pagerank(H, max_iter=10, precision="fp32", out="host", method="segmented")
    assert np.abs(r - ref_r).sum() <= 1e-6
    lvb, _ = G.bfs_batch(H, srcs, out="host")
    db, _ = G.sssp_batch(H, srcs, out="host")
    for row, x in enumerate(srcs):
        assert np.array_equal(lvb[row], oracle.bfs(g.n, g.offsets, g.cols, x)[0])
        assert np.array_equal(db[row], oracle.sssp(g.n, g.offsets, g.cols, g.weights, x))
    sc, _ = G.betweenness(H, srcs[:2], out="host")
    ref_b, _ = oracle.bc(g.n, g.offsets, g.cols, srcs[:2])
    assert (np.abs(sc - ref_b) / np.maximum(1.0, np.abs(ref_b))).max() <= 1e-9
    hl, hp, _ = G.bfs_hybrid(H, s, out="host", cpu_threads=4)
    assert np.array_equal(hl, ref_l)
    hd, _ = G.sssp_hybrid(H, s, out="host", cpu_threads=4)
    assert np.array_equal(hd, ref_d)
    hr, _ = G.pagerank_hybrid(H, max_iter=10, precision="fp32", out="host", cpu_threads=4)
    assert np.abs(hr - ref_r).sum() <= 1e-6


@pytest.mark.parametrize("which", ["part0", "part1", ["part0", "part1", "input"]])
def test_algorithms_with_host_resident_edges(gpu, which):
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=32)
    gpu.graph_set_edge_memory(H, which, "host")
    placed = gpu.graph_get_edge_memory(H)
    for w in ([which] if isinstance(which, str) else which):
        assert placed[w] == "host"
    check_all(gpu, H, g)
    # back to device memory: the same partition, the same results
    gpu.graph_set_edge_memory(H, which, "device")
    assert set(gpu.graph_get_edge_memory(H).values()) == {"device"}
    check_all(gpu, H, g)
    H.free()


def test_partition_from_host_resident_input_and_server(gpu):
    import torch
    g = rmat_graph(12, seed=3)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_set_edge_memory(H, "input", "host")        # before any partition
    asg = synth.random_assignment(g.n, 0.4, 7)
    gpu.graph_partition(H, "explicit", assignment=asg)
    ref = oracle.partition(g.n, g.offsets, g.cols, asg, g.weights)
    for p in (0, 1):
        got = gpu.graph_export_partition(H, p, weights=True)
        assert np.array_equal(got["E"], ref["parts"][p]["E"])
        assert np.array_equal(got["W"], ref["parts"][p]["W"])
        assert np.array_equal(got["off"], ref["parts"][p]["off"])
    gpu.graph_set_edge_memory(H, ["part0", "part1"], "host")
    for p in (0, 1):   # export reads the host-resident arrays
        got = gpu.graph_export_partition(H, p, weights=True)
        assert np.array_equal(got["E"], ref["parts"][p]["E"])
    srcs = [int(s) for s in synth.sources(g, 12, seed=5)]
    outs = []
    with gpu.Server(H, out="device", sssp_batch=True) as srv:
        for i, s in enumerate(srcs):
            buf = torch.empty(g.n, dtype=torch.int32, device="cuda")
            srv.submit("bfs" if i % 2 else "sssp", s, buf)
            outs.append(buf)
        done = []
        while len(done) < len(srcs):
            done += srv.poll(cap=64, wait_ms=20)
    for c in done:
        assert c["status"] == 0
        got = gpu.as_numpy_u32(c["out"])
        ref_v = (oracle.bfs(g.n, g.offsets, g.cols, c["source"])[0] if c["kind"] == "bfs"
                 else oracle.sssp(g.n, g.offsets, g.cols, g.weights, c["source"]))
        assert np.array_equal(got, ref_v)
    # re-partitioning from the host-resident input puts the new partitions on the device
    gpu.graph_partition(H, "degree", degree_threshold=16)
    m = gpu.graph_get_edge_memory(H)
    assert m == {"part0": "device", "part1": "device", "input": "host"}
    lv, _, _ = gpu.bfs(H, srcs[0], out="host")
    assert np.array_equal(lv, oracle.bfs(g.n, g.offsets, g.cols, srcs[0])[0])
    H.free()


def test_edge_memory_bad_arguments(gpu):
    from paper_1312_3018_gb300 import _lib
    g = rmat_graph(10)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    lib = _lib.load()
    assert lib.graph_set_edge_memory(H.handle, 1, _lib.GRAPH_MEM_HOST) == _lib.GRAPH_ESTATE
    for which, mem in ((0, _lib.GRAPH_MEM_HOST), (8, _lib.GRAPH_MEM_HOST), (1, 7)):
        assert lib.graph_set_edge_memory(H.handle, which, mem) == _lib.GRAPH_EINVAL
    assert lib.graph_get_edge_memory(H.handle, None) == _lib.GRAPH_EINVAL
    gpu.graph_set_edge_memory(H, "input", "host")
    gpu.graph_set_edge_memory(H, "input", "host")       # already there: no change
    gpu.graph_partition(H, "none")
    lv, _, _ = gpu.bfs(H, 0, out="host")
    assert np.array_equal(lv, oracle.bfs(g.n, g.offsets, g.cols, 0)[0])
    H.free()
