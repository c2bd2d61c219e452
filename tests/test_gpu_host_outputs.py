"""Results delivered to host memory. A page-locked (pinned) host array is written by the
collect kernel directly over the host link; a pageable array goes through the device
staging buffer and a copy. Both must hold exactly what a device output holds, for BFS
(levels, and parents as a valid BFS tree), SSSP, connected components and PageRank, on two partitions, also
when only one of two host outputs is pinned."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import rmat_graph

pytestmark = pytest.mark.gpu


def pinned(torch, n, dtype):
    return torch.empty(n, dtype=dtype, pin_memory=True).numpy()


@pytest.mark.parametrize("T", [64, 1 << 30])
def test_host_outputs_pinned_and_pageable(gpu, T):
    import torch
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=T)
    s = int(synth.sources(g, 1, seed=2)[0])
    lv_d, pa_d, _ = gpu.bfs(H, s, out="device")
    lv_d, pa_d = gpu.as_numpy_u32(lv_d), gpu.as_numpy_u32(pa_d)
    assert np.array_equal(lv_d, oracle.bfs(g.n, g.offsets, g.cols, s)[0])
    pl, pp = pinned(torch, g.n, torch.int32).view(np.uint32), pinned(torch, g.n, torch.int32).view(np.uint32)
    ql, qp = np.zeros(g.n, np.uint32), np.zeros(g.n, np.uint32)
    for levels, parents in ((pl, pp), (ql, qp), (pl, qp), (ql, pp)):
        levels[:] = 7
        parents[:] = 7
        gpu.bfs(H, s, levels, parents, out="host")
        assert np.array_equal(levels, lv_d)
        # parents form one valid BFS tree; which one can differ from call to call
        assert oracle.check_bfs(g.n, g.offsets, g.cols, s, levels, parents) == 0
    d_d, _ = gpu.sssp(H, s, out="device")
    d_d = gpu.as_numpy_u32(d_d)
    assert np.array_equal(d_d, oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
    for dist in (pinned(torch, g.n, torch.int32).view(np.uint32), np.zeros(g.n, np.uint32)):
        _, st = gpu.sssp(H, s, dist, out="host")
        assert np.array_equal(dist, d_d)
        assert st["edges_traversed"] == oracle.traversed(g.n, g.offsets, d_d)
    c_d, _ = gpu.connected_components(H, out="device")
    c_d = gpu.as_numpy_u32(c_d)
    for lab in (pinned(torch, g.n, torch.int32).view(np.uint32), np.zeros(g.n, np.uint32)):
        gpu.connected_components(H, lab, out="host")
        assert np.array_equal(lab, c_d)
    r_d, _ = gpu.pagerank(H, max_iter=10, precision="fp32", out="device")
    r_d = r_d.cpu().numpy()
    for ranks in (pinned(torch, g.n, torch.float64), np.zeros(g.n)):
        gpu.pagerank(H, ranks=ranks, max_iter=10, precision="fp32", out="host")
        assert np.array_equal(ranks, r_d)
    H.free()


def test_host_outputs_batched_sssp_and_betweenness(gpu):
    import torch
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=32)
    srcs = [int(s) for s in synth.sources(g, 5, seed=6)]
    d_d, _ = gpu.sssp_batch(H, srcs, out="device")
    d_d = gpu.as_numpy_u32(d_d)
    for row, s in enumerate(srcs):
        assert np.array_equal(d_d[row], oracle.sssp(g.n, g.offsets, g.cols, g.weights, s))
    for dist in (pinned(torch, len(srcs) * g.n, torch.int32).view(np.uint32).reshape(len(srcs), g.n),
                 np.zeros((len(srcs), g.n), np.uint32)):
        gpu.sssp_batch(H, srcs, dist, out="host")
        assert np.array_equal(dist, d_d)
    b_d, _ = gpu.betweenness(H, srcs[:3], out="device")
    b_d = b_d.cpu().numpy()
    for sc in (pinned(torch, g.n, torch.float64), np.zeros(g.n)):
        gpu.betweenness(H, srcs[:3], sc, out="host")
        assert np.allclose(sc, b_d, rtol=1e-12, atol=0)
    H.free()
