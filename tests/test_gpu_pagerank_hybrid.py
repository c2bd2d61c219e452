"""Hybrid PageRank (partition 0 on the host's cores, partition 1 on the GPU; the paper's
hybrid placement, Section 4.1 and Section 6.2) against the FP64 oracle (Section 7.1,
Figure 14), with the tolerances of the GPU-only path:
  FP64  1e-12 in L1: only the summation order differs (the host sums four interleaved
        partial sums per vertex, the GPU its own tree);
  FP32  1e-6 in L1: the stated target for FP32 gathers with FP32 accumulation.
Every partition setting, both dangling modes, host and device outputs, one and several
host threads, the tolerance stop, the two degenerate placements (everything on the GPU,
everything on the host), and interleaving with the GPU-only call."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-6}


def run_hyb(G, H, prec, iters, threads=4, dangling=True, out="host", tol=0.0):
    r, st = G.pagerank_hybrid(H, cpu_threads=threads, max_iter=iters, precision=prec,
                              dangling=dangling, out=out, tol=tol, timing=True)
    if out == "device":
        r = r.cpu().numpy()
    return r, st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hybrid_rmat14_twenty_iterations(gpu, p, prec):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    info, asg = apply_partition(gpu, H, g, p)
    ref, res, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=20)
    r, st = run_hyb(gpu, H, prec, 20, out="device" if prec == "fp32" else "host")
    l1 = np.abs(r - ref).sum()
    assert l1 <= TOL[prec], f"{prec} L1 {l1:.3e}"
    assert st["supersteps"] == 20 and st["edges_traversed"] == 20 * g.m
    if prec == "fp64":
        assert abs(st["residual"] - res[-1]) <= 1e-12
    h = st["hybrid"]
    deg = np.diff(g.offsets)
    assert h["cpu_vertices"] == int((asg == 0).sum())
    assert h["cpu_vertices"] + h["gpu_vertices"] == g.n
    assert h["cpu_edges"] == int(deg[asg == 0].sum())
    assert h["cpu_edges"] + h["gpu_edges"] == g.m
    assert st["messages"] == 20 * (info["nout"][0] + info["nout"][1])
    H.free()


@pytest.mark.parametrize("dangling", [True, False])
@pytest.mark.parametrize("threads", [1, 3, 16])
def test_hybrid_dangling_modes_and_thread_counts(gpu, dangling, threads):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=32)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=15,
                                dangling=int(dangling))
    r, st = run_hyb(gpu, H, "fp64", 15, threads=threads, dangling=dangling)
    assert np.abs(r - ref).sum() <= 1e-12
    assert st["hybrid"]["cpu_threads"] == threads
    H.free()


def test_hybrid_tolerance_stop_matches_oracle(gpu):
    """The FP64 run stops on its own residual at the oracle's first iteration below tol."""
    g = rmat_graph(13, seed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", edge_share=0.4)
    ref, res, k = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=1000, tol=1e-9)
    r, st = run_hyb(gpu, H, "fp64", 1000, tol=1e-9)
    # same stopping iteration unless the residual sits within rounding of the tolerance
    if st["supersteps"] != k:
        assert abs(res[min(st["supersteps"], k) - 1] - 1e-9) < 1e-20
    else:
        assert np.abs(r - ref).sum() <= 1e-12
    H.free()


def test_hybrid_multi_chunk_hub_on_either_side(gpu):
    """A hub with many chunks on the host (degree split) and on the GPU (explicit split
    with the hub in partition 1)."""
    g = star_plus(20000, extra_seed=8)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=25)
    gpu.graph_partition(H, "degree", degree_threshold=3)
    for prec in ("fp64", "fp32"):
        r, _ = run_hyb(gpu, H, prec, 25)
        assert np.abs(r - ref).sum() <= TOL[prec]
    asg = synth.random_assignment(g.n, 0.5, 9)
    asg[0] = 1
    gpu.graph_partition(H, "explicit", assignment=asg)
    r, _ = run_hyb(gpu, H, "fp64", 25)
    assert np.abs(r - ref).sum() <= 1e-12
    H.free()


def test_hybrid_all_on_one_side(gpu):
    """Everything on the GPU (no host vertices) and everything on the host (no GPU
    vertices): the result does not depend on the placement."""
    g = rmat_graph(12, seed=6)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=12)
    for asg in (np.ones(g.n, np.uint8), np.zeros(g.n, np.uint8)):
        gpu.graph_partition(H, "explicit", assignment=asg)
        for prec in ("fp64", "fp32"):
            r, st = run_hyb(gpu, H, prec, 12)
            assert np.abs(r - ref).sum() <= TOL[prec]
            assert st["hybrid"]["cpu_vertices"] == int((asg == 0).sum())
    H.free()


def test_hybrid_interleaved_with_gpu_only_and_repartition(gpu):
    """Hybrid and GPU-only calls share the workspace: each call resolves the work items of
    its own placement, a precision change rebuilds the workspace and a re-partition the
    host copies."""
    g = rmat_graph(13, seed=2)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=10)
    gpu.graph_partition(H, "degree", degree_threshold=16)
    for _ in range(2):
        for call in ("hybrid", "gpu"):
            for prec in ("fp64", "fp32", "fp64"):
                if call == "hybrid":
                    r, _ = run_hyb(gpu, H, prec, 10)
                else:
                    r, _ = gpu.pagerank(H, max_iter=10, precision=prec, out="host")
                assert np.abs(r - ref).sum() <= TOL[prec], (call, prec)
        gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.6, 4))
    H.free()


def test_hybrid_rejects_bad_arguments(gpu):
    g = synth.path(8)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="graph_partition"):
        gpu.pagerank_hybrid(H, out="host")
    gpu.graph_partition(H, "degree", degree_threshold=2)
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.pagerank_hybrid(H, precision="fp16", out="host")
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.pagerank_hybrid(H, cpu_threads=4096, out="host")
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.pagerank_hybrid(H, max_iter=0, out="host")
    r, _ = gpu.pagerank_hybrid(H, cpu_threads=2, max_iter=5, precision="fp64", out="host")
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=5)
    assert np.abs(r - ref).sum() <= 1e-12
    H.free()
