"""PageRank on the GPU against the FP64 oracle (Section 7.1, Figure 14).

Tolerances (L1 = sum of |r_gpu - r_oracle| over all vertices, ranks sum to 1):
  FP64  1e-12: only the summation order differs (hub chunks, shuffle trees); each rank
        carries a relative error of a few ulps (~1e-15) and the L1 over ranks summing to
        one stays near 1e-14; 1e-12 leaves a wide margin.
  FP32  1e-6: the stated target for FP32 gathers with FP32 accumulation.
  FP16  1e-3: contributions rounded to 11-bit mantissas (relative 2^-11 ~ 5e-4 each);
        reported, no target is claimed.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3}


def run_pr(G, H, prec, iters, dangling=True, out="host"):
    r, st = G.pagerank(H, max_iter=iters, precision=prec, dangling=dangling, out=out)
    if out == "device":
        r = r.cpu().numpy()
    return r, st


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_pagerank_rmat14_twenty_iterations(gpu, p, prec):
    """Small-config workload: RMAT scale 14, damping 0.85, 20 iterations."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    ref, res, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=20)
    r, st = run_pr(gpu, H, prec, 20, out={"fp64": "host", "fp32": "device", "fp16": "host"}[prec])
    l1 = np.abs(r - ref).sum()
    assert l1 <= TOL[prec], f"{prec} L1 {l1:.3e}"
    assert st["supersteps"] == 20 and st["edges_traversed"] == 20 * g.m
    if prec == "fp64":
        assert abs(st["residual"] - res[-1]) <= 1e-12
    H.free()


@pytest.mark.parametrize("dangling", [True, False])
def test_pagerank_dangling_modes(gpu, dangling):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=32)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=15,
                                dangling=int(dangling))
    r, _ = run_pr(gpu, H, "fp64", 15, dangling=dangling)
    assert np.abs(r - ref).sum() <= 1e-12
    H.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pagerank_multi_chunk_hub(gpu, prec):
    g = star_plus(20000, extra_seed=8)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=12)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        r, _ = run_pr(gpu, H, prec, 12)
        assert np.abs(r - ref).sum() <= TOL[prec]
    H.free()


def test_pagerank_cycle_uniform_and_star_closed_form(gpu):
    g = synth.cycle(1001)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "explicit", assignment=synth.random_assignment(g.n, 0.5, 1))
    r, _ = run_pr(gpu, H, "fp64", 9)
    assert np.allclose(r, 1 / 1001, rtol=0, atol=1e-15)
    H.free()
    k, d = 5000, 0.85
    g = synth.star(k)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=2048)
    r, _ = run_pr(gpu, H, "fp64", 300)
    n = k + 1
    rc = (1 + d * k) / (n * (1 + d))
    assert abs(r[0] - rc) < 1e-13
    assert np.allclose(r[1:], (1 - d) / n + d * rc / k, rtol=0, atol=1e-15)
    H.free()


def test_pagerank_tolerance_stops_like_the_oracle(gpu):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    ref, res, k = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=1000, tol=1e-9)
    r, st = gpu.pagerank(H, max_iter=1000, tol=1e-9, precision="fp64", out="host")
    # same stopping iteration unless the residual sits within rounding of the tolerance
    if st["supersteps"] != k:
        assert abs(res[min(st["supersteps"], k) - 1] - 1e-9) < 1e-20
    assert np.abs(r - ref).sum() <= 1e-12 or st["supersteps"] != k
    H.free()


def test_pagerank_rejects_bad_attributes(gpu):
    g = synth.path(5)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "none")
    with pytest.raises(gpu.GraphError):
        gpu.pagerank(H, damping=1.5)
    with pytest.raises(gpu.GraphError):
        gpu.pagerank(H, max_iter=0)
    H.free()
