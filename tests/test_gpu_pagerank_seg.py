"""Segmented PageRank (method "segmented", FP32 and FP16) against the FP64 oracle and
against the per-edge gather kernel (Section 7.1, Figure 14).

The segmented method forms the same neighbour sums in another order: per (segment,
destination) partial sums from shared memory, then each destination's partials in segment
order. Tolerances are the FP32 / FP16 ones of the other PageRank tests (L1 over ranks
summing to one: FP32 1e-6, FP16 1e-3 against FP64). Small layout parameters (segments of
64 sources, chunks of 64 entries, bins of 64 partial sums) make small graphs exercise
many segments per partition, rows split across chunks, several passes per bin and many
bins; the defaults are exercised too. Ranks must repeat bit for bit from call to call.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-6, "fp16": 1e-3}
TINY = dict(seg_log2=6, seg_chunk=64, seg_bin=64)
LAYOUTS = {"default": {}, "tiny": TINY, "mid": dict(seg_log2=9, seg_chunk=1000, seg_bin=700)}


def pr(G, H, prec, iters, **kw):
    r, st = G.pagerank(H, max_iter=iters, precision=prec, out="host", **kw)
    return r, st


@pytest.mark.parametrize("layout", list(LAYOUTS))
@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
def test_segmented_rmat14_all_partitions(gpu, p, layout):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    apply_partition(gpu, H, g, p)
    ref, res, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=20)
    for prec in ("fp32", "fp16"):
        r, st = pr(gpu, H, prec, 20, method="segmented", **LAYOUTS[layout])
        l1 = np.abs(r - ref).sum()
        assert l1 <= TOL[prec], f"{prec} L1 {l1:.3e}"
        assert st["supersteps"] == 20 and st["edges_traversed"] == 20 * g.m
        if prec == "fp32":
            assert abs(st["residual"] - res[-1]) <= 1e-6
    info = gpu.pagerank_plan(H)
    assert info["built"] == 1 and info["usable"] == 1
    assert 0 < info["partials"] <= g.m + info["chunks"]
    H.free()


@pytest.mark.parametrize("layout", ["default", "tiny"])
def test_segmented_agrees_with_gather_and_repeats(gpu, layout):
    g = rmat_graph(15)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    rg, _ = pr(gpu, H, "fp32", 10, method="gather")
    r1, _ = pr(gpu, H, "fp32", 10, method="segmented", **LAYOUTS[layout])
    r2, _ = pr(gpu, H, "fp32", 10, method="segmented", **LAYOUTS[layout])
    assert np.array_equal(r1, r2), "segmented ranks differ between two calls"
    assert np.abs(r1 - rg).sum() <= 1e-6
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=10)
    assert np.abs(r1 - ref).sum() <= 1e-6
    H.free()


def test_segmented_dangling_tolerance_and_device_output(gpu):
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=16)
    for dangling in (True, False):
        ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=25,
                                    dangling=int(dangling))
        r, _ = pr(gpu, H, "fp32", 25, dangling=dangling, method="segmented", **TINY)
        assert np.abs(r - ref).sum() <= 1e-6
    # tolerance stop: the FP32 residual reaches 1e-6 after the oracle's iteration count
    ref, res, k = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=200, tol=1e-6)
    r, st = pr(gpu, H, "fp32", 200, tol=1e-6, method="segmented")
    assert abs(st["supersteps"] - k) <= 1
    assert np.abs(r - ref).sum() <= 1e-6
    rd, _ = gpu.pagerank(H, max_iter=8, precision="fp32", out="device", method="segmented")
    rh, _ = pr(gpu, H, "fp32", 8, method="segmented")
    assert np.array_equal(rd.cpu().numpy(), rh)
    H.free()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_segmented_hub_rows_split_over_chunks(gpu, prec):
    """A 20,000-leaf hub: its row in a segment spans many chunks (split rows) and its
    partial sums span several passes of its bin."""
    g = star_plus(20000, extra_seed=8)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=12)
    for T in (3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        for lay in ({}, dict(seg_log2=10, seg_chunk=256, seg_bin=64)):
            r, _ = pr(gpu, H, prec, 12, method="segmented", **lay)
            assert np.abs(r - ref).sum() <= TOL[prec], f"T={T} {lay}"
    H.free()


def test_segmented_edge_cases(gpu):
    # no edges at all: every vertex keeps the constant term
    g = synth.from_edges(50, [])
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=4)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=5)
    r, _ = pr(gpu, H, "fp32", 5, method="segmented")
    assert np.abs(r - ref).sum() <= 1e-6
    H.free()
    # one edge, a path, a cycle, everything in partition 0 or in partition 1
    for g in (synth.from_edges(7, [(2, 5)]), synth.path(300), synth.cycle(257)):
        ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=30)
        H = gpu.graph_load_csr(g.offsets, g.cols)
        for name, kw in (("degree", dict(degree_threshold=0)), ("none", {}),
                         ("degree", dict(degree_threshold=2))):
            gpu.graph_partition(H, name, **kw)
            for lay in ({}, TINY):
                r, _ = pr(gpu, H, "fp32", 30, method="segmented", **lay)
                assert np.abs(r - ref).sum() <= 1e-6
        H.free()


def test_segmented_limits_and_bad_arguments(gpu):
    from paper_1312_3018_gb300 import _lib
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    for kw in (dict(seg_log2=5), dict(seg_log2=16), dict(seg_chunk=63), dict(seg_chunk=9000),
               dict(seg_bin=63), dict(seg_bin=14337)):
        with pytest.raises(_lib.GraphError) as e:
            pr(gpu, H, "fp32", 3, method="segmented", **kw)
        assert e.value.status == _lib.GRAPH_EINVAL
    with pytest.raises(_lib.GraphError) as e:
        pr(gpu, H, "fp64", 3, method="segmented")
    assert e.value.status == _lib.GRAPH_EINVAL
    attr = _lib.pagerank_attr(0.85, 3, 0.0, 0, 1, 0, 0, 7, 0, 0, 0)   # unknown method
    r = np.zeros(g.n)
    assert _lib.load().pagerank(H.handle, attr, r.ctypes.data, None) == _lib.GRAPH_EINVAL
    H.free()
    # a hub adjacent to more than 2,047 segments of 64 sources exceeds the layout: the
    # segmented method is refused (the plan records it), the gather method is right
    g = star_plus(300000, extra_seed=3)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "none")
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=6)
    with pytest.raises(_lib.GraphError) as e:
        pr(gpu, H, "fp32", 6, method="segmented", seg_log2=6)
    assert e.value.status == _lib.GRAPH_EINVAL
    info = gpu.pagerank_plan(H)
    assert info["built"] == 1 and info["usable"] == 0
    r, _ = pr(gpu, H, "fp32", 6)   # auto: gather
    assert np.abs(r - ref).sum() <= 1e-6
    r, _ = pr(gpu, H, "fp32", 6, method="segmented")   # default segments: fits
    assert gpu.pagerank_plan(H)["usable"] == 1
    assert np.abs(r - ref).sum() <= 1e-6
    H.free()


def test_segmented_plan_follows_the_partition(gpu):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=10)
    gpu.graph_partition(H, "degree", degree_threshold=8)
    assert gpu.pagerank_plan(H)["built"] == 0
    pr(gpu, H, "fp32", 10)                         # auto gathers: no plan
    assert gpu.pagerank_plan(H)["built"] == 0
    pr(gpu, H, "fp32", 10, method="segmented")
    a = gpu.pagerank_plan(H)
    gpu.graph_partition(H, "degree", degree_threshold=256)
    assert gpu.pagerank_plan(H)["built"] == 0      # re-partition drops the plan
    r, _ = pr(gpu, H, "fp32", 10, method="segmented")
    b = gpu.pagerank_plan(H)
    assert a["built"] == b["built"] == 1 and a["partials"] != b["partials"]
    assert np.abs(r - ref).sum() <= 1e-6
    # interleaved precisions and methods reuse the plan
    for prec, m in (("fp64", "auto"), ("fp16", "segmented"), ("fp32", "gather"),
                    ("fp32", "segmented")):
        r, _ = pr(gpu, H, prec, 10, method=m)
        assert np.abs(r - ref).sum() <= (1e-12 if prec == "fp64" else TOL[prec])
    assert gpu.pagerank_plan(H)["partials"] == b["partials"]
    H.free()
