"""Many-graph PageRank on the GPU: every component of a disjoint union against the FP64
oracle run on that graph alone (Section 7.1, Figure 14 per component; the union only shares
the supersteps and their CUDA graph).

Tolerances per component (L1 over the component's ranks, which sum to 1) are those of the
single-graph tests: FP64 1e-12, FP32 1e-6, FP16 1e-3. The last-iteration residual of a
component is a sum of |r_K - r_{K-1}|, so it may differ from the oracle's by the L1 error
of both iterates: within 2 x the tolerance."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, star_plus

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-6, "fp16": 1e-3}


def family():
    """Uneven components: RMAT graphs of several scales and edge factors, closed-form
    shapes, a multi-chunk hub, isolated vertices and an empty component."""
    gs = synth.rmat_family(12, scales=(5, 12), edge_factors=(4, 32), seed=3)
    gs += [synth.cycle(7), synth.star(40), synth.complete(6), synth.path(1),
           synth.from_edges(5, [(0, 1)]), star_plus(3000, extra_seed=2),
           synth.from_edges(0, []), synth.grid(9, 4)]
    order = np.random.default_rng(5).permutation(len(gs))
    return [gs[i] for i in order]


_FAM = {}


def union():
    if "u" not in _FAM:
        gs = family()
        u, vb = synth.disjoint_union(gs)
        _FAM["u"] = (gs, u, vb)
    return _FAM["u"]


def check_multi(G, H, gs, vb, prec, K, dangling=True, out="host", damping=0.85):
    r, res, st = G.pagerank_multi(H, vb, max_iter=K, precision=prec, dangling=dangling,
                                  out=out, damping=damping)
    r = r.cpu().numpy() if out == "device" else r
    for i, g in enumerate(gs):
        if g.n == 0:
            continue
        ref, rres, _ = oracle.pagerank(g.n, g.offsets, g.cols, damping, max_iter=K,
                                       dangling=int(dangling))
        seg = r[vb[i]:vb[i + 1]]
        l1 = np.abs(seg - ref).sum()
        assert l1 <= TOL[prec], f"component {i} (n={g.n}) {prec} L1 {l1:.3e}"
        assert abs(res[i] - rres[-1]) <= 2 * TOL[prec], f"component {i} residual"
    assert st["supersteps"] == K
    return r, res, st


@pytest.mark.parametrize("p", [PARTITIONS[0], PARTITIONS[2], PARTITIONS[3], PARTITIONS[6]],
                         ids=part_id)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_multi_components_match_oracle(gpu, p, prec):
    gs, u, vb = union()
    H = gpu.graph_load_csr(u.offsets, u.cols)
    apply_partition(gpu, H, u, p)
    check_multi(gpu, H, gs, vb, prec, 30, out={"fp64": "host", "fp32": "device", "fp16": "host"}[prec])
    H.free()


@pytest.mark.parametrize("dangling", [True, False])
def test_multi_dangling_modes(gpu, dangling):
    gs, u, vb = union()
    H = gpu.graph_load_csr(u.offsets, u.cols)
    gpu.graph_partition(H, "degree", degree_threshold=16)
    check_multi(gpu, H, gs, vb, "fp64", 15, dangling=dangling)
    H.free()


def test_multi_one_component_is_plain_pagerank(gpu):
    g = synth.rmat(12, seed=4)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    check_multi(gpu, H, [g], np.array([0, g.n], np.uint32), "fp64", 20)
    H.free()


def test_multi_replay_and_recapture(gpu):
    """A second call with the same layout and count replays the captured graph (same
    result, bit for bit); a new count or a new damping recaptures, and going back to the
    first settings gives the first result again."""
    gs, u, vb = union()
    H = gpu.graph_load_csr(u.offsets, u.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    a, ra, _ = check_multi(gpu, H, gs, vb, "fp32", 30)
    b, rb, _ = check_multi(gpu, H, gs, vb, "fp32", 30)
    assert np.array_equal(a, b) and np.array_equal(ra, rb)
    check_multi(gpu, H, gs, vb, "fp32", 7)
    check_multi(gpu, H, gs, vb, "fp32", 7, damping=0.5)
    # plain pagerank on the same handle still ranks the whole union as one graph
    ref, _, _ = oracle.pagerank(u.n, u.offsets, u.cols, 0.85, max_iter=5)
    r, _ = gpu.pagerank(H, max_iter=5, precision="fp64", out="host")
    assert np.abs(r - ref).sum() <= 1e-12
    check_multi(gpu, H, gs, vb, "fp32", 7)
    c, rc, _ = check_multi(gpu, H, gs, vb, "fp32", 30)
    assert np.array_equal(a, c) and np.array_equal(ra, rc)
    H.free()


def test_multi_rejects_bad_layouts(gpu):
    g = synth.path(10)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="out of order"):
        gpu.pagerank_multi(H, [0, 10])
    gpu.graph_partition(H, "none")
    for bad in ([0, 5, 10], [1, 10], [0, 9], [0, 6, 4, 10]):
        with pytest.raises(gpu.GraphError, match="invalid argument"):
            gpu.pagerank_multi(H, bad)
    r, res, _ = gpu.pagerank_multi(H, [0, 0, 10, 10], out="host", max_iter=12,
                                   precision="fp64")
    ref, rres, _ = oracle.pagerank(10, g.offsets, g.cols, 0.85, max_iter=12)
    assert np.abs(r - ref).sum() <= 1e-12 and res[0] == 0 and res[2] == 0
    assert abs(res[1] - rres[-1]) <= 1e-12
    H.free()
