"""Degree-threshold autotuner: picks one of its candidates, leaves the graph partitioned
with it, caches the choice, and results stay exact."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import rmat_graph

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_caches(gpu, tmp_path):
    from paper_1312_3018_gb300 import autotune
    g = rmat_graph(13)
    s = int(synth.sources(g, 1, seed=2)[0])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    cands = (64, 512, 1 << 31)
    cache = str(tmp_path / "tune.json")
    r1 = autotune.autotune_threshold(gpu, H, s, weighted=True, candidates=cands, cache=cache)
    assert r1["T"] in cands and not r1["cached"]
    assert gpu.graph_get_partition_info(H)["threshold"] == r1["T"]
    lv, pa, _ = gpu.bfs(H, s, out="host")
    assert np.array_equal(lv, oracle.bfs(g.n, g.offsets, g.cols, s)[0])
    r2 = autotune.autotune_threshold(gpu, H, s, weighted=True, candidates=cands, cache=cache)
    assert r2["cached"] and r2["T"] == r1["T"]
    r3 = autotune.autotune_threshold(gpu, H, s, weighted=True, candidates=cands, cache=cache,
                                     retune=True)
    assert not r3["cached"] and r3["T"] in cands
    H.free()


def test_autotune_reports_but_never_picks_reported_thresholds(gpu, tmp_path):
    from paper_1312_3018_gb300 import autotune
    g = rmat_graph(12)
    s = int(synth.sources(g, 1, seed=2)[0])
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    cache = str(tmp_path / "tune.json")
    r = autotune.autotune_threshold(gpu, H, s, weighted=True, candidates=(64, 512),
                                    cache=cache, report=(1 << 31,))
    assert r["T"] in (64, 512) and str(1 << 31) in r["reported"]
    assert r["measured_on"]
    r2 = autotune.autotune_threshold(gpu, H, s, weighted=True, candidates=(64, 512),
                                     cache=cache, report=(1 << 31,))
    assert r2["cached"] and r2["measured_on"] == r["measured_on"]
    assert str(1 << 31) in r2["reported"]            # re-timed even from the cache
    assert gpu.graph_get_partition_info(H)["threshold"] == r2["T"]
    H.free()


def test_tune_pagerank_and_bfs_pick_working_parameters(gpu):
    from paper_1312_3018_gb300 import autotune
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    t = autotune.tune_pagerank(gpu, H)
    assert t["best"] is not None and t["best"]["method"] in ("gather", "segmented")
    assert all(v is None or v > 0 for v in t["ms_per_iter"].values())
    r, _ = gpu.pagerank(H, max_iter=20, precision="fp32", out="host", **t["best"])
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=20)
    assert np.abs(r - ref).sum() <= 1e-6
    srcs = synth.sources(g, 3, seed=2)
    b = autotune.tune_bfs(gpu, H, srcs, alphas=(5.0, 15.0), betas=(18.0,))
    assert b["alpha"] in (5.0, 15.0) and b["beta"] == 18.0 and len(b["ms"]) == 2
    for s in srcs:
        lv, pa, _ = gpu.bfs(H, int(s), out="host", alpha=b["alpha"], beta=b["beta"])
        assert np.array_equal(lv, oracle.bfs(g.n, g.offsets, g.cols, int(s))[0])
    H.free()
