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
