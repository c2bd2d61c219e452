"""The timed CPU baseline (baseline/, OpenMP) against the oracle: it must compute what the
benchmark step computes before its time means anything. BFS levels and SSSP distances are
unique, so they are compared element by element; PageRank (FP32 sums) within the FP32
target L1 <= 1e-6 against the FP64 oracle."""
import numpy as np
import pytest

import baseline
import oracle
import synth


@pytest.fixture(scope="module")
def g():
    g = synth.rmat(14, seed=1)
    synth.weights(g, 64, seed=3)
    return g


def test_omp_bfs_matches_oracle(g):
    for s in synth.sources(g, 4, seed=2):
        lv, levels = baseline.bfs(g.n, g.offsets, g.cols, int(s))
        ref, _ = oracle.bfs(g.n, g.offsets, g.cols, int(s), want_parents=False)
        assert np.array_equal(lv, ref)
        assert levels == int(ref[ref != oracle.INF].max()) + 1


def test_omp_sssp_matches_oracle(g):
    for s in synth.sources(g, 4, seed=2):
        d, rounds = baseline.sssp(g.n, g.offsets, g.cols, g.weights, int(s))
        assert np.array_equal(d, oracle.sssp(g.n, g.offsets, g.cols, g.weights, int(s)))
        assert rounds >= 1


@pytest.mark.parametrize("dangling", [True, False])
def test_omp_pagerank_matches_oracle(g, dangling):
    r, res = baseline.pagerank(g.n, g.offsets, g.cols, 0.85, 20, dangling)
    ref, rres, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=20,
                                   dangling=int(dangling))
    assert np.abs(r - ref).sum() <= 1e-6
    assert abs(res - rres[-1]) <= 1e-6


def test_omp_small_graphs():
    p = synth.path(50)
    lv, levels = baseline.bfs(p.n, p.offsets, p.cols, 0)
    assert lv.tolist() == list(range(50)) and levels == 50
    st = synth.star(10)
    lv, _ = baseline.bfs(st.n, st.offsets, st.cols, 3)
    assert lv[0] == 1 and lv[3] == 0 and np.all(lv[1:][np.arange(1, 11) != 3] == 2)
    c = synth.cycle(64)
    r, _ = baseline.pagerank(c.n, c.offsets, c.cols, 0.85, 7)
    assert np.allclose(r, 1 / 64, rtol=0, atol=1e-9)
    assert baseline.threads() >= 1
