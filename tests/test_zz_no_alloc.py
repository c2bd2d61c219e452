"""The allocation-free BFS entry point (bfs_csr_noalloc) against the regular bfs() and the
oracle.

bfs_csr_noalloc exists for callers that cannot allocate device memory when they search
(allocation forbidden in their context, such as host callbacks or driver hooks, or a
device-memory budget fixed at start-up): it keeps all of its scratch in one fixed device
array and allocates nothing. These tests call it through the C ABI on a CSR already in
device memory, twice in a row (the shared scratch array must be cleared between calls), and
check that its levels equal those of the regular entry point and of the oracle bit for bit
and that its parents form a valid BFS tree; then the edge cases of its fixed scratch (a
graph of exactly the vertex limit, a frontier of almost every vertex), calls without
parents, graphs without edges, an isolated source, and the Python wrapper with its input
checks. This file runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def device_csr(torch, g):
    off = torch.from_numpy(np.asarray(g.offsets, dtype=np.int64).copy()).cuda()
    cols = torch.from_numpy(np.asarray(g.cols, dtype=np.uint32).view(np.int32).copy()).cuda()
    return off, cols


def call_noalloc(torch, off, cols, source, levels, parents):
    """Direct C-ABI call with preallocated outputs (the wrapper allocates nothing either)."""
    from paper_1312_3018_gb300 import _lib
    st = _lib.load().bfs_csr_noalloc(off.numel() - 1, cols.numel() if cols is not None else 0,
                                     off.data_ptr(),
                                     cols.data_ptr() if cols is not None else None,
                                     int(source), levels.data_ptr(),
                                     parents.data_ptr() if parents is not None else None,
                                     torch.cuda.current_stream().cuda_stream)
    _lib.check(st, "bfs_csr_noalloc")
    torch.cuda.synchronize()
    lv = levels.cpu().numpy().view(np.uint32)
    return lv, (parents.cpu().numpy().view(np.uint32) if parents is not None else None)


@pytest.mark.parametrize("scale", [12, 16])
def test_noalloc_matches_bfs_twice_in_a_row(gpu, scale):
    import torch
    g = synth.rmat(scale, seed=21)
    off, cols = device_csr(torch, g)
    levels = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parents = torch.empty(g.n, dtype=torch.int32, device="cuda")
    H = gpu.graph_load_csr(g.offsets, g.cols)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    for s in synth.sources(g, 2, seed=22):       # two calls in a row share the scratch
        lv, pa = call_noalloc(torch, off, cols, int(s), levels, parents)
        ref, _, _ = gpu.bfs(H, int(s), out="host")
        assert np.array_equal(lv, ref)
        want, _ = oracle.bfs(g.n, g.offsets, g.cols, int(s), want_parents=False)
        assert np.array_equal(lv, want)
        assert oracle.check_bfs(g.n, g.offsets, g.cols, int(s), lv, pa) == 0
    H.free()


def test_noalloc_at_the_vertex_limit(gpu):
    """n = 2^21 exactly (RMAT scale 21), twice in a row, against the oracle: the bitmap and
    both queues are used up to their last word."""
    import torch
    from paper_1312_3018_gb300 import _lib
    g = synth.rmat(21, seed=23)
    assert g.n == _lib.GRAPH_NOALLOC_MAX_VERTICES
    off, cols = device_csr(torch, g)
    levels = torch.empty(g.n, dtype=torch.int32, device="cuda")
    parents = torch.empty(g.n, dtype=torch.int32, device="cuda")
    for s in synth.sources(g, 2, seed=24):
        lv, pa = call_noalloc(torch, off, cols, int(s), levels, parents)
        want, _ = oracle.bfs(g.n, g.offsets, g.cols, int(s), want_parents=False)
        assert np.array_equal(lv, want)
        assert oracle.check_bfs(g.n, g.offsets, g.cols, int(s), lv, pa) == 0


def test_noalloc_star_at_the_vertex_limit(gpu):
    """A star with 2^21 - 1 leaves searched from a leaf: the third level holds every other
    vertex, the largest frontier the queues can be asked to hold."""
    import torch
    from paper_1312_3018_gb300 import _lib
    n = _lib.GRAPH_NOALLOC_MAX_VERTICES
    off = np.concatenate([[0], np.arange(n - 1, 2 * n - 1, dtype=np.int64)])
    g = synth.Csr(n, off, np.concatenate([np.arange(1, n), np.zeros(n - 1)]).astype(np.uint32))
    off, cols = device_csr(torch, g)
    levels = torch.empty(n, dtype=torch.int32, device="cuda")
    lv, _ = call_noalloc(torch, off, cols, 5, levels, None)   # parents = NULL
    want = np.full(n, 2, np.uint32)
    want[0], want[5] = 1, 0
    assert np.array_equal(lv, want)


def test_noalloc_without_parents_and_without_edges(gpu):
    import torch
    g = synth.rmat(12, seed=25)
    off, cols = device_csr(torch, g)
    levels = torch.empty(g.n, dtype=torch.int32, device="cuda")
    s = int(synth.sources(g, 1, seed=26)[0])
    lv, pa = call_noalloc(torch, off, cols, s, levels, None)
    assert pa is None
    want, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
    assert np.array_equal(lv, want)
    # an isolated source reaches only itself
    iso = int(np.flatnonzero(np.diff(g.offsets) == 0)[0])
    lv, _ = call_noalloc(torch, off, cols, iso, levels, None)
    assert lv[iso] == 0 and np.count_nonzero(lv != oracle.INF) == 1
    # a graph with no edges at all: m = 0 and cols = NULL
    off0 = torch.zeros(6, dtype=torch.int64, device="cuda")
    lv0 = torch.empty(5, dtype=torch.int32, device="cuda")
    out, _ = call_noalloc(torch, off0, None, 3, lv0, None)
    assert out.tolist() == [oracle.INF, oracle.INF, oracle.INF, 0, oracle.INF]


def test_noalloc_python_wrapper_and_its_checks(gpu):
    import torch
    g = synth.rmat(13, seed=27)
    off, cols = device_csr(torch, g)
    s = int(synth.sources(g, 1, seed=28)[0])
    lv, pa = gpu.bfs_csr_noalloc(off, cols, s)
    want, _ = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)
    got = lv.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    assert oracle.check_bfs(g.n, g.offsets, g.cols, s, got, pa.cpu().numpy().view(np.uint32)) == 0
    lv2, pa2 = gpu.bfs_csr_noalloc(off, cols, s, want_parents=False)
    assert pa2 is None and np.array_equal(lv2.cpu().numpy().view(np.uint32), want)
    with pytest.raises(ValueError, match="dtype"):
        gpu.bfs_csr_noalloc(off.to(torch.int32), cols, s)          # 32-bit offsets
    with pytest.raises(ValueError, match="CUDA"):
        gpu.bfs_csr_noalloc(off.cpu(), cols, s)                    # host tensor
    with pytest.raises(ValueError, match="contiguous"):
        gpu.bfs_csr_noalloc(off, torch.stack([cols, cols], 1)[:, 0], s)
    with pytest.raises(ValueError, match="elements"):
        gpu.bfs_csr_noalloc(off, cols, s, torch.empty(g.n - 1, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError, match="dtype"):
        gpu.bfs_csr_noalloc(off, cols, s, torch.empty(g.n, dtype=torch.int64, device="cuda"))


def test_noalloc_rejects_too_many_vertices(gpu):
    import torch
    from paper_1312_3018_gb300 import _lib
    n = _lib.GRAPH_NOALLOC_MAX_VERTICES + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    st = _lib.load().bfs_csr_noalloc(n, 0, off.data_ptr(), None, 0, lv.data_ptr(), None, None)
    assert st == _lib.GRAPH_EINVAL
    assert b"allocation-free limit" in _lib.load().graph_last_error()


def test_noalloc_rejects_invalid_csr(gpu):
    import torch
    from paper_1312_3018_gb300 import _lib
    off = torch.tensor([0, 1, 2, 3], dtype=torch.int64, device="cuda")
    cols = torch.tensor([1, 9, 0], dtype=torch.int32, device="cuda")     # id 9 >= n
    lv = torch.empty(3, dtype=torch.int32, device="cuda")
    st = _lib.load().bfs_csr_noalloc(3, 3, off.data_ptr(), cols.data_ptr(), 0, lv.data_ptr(),
                                     None, None)
    assert st == _lib.GRAPH_EINVAL
    assert b"column id" in _lib.load().graph_last_error()
