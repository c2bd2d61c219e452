"""The allocation-free BFS entry point (bfs_csr_noalloc) against the regular bfs().

bfs_csr_noalloc exists for callers that cannot allocate device memory when they search
(allocation forbidden in their context, or a device-memory budget fixed at start-up): it
keeps all of its scratch in one fixed device array and allocates nothing. These tests call
it through the C ABI on a CSR already in device memory, twice in a row (the shared scratch
array must be cleared between calls), and check that its levels equal those of the regular
entry point bit for bit and that its parents form a valid BFS tree. This file runs last so
that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def device_csr(torch, g):
    off = torch.from_numpy(np.asarray(g.offsets, dtype=np.int64).copy()).cuda()
    cols = torch.from_numpy(np.asarray(g.cols, dtype=np.uint32).view(np.int32).copy()).cuda()
    return off, cols


def call_noalloc(G, torch, off, cols, source, levels, parents):
    """Direct C-ABI call with preallocated outputs (the wrapper allocates nothing either)."""
    from paper_1312_3018_gb300 import _lib
    st = _lib.load().bfs_csr_noalloc(off.numel() - 1, cols.numel(), off.data_ptr(),
                                     cols.data_ptr(), int(source), levels.data_ptr(),
                                     parents.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    _lib.check(st, "bfs_csr_noalloc")
    torch.cuda.synchronize()
    return levels.cpu().numpy().view(np.uint32), parents.cpu().numpy().view(np.uint32)


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
        lv, pa = call_noalloc(gpu, torch, off, cols, int(s), levels, parents)
        ref, _, _ = gpu.bfs(H, int(s), out="host")
        assert np.array_equal(lv, ref)
        assert oracle.check_bfs(g.n, g.offsets, g.cols, int(s), lv, pa) == 0
    H.free()


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
