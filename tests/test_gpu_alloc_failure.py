"""Allocation failure through the caller's allocator hooks (graph_runtime): an allocator
that returns NULL once it has served K allocations makes the call that needed the next
one return GRAPH_ENOMEM (no other status, no fault). The handle stays usable: the same
call succeeds once the allocator serves again, every result then equals the oracle's, and
graph_free returns every byte. K runs over every allocation point of a load, a partition,
a BFS, an SSSP, an FP32 PageRank, a hybrid FP64 PageRank, a batched BFS and SSSP (their
graph-driven loops), betweenness, hybrid BFS and SSSP, connected components and a round
trip of partition 0's edge arrays through host memory."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_common import rmat_graph

pytestmark = pytest.mark.gpu


class LimitedAllocator:
    """The torch caching allocator behind a counter: `left` allocations are served, then
    NULL is returned (None: unlimited)."""

    def __init__(self, torch, lib, stream):
        self.left = None
        self.count = 0
        self.live = {}
        self.bad_frees = []
        dev = torch.cuda.current_device()

        @lib.ALLOC_FN
        def alloc(nbytes, ctx):
            if self.left is not None:
                if self.left <= 0:
                    return None
                self.left -= 1
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
            except Exception:
                return None
            self.count += 1
            self.live[p] = int(nbytes)
            return p

        @lib.FREE_FN
        def free(ptr, nbytes, ctx):
            # an exception would not cross the C callback boundary: record and check later
            if self.live.pop(ptr, None) != int(nbytes):
                self.bad_frees.append((ptr, int(nbytes)))
            torch.cuda.caching_allocator_delete(ptr)

        self.keep = [alloc, free]
        self.rt = lib.graph_runtime(alloc, free, None, stream)


def test_every_allocation_point_fails_cleanly(gpu):
    import torch
    from paper_1312_3018_gb300 import _lib

    lib = _lib.load()
    g = rmat_graph(10)
    stream = torch.cuda.current_stream().cuda_stream
    A = LimitedAllocator(torch, _lib, stream)
    src = int(synth.sources(g, 1, seed=2)[0])
    ref_lv, _ = oracle.bfs(g.n, g.offsets, g.cols, src)
    ref_d = oracle.sssp(g.n, g.offsets, g.cols, g.weights, src)
    ref_pr, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=10)
    srcs = [int(x) for x in synth.sources(g, 3, seed=5)]
    ref_rows = [oracle.bfs(g.n, g.offsets, g.cols, x)[0] for x in srcs]
    ref_drows = [oracle.sssp(g.n, g.offsets, g.cols, g.weights, x) for x in srcs]
    ref_bc, _ = oracle.bc(g.n, g.offsets, g.cols, srcs[:2])
    ref_cc = oracle.cc(g.n, g.offsets, g.cols)
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.uint32)
    w = np.ascontiguousarray(g.weights, dtype=np.uint32)

    def load():
        out = C.c_void_p(0)
        st = lib.graph_load_csr(g.n, g.m, off.ctypes.data, col.ctypes.data, w.ctypes.data,
                                _lib.GRAPH_MEM_HOST, C.byref(A.rt), C.byref(out))
        if st != _lib.GRAPH_OK:
            assert out.value is None
            raise gpu.GraphError(st, "graph_load_csr")
        return gpu.Graph(out.value, g.n, g.m, stream, A.keep)

    def run_all(H):
        return [
            ("partition", lambda: gpu.graph_partition(H, "degree", degree_threshold=32)),
            ("bfs", lambda: gpu.bfs(H, src, out="host")),
            ("sssp", lambda: gpu.sssp(H, src, out="host")),
            ("pagerank", lambda: gpu.pagerank(H, max_iter=10, precision="fp32", out="host")),
            ("hybrid", lambda: gpu.pagerank_hybrid(H, cpu_threads=2, max_iter=10,
                                                   precision="fp64", out="host")),
            ("bfs_batch", lambda: gpu.bfs_batch(H, srcs, out="host")),
            ("sssp_batch", lambda: gpu.sssp_batch(H, srcs, out="host")),
            ("betweenness", lambda: gpu.betweenness(H, srcs[:2], out="host")),
            ("bfs_hybrid", lambda: gpu.bfs_hybrid(H, src, out="host", cpu_threads=2)),
            ("sssp_hybrid", lambda: gpu.sssp_hybrid(H, src, out="host", cpu_threads=2)),
            ("cc", lambda: gpu.connected_components(H, out="host")),
            ("edges", lambda: (gpu.graph_set_edge_memory(H, "part0", "host"),
                               gpu.graph_set_edge_memory(H, "part0", "device"))),
        ]

    failed = set()  # calls that met a failing allocation somewhere in the sweep

    def attempt(name, fn):
        """Runs fn; on ENOMEM lifts the limit and runs it again. Returns its result."""
        try:
            return fn()
        except gpu.GraphError as e:
            assert e.status == _lib.GRAPH_ENOMEM, str(e)
            failed.add(name)
            A.left = None
            return fn()

    total = None
    K = 0
    while total is None or K <= total:
        A.left, A.count = K, 0
        H = attempt("load", load)
        res = [attempt(name, f) for name, f in run_all(H)]
        lv = res[1][0]
        assert np.array_equal(lv, ref_lv), f"BFS levels differ at K={K}"
        assert np.array_equal(res[2][0], ref_d), f"SSSP distances differ at K={K}"
        assert np.abs(res[3][0] - ref_pr).sum() <= 1e-6, f"PageRank FP32 differs at K={K}"
        assert np.abs(res[4][0] - ref_pr).sum() <= 1e-12, f"hybrid FP64 differs at K={K}"
        for row in range(len(srcs)):
            assert np.array_equal(res[5][0][row], ref_rows[row]), f"bfs_batch at K={K}"
            assert np.array_equal(res[6][0][row], ref_drows[row]), f"sssp_batch at K={K}"
        assert (np.abs(res[7][0] - ref_bc) / np.maximum(1.0, np.abs(ref_bc))).max() <= 1e-9
        assert np.array_equal(res[8][0], ref_lv), f"bfs_hybrid at K={K}"
        assert np.array_equal(res[9][0], ref_d), f"sssp_hybrid at K={K}"
        assert np.array_equal(res[10][0], ref_cc), f"cc at K={K}"
        H.free()
        assert not A.live, f"{len(A.live)} allocations not returned at K={K}"
        assert not A.bad_frees, f"frees of unknown pointers or sizes at K={K}"
        if total is None:
            total = A.count  # allocations of a run that never failed (K = 0 failed first)
        K += 1
    # (calls that reuse a workspace an earlier call made may never meet a failure)
    assert failed >= {"load", "partition", "bfs", "sssp", "pagerank", "hybrid", "bfs_batch",
                      "sssp_batch", "betweenness", "edges"}, failed
