"""GPU partition (device relabel, local-first CSR, outbox/inbox) equals the oracle's
partition bit for bit (Section 4.3.1-4.3.2, Figure 6; Section 6.2-6.3.1)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph, star_plus

pytestmark = pytest.mark.gpu


def compare(G, H, g, asg):
    ref = oracle.partition(g.n, g.offsets, g.cols, asg, g.weights)
    for p in (0, 1):
        got = G.graph_export_partition(H, p, weights=g.weights is not None)
        exp = ref["parts"][p]
        assert got["nv"] == exp["nv"]
        assert got["ne"] == exp["ne"]
        assert np.array_equal(got["l2g"], exp["l2g"]), f"l2g differs in partition {p}"
        assert np.array_equal(got["off"], exp["off"]), f"offsets differ in partition {p}"
        assert np.array_equal(got["E"], exp["E"]), f"E differs in partition {p}"
        if g.weights is not None:
            assert np.array_equal(got["W"], exp["W"]), f"W differs in partition {p}"
        assert np.array_equal(got["outbox"], exp["outbox"]), f"outbox differs in {p}"
        assert np.array_equal(got["cls_end"], exp["cls_end"]), f"class ranges differ in {p}"
        assert np.array_equal(got["g2l"], ref["g2l"])


@pytest.mark.parametrize("p", PARTITIONS, ids=part_id)
@pytest.mark.parametrize("scale", [10, 14])
def test_partition_matches_oracle_rmat(gpu, scale, p):
    g = rmat_graph(scale)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    info, asg = apply_partition(gpu, H, g, p)
    compare(gpu, H, g, asg)
    H.free()


def test_partition_with_multi_chunk_hub(gpu):
    g = star_plus(20000)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    for T in (0, 3, 2048, 1 << 30):
        gpu.graph_partition(H, "degree", degree_threshold=T)
        compare(gpu, H, g, oracle.degree_assignment(g.offsets, T))
    H.free()


@pytest.mark.parametrize("share", [0.05, 0.25, 0.5, 0.8, 1.0])
def test_edge_share_threshold_matches_oracle(gpu, share):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    info = gpu.graph_partition(H, "degree", edge_share=share)
    assert info["threshold"] == oracle.edge_share_threshold(g.offsets, share)
    H.free()


def test_partition_space_formula(gpu):
    """bytes_graph follows Section 4.3.3: eid|V_p| + vid|E_p| + w|E_p| + vid(|V_i|+|V_o|)."""
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    info = gpu.graph_partition(H, "degree", degree_threshold=64)
    ref = oracle.partition(g.n, g.offsets, g.cols, oracle.degree_assignment(g.offsets, 64))
    exp = 0
    for p in (0, 1):
        P, Q = ref["parts"][p], ref["parts"][1 - p]
        exp += 8 * (P["nv"] + 1) + 4 * P["ne"] + 4 * P["ne"] + 4 * (len(P["outbox"]) +
                                                                   len(Q["outbox"]))
    assert info["bytes_graph"] == exp
    H.free()


def test_partition_rejects_bad_assignment(gpu):
    g = synth.path(10)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="invalid argument"):
        gpu.graph_partition(H, "explicit", assignment=np.full(10, 2, np.uint8))
    with pytest.raises(gpu.GraphError):
        gpu.graph_partition(H, "degree", edge_share=1.5)
    H.free()


def test_load_rejects_invalid_csr(gpu):
    off = np.array([0, 2, 1, 3], np.int64)          # decreasing
    cols = np.array([1, 2, 0], np.uint32)
    with pytest.raises(gpu.GraphError, match="flags 0x2:"):
        gpu.graph_load_csr(off, cols)
    off = np.array([0, 1, 2, 3], np.int64)
    cols = np.array([1, 7, 0], np.uint32)            # id >= n
    with pytest.raises(gpu.GraphError, match="flags 0x8:"):
        gpu.graph_load_csr(off, cols)
    with pytest.raises(gpu.GraphError, match="flags 0x10:"):
        gpu.graph_load_csr(off, np.array([1, 2, 0], np.uint32), np.array([1, 0, 1], np.uint32))


def test_algorithms_before_partition_are_rejected(gpu):
    g = synth.path(5)
    H = gpu.graph_load_csr(g.offsets, g.cols)
    with pytest.raises(gpu.GraphError, match="out of order"):
        gpu.bfs(H, 0)
    H.free()


def test_device_inputs_and_cuda_allocator(gpu):
    import torch
    g = rmat_graph(10)
    off = torch.from_numpy(np.asarray(g.offsets, dtype=np.int64).copy()).cuda()
    cols = torch.from_numpy(np.asarray(g.cols).view(np.int32).copy()).cuda()
    H = gpu.graph_load_csr(off, cols, allocator="cuda")
    gpu.graph_partition(H, "degree", degree_threshold=16)
    compare_g = synth.Csr(g.n, g.offsets, g.cols)
    compare(gpu, H, compare_g, oracle.degree_assignment(g.offsets, 16))
    H.free()
