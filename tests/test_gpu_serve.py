"""Query server on the GPU: continuous batching of BFS and SSSP queries. Every result is
compared element by element with the oracle (BFS levels and SSSP distances are unique), so
a result is the same alone and in the mix; the tests also check that queries really ran
concurrently (lanes joined while others were in flight, SSSP slots overlapped) and that
the memory budget bounds the slots."""
import time

import numpy as np
import pytest

import oracle
import synth
from gpu_common import PARTITIONS, apply_partition, part_id, rmat_graph

pytestmark = pytest.mark.gpu


def expected(g, kind, s, cache):
    key = (kind, s)
    if key not in cache:
        if kind == "bfs":
            cache[key] = oracle.bfs(g.n, g.offsets, g.cols, s, want_parents=False)[0]
        else:
            cache[key] = oracle.sssp(g.n, g.offsets, g.cols, g.weights, s)
    return cache[key]


def drain(G, srv, count, timeout_s=120.0):
    done = []
    t_end = time.time() + timeout_s
    while len(done) < count:
        assert time.time() < t_end, f"only {len(done)} of {count} queries completed"
        done += srv.poll(cap=256, wait_ms=20)
    return done


def as_u32(G, a):
    return G.as_numpy_u32(a) if not isinstance(a, np.ndarray) else a.view(np.uint32)


def mixed_queries(g, count, seed):
    rng = np.random.default_rng(seed)
    srcs = synth.sources(g, 24, seed=seed)
    kinds = np.where(rng.random(count) < 0.7, "bfs", "sssp")
    picks = rng.integers(0, len(srcs), size=count)
    return [(str(k), int(srcs[p])) for k, p in zip(kinds, picks)]


def run_mix(G, H, g, queries, out="device", gap_s=0.0, **kw):
    import torch
    cache = {}
    outs = []
    with G.Server(H, out=out, **kw) as srv:
        for kind, s in queries:
            buf = (torch.empty(g.n, dtype=torch.int32, device="cuda") if out == "device"
                   else torch.empty(g.n, dtype=torch.int32, pin_memory=True).numpy())
            srv.submit(kind, s, buf)
            outs.append(buf)
            if gap_s:
                time.sleep(gap_s)
        done = drain(G, srv, len(queries))
        info = srv.info()
    assert len(done) == len(queries) == info["completed"]
    for c in done:
        assert c["status"] == 0, c
        assert c["t_submit_ms"] <= c["t_admit_ms"] <= c["t_done_ms"]
        ref = expected(g, c["kind"], c["source"], cache)
        got = as_u32(G, c["out"] if out == "host" else c["out"].cpu().numpy())
        assert np.array_equal(got, ref), f"{c['kind']} from {c['source']} differs"
    return done, info


def test_server_mix_matches_oracle(gpu):
    """A burst of 150 mixed queries (70% BFS, 30% SSSP, repeated sources included)."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    done, info = run_mix(gpu, H, g, mixed_queries(g, 150, 4))
    assert info["max_lanes_busy"] > 1 and info["max_slots_busy"] > 1
    H.free()


def test_server_near_far_sssp_matches_oracle(gpu):
    """SSSP jobs in near-far order (sssp_delta > 0): the same distances as the oracle, in a
    mix with BFS queries."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    done, info = run_mix(gpu, H, g, mixed_queries(g, 80, 9), sssp_delta=16)
    assert any(c["kind"] == "sssp" for c in done)
    H.free()


def test_server_batched_sssp_matches_oracle(gpu):
    """A burst of SSSP-heavy queries with batched SSSP jobs enabled: queries that wait
    together share sssp_batch searches, and every result still equals the oracle's."""
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    qs = [("sssp" if i % 3 else "bfs", s) for i, (_, s) in enumerate(mixed_queries(g, 120, 12))]
    done, info = run_mix(gpu, H, g, qs, sssp_batch=True, max_sssp=2)
    assert info["sssp_batch_slots"] > 0
    assert info["sssp_batched"] > 0, "no query ran on a batched job"
    H.free()


def test_server_batched_sssp_host_outputs_and_partitions(gpu):
    g = rmat_graph(13, seed=5, wmax=255, wseed=7)
    for p in (PARTITIONS[0], PARTITIONS[4], PARTITIONS[6]):
        H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
        apply_partition(gpu, H, g, p)
        qs = [("sssp", s) for _, s in mixed_queries(g, 40, 13)]
        done, info = run_mix(gpu, H, g, qs, out="host", sssp_batch=True, max_sssp=1)
        assert info["sssp_batched"] > 0
        H.free()


def test_server_lanes_join_while_others_run(gpu):
    """Staggered arrivals: some BFS query is admitted while another is still in flight, and
    both results are exact."""
    g = rmat_graph(15)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=2048)
    qs = [("bfs", s) for _, s in mixed_queries(g, 60, 6)]
    done, info = run_mix(gpu, H, g, qs, gap_s=0.0003)
    bfs = sorted(done, key=lambda c: c["t_admit_ms"])
    overlapped = any(a["t_admit_ms"] < b["t_admit_ms"] < a["t_done_ms"]
                     for a, b in zip(bfs, bfs[1:]))
    assert overlapped, "no BFS query joined while another was running"
    H.free()


def test_server_same_result_alone_and_in_the_mix(gpu):
    g = rmat_graph(14)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=256)
    s = int(synth.sources(g, 1, seed=21)[0])
    alone_b, _ = run_mix(gpu, H, g, [("bfs", s)])
    alone_s, _ = run_mix(gpu, H, g, [("sssp", s)])
    mix = mixed_queries(g, 80, 9)
    mix[17] = ("bfs", s)
    mix[42] = ("sssp", s)
    done, _ = run_mix(gpu, H, g, mix)
    ab = alone_b[0]["out"].cpu().numpy()
    as_ = alone_s[0]["out"].cpu().numpy()
    for c in done:
        if c["source"] == s:
            ref = ab if c["kind"] == "bfs" else as_
            assert np.array_equal(c["out"].cpu().numpy(), ref)
    H.free()


def test_server_admission_by_memory(gpu):
    """A budget for the lanes and two SSSP jobs gives two slots; ten SSSP queries then never
    run more than two at a time, and all complete exactly."""
    g = rmat_graph(13)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=64)
    with gpu.Server(H, bfs_lanes=8) as probe:
        inf = probe.info()
    budget = inf["bytes_lanes"] + 2 * inf["bytes_per_sssp"] + 1024
    qs = [("sssp", s) for _, s in mixed_queries(g, 10, 3)] + [("bfs", 0)]
    done, info = run_mix(gpu, H, g, qs, bfs_lanes=8, mem_budget=budget)
    assert info["sssp_slots"] == 2 and info["max_slots_busy"] <= 2
    assert info["bfs_lanes"] == 8
    with pytest.raises(gpu.GraphError, match="out of memory"):
        gpu.Server(H, mem_budget=1024)
    H.free()


@pytest.mark.parametrize("p", [PARTITIONS[0], PARTITIONS[3], PARTITIONS[6]], ids=part_id)
def test_server_partitions_and_host_outputs(gpu, p):
    g = rmat_graph(12)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    apply_partition(gpu, H, g, p)
    run_mix(gpu, H, g, mixed_queries(g, 40, 11), out="host")
    H.free()


def test_server_rejects_bad_requests(gpu):
    g = rmat_graph(11)
    H = gpu.graph_load_csr(g.offsets, g.cols)   # no weights: no SSSP slots
    with pytest.raises(gpu.GraphError, match="out of order"):
        gpu.Server(H)
    gpu.graph_partition(H, "none")
    import torch
    buf = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with gpu.Server(H) as srv:
        assert srv.info()["sssp_slots"] == 0
        with pytest.raises(gpu.GraphError, match="invalid argument"):
            srv.submit("sssp", 0, buf)
        with pytest.raises(gpu.GraphError, match="invalid argument"):
            srv.submit("bfs", g.n, buf)
        with pytest.raises(ValueError):
            srv.submit("bfs", 0, np.empty(g.n, np.uint32))
        srv.submit("bfs", 3, buf)
        (c,) = drain(gpu, srv, 1)
        ref = oracle.bfs(g.n, g.offsets, g.cols, 3, want_parents=False)[0]
        assert np.array_equal(buf.cpu().numpy().view(np.uint32), ref)
    H.free()


def test_server_rmat23_serving_workload_sampled_parity(gpu):
    """The serving workload the benchmark measures: RMAT scale 23 (8.4M vertices, ~260M
    edge entries, weights 1..64), degree threshold 2048, near-far SSSP width 16, batched
    SSSP jobs on, 300 queries (70% BFS, 30% SSSP) submitted as one burst so that BFS lanes
    and SSSP slots and batches all fill. Every query must complete without error; a sample
    of the completed queries (four BFS, three SSSP, different sources) is compared with the
    oracle element by element."""
    import torch
    g = rmat_graph(23)
    H = gpu.graph_load_csr(g.offsets, g.cols, g.weights)
    gpu.graph_partition(H, "degree", degree_threshold=2048)
    srcs = synth.sources(g, 4096, seed=5)
    rng = np.random.default_rng(11)
    kinds = np.where(rng.random(300) < 0.7, "bfs", "sssp")
    picks = srcs[rng.integers(len(srcs), size=300)]
    with gpu.Server(H, out="device", sssp_delta=16, sssp_batch=True) as srv:
        for k, s in zip(kinds, picks):
            srv.submit(str(k), int(s), torch.empty(g.n, dtype=torch.int32, device="cuda"))
        done = drain(gpu, srv, len(kinds), timeout_s=300.0)
        info = srv.info()
    assert all(c["status"] == 0 for c in done)
    assert info["max_lanes_busy"] > 1 and info["sssp_batched"] > 0
    sample, seen = [], set()
    for kind, want in (("bfs", 4), ("sssp", 3)):
        for c in done:
            if c["kind"] == kind and c["source"] not in seen and want > 0:
                sample.append(c)
                seen.add(c["source"])
                want -= 1
    assert len(sample) == 7
    cache = {}
    for c in sample:
        got = as_u32(gpu, c["out"].cpu().numpy())
        ref = expected(g, c["kind"], c["source"], cache)
        assert np.array_equal(got, ref), f"{c['kind']} from {c['source']} differs"
    H.free()
