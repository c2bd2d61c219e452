"""The benchmark's host-side contract, checked without a GPU: the reference arm (the CPU
oracle) prints one JSON line with the keys the GPU arm's line carries, only rank 0 prints
it under a multi-rank launch, and the GPU arm fails loudly when no GPU is present."""
import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--scale", "11", "--steps", "2", "--warmup", "1"]


def run_bench(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=timeout)


def json_lines(out):
    return [json.loads(s) for s in out.splitlines() if s.startswith("{")]


def test_reference_arm_line():
    r = run_bench(["--impl", "reference"] + SMALL)
    assert r.returncode == 0, r.stderr
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["n"] == 2048 and d["config"]["m"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_only_rank_zero_prints():
    r = run_bench(["--impl", "reference", "--gpus", "2"] + SMALL,
                  env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert json_lines(r.stdout) == []


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_gpu_arm_fails_loudly_without_gpu():
    r = run_bench(SMALL + ["--no-serve", "--no-batch", "--no-cpu-baseline"])
    assert r.returncode != 0
    assert json_lines(r.stdout) == []


def _bench_module():
    import importlib
    import sys
    sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_cpu_baseline_leg_returns_the_oracle_ranks_for_the_precision_report():
    """The oracle runs only in the CPU-baseline leg: that leg returns the FP64 ranks after
    its PageRank iterations, and the precision report compares against exactly those."""
    import numpy as np
    import oracle
    import synth
    bench = _bench_module()
    g = synth.rmat(10, seed=1)
    synth.weights(g, 255, seed=3)
    cpu, ranks = bench.cpu_baseline(g, int(synth.sources(g, 1, seed=2)[0]), 25.0, pr_iters=3)
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0
    assert "3 FP64 PageRank iterations" in cpu["sample"]
    ref, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=3)
    assert np.array_equal(ranks, ref)

    class FakeLib:
        """Stands in for the GPU library: returns the oracle's ranks rounded to the
        requested precision, so the report's arithmetic can be checked on the host."""
        def pagerank(self, H, max_iter, precision, out):
            r, _, _ = oracle.pagerank(g.n, g.offsets, g.cols, 0.85, max_iter=max_iter)
            dt = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16}[precision]
            return r.astype(dt).astype(np.float64), {}

    rep = bench.precision_report(FakeLib(), None, g, ranks, iters_oracle=3, iters_step=5)
    assert list(rep) == ["vs_oracle", "vs_gpu_fp64", "target"]
    assert rep["vs_oracle"]["fp64"]["l1"] == 0.0
    l1_32 = float(np.abs(ref.astype(np.float32).astype(np.float64) - ref).sum())
    assert rep["vs_oracle"]["fp32"]["l1"] == l1_32
    assert rep["vs_oracle"]["fp16"]["l1"] > rep["vs_oracle"]["fp32"]["l1"]
    rep = bench.precision_report(FakeLib(), None, g, None, iters_step=5)
    assert "vs_oracle" not in rep and rep["vs_gpu_fp64"]["iterations"] == 5


def test_hybrid_report_fields():
    """The hybrid object: one point per host edge share, with the per-processor times of
    the library's info turned into per-iteration figures."""
    bench = _bench_module()

    class FakeTensor:
        def __init__(self, v):
            self.v = v

        def __sub__(self, o):
            return FakeTensor(self.v - o.v)

        def abs(self):
            return FakeTensor(abs(self.v))

        def sum(self):
            return self.v

        def __float__(self):
            return float(self.v)

    class FakeTorch:
        float64 = "f64"

        class cuda:
            @staticmethod
            def synchronize():
                pass

        @staticmethod
        def empty(n, dtype, device):
            return FakeTensor(0.0)

    class FakeLib:
        def graph_partition(self, H, strategy, edge_share):
            return {"threshold": int(1000 * (1 - edge_share))}

        def pagerank(self, H, max_iter, precision, ranks, out):
            ranks.v = 1.0
            return ranks, {}

        def pagerank_hybrid(self, H, max_iter, precision, ranks, out, timing=False):
            ranks.v = 1.0 + 1e-9
            info = {"cpu_vertices": 10, "cpu_edges": 250, "ms_cpu_compute": 5.0 * max_iter,
                    "ms_gpu_compute": 1.0 * max_iter, "ms_exchange": 0.5 * max_iter}
            return ranks, {"hybrid": info, "messages": 70 * max_iter, "supersteps": max_iter}

    class FakeGraph:
        n = 100

    rep = bench.hybrid_report(FakeLib(), FakeGraph(), 1000, FakeTorch, shares=(0.05, 0.25),
                              iters=5)
    assert rep["iters"] == 5 and len(rep["points"]) == 2
    p = rep["points"][1]
    assert p["edge_share"] == 0.25 and p["T"] == 750
    assert p["cpu_edge_share"] == 0.25
    assert p["cpu_compute_ms_per_iter"] == 5.0 and p["gpu_compute_ms_per_iter"] == 1.0
    assert p["exchange_ms_per_iter"] == 0.5 and p["messages_per_iter"] == 70
    assert abs(p["l1_vs_gpu_only"] - 1e-9) < 1e-15
    assert p["hybrid_ms_per_iter"] >= 0 and p["gpu_only_ms_per_iter"] >= 0


def test_host_edges_report_fields_and_restores_placement():
    """The host-edges object: device, partition-0-on-host and all-on-host timings, the link
    rate of the PageRank iterations, and the placement moved back to the device."""
    bench = _bench_module()
    calls = []

    class FakeTorch:
        class cuda:
            @staticmethod
            def synchronize():
                pass

    class FakeLib:
        def graph_get_partition_info(self, H):
            return {"ne": [3000, 1000]}

        def graph_set_edge_memory(self, H, which, mem):
            calls.append((which, mem))

        def bfs(self, H, s, want_parents):
            return None

        def sssp(self, H, s, delta):
            return None

        def pagerank(self, H, max_iter, precision):
            return None

    rep = bench.host_edges_report(FakeLib(), object(), FakeTorch, 5, pr_iters=5)
    for k in ("device", "part0_host", "all_host"):
        assert set(rep[k]) == {"bfs_ms", "sssp_ms", "pagerank_ms_per_iter"}
    assert set(rep["pagerank_link_gbs"]) == {"part0_host", "all_host"}
    assert calls[0] == ("part0", "host")
    assert calls[-1] == (["part0", "part1", "input"], "device")
