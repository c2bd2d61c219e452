"""The committed autotuner cache that the benchmark reads (no GPU needed)."""
import json
import os


def test_committed_threshold_cache_is_well_formed():
    """The benchmark's autotuner cache: each entry names one of the split candidates and
    holds a step-time estimate for every candidate of its signature."""
    from paper_1312_3018_gb300 import autotune
    path = os.path.join(os.path.dirname(autotune.__file__), "tuned_thresholds.json")
    table = json.load(open(path))
    assert table
    for key, entry in table.items():
        sig = json.loads(key)
        cands = [p[0] for p in sig["parts"]]
        assert entry["T"] in cands and set(cands) <= set(autotune.SPLIT_CANDIDATES)
        assert sorted(int(t) for t in entry["ms"]) == sorted(cands)
        assert min(entry["ms"], key=entry["ms"].get) == str(entry["T"])
