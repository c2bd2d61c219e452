"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of
oracle.c (on the CPU), builds it, swaps it in, and requires at least one pin of
test_oracle_pins.py to fail. A pin set that let one of these through would not be
strong enough to trust the oracle."""
import ctypes
import os
import subprocess
import sys

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text to replace, replacement, pins that exercise the function)
BFS_PINS = [lambda: pins.test_bfs_path_levels_are_distance_along_path(17, 8),
            lambda: pins.test_bfs_grid_levels_are_manhattan(7, 5, 17),
            lambda: pins.test_bfs_star_from_centre_and_leaf(),
            lambda: pins.test_bfs_brute_force_floyd_warshall(1)]
SSSP_PINS = [lambda: pins.test_sssp_weighted_path_is_prefix_sum(),
             lambda: pins.test_sssp_uniform_weight_is_weight_times_hops(7),
             lambda: pins.test_sssp_brute_force_floyd_warshall(2),
             lambda: pins.test_sssp_overflow_is_reported()]
PR_PINS = [lambda: pins.test_pagerank_cycle_is_uniform_every_iteration(10),
           lambda: pins.test_pagerank_star_closed_form(3),
           lambda: pins.test_pagerank_iterates_match_dense_matrix_iteration(0, 1),
           lambda: pins.test_pagerank_iterates_match_dense_matrix_iteration(2, 0),
           lambda: pins.test_pagerank_converges_to_dense_solve(10, 1),
           lambda: pins.test_pagerank_path3_golden()]
PART_PINS = [lambda: pins.test_partition_is_an_exact_relabelling("deg16"),
             lambda: pins.test_partition_is_an_exact_relabelling("random")]
CHECK_PINS = [lambda: pins.test_bfs_validator_rejects_planted_mistakes(),
              lambda: pins.test_bfs_validator_rejects_level_jump_on_a_non_tree_edge(),
              lambda: pins.test_sssp_certificate_rejects_planted_mistakes()]
BC_PINS = [lambda: pins.test_bc_path_closed_form(6),
           lambda: pins.test_bc_star_closed_form(9),
           lambda: pins.test_bc_matches_pair_dependency_definition(0),
           lambda: pins.test_bc_sum_is_total_interior_length()]
CC_PINS = [lambda: pins.test_cc_closed_forms(),
           lambda: pins.test_cc_matches_scipy(12, 2)]

MUTANTS = [
    ("bfs level +2", "level[u] = level[v] + 1;", "level[u] = level[v] + 2;", BFS_PINS),
    ("bfs parent self", "if (parent) parent[u] = v;", "if (parent) parent[u] = u;", BFS_PINS),
    ("bfs source level 1", "level[source] = 0;", "level[source] = 1;", BFS_PINS),
    ("sssp ignores weights", "uint64_t nd = dv + (uint64_t)w[e];", "uint64_t nd = dv + 1;",
     SSSP_PINS),
    ("sssp heap order", "if (h->key[h->heap[p]] <= h->key[h->heap[i]]) break;",
     "if (h->key[h->heap[p]] >= h->key[h->heap[i]]) break;", SSSP_PINS),
    ("sssp no overflow report", "rc = ORC_ERANGE;", "rc = ORC_OK;", SSSP_PINS),
    ("pr no degree division", "x[u] = r[u] / (double)deg;", "x[u] = r[u];", PR_PINS),
    ("pr dangling dropped", "if (dangling_mode == 1) D += r[u];", "if (dangling_mode == 2) D += r[u];",
     PR_PINS),
    ("pr teleport not divided", "rn[v] = (1.0 - d) / (double)n + d * (s + D / (double)n);",
     "rn[v] = (1.0 - d) + d * (s + D / (double)n);", PR_PINS),
    ("pr dangling not divided", "rn[v] = (1.0 - d) / (double)n + d * (s + D / (double)n);",
     "rn[v] = (1.0 - d) / (double)n + d * (s + D);", PR_PINS),
    ("pr damping misplaced", "rn[v] = (1.0 - d) / (double)n + d * (s + D / (double)n);",
     "rn[v] = (1.0 - d) / (double)n + d * s + D / (double)n;", PR_PINS),
    ("pr initial rank", "for (uint32_t v = 0; v < n; ++v) r[v] = 1.0 / (double)n;",
     "for (uint32_t v = 0; v < n; ++v) r[v] = 1.0;", PR_PINS),
    ("partition remote first", "if (assign[u] == p) {\n          pE[p][pos] = g2l[u] & 0x7FFFFFFFu;",
     "if (assign[u] != p) {\n          pE[p][pos] = g2l[u] & 0x7FFFFFFFu;", PART_PINS),
    ("partition outbox index +1", "index[ql] = k;", "index[ql] = k + 1;", PART_PINS),
    ("partition class ascending", "for (c = ORC_NCLASS - 2; c >= 0; --c) {\n      next[p][c] = run;",
     "for (c = 0; c <= ORC_NCLASS - 2; ++c) {\n      next[p][c] = run;", PART_PINS),
    ("bfs validator loose", "if (diff > 1 || diff < -1) return 3;", "if (diff > 2 || diff < -2) return 3;",
     CHECK_PINS),
    ("bfs validator skips parent edge", "if (!has_edge(off, col, v, p)) return 4;", "",
     CHECK_PINS),
    ("sssp certificate skips tightness", "if (!tight) return 3;", "", CHECK_PINS),
    ("bc drops the 1 +", "* (1.0 + delta[w]);", "* delta[w];", BC_PINS),
    ("bc scores the source", "if (v != s) bc[v] += delta[v];", "bc[v] += delta[v];", BC_PINS),
    ("bc copies sigma", "if (dist[w] == dist[v] + 1) sigma[w] += sigma[v];",
     "if (dist[w] == dist[v] + 1) sigma[w] = sigma[v];", BC_PINS),
    ("bc ratio inverted", "delta[v] += sigma[v] / sigma[w]", "delta[v] += sigma[w] / sigma[v]",
     BC_PINS),
    ("cc labels by largest id", "for (uint32_t r = 0; r < n; ++r) {\n    if (label[r] != ORC_INF)",
     "for (uint32_t r = n; r-- > 0;) {\n    if (label[r] != ORC_INF)", CC_PINS),
]


@pytest.fixture(scope="module")
def source_text():
    return open(SRC).read()


def run_checks(so_path, mutant_index):
    """Run one mutant's pins; returns how many of them failed. Runs in a child process so
    that a mutant that crashes (for instance by writing out of bounds) cannot take the
    test session down; a crash counts as caught."""
    oracle._lib = oracle._configure(ctypes.CDLL(so_path))
    caught = 0
    for check in MUTANTS[mutant_index][3]:
        try:
            check()
        except BaseException as e:  # noqa: B902 - pytest.fail raises a BaseException
            if isinstance(e, KeyboardInterrupt):
                raise
            caught += 1
    return caught


@pytest.mark.parametrize("idx", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, source_text, idx):
    name, old, new, _ = MUTANTS[idx]
    assert old in source_text, f"mutation anchor not found for {name}"
    mutant = tmp_path / "oracle_mutant.c"
    mutant.write_text(source_text.replace(old, new, 1))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(mutant), "-o",
                           str(so), "-lm"])
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_oracle_mutations as t; "
            "print('CAUGHT', t.run_checks(%r, %d))" % (tests_dir, os.path.dirname(tests_dir),
                                                       str(so), idx))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=300)
    if r.returncode != 0:
        return  # the mutant crashed under its pins: caught
    caught = int(r.stdout.strip().split()[-1])
    assert caught > 0, f"no pin caught the planted mistake '{name}'"
