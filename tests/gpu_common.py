"""Helpers shared by the GPU parity tests (inputs come from `synth`, expected values from
`oracle`; nothing here computes a graph algorithm)."""
import functools

import numpy as np

import oracle
import synth

# Partition settings every algorithm must be independent of (Section 4.3: the result of a
# BSP run does not depend on how vertices are split): one partition, degree splits at
# several thresholds (every vertex a hub, a low threshold, the CTA-per-hub threshold), the
# HIGH edge-share rule, and a seeded random split (RAND).
PARTITIONS = [
    ("none", {}),
    ("degree", dict(degree_threshold=0)),
    ("degree", dict(degree_threshold=4)),
    ("degree", dict(degree_threshold=64)),
    ("degree", dict(degree_threshold=2048)),
    ("degree", dict(edge_share=0.5)),
    ("explicit", dict(share=0.3, seed=5)),
]


def part_id(p):
    name, kw = p
    return name + "".join(f"-{k}{v}" for k, v in kw.items())


def apply_partition(G, H, g, p):
    name, kw = p
    if name == "explicit":
        asg = synth.random_assignment(g.n, kw["share"], kw["seed"])
        return G.graph_partition(H, "explicit", assignment=asg), asg
    info = G.graph_partition(H, name, **kw)
    if name == "none":
        asg = np.ones(g.n, np.uint8)
    else:
        T = info["threshold"]
        asg = oracle.degree_assignment(g.offsets, T)
    return info, asg


@functools.lru_cache(maxsize=None)
def rmat_graph(scale, seed=1, wmax=64, wseed=3):
    g = synth.rmat(scale, seed=seed)
    synth.weights(g, wmax, seed=wseed)
    return g


def star_plus(k, extra_seed=0):
    """A star with k leaves whose leaves also form a sparse random graph, plus isolated
    vertices: one very high-degree hub (several hub chunks) next to low-degree vertices."""
    rng = np.random.default_rng(extra_seed)
    n = k + 1 + 16
    edges = [(0, i) for i in range(1, k + 1)]
    a = rng.integers(1, k + 1, size=k)
    b = rng.integers(1, k + 1, size=k)
    edges += list(zip(a.tolist(), b.tolist()))
    g = synth.from_edges(n, edges)
    synth.weights(g, 64, seed=extra_seed + 1)
    return g
