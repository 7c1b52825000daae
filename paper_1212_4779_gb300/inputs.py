"""Seeded synthetic graph generators (COO arc lists) shared by the tests,
the oracle checks and the benchmark.

This module only draws random graphs.  It holds none of the method's
arithmetic: no live-edge hash, no thresholds, no canonicalisation beyond
what a generator needs to hit an exact arc count.  Every generator returns
``(n, src, dst)`` with ``src``/``dst`` int32 numpy arrays of equal length;
both the CUDA library and the oracle canonicalise that list on their own.

The graph families stand in for the shapes of the paper's networks
(Table 2 of the paper: collaboration networks such as NetHEPT with 15K
nodes / 59K undirected edges, and directed social networks); the real
datasets are not available, so seeded synthetic graphs replace them.
All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "er_directed",
    "chung_lu_undirected",
    "rmat",
    "path_graph",
    "out_star",
    "out_tree",
    "random_small",
    "batch_queries",
    "WorkloadGraph",
    "workload",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _unique_in_order(keys: np.ndarray) -> np.ndarray:
    """Unique keys, keeping each key's first occurrence, in draw order."""
    _, first = np.unique(keys, return_index=True)
    return keys[np.sort(first)]


def er_directed(n: int, m: int, seed: int):
    """Directed Erdos-Renyi graph with exactly ``m`` distinct arcs.

    Endpoints are uniform over ``[0, n)``; self-loops and repeated arcs are
    rejected and drawing continues until ``m`` distinct arcs exist.
    """
    if m > n * (n - 1):
        raise ValueError("too many arcs for a simple digraph")
    rng = _rng(seed)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        b = max(1024, 2 * need)
        u = rng.integers(0, n, size=b, dtype=np.int64)
        v = rng.integers(0, n, size=b, dtype=np.int64)
        ok = u != v
        keys = _unique_in_order(np.concatenate([keys, (u[ok] << 32) | v[ok]]))
    keys = keys[:m]
    return n, (keys >> 32).astype(np.int32), (keys & 0xFFFFFFFF).astype(np.int32)


def chung_lu_undirected(n: int, n_edges: int, beta: float, mean_deg: float, seed: int):
    """Undirected Chung-Lu power-law graph, stored as both arcs.

    Node weights are ``w_i = (i+1)^(-1/(beta-1))`` scaled so that
    ``sum(w) = n * mean_deg``; endpoint pairs are drawn with probability
    proportional to ``w_u * w_v`` (each endpoint independently by weight)
    until exactly ``n_edges`` distinct undirected non-loop edges exist.
    Returns ``2 * n_edges`` arcs.
    """
    rng = _rng(seed)
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-1.0 / (beta - 1.0))
    w *= n * mean_deg / w.sum()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    keys = np.empty(0, dtype=np.int64)
    while keys.size < n_edges:
        need = n_edges - keys.size
        b = max(1024, 2 * need)
        u = np.searchsorted(cdf, rng.random(b), side="right").astype(np.int64)
        v = np.searchsorted(cdf, rng.random(b), side="right").astype(np.int64)
        np.minimum(u, n - 1, out=u)
        np.minimum(v, n - 1, out=v)
        ok = u != v
        lo = np.minimum(u[ok], v[ok])
        hi = np.maximum(u[ok], v[ok])
        keys = _unique_in_order(np.concatenate([keys, (lo << 32) | hi]))
    keys = keys[:n_edges]
    a = (keys >> 32).astype(np.int32)
    b_ = (keys & 0xFFFFFFFF).astype(np.int32)
    return n, np.concatenate([a, b_]), np.concatenate([b_, a])


def rmat(scale: int, m: int, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0):
    """Directed R-MAT graph on ``2^scale`` nodes with exactly ``m`` distinct arcs.

    Each arc picks one quadrant per bit level with probabilities
    ``(a, b, c, d)`` (no noise, ids not permuted).  Self-loops and repeats
    are dropped and drawing tops up until ``m`` distinct arcs exist.
    """
    n = 1 << scale
    a, b, c, d = abcd
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    rng = _rng(seed)
    keys = np.empty(0, dtype=np.int64)
    # quadrant thresholds on one uniform draw: [0,a)->(0,0) [a,a+b)->(0,1) ...
    t1, t2, t3 = a, a + b, a + b + c
    while keys.size < m:
        need = m - keys.size
        bsz = max(1 << 16, int(need * 1.12) + 1024)
        u = np.zeros(bsz, dtype=np.int64)
        v = np.zeros(bsz, dtype=np.int64)
        for _lvl in range(scale):
            x = rng.random(bsz)
            ubit = (x >= t2).astype(np.int64)
            vbit = (((x >= t1) & (x < t2)) | (x >= t3)).astype(np.int64)
            u = (u << 1) | ubit
            v = (v << 1) | vbit
        ok = u != v
        keys = _unique_in_order(np.concatenate([keys, (u[ok] << 32) | v[ok]]))
    keys = keys[:m]
    return n, (keys >> 32).astype(np.int32), (keys & 0xFFFFFFFF).astype(np.int32)


# ---------------------------------------------------------------- small shapes


def path_graph(n: int):
    """Directed path 0 -> 1 -> ... -> n-1."""
    s = np.arange(n - 1, dtype=np.int32)
    return n, s, s + 1


def out_star(n: int, centre: int = 0):
    """Out-star: ``centre`` has an arc to every other node."""
    d = np.array([i for i in range(n) if i != centre], dtype=np.int32)
    return n, np.full(d.size, centre, dtype=np.int32), d


def out_tree(n: int, seed: int):
    """Random rooted out-tree on ``n`` nodes with root 0 (parent < child)."""
    rng = _rng(seed)
    child = np.arange(1, n, dtype=np.int64)
    parent = np.array([rng.integers(0, c) for c in child], dtype=np.int64)
    return n, parent.astype(np.int32), child.astype(np.int32)


def random_small(n: int, m: int, seed: int, loops_and_dups: bool = False):
    """Random small directed arc list; optionally keeps self-loops and
    repeated arcs so that canonicalisation has work to do."""
    rng = _rng(seed)
    u = rng.integers(0, n, size=m, dtype=np.int64)
    v = rng.integers(0, n, size=m, dtype=np.int64)
    if not loops_and_dups:
        keys = _unique_in_order((u << 32) | v)
        keys = keys[(keys >> 32) != (keys & 0xFFFFFFFF)]
        u, v = keys >> 32, keys & 0xFFFFFFFF
    return n, u.astype(np.int32), v.astype(np.int32)


def symmetric(n: int, src, dst):
    """Both arcs of every (non-loop) pair: an undirected graph stored as a
    symmetric arc list."""
    src = np.asarray(src, dtype=np.int32)
    dst = np.asarray(dst, dtype=np.int32)
    keep = src != dst
    return n, np.concatenate([src[keep], dst[keep]]), np.concatenate([dst[keep], src[keep]])


# ------------------------------------------------------------- named workloads


@dataclass(frozen=True)
class WorkloadGraph:
    """One named workload: a graph recipe plus the selection query."""

    name: str
    model: str  # "uic" or "wic"
    p: float  # UIC probability (ignored for WIC)
    R: int
    k: int
    seed: int  # live-edge hash seed

    def graph(self):
        return _WORKLOAD_GRAPHS[self.name.split(":")[0]]()


_WORKLOAD_GRAPHS = {
    # directed ER, n=2,000, m=10,000, generator seed 101
    "er2k": lambda: er_directed(2000, 10000, 101),
    # undirected Chung-Lu, n=15,000, 58,000 edges (116,000 arcs), beta=2.5,
    # mean degree 7.7, generator seed 102 (NetHEPT-shaped, Table 2)
    "cl15k": lambda: chung_lu_undirected(15000, 58000, 2.5, 7.7, 102),
    # directed R-MAT scale 20, 8,388,608 arcs, (0.57,0.19,0.19,0.05), seed 103
    "rmat20": lambda: rmat(20, 8388608, (0.57, 0.19, 0.19, 0.05), 103),
    # the scale-20 recipe at scale 18 (2,097,152 arcs): a small case of the
    # same kernels, for profiler captures
    "rmat18": lambda: rmat(18, 2097152, (0.57, 0.19, 0.19, 0.05), 103),
    "rmat19": lambda: rmat(19, 4194304, (0.57, 0.19, 0.19, 0.05), 103),
    # directed R-MAT scale 22, 67,108,864 arcs, seed 105 (served graph)
    "rmat22": lambda: rmat(22, 67108864, (0.57, 0.19, 0.19, 0.05), 105),
}

_WORKLOADS = {
    "er2k_uic0.1": WorkloadGraph("er2k", "uic", 0.1, 100, 10, 1),
    "cl15k_uic0.01": WorkloadGraph("cl15k", "uic", 0.01, 100, 50, 7),
    "cl15k_wic": WorkloadGraph("cl15k", "wic", 0.0, 100, 50, 7),
    "rmat20_wic": WorkloadGraph("rmat20", "wic", 0.0, 256, 50, 11),
    "rmat18_wic": WorkloadGraph("rmat18", "wic", 0.0, 256, 50, 11),
    "rmat19_wic": WorkloadGraph("rmat19", "wic", 0.0, 256, 50, 11),
}


def workload(name: str) -> WorkloadGraph:
    return _WORKLOADS[name]


def batch_queries(count: int = 256, first: int = 0):
    """Recipes for the batched workload: query ``i`` uses generator seed
    ``2000+i`` and hash seed ``1000+i``; n is log-uniform in [1e3, 2e5],
    mean degree uniform in [4, 20] (Chung-Lu, beta 2.5, undirected); the
    model is uniform over {UIC 0.01, 0.02, 0.05, WIC}; R over {64, 128, 256};
    k uniform in [10, 100].  Returns a list of dicts (graph built lazily by
    :func:`batch_graph`)."""
    out = []
    for i in range(first, first + count):
        rng = _rng(2000 + i)
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        deg = float(rng.uniform(4.0, 20.0))
        choice = int(rng.integers(0, 4))
        model, p = [("uic", 0.01), ("uic", 0.02), ("uic", 0.05), ("wic", 0.0)][choice]
        R = int([64, 128, 256][int(rng.integers(0, 3))])
        k = int(rng.integers(10, 101))
        n_edges = int(round(n * deg / 2))
        out.append(dict(index=i, n=n, mean_deg=deg, n_edges=n_edges, model=model,
                        p=p, R=R, k=min(k, n), seed=1000 + i, gen_seed=2000 + i))
    return out


def batch_graph(q: dict):
    """The Chung-Lu graph of one batched-query recipe."""
    return chung_lu_undirected(q["n"], q["n_edges"], 2.5, q["mean_deg"], q["gen_seed"] + 500000)
