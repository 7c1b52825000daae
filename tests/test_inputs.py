"""The seeded generators produce the shapes the workloads are stated with:
exact arc counts, no self-loops or repeats where promised, the same graph
for the same seed, and the named workloads' queries."""

import numpy as np
import pytest

from paper_1212_4779_gb300 import inputs


def _keys(s, d):
    return (s.astype(np.int64) << 32) | d.astype(np.int64)


def _simple(n, s, d, m):
    assert s.dtype == np.int32 and d.dtype == np.int32 and s.size == d.size == m
    assert (s >= 0).all() and (s < n).all() and (d >= 0).all() and (d < n).all()
    assert (s != d).all()
    assert np.unique(_keys(s, d)).size == m


def test_er_exact_and_deterministic():
    n, s, d = inputs.er_directed(500, 4000, 7)
    _simple(n, s, d, 4000)
    n2, s2, d2 = inputs.er_directed(500, 4000, 7)
    assert n2 == n and np.array_equal(s, s2) and np.array_equal(d, d2)
    _, s3, _ = inputs.er_directed(500, 4000, 8)
    assert not np.array_equal(s, s3)
    with pytest.raises(ValueError):
        inputs.er_directed(3, 7, 1)  # a simple digraph on 3 nodes has 6 arcs


def test_chung_lu_symmetric_exact_edges_and_skewed():
    n, s, d = inputs.chung_lu_undirected(3000, 12000, 2.5, 8.0, 4)
    _simple(n, s, d, 24000)
    assert np.array_equal(np.sort(_keys(s, d)), np.sort(_keys(d, s)))  # every arc's reverse
    deg = np.bincount(s, minlength=n)
    # weights fall with the id: node 0 carries the largest weight, degrees are heavy-tailed
    assert deg[:30].mean() > 5 * deg.mean() and deg.max() > 20 * np.median(deg)


def test_rmat_exact_arcs_and_quadrant_skew():
    scale = 12
    n, s, d = inputs.rmat(scale, 8 << scale, (0.57, 0.19, 0.19, 0.05), 103)
    assert n == 1 << scale
    _simple(n, s, d, 8 << scale)
    # a = 0.57 puts mass in the low ids of both endpoints; d = 0.05 keeps
    # the high-high quadrant sparse
    half = n // 2
    low_low = np.mean((s < half) & (d < half))
    high_high = np.mean((s >= half) & (d >= half))
    assert low_low > 0.45 and high_high < 0.10
    with pytest.raises(ValueError):
        inputs.rmat(4, 10, (0.5, 0.2, 0.2, 0.2))


def test_small_shapes():
    n, s, d = inputs.path_graph(6)
    assert list(s) == [0, 1, 2, 3, 4] and list(d) == [1, 2, 3, 4, 5]
    n, s, d = inputs.out_star(5, centre=2)
    assert set(s) == {2} and sorted(d) == [0, 1, 3, 4]
    n, s, d = inputs.out_tree(50, 3)
    assert (s < d).all() and sorted(d) == list(range(1, 50))
    n, s, d = inputs.random_small(30, 400, 5, loops_and_dups=True)
    assert s.size == 400 and ((s == d).any() or np.unique(_keys(s, d)).size < 400)
    n, s, d = inputs.random_small(30, 400, 5)
    assert (s != d).all() and np.unique(_keys(s, d)).size == s.size


def test_symmetric_doubles_and_drops_loops():
    n, s, d = inputs.symmetric(4, np.array([0, 1, 2]), np.array([1, 1, 3]))
    assert sorted(zip(s.tolist(), d.tolist())) == [(0, 1), (1, 0), (2, 3), (3, 2)]


def test_named_workloads_carry_their_queries():
    want = {
        "er2k_uic0.1": ("uic", 0.1, 100, 10, 1),
        "cl15k_uic0.01": ("uic", 0.01, 100, 50, 7),
        "cl15k_wic": ("wic", 0.0, 100, 50, 7),
        "rmat20_wic": ("wic", 0.0, 256, 50, 11),
        "rmat18_wic": ("wic", 0.0, 256, 50, 11),
        "rmat19_wic": ("wic", 0.0, 256, 50, 11),
    }
    for name, (model, p, R, k, seed) in want.items():
        wl = inputs.workload(name)
        assert (wl.model, wl.p, wl.R, wl.k, wl.seed) == (model, p, R, k, seed)
    n, s, d = inputs.workload("er2k_uic0.1").graph()
    _simple(n, s, d, 10000)
    assert n == 2000
    n, s, d = inputs.workload("cl15k_wic").graph()
    _simple(n, s, d, 116000)
    assert n == 15000


def test_batch_recipes_are_deterministic_and_in_range():
    qs = inputs.batch_queries(64)
    assert qs == inputs.batch_queries(64)
    assert inputs.batch_queries(8, first=10) == qs[10:18]
    for q in qs:
        assert 1000 <= q["n"] <= 200000 and 4.0 <= q["mean_deg"] <= 20.0
        assert (q["model"], q["p"]) in {("uic", 0.01), ("uic", 0.02), ("uic", 0.05), ("wic", 0.0)}
        assert q["R"] in (64, 128, 256) and 10 <= q["k"] <= 100
        assert q["seed"] == 1000 + q["index"] and q["gen_seed"] == 2000 + q["index"]
    n, s, d = inputs.batch_graph(qs[0])
    _simple(n, s, d, 2 * qs[0]["n_edges"])
