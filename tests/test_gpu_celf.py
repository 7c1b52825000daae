"""StaticGreedyCELF on the GPU (sg_select_celf) returns the oracle's CELF
seeds, gains and number of lazy evaluations, and the same seeds and gains
as the dynamic update; integers, so the tolerance is zero."""

import numpy as np
import pytest

import oracle
from paper_1212_4779_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4779_gb300 import sg as _sg

    return _sg


@pytest.mark.parametrize("name", ["er2k_uic0.1", "cl15k_uic0.01", "cl15k_wic"])
def test_celf_matches_oracle(sg, name):
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    ref = o.select(wl.R, wl.k, wl.seed, mode=oracle.CELF)
    res, evals = g.select_celf(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    assert evals == ref["evals"]
    assert [res.stats["init_edges"], res.stats["fwd_edges"]] == [int(x) for x in ref["counters"][:2]]
    du = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed)
    assert np.array_equal(du.seeds, res.seeds) and np.array_equal(du.gains, res.gains)


def test_celf_after_other_queries_on_the_same_graph(sg):
    """Per-query caches (index, lists, landmarks) are rebuilt for each
    query's coins: CELF after selections with other seeds and R, and a
    selection after CELF, still equal the oracle."""
    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    g.select(130, 12, wl.model, wl.p, 99)
    ref = o.select(wl.R, 15, 4242, mode=oracle.CELF)
    res, evals = g.select_celf(wl.R, 15, wl.model, wl.p, 4242)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    assert evals == ref["evals"]
    ref2 = o.select(70, 9, 17, mode=oracle.DU)
    du = g.select(70, 9, wl.model, wl.p, 17)
    assert np.array_equal(du.seeds, ref2["seeds"]) and np.array_equal(du.gains, ref2["gains"])


def test_celf_closed_forms(sg):
    n, s, d = inputs.path_graph(12)
    g = sg.Graph.from_coo(n, s, d)
    res, evals = g.select_celf(3, 4, "uic", 1.0, 5)
    assert list(res.seeds) == [0, 1, 2, 3] and list(res.gains) == [36, 0, 0, 0] and evals == 13
    n, s, d = inputs.out_star(9, centre=4)
    g = sg.Graph.from_coo(n, s, d)
    res, evals = g.select_celf(2, 4, "uic", 1.0, 1)
    assert list(res.seeds) == [4, 0, 1, 2] and list(res.gains) == [18, 0, 0, 0] and evals == 10


@pytest.mark.parametrize("cache,heavy", [(1, 2), (0, 0), (1, 0)])
def test_celf_with_caches(sg, cache, heavy):
    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    try:
        sg.sg_set_heavy_threshold(heavy)
        sg.sg_set_mask_cache(cache)
        g = sg.Graph.from_coo(n, s, d)
        o = oracle.Graph(n, s, d, wl.model, wl.p)
        ref = o.select(wl.R, 20, wl.seed, mode=oracle.CELF)
        res, evals = g.select_celf(wl.R, 20, wl.model, wl.p, wl.seed)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        assert evals == ref["evals"]
    finally:
        sg.sg_set_heavy_threshold(2)
        sg.sg_set_mask_cache(0)


def test_celf_device_outputs(sg):
    import torch

    wl = inputs.workload("er2k_uic0.1")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    so = torch.zeros(wl.k, dtype=torch.int32, device="cuda")
    go = torch.zeros(wl.k, dtype=torch.int64, device="cuda")
    ev, _ = sg.sg_select_celf(g.handle, wl.R, wl.k, wl.model, wl.p, wl.seed, so, go)
    ref = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed)
    assert np.array_equal(so.cpu().numpy(), ref.seeds) and np.array_equal(go.cpu().numpy(), ref.gains)
    assert ev > 0


def test_celf_rejects_bad_queries(sg):
    n, s, d = inputs.path_graph(10)
    g = sg.Graph.from_coo(n, s, d)
    for R, k in ((0, 2), (4, 0), (4, 11)):
        with pytest.raises(sg.SGError) as ei:
            g.select_celf(R, k, "uic", 0.5, 1)
        assert ei.value.status == sg.SG_EINVAL


def test_celf_rmat20_equals_dynamic_update(sg):
    """Full size: the 50 CELF seeds and gains on R-MAT scale 20 (weighted
    cascade, R = 256) equal the dynamic update's, whose gains the parity
    tests tie to the oracle."""
    wl = inputs.workload("rmat20_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    du = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
    res, evals = g.select_celf(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
    assert np.array_equal(res.seeds, du.seeds) and np.array_equal(res.gains, du.gains)
    assert res.stats["init_edges"] == du.stats["init_edges"] and res.stats["fwd_edges"] == du.stats["fwd_edges"]
    assert evals >= wl.k - 1
