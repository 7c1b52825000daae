"""The linear threshold model in its live-edge form (SG_LT; Kempe, Kleinberg
and Tardos 2003, weights 1/indeg, named by the paper as StaticGreedy's LT
generalisation) on the GPU against the oracle: live masks bit for bit,
initial gains element by element, seeds, gains and the three snapshot-edge
counters, spread and lazy-forward selection; integers, so equal."""

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


GRAPHS = {
    "er": lambda: inputs.er_directed(2000, 10000, 101),
    "cl": lambda: inputs.chung_lu_undirected(15000, 58000, 2.5, 7.7, 102),
    "small": lambda: inputs.random_small(60, 400, 7, loops_and_dups=True),
    "star": lambda: (9, np.array([0, 1, 2, 3, 4, 5, 6, 7], np.int32), np.array([8] * 8, np.int32)),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("R", [1, 65, 130])
def test_lt_live_masks_bit_exact(sg, name, R):
    n, s, d = GRAPHS[name]()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, "lt")
    assert np.array_equal(g.live_masks(R, "lt", 0.0, 77 + R), o.live_masks(R, 77 + R))
    g.close()


@pytest.mark.parametrize("name,R,k", [("er", 100, 10), ("cl", 100, 30), ("small", 70, 8), ("star", 64, 3)])
def test_lt_select_matches_oracle(sg, name, R, k):
    n, s, d = GRAPHS[name]()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, "lt")
    ref = o.select(R, k, 5, mode=oracle.DU, want_init=True)
    s_gpu, ed = g.init_gains(R, "lt", 0.0, 5)
    assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
    res = g.select(R, k, "lt", 0.0, 5, stats=True)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]]
    assert res.stats["status_flags"] == 0 and res.stats["mask_cache"] == 1
    tot, edges = g.spread(R + 200, "lt", 0.0, 9, res.seeds)
    assert (tot, edges) == o.spread(R + 200, 9, res.seeds, want_edges=True)
    (cres, evals) = g.select_celf(R, k, "lt", 0.0, 5)
    cref = o.select(R, k, 5, mode=oracle.CELF)
    assert np.array_equal(cres.seeds, cref["seeds"]) and np.array_equal(cres.gains, cref["gains"])
    assert evals == cref["evals"]
    g.close()


def test_lt_every_walk_setting_and_tier_agrees(sg):
    """Engine tiers, walk splits and the direction switch with LT coins (read
    from the cache in both arc orders): identical to the oracle."""
    n, s, d = GRAPHS["cl"]()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, "lt")
    ref = o.select(128, 12, 3, mode=oracle.DU)
    try:
        for t1, t2, groups, mode in [(256, 2048, 32, 1), (2, 16, 8, 2), (16, 300, 64, 0)]:
            sg.sg_set_engine_limits(t1, t2)
            sg.sg_set_walk_groups(groups)
            sg.sg_set_direction(mode, 4 if mode != 2 else 1)
            g.trim()
            res = g.select(128, 12, "lt", 0.0, 3, stats=True)
            assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
            got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
            assert got == [int(x) for x in ref["counters"]]
    finally:
        sg.sg_set_engine_limits(64, 2048)
        sg.sg_set_walk_groups(64)
        sg.sg_set_direction(1, 4)
    g.close()


def test_lt_in_a_batch_equals_oracle(sg):
    import torch

    graphs, items, outs, refs, wss = [], [], [], [], []
    for name, R, k in (("er", 100, 10), ("cl", 192, 20)):
        n, s, d = GRAPHS[name]()
        g = sg.Graph.from_coo(n, s, d)
        graphs.append(g)
        refs.append(oracle.Graph(n, s, d, "lt").select(R, k, 21, mode=oracle.CELF))
        wss.append(sg.sg_workspace_create(g.handle, R, k))
        so = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        go = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        outs.append((so, go))
        items.append((g.handle, wss[-1], R, k, "lt", 0.0, 21, so, go))
    try:
        st = sg.sg_select_batch(items, concurrency=2)
        torch.cuda.synchronize()
        assert all(x == sg.SG_OK for x in st)
        for (so, go), ref in zip(outs, refs):
            assert np.array_equal(so.cpu().numpy(), ref["seeds"]) and np.array_equal(go.cpu().numpy(), ref["gains"])
    finally:
        for w in wss:
            sg.sg_workspace_free(w)
        for g in graphs:
            g.close()
