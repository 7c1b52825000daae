"""The autotuner (no counterpart in the paper): it times whole selections
under candidate knob settings and must find settings whose results are the
oracle's; its JSON-lines cache returns the same tuning without timing; and
batches accept a tuning per query with results equal to the oracle's."""

import os

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


def test_autotune_keeps_results_and_caches(sg, tmp_path):
    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    ref = oracle.Graph(n, s, d, wl.model, wl.p).select(wl.R, 20, wl.seed, mode=oracle.DU)
    before = sg.sg_get_tuning().as_dict()
    cache = str(tmp_path / "tuning.jsonl")
    t, ms = sg.sg_autotune(g.handle, wl.R, 20, wl.model, wl.p, wl.seed, cache_path=cache)
    assert ms > 0
    assert sg.sg_get_tuning().as_dict() == before  # the process-wide knobs are untouched
    td = t.as_dict()
    assert td["walk_groups"] in (8, 16, 32, 64) and 0 <= td["landmarks"] <= 8
    with open(cache) as f:
        lines = f.readlines()
    assert len(lines) == 1 and '"walk_groups": %d' % td["walk_groups"] in lines[0]
    t2, ms2 = sg.sg_autotune(g.handle, wl.R, 20, wl.model, wl.p, wl.seed, cache_path=cache)
    assert t2.as_dict() == td and abs(ms2 - ms) < 1e-2
    with open(cache) as f:
        assert len(f.readlines()) == 1  # answered from the cache
    sg.sg_set_tuning(t)
    try:
        res = g.select(wl.R, 20, wl.model, wl.p, wl.seed)
    finally:
        sg.sg_set_tuning(sg.sg_tuning(**before))
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    g.close()


def test_batch_with_per_query_tunings_equals_oracle(sg):
    import torch

    qs = [q for q in inputs.batch_queries(12) if q["n"] <= 60000][:6]
    graphs, wss, items, outs, refs = [], [], [], [], []
    variants = [dict(walk_groups=8, direction_mode=0, direction_div=4, tier1_keys=256, tier2_keys=2048,
                     landmarks=8, scc=1, forward_lists=1, word_major=1, tier1_direct=16),
                dict(walk_groups=32, direction_mode=2, direction_div=1, tier1_keys=16, tier2_keys=300,
                     landmarks=0, scc=0, forward_lists=0, word_major=0, tier1_direct=0),
                dict(walk_groups=64, direction_mode=1, direction_div=16, tier1_keys=64, tier2_keys=1024,
                     landmarks=4, scc=1, forward_lists=1, word_major=1, tier1_direct=1)]
    sg.sg_set_walk_groups(64)  # workspaces sized for every split
    try:
        for i, q in enumerate(qs):
            n, s, d = inputs.batch_graph(q)
            g = sg.Graph.from_coo(n, s, d)
            graphs.append(g)
            wss.append(sg.sg_workspace_create(g.handle, q["R"], q["k"]))
            refs.append(oracle.Graph(n, s, d, q["model"], q["p"]).select(q["R"], q["k"], q["seed"],
                                                                        mode=oracle.CELF))
            so = torch.full((q["k"],), -1, dtype=torch.int32, device="cuda")
            go = torch.full((q["k"],), -1, dtype=torch.int64, device="cuda")
            outs.append((so, go))
            tun = sg.sg_tuning(**variants[i % len(variants)])
            items.append((g.handle, wss[-1], q["R"], q["k"], q["model"], q["p"], q["seed"], so, go, tun))
    finally:
        sg.sg_set_walk_groups(64)
    try:
        st = sg.sg_select_batch(items, concurrency=4)
        torch.cuda.synchronize()
        assert all(x == sg.SG_OK for x in st)
        for (so, go), ref in zip(outs, refs):
            assert np.array_equal(so.cpu().numpy(), ref["seeds"])
            assert np.array_equal(go.cpu().numpy(), ref["gains"])
        bad = list(items[0])
        bad[9] = sg.sg_tuning(**dict(variants[0], walk_groups=12))
        with pytest.raises(sg.SGError) as e:
            sg.sg_select_batch([tuple(bad)])
        assert e.value.status == sg.SG_EINVAL
    finally:
        for w in wss:
            sg.sg_workspace_free(w)
        for g in graphs:
            g.close()
