"""Seed-set spread on fresh snapshots (sg_spread) equals the oracle's
multi-source count bit for bit: the total sum_r |R(G'_r, S)| and the
snapshot-edge count."""

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


@pytest.mark.parametrize("R", [1, 63, 64, 65, 200, 777])
@pytest.mark.parametrize("name", ["er2k_uic0.1", "cl15k_uic0.01", "cl15k_wic"])
def test_spread_matches_oracle(sg, name, R):
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    S = o.select(wl.R, 10, wl.seed, mode=oracle.DU)["seeds"]
    for seed in (wl.seed + 1000, 5):
        got = g.spread(R, wl.model, wl.p, seed, S)
        assert got == o.spread(R, seed, S, want_edges=True)


def test_spread_edge_cases(sg):
    n, s, d = inputs.path_graph(300)
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, "uic", 1.0)
    assert g.spread(70, "uic", 1.0, 3, []) == (0, 0)
    assert g.spread(70, "uic", 1.0, 3, [0]) == (70 * 300, 70 * 299)
    assert g.spread(70, "uic", 1.0, 3, [299, 299, 299]) == (70, 0)  # repeated seeds count once
    assert g.spread(70, "uic", 1.0, 3, list(range(300))) == (70 * 300, 70 * 299)
    o0 = oracle.Graph(n, s, d, "uic", 0.0)
    assert g.spread(65, "uic", 0.0, 3, [5, 9]) == o0.spread(65, 3, [5, 9], want_edges=True) == (130, 130)
    o5 = oracle.Graph(n, s, d, "uic", 0.5)
    assert g.spread(129, "uic", 0.5, 11, [0, 100, 200]) == o5.spread(129, 11, [0, 100, 200], want_edges=True)
    del o


def test_spread_device_seed_list(sg):
    import torch

    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    S = torch.tensor([3, 77, 1200, 14999], dtype=torch.int32, device="cuda")
    assert g.spread(130, wl.model, wl.p, 42, S) == o.spread(130, 42, S.cpu().numpy(), want_edges=True)


def test_spread_rejects_bad_arguments(sg):
    n, s, d = inputs.path_graph(10)
    g = sg.Graph.from_coo(n, s, d)
    for bad in ([10], [-1], [3, 11]):
        with pytest.raises(sg.SGError) as ei:
            g.spread(4, "uic", 0.5, 1, bad)
        assert ei.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SGError):
        g.spread(0, "uic", 0.5, 1, [1])
    with pytest.raises(sg.SGError):
        g.spread(4, "uic", 1.5, 1, [1])


def test_spread_rmat20_many_snapshots(sg):
    """R-MAT scale 20 (weighted cascade), 20,000 snapshots: 313 words, more
    than one launch of words; seeds are the top out-degree nodes."""
    wl = inputs.workload("rmat20_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    S = np.argsort(-np.diff(o.rp), kind="stable")[:20].astype(np.int32)
    got = g.spread(20000, wl.model, wl.p, 777, S)
    assert got == o.spread(20000, 777, S, want_edges=True)
