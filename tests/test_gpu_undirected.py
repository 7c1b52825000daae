"""The undirected variant (one coin per undirected edge, SG_UIC_UNDIRECTED):
the GPU's union-find path gives the oracle's seeds, gains, initial gains,
spreads, live masks and snapshot-edge counters bit for bit."""

import numpy as np
import pytest

import oracle
from paper_1212_4779_gb300 import inputs

pytestmark = pytest.mark.gpu
UND = "uic_undirected"


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4779_gb300 import sg as _sg

    return _sg


@pytest.mark.parametrize("p,R,k", [(0.01, 100, 50), (0.05, 100, 30), (0.2, 20, 12), (0.5, 1, 5)])
def test_undirected_matches_oracle(sg, p, R, k):
    """Giant components (p >= 0.2) use the oracle's covered-set route (its
    dynamic update is quadratic in the component size), which counts no
    reverse snapshot-edges; the others compare all three counters."""
    n, s, d = inputs.workload("cl15k_uic0.01").graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, UND, p)
    mode = oracle.DU if p < 0.1 else oracle.COVER
    ref = o.select(R, k, 7, mode=mode, want_init=True)
    res = g.select(R, k, UND, p, 7, stats=True)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    ncmp = 3 if mode == oracle.DU else 2
    assert got[:ncmp] == [int(x) for x in ref["counters"][:ncmp]]
    s_gpu, ed = g.init_gains(R, UND, p, 7)
    assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
    S = ref["seeds"][: min(k, 10)]
    assert g.spread(R + 3, UND, p, 99, S) == o.spread(R + 3, 99, S, want_edges=True)


@pytest.mark.parametrize("qi", [3, 100, 200])
def test_undirected_batch_recipes(sg, qi):
    """Batched-recipe Chung-Lu graphs (giant components at p = 0.05)."""
    q = inputs.batch_queries(1, first=qi)[0]
    n, s, d = inputs.batch_graph(q)
    if n > 60000:
        pytest.skip("oracle too slow for this size")
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, UND, 0.05)
    ref = o.select(64, 12, q["seed"], mode=oracle.DU)
    res = g.select(64, 12, UND, 0.05, q["seed"], stats=True)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    assert [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]] == \
        [int(x) for x in ref["counters"]]


def test_undirected_closed_forms_and_masks(sg):
    n, s0, d0 = inputs.chung_lu_undirected(400, 1500, 2.5, 7.0, 5)
    p_ = np.arange(n - 1, dtype=np.int32)   # a path keeps it connected
    s = np.concatenate([s0, p_, p_ + 1])
    d = np.concatenate([d0, p_ + 1, p_])
    g = sg.Graph.from_coo(n, s, d)
    res = g.select(9, 4, UND, 1.0, 3)
    assert list(res.seeds) == [0, 1, 2, 3] and list(res.gains) == [9 * n, 0, 0, 0]
    res = g.select(9, 4, UND, 0.0, 3)
    assert list(res.seeds) == [0, 1, 2, 3] and list(res.gains) == [9] * 4
    o = oracle.Graph(n, s, d, UND, 0.3)
    assert np.array_equal(g.live_masks(130, UND, 0.3, 8), o.live_masks(130, 8))


def test_undirected_rejections(sg):
    n, s, d = inputs.path_graph(20)          # directed: not symmetric
    g = sg.Graph.from_coo(n, s, d)
    with pytest.raises(sg.SGError) as ei:
        g.select(10, 3, UND, 0.5, 1)
    assert ei.value.status == sg.SG_EINVAL
    n, s, d = inputs.workload("cl15k_uic0.01").graph()
    g = sg.Graph.from_coo(n, s, d)
    with pytest.raises(sg.SGError) as ei:
        g.select_celf(10, 3, UND, 0.5, 1)
    assert ei.value.status == sg.SG_EINVAL


def test_undirected_in_a_batch(sg):
    import torch

    n, s, d = inputs.workload("cl15k_uic0.01").graph()
    g = sg.Graph.from_coo(n, s, d)
    qs = [(UND, 0.05, 100, 20, 1), ("uic", 0.05, 100, 20, 1), (UND, 0.02, 64, 10, 2)]
    alone = [g.select(R, k, m, p, sd) for m, p, R, k, sd in qs]
    wss = [sg.sg_workspace_create(g.handle, R, k) for _, _, R, k, _ in qs]
    try:
        outs = [(torch.zeros(k, dtype=torch.int32, device="cuda"), torch.zeros(k, dtype=torch.int64, device="cuda"))
                for _, _, _, k, _ in qs]
        items = [(g.handle, w, R, k, m, p, sd, so, go) for (m, p, R, k, sd), w, (so, go) in zip(qs, wss, outs)]
        sg.sg_select_batch(items, concurrency=3)
        torch.cuda.synchronize()
        for (so, go), a in zip(outs, alone):
            assert np.array_equal(so.cpu().numpy(), a.seeds) and np.array_equal(go.cpu().numpy(), a.gains)
    finally:
        for w in wss:
            sg.sg_workspace_free(w)
