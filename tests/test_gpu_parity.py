"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Every comparison is exact: coins, canonical CSR, initial gains, seeds,
integer gains and the implementation-independent snapshot-edge counters
are integers, so the tolerance is zero."""

import numpy as np
import pytest

import oracle
from paper_1212_4779_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def sg():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4779_gb300 import sg as _sg

    return _sg


def _both(sg, n, s, d, model, p):
    return sg.Graph.from_coo(n, s, d), oracle.Graph(n, s, d, model, p)


# ------------------------------------------------------------------- coins


@pytest.mark.parametrize("gen,model,p,R,seed", [
    (lambda: inputs.er_directed(500, 3000, 1), "uic", 0.1, 100, 1),
    (lambda: inputs.chung_lu_undirected(800, 3000, 2.5, 7.0, 2), "wic", 0.0, 130, 7),
    (lambda: inputs.random_small(40, 500, 3, loops_and_dups=True), "uic", 0.5, 64, 2**63 + 5),
    (lambda: inputs.er_directed(300, 900, 4), "uic", 1.0, 1, 9),
    (lambda: inputs.er_directed(300, 900, 4), "uic", 0.0, 70, 9),
])
def test_live_masks_bit_exact(sg, gen, model, p, R, seed):
    n, s, d = gen()
    g, o = _both(sg, n, s, d, model, p)
    assert g.m == o.m
    got = g.live_masks(R, model, p, seed)
    want = o.live_masks(R, seed)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_canonical_csr_matches_oracle(sg):
    for seed in range(3):
        n, s, d = inputs.random_small(50, 900, seed, loops_and_dups=True)
        g, o = _both(sg, n, s, d, "uic", 0.3)
        rp, col = g.csr()
        assert np.array_equal(rp, o.rp)
        assert np.array_equal(col, o.col[: o.m])


def test_csr_input_is_canonicalised(sg):
    n, s, d = inputs.random_small(60, 700, 11, loops_and_dups=True)
    order = np.argsort(s, kind="stable")
    s2, d2 = s[order], d[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, s2.astype(np.int64) + 1, 1)
    rp = np.cumsum(rp)
    g = sg.Graph.from_csr(n, rp, d2)
    o = oracle.Graph(n, s, d, "wic")
    rpg, colg = g.csr()
    assert np.array_equal(rpg, o.rp) and np.array_equal(colg, o.col[: o.m])
    res = g.select(70, 5, "wic", 0.0, 3)
    ref = o.select(70, 5, 3, mode=oracle.DU)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])


# ----------------------------------------------------------- initial gains


INIT_CASES = [
    ("er2k_uic0.1", None),
    ("cl15k_uic0.01", None),
    ("cl15k_wic", None),
    ("cl15k_wic", 1),
    ("cl15k_wic", 65),
    ("er2k_uic0.1", 200),
]


@pytest.mark.parametrize("name,R", INIT_CASES)
def test_init_gains_match_oracle(sg, name, R):
    wl = inputs.workload(name)
    R = R or wl.R
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    got, ed = g.init_gains(R, wl.model, wl.p, wl.seed)
    want, ed_want = o.init_gains(R, wl.seed)
    assert np.array_equal(got, want)
    assert ed == ed_want


@pytest.mark.parametrize("name", ["cl15k_wic", "er2k_uic0.1"])
def test_init_gains_per_word_partial_sums(sg, name):
    """Per-word partial sums of the initial gains: the gains over R = 192
    snapshots minus those over R = 128 (a snapshot's coins do not depend
    on R) are word 2's sums, equal to the oracle's over snapshots 128..191;
    likewise word 0 against R = 64."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    s64, _ = g.init_gains(64, wl.model, wl.p, wl.seed)
    s128, _ = g.init_gains(128, wl.model, wl.p, wl.seed)
    s192, _ = g.init_gains(192, wl.model, wl.p, wl.seed)
    assert np.array_equal(s64, o.init_gains(192, wl.seed, 0, 64)[0])
    assert np.array_equal(s192 - s128, o.init_gains(192, wl.seed, 128, 192)[0])


@pytest.mark.parametrize("lmk", [0, 8])
def test_big_tasks_take_the_upper_tiers_and_agree(sg, limits, lmk):
    """High-probability cascade: most sources reach hundreds of nodes per
    64-snapshot word, so without landmarks the shared-memory warp tables
    overflow and tasks move to the upper tiers; with landmarks the sources
    are credited with the giant component's reach and stay small."""
    n, s, d = inputs.chung_lu_undirected(3000, 12000, 2.5, 8.0, 31)
    g, o = _both(sg, n, s, d, "uic", 0.3)
    sg.sg_set_landmarks(lmk)
    _set_tier1_direct(sg, 0)  # every overflow passes through the block-shared tier
    res = g.select(96, 8, "uic", 0.3, 4, stats=True)
    ref = o.select(96, 8, 4, mode=oracle.DU)
    if lmk == 0:
        assert res.stats["init_tier2_tasks"] > 0
    assert np.array_equal(res.seeds, ref["seeds"])
    assert np.array_equal(res.gains, ref["gains"])
    assert [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]] == list(map(int, ref["counters"]))


@pytest.fixture
def limits(sg):
    yield sg.sg_set_engine_limits
    sg.sg_set_engine_limits(64, 2048)
    sg.sg_set_heavy_threshold(2)
    sg.sg_set_landmarks(8)
    sg.sg_set_snapshot_lists(1)
    sg.sg_set_mask_cache(0)
    sg.sg_set_forward_lists(1)
    sg.sg_set_walk_groups(64)
    sg.sg_set_direction(1, 4)
    sg.sg_set_scc_condensation(1)
    _set_tier1_direct(sg, 16)


def _set_tier1_direct(sg, v):
    """Warp-tier overflows with >= v frontier entries left skip the
    block-shared tier (0: never); set through the tuning struct."""
    t = sg.sg_get_tuning()
    t.tier1_direct = v
    sg.sg_set_tuning(t)


@pytest.mark.parametrize("t1,t2", [(256, 4096), (2, 16)])
def test_scc_condensation_is_exact_and_skips_work(sg, limits, t1, t2):
    """UIC 0.05 on a Chung-Lu graph with a giant strongly connected component
    holding the hubs: sources inside a landmark's component skip those
    snapshots' walks.  With condensation on and off the initial gains,
    seeds, gains and counters equal the oracle's, and on expands fewer
    elements; also on the named workloads."""
    n, s, d = inputs.chung_lu_undirected(4000, 30000, 2.5, 15.0, 77)
    g, o = _both(sg, n, s, d, "uic", 0.05)
    ref = o.select(128, 8, 99, mode=oracle.DU, want_init=True)
    limits(t1, t2)
    elems = {}
    for on in (0, 1):
        sg.sg_set_scc_condensation(on)
        s_gpu, ed = g.init_gains(128, "uic", 0.05, 99)
        assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
        res = g.select(128, 8, "uic", 0.05, 99, stats=True)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]
        elems[on] = sum(res.stats["work_elems"][0])
    assert elems[1] < elems[0], elems
    for name in ("cl15k_wic", "cl15k_uic0.01"):
        wl = inputs.workload(name)
        n, s, d = wl.graph()
        g, o = _both(sg, n, s, d, wl.model, wl.p)
        ref = o.select(wl.R, 10, wl.seed, mode=oracle.DU, want_init=True)
        for on in (0, 1):
            sg.sg_set_scc_condensation(on)
            s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
            assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])


@pytest.mark.parametrize("mode,div", [(0, 4), (1, 4), (1, 64), (2, 1)])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1", "giant"])
def test_direction_optimising_gives_identical_results(sg, limits, name, mode, div):
    """Top-down only, switching by frontier size, and bottom-up forced after
    the first level: the forward update's walk and ancestor walk and the
    landmark walks reach the same (node, snapshot) pairs, so initial gains,
    seeds, gains and all three counters equal the oracle's; so does the
    spread of the chosen seeds.  "giant" is UIC 0.05 on a Chung-Lu graph with
    a giant component, where frontiers pass n / 4 and the switch is taken."""
    if name == "giant":
        n, s, d = inputs.chung_lu_undirected(4000, 30000, 2.5, 15.0, 77)
        model, p, R, seed = "uic", 0.05, 128, 99
    else:
        wl = inputs.workload(name)
        n, s, d = wl.graph()
        model, p, R, seed = wl.model, wl.p, wl.R, wl.seed
    sg.sg_set_direction(mode, div)
    for groups in (8, 32):
        sg.sg_set_walk_groups(groups)
        g, o = _both(sg, n, s, d, model, p)
        ref = o.select(R, 12, seed, mode=oracle.DU, want_init=True)
        s_gpu, ed = g.init_gains(R, model, p, seed)
        assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
        res = g.select(R, 12, model, p, seed, stats=True)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]
        tot, edges = g.spread(R + 64, model, p, seed + 1, res.seeds)
        want_t, want_e = o.spread(R + 64, seed + 1, res.seeds, want_edges=True)
        assert tot == want_t and edges == want_e
        g.close()


@pytest.mark.parametrize("groups", [8, 16, 32, 64])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1"])
def test_walk_groups_give_identical_results(sg, limits, name, groups):
    """The forward update's walk and the landmark walks split each 64-snapshot
    word over 8 to 64 blocks (bit-disjoint atomics on shared words): the
    oracle's initial gains, seeds, gains and counters for every split."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    sg.sg_set_walk_groups(groups)
    g, o = _both(sg, n, s, d, wl.model, wl.p)  # the workspace's queues are sized for this split
    ref = o.select(wl.R, 12, wl.seed, mode=oracle.DU, want_init=True)
    s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
    assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
    res = g.select(wl.R, 12, wl.model, wl.p, wl.seed, stats=True)
    assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]]


@pytest.mark.parametrize("fl", [0, 1])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1"])
def test_forward_lists_give_identical_results(sg, limits, name, fl):
    """Sparse expansions through the forward per-snapshot lists (one bit at
    a time, the rest re-queued) give the oracle's initial gains, seeds,
    gains and counters in every tier, with the lists on and off."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    sg.sg_set_forward_lists(fl)
    ref = o.select(wl.R, 10, wl.seed, mode=oracle.DU, want_init=True)
    for t1, t2 in [(256, 4096), (2, 16)]:
        limits(t1, t2)
        for lmk in (0, 8):
            sg.sg_set_landmarks(lmk)
            s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
            assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
            res = g.select(wl.R, 10, wl.model, wl.p, wl.seed, stats=True)
            assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
            got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
            assert got == [int(x) for x in ref["counters"]]


@pytest.mark.parametrize("heavy", [0, 2])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1"])
def test_mask_cache_gives_identical_results(sg, limits, name, heavy):
    """The live-mask cache holds the same coins, evaluated once per query:
    identical initial gains, seeds, gains and counters in every tier, with
    and without the heavy-row index on top of it."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    sg.sg_set_heavy_threshold(heavy)
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    sg.sg_set_mask_cache(1)
    ref = o.select(wl.R, 10, wl.seed, mode=oracle.DU, want_init=True)
    for t1, t2 in [(256, 4096), (2, 16)]:
        limits(t1, t2)
        s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
        assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
        res = g.select(wl.R, 10, wl.model, wl.p, wl.seed, stats=True)
        assert res.stats["mask_cache"] == 1
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]


def test_mask_cache_bytes_are_reported(sg, limits):
    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    off = sg.sg_workspace_bytes(g.handle, 128, 10)
    sg.sg_set_mask_cache(1)
    on = sg.sg_workspace_bytes(g.handle, 128, 10)
    assert on - off == 2 * 2 * g.m * 8


@pytest.mark.parametrize("lists", [0, 1])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01"])
def test_snapshot_lists_give_identical_results(sg, limits, name, lists):
    """Per-snapshot live in-lists of heavy rows are a cache of the same
    coins: identical seeds, gains and counters with them on or off, with a
    low heavy threshold so that many rows use them."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    sg.sg_set_heavy_threshold(4)
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    sg.sg_set_snapshot_lists(lists)
    ref = o.select(wl.R, 12, wl.seed, mode=oracle.DU)
    for t1, t2 in [(256, 4096), (2, 16)]:
        limits(t1, t2)
        res = g.select(wl.R, 12, wl.model, wl.p, wl.seed, stats=True)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]


@pytest.mark.parametrize("lmk", [0, 1, 3, 8])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1"])
def test_landmark_gives_identical_results(sg, limits, name, lmk):
    """Crediting the landmark's reach set is exact: same initial gains, seeds,
    gains and snapshot-edge counters with and without it, in every tier."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    sg.sg_set_landmarks(lmk)
    ref = o.select(wl.R, 8, wl.seed, mode=oracle.DU, want_init=True)
    for t1, t2 in [(256, 4096), (2, 16)]:
        limits(t1, t2)
        s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
        assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
        res = g.select(wl.R, 8, wl.model, wl.p, wl.seed, stats=True)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]


@pytest.mark.parametrize("direct", [0, 1, 16])
@pytest.mark.parametrize("t1,t2", [(1, 1), (4, 32), (16, 300), (256, 4096)])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01"])
def test_every_tier_gives_identical_results(sg, limits, name, t1, t2, direct):
    """Tiny table limits push tasks through all three engine tiers, with the
    warp tier's overflows routed through the block-shared tier (direct 0) or
    straight to the dense tier past 1 or 16 frontier entries; the seeds,
    gains and counters must not change."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    limits(t1, t2)
    _set_tier1_direct(sg, direct)
    k = 12
    res = g.select(wl.R, k, wl.model, wl.p, wl.seed, stats=True)
    ref = o.select(wl.R, k, wl.seed, mode=oracle.DU)
    assert np.array_equal(res.seeds, ref["seeds"])
    assert np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]]
    if t2 <= 32:
        assert res.stats["init_tier3_tasks"] > 0 and res.stats["rev_tier3_tasks"] > 0
    if t1 <= 4 and direct == 0:
        assert res.stats["init_tier2_tasks"] > 0 and res.stats["rev_tier2_tasks"] > 0


@pytest.mark.parametrize("heavy", [0, 2, 8, 64])
@pytest.mark.parametrize("name", ["cl15k_wic", "cl15k_uic0.01", "er2k_uic0.1"])
def test_heavy_index_threshold_gives_identical_results(sg, limits, name, heavy):
    """The per-query live index of heavy rows is a cache of the same coins:
    any threshold (0 = none, 2 = nearly every row) gives the same result."""
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    sg.sg_set_heavy_threshold(heavy)
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    k = 10
    res = g.select(wl.R, k, wl.model, wl.p, wl.seed, stats=True)
    ref = o.select(wl.R, k, wl.seed, mode=oracle.DU)
    maxdeg = max(np.bincount(o.col[: o.m], minlength=n).max(), np.diff(o.rp).max())
    assert res.stats["heavy_index"] == (1 if 0 < heavy <= maxdeg else 0)
    assert np.array_equal(res.seeds, ref["seeds"])
    assert np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]]
    s_gpu, ed = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
    s_ref, ed_ref = o.init_gains(wl.R, wl.seed)
    assert np.array_equal(s_gpu, s_ref) and ed == ed_ref


def test_giant_component_reaches_tier3_and_agrees(sg, limits):
    """p = 1 on a connected graph: every task reaches all n > 4096 nodes.
    Without the landmark, initial-gain tasks run in the dense tier-3
    engine; with it, every source is credited with the landmark's reach."""
    n, s, d = inputs.chung_lu_undirected(9000, 30000, 2.5, 6.0, 41)
    p_ = np.arange(n - 1, dtype=np.int32)
    s = np.concatenate([s, p_, p_ + 1])
    d = np.concatenate([d, p_ + 1, p_])
    g, o = _both(sg, n, s, d, "uic", 1.0)
    ref = o.select(2, 3, 5, mode=oracle.DU)
    for lmk in (0, 1, 8):
        sg.sg_set_landmarks(lmk)
        res = g.select(2, 3, "uic", 1.0, 5, stats=True)
        if lmk == 0:
            assert res.stats["init_tier3_tasks"] > 0
        assert list(res.gains) == [2 * n, 0, 0] and list(res.seeds) == [0, 1, 2]
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]


@pytest.mark.parametrize("t1,t2", [(256, 4096), (2, 16)])
def test_landmark_credit_in_a_giant_component(sg, limits, t1, t2):
    """UIC 0.05 on a Chung-Lu graph with a giant component (about 1,000
    nodes per snapshot): sources that reach a landmark are credited with its
    reach set from the start and stop at its boundary.  Results equal the
    oracle with 0, 1 and 8 landmarks, and the landmarks remove most of the
    traversal."""
    n, s, d = inputs.chung_lu_undirected(4000, 30000, 2.5, 15.0, 77)
    g, o = _both(sg, n, s, d, "uic", 0.05)
    ref = o.select(128, 8, 99, mode=oracle.DU, want_init=True)
    limits(t1, t2)
    elems = {}
    for lmk in (0, 1, 8):
        sg.sg_set_landmarks(lmk)
        s_gpu, ed = g.init_gains(128, "uic", 0.05, 99)
        assert np.array_equal(s_gpu, ref["s_init"]) and ed == int(ref["counters"][0])
        res = g.select(128, 8, "uic", 0.05, 99, stats=True)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])
        got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
        assert got == [int(x) for x in ref["counters"]]
        elems[lmk] = sum(res.stats["work_elems"][0])
    assert elems[8] < 0.5 * elems[0], elems


# ---------------------------------------------------------- full selection


@pytest.mark.parametrize("name", ["er2k_uic0.1", "cl15k_uic0.01", "cl15k_wic"])
def test_select_matches_oracle_on_workloads(sg, name):
    wl = inputs.workload(name)
    n, s, d = wl.graph()
    g, o = _both(sg, n, s, d, wl.model, wl.p)
    res = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
    ref = o.select(wl.R, wl.k, wl.seed, mode=oracle.DU)
    assert np.array_equal(res.seeds, ref["seeds"])
    assert np.array_equal(res.gains, ref["gains"])
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]]
    assert res.stats["status_flags"] == 0


EDGE_CASES = [
    # (label, graph, model, p, R, k)
    ("single_node", lambda: (1, np.zeros(0, np.int32), np.zeros(0, np.int32)), "uic", 0.5, 10, 1),
    ("no_arcs", lambda: (7, np.zeros(0, np.int32), np.zeros(0, np.int32)), "wic", 0.0, 70, 7),
    ("p0", lambda: inputs.er_directed(100, 500, 5), "uic", 0.0, 33, 6),
    ("p1_path", lambda: inputs.path_graph(40), "uic", 1.0, 64, 5),
    ("p1_star", lambda: inputs.out_star(300, centre=17), "uic", 1.0, 65, 4),
    ("k_equals_n", lambda: inputs.random_small(25, 80, 6), "uic", 0.4, 129, 25),
    ("R1", lambda: inputs.er_directed(200, 1000, 7), "uic", 0.2, 1, 10),
    ("R64", lambda: inputs.er_directed(200, 1000, 7), "wic", 0.0, 64, 10),
    ("loops_dups", lambda: inputs.random_small(80, 1500, 8, loops_and_dups=True), "wic", 0.0, 100, 12),
    ("two_trees", lambda: (50, np.r_[inputs.out_tree(20, 2)[1], inputs.out_tree(30, 1)[1] + 20],
                           np.r_[inputs.out_tree(20, 2)[2], inputs.out_tree(30, 1)[2] + 20]), "uic", 1.0, 3, 3),
]


def _coverage_reference(o, n, R, seed, S):
    """Coverage of S in every snapshot from the oracle's live masks (bits
    pinned to the coin definition) and a library breadth-first search:
    cov[w, u] bit b = u reached from S in snapshot 64w + b."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order

    W = (R + 63) // 64
    masks = o.live_masks(R, seed)
    src = np.repeat(np.arange(n), np.diff(o.rp)).astype(np.int64)
    dst = o.col[: o.m].astype(np.int64)
    cov = np.zeros((W, n), dtype=np.uint64)
    for r in range(R):
        live = ((masks[:, r // 64] >> np.uint64(r % 64)) & np.uint64(1)).astype(bool)
        # a virtual root n with an arc to every seed: one search from S
        rows = np.concatenate([src[live], np.full(len(S), n)])
        cols = np.concatenate([dst[live], np.asarray(S, dtype=np.int64)])
        A = sp.csr_matrix((np.ones(rows.size, dtype=np.int8), (rows, cols)), shape=(n + 1, n + 1))
        reached = breadth_first_order(A, n, directed=True, return_predecessors=False)
        reached = reached[reached < n]
        cov[r // 64, reached] |= np.uint64(1) << np.uint64(r % 64)
    return cov


@pytest.mark.parametrize("name,model,p,R,k", [("er2k", "uic", 0.1, 100, 10), ("cl15k", "wic", 0.0, 100, 20),
                                              ("cl15k", "lt", 0.0, 130, 12)])
def test_state_after_k_rounds_matches_oracle(sg, name, model, p, R, k):
    """The state Algorithm 2 maintains (Section 4) after its k rounds: the
    whole gain vector equals the oracle's DU vector (every non-seed's
    marginal gain f(S + u) - f(S), checked on a sample against the oracle's
    spread too; seeds negative), and the coverage bitsets equal the reach
    of S in every snapshot, from the oracle's live masks and a library
    breadth-first search (the last word masked to R mod 64)."""
    gens = {"er2k": lambda: inputs.er_directed(2000, 10000, 101),
            "cl15k": lambda: inputs.chung_lu_undirected(15000, 58000, 2.5, 7.7, 102)}
    n, s, d = gens[name]()
    g, o = _both(sg, n, s, d, model, p)
    seed = 77
    sel, s_gpu, cov = g.select_state(R, k, model, p, seed)
    ref = o.select(R, k, seed, mode=oracle.DU, want_hist=True)
    assert np.array_equal(sel.seeds, ref["seeds"]) and np.array_equal(sel.gains, ref["gains"])
    S = sel.seeds
    nonseed = np.ones(n, dtype=bool)
    nonseed[S] = False
    assert np.array_equal(s_gpu[nonseed], ref["s_hist"][k - 1][nonseed])
    assert np.all(s_gpu[S] < 0)
    fS = o.spread(R, seed, S)
    assert fS == int(sel.gains.sum())
    rng = np.random.default_rng(5)
    for u in rng.choice(np.flatnonzero(nonseed), 8, replace=False):
        assert s_gpu[u] == o.spread(R, seed, np.append(S, u)) - fS
    assert np.array_equal(cov, _coverage_reference(o, n, R, seed, S))
    assert sum(bin(int(x)).count("1") for x in cov.ravel()) == fS


@pytest.mark.parametrize("label,gen,model,p,R,k", EDGE_CASES, ids=[c[0] for c in EDGE_CASES])
def test_select_edge_cases(sg, label, gen, model, p, R, k):
    n, s, d = gen()
    g, o = _both(sg, n, s, d, model, p)
    res = g.select(R, k, model, p, 12345, stats=True)
    ref = o.select(R, k, 12345, mode=oracle.DU)
    assert np.array_equal(res.seeds, ref["seeds"]), label
    assert np.array_equal(res.gains, ref["gains"]), label
    got = [res.stats["init_edges"], res.stats["fwd_edges"], res.stats["rev_edges"]]
    assert got == [int(x) for x in ref["counters"]], label


def test_workspace_reuse_across_queries(sg):
    n, s, d = inputs.chung_lu_undirected(2000, 8000, 2.5, 8.0, 12)
    g = sg.Graph.from_coo(n, s, d)
    queries = [("wic", 0.0, 100, 10, 1), ("uic", 0.05, 256, 20, 2), ("uic", 0.02, 64, 5, 3), ("wic", 0.0, 130, 15, 4)]
    for model, p, R, k, seed in queries + queries[::-1]:
        res = g.select(R, k, model, p, seed)
        ref = oracle.Graph(n, s, d, model, p).select(R, k, seed, mode=oracle.DU)
        assert np.array_equal(res.seeds, ref["seeds"]) and np.array_equal(res.gains, ref["gains"])


def test_trim_releases_and_rebuilds_the_workspace(sg):
    wl = inputs.workload("cl15k_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    a = g.select(wl.R, 12, wl.model, wl.p, wl.seed)
    g.trim()
    g.trim()  # twice is fine
    b = g.select(wl.R, 12, wl.model, wl.p, wl.seed)
    assert np.array_equal(a.seeds, b.seeds) and np.array_equal(a.gains, b.gains)
    with pytest.raises(sg.SGError):
        sg.sg_graph_trim(None)


def test_device_outputs_and_stream(sg):
    import torch

    wl = inputs.workload("er2k_uic0.1")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    st = torch.cuda.Stream()
    seeds = torch.zeros(wl.k, dtype=torch.int32, device="cuda")
    gains = torch.zeros(wl.k, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(st):
        sg.sg_select(g.handle, wl.R, wl.k, wl.model, wl.p, wl.seed, seeds, gains, stream=st)
    st.synchronize()
    ref = oracle.Graph(n, s, d, wl.model, wl.p).select(wl.R, wl.k, wl.seed, mode=oracle.DU)
    assert np.array_equal(seeds.cpu().numpy(), ref["seeds"])
    assert np.array_equal(gains.cpu().numpy(), ref["gains"])


def test_invalid_queries_are_rejected(sg):
    n, s, d = inputs.er_directed(50, 200, 3)
    g = sg.Graph.from_coo(n, s, d)
    for R, k, model, p in [(0, 1, "uic", 0.1), (1 << 24, 1, "uic", 0.1), (10, 0, "uic", 0.1), (10, 51, "uic", 0.1),
                           (10, 1, "uic", 1.5), (10, 1, "uic", float("nan")), (10, 1, "uic", -0.1)]:
        with pytest.raises(sg.SGError) as ei:
            g.select(R, k, model, p, 1)
        assert ei.value.status == sg.SG_EINVAL
    with pytest.raises(sg.SGError):
        sg.Graph.from_coo(5, np.array([0, 7], np.int32), np.array([1, 2], np.int32))


# ------------------------------------------------- full size (R-MAT scale 20)


@pytest.fixture(scope="module")
def rmat20(sg):
    wl = inputs.workload("rmat20_wic")
    n, s, d = wl.graph()
    g = sg.Graph.from_coo(n, s, d)
    o = oracle.Graph(n, s, d, wl.model, wl.p)
    res = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
    return wl, g, o, res


@pytest.fixture(scope="module")
def rmat20_oracle(rmat20):
    """The oracle's whole selection on the full R-MAT scale-20 query (R = 256,
    k = 50, hash seed 11) by lazy forward evaluation (StaticGreedyCELF, the
    route the pins prove equal to Algorithm 2), with its initial gains."""
    wl, g, o, res = rmat20
    return o.select(wl.R, wl.k, wl.seed, mode=oracle.CELF, want_init=True)


def test_rmat20_seeds_and_gains_equal_oracle(sg, rmat20, rmat20_oracle):
    """Full size, no sampling: all 50 seeds and gains of sg_select equal the
    oracle's, as do the initial and forward snapshot-edge counters."""
    wl, g, o, res = rmat20
    ref = rmat20_oracle
    assert np.array_equal(res.seeds, ref["seeds"])
    assert np.array_equal(res.gains, ref["gains"])
    assert res.stats["init_edges"] == int(ref["counters"][0])
    assert res.stats["fwd_edges"] == int(ref["counters"][1])
    assert res.stats["status_flags"] == 0


def test_rmat20_full_initial_gains_equal_oracle(sg, rmat20, rmat20_oracle):
    """The whole 1,048,576-entry initial-gain vector (Algorithm 2, first
    loop) against the oracle's, element by element."""
    wl, g, o, res = rmat20
    s_gpu, e_gpu = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
    assert np.array_equal(s_gpu, rmat20_oracle["s_init"])
    assert e_gpu == int(rmat20_oracle["counters"][0])


def test_rmat20_served_requests_equal_oracle(sg, rmat20):
    """Full size through the server: two requests of the served trace's
    shape (R in {100, 200}, hash seeds 100000 + j) on the R-MAT scale-20
    graph, submitted together so that they overlap on the device; each
    one's seeds and gains equal the oracle's selection for the same query."""
    import time

    wl, g, o, res = rmat20
    reqs = [(100, 12, 100000), (200, 20, 100001)]
    srv = sg.sg_server_create(max_running=2, k_cap=32)
    try:
        ids = [(sg.sg_server_submit(srv, g.handle, R, k, wl.model, wl.p, seed), R, k, seed) for R, k, seed in reqs]
        got = {}
        deadline = time.time() + 300
        while len(got) < len(ids) and time.time() < deadline:
            for rid, R, k, seed in ids:
                if rid in got:
                    continue
                done, seeds, gains, _ = sg.sg_server_poll(srv, rid, k)
                if done:
                    got[rid] = (seeds, gains)
            time.sleep(0.01)
        assert len(got) == len(ids)
    finally:
        sg.sg_server_destroy(srv)
    for rid, R, k, seed in ids:
        ref = o.select(R, k, seed, mode=oracle.CELF)
        seeds, gains = got[rid]
        assert np.array_equal(seeds, ref["seeds"]), (R, k)
        assert np.array_equal(gains, ref["gains"]), (R, k)


def test_rmat20_gains_are_exact_marginals(sg, rmat20):
    wl, g, o, res = rmat20
    gains = res.gains
    assert np.all(np.diff(gains) <= 0)
    assert len(set(res.seeds.tolist())) == wl.k
    assert res.stats["status_flags"] == 0
    prev = 0
    for i in (1, 2, 5, 10, 25, 50):
        f = o.spread(wl.R, wl.seed, res.seeds[:i])
        assert f == int(gains[:i].sum()), i
        prev = f
    assert prev == int(gains.sum())


def test_rmat20_mask_cache_equals_in_register_coins(sg, rmat20, rmat20_oracle):
    """Full size: the live-mask cache gives the same seeds, gains and
    counters as in-register hashing, and the same full initial-gain vector
    as the oracle."""
    wl, g, o, res = rmat20
    sg.sg_set_mask_cache(1)
    try:
        r2 = g.select(wl.R, wl.k, wl.model, wl.p, wl.seed, stats=True)
        s_gpu, _ = g.init_gains(wl.R, wl.model, wl.p, wl.seed)
    finally:
        sg.sg_set_mask_cache(0)
    assert r2.stats["mask_cache"] == 1 and r2.stats["status_flags"] == 0
    assert np.array_equal(r2.seeds, res.seeds) and np.array_equal(r2.gains, res.gains)
    for key in ("init_edges", "fwd_edges", "rev_edges"):
        assert r2.stats[key] == res.stats[key]
    assert np.array_equal(s_gpu, rmat20_oracle["s_init"])


def test_rmat20_greedy_choice_beats_sampled_candidates(sg, rmat20):
    wl, g, o, res = rmat20
    rng = np.random.default_rng(7)
    for i in (0, 1, 9, 30):
        S = res.seeds[:i]
        fS = o.spread(wl.R, wl.seed, S) if i else 0
        for u in rng.choice(g.n, 12, replace=False):
            if u in res.seeds[: i + 1]:
                continue
            du = o.spread(wl.R, wl.seed, np.append(S, u)) - fS
            assert du < res.gains[i] or (du == res.gains[i] and u > res.seeds[i])
