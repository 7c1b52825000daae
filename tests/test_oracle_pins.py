"""Pins for the CPU oracle: each checks it against something other than
itself -- published test vectors, exact arithmetic, closed forms on graphs
whose reach sets are known, a pure-Python brute force over all subsets,
exact expectations over all live-edge worlds, and the monotone/submodular
invariants of Section 3.2 of the paper.

These tests need no GPU."""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1212_4779_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ the hash


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(t, 0) for t in line.split()])
    return rows


def test_splitmix64_published_vectors(oracle_mod):
    rows = _golden_rows("splitmix64.txt")
    assert len(rows) == 4
    for x, want in rows:
        assert oracle.splitmix64(x) == want
        assert brute.splitmix64(x) == want


def test_coin_word_layout(oracle_mod):
    """The coin of (e, r) hashes seed XOR (r << 40) XOR e and keeps the arc
    iff the high 32 bits are below thr; checked against the Python restatement
    for ids beyond 2^32, snapshots up to 2^24 - 1 and the threshold ends."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        seed = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        r = int(rng.integers(0, 2**24))
        e = int(rng.integers(0, 2**40))
        thr = int(rng.integers(0, 2**32 + 1))
        assert oracle.live(seed, r, e, thr) == brute.coin(seed, r, e, thr)
        assert oracle.live(seed, r, e, 1 << 32)
        assert not oracle.live(seed, r, e, 0)
    # the high word alone decides: a value just above / at the hash's hi32
    x = 0x1234 ^ (77 << 40) ^ 99
    hi = brute.splitmix64(x) >> 32
    assert oracle.live(0x1234, 77, 99, hi + 1)
    assert not oracle.live(0x1234, 77, 99, hi)


@pytest.mark.parametrize("R", [1, 63, 64, 65, 130])
@pytest.mark.parametrize("model,p", [("uic", 0.3), ("wic", 0.0), ("uic_undirected", 0.4), ("lt", 0.0)])
def test_live_masks_bit_by_bit(oracle_mod, R, model, p):
    """or_live_masks against the pure-Python coin, bit by bit: bit b of word
    w of arc e is the coin of snapshot 64w + b (Section 3.1 snapshot; reading
    A9: snapshots 0..R-1, the last word masked to R mod 64 bits), for every
    arc and snapshot of a small graph, including the word boundary cases."""
    if model == "uic_undirected":
        n, s, d = inputs.chung_lu_undirected(40, 90, 2.5, 4.0, 11)
    else:
        n, s, d = inputs.random_small(40, 160, 9)
    g = oracle.Graph(n, s, d, model, p)
    seed = 0xF00DFACE12345 ^ R
    masks = g.live_masks(R, seed)
    W = (R + 63) // 64
    assert masks.shape == (g.m, W)
    arcs = brute.canonical_arcs(s, d)
    assert len(arcs) == g.m
    iv = brute.intervals(n, arcs, model, p)
    cid = brute.coin_ids(arcs, model)
    for e in range(g.m):
        for w in range(W):
            want = 0
            for b in range(64):
                r = 64 * w + b
                if r < R and brute.coin_range(seed, r, cid[e], *iv[e]):
                    want |= 1 << b
            assert int(masks[e, w]) == want, (e, w)


@pytest.mark.parametrize("p,want", [(0.1, 429496729), (0.01, 42949672), (0.02, 85899345),
                                    (0.05, 214748364), (0.0, 0), (1.0, 1 << 32), (0.5, 1 << 31)])
def test_uic_threshold_exact(oracle_mod, p, want):
    g = oracle.Graph(3, [0, 1], [1, 2], "uic", p)
    assert math.floor(Fraction(p) * (1 << 32)) == want
    assert list(g.thr[: g.m]) == [want, want]


def test_wic_threshold_is_integer_quotient(oracle_mod):
    # node 4 has in-degree 1, node 5 in-degree 3, node 6 in-degree 7
    src = [0, 0, 1, 2, 0, 1, 2, 3, 7, 8, 9]
    dst = [4, 5, 5, 5, 6, 6, 6, 6, 6, 6, 6]
    g = oracle.Graph(10, src, dst, "wic")
    want = {4: 1 << 32, 5: 1431655765, 6: 613566756}
    for e in range(g.m):
        assert int(g.thr[e]) == want[int(g.col[e])] == (1 << 32) // {4: 1, 5: 3, 6: 7}[int(g.col[e])]


def _sigma_check(count, mean, var, k=6.0):
    assert abs(count - mean) <= k * math.sqrt(var) + 1e-9, (count, mean, var)


def test_coin_frequency_uic(oracle_mod):
    """~10^6 coins at p = 0.1: the kept fraction, per 64-snapshot word and per
    out-degree bucket, is within 6 sigma of the binomial expectation."""
    n, s, d = inputs.er_directed(4000, 7813, 3)
    g = oracle.Graph(n, s, d, "uic", 0.1)
    R = 128
    masks = g.live_masks(R, seed=12345)
    q = 429496729 / 2**32
    bits = np.unpackbits(masks.view(np.uint8), axis=1)  # (m, 16*8)
    tot = int(bits.sum())
    N = g.m * R
    _sigma_check(tot, N * q, N * q * (1 - q))
    for w in range(2):
        cw = int(np.unpackbits(np.ascontiguousarray(masks[:, w]).view(np.uint8)).sum())
        _sigma_check(cw, g.m * 64 * q, g.m * 64 * q * (1 - q))
    outdeg = np.diff(g.rp)
    src_of = np.repeat(np.arange(n), outdeg)
    per_arc = bits.sum(axis=1)
    for lo, hi in [(0, 2), (2, 4), (4, 100)]:
        sel = (outdeg[src_of] >= lo) & (outdeg[src_of] < hi)
        c = int(per_arc[sel].sum())
        N2 = int(sel.sum()) * R
        _sigma_check(c, N2 * q, N2 * q * (1 - q))


def test_coin_frequency_wic(oracle_mod):
    n, s, d = inputs.chung_lu_undirected(3000, 12000, 2.5, 8.0, 4)
    g = oracle.Graph(n, s, d, "wic")
    R = 64
    masks = g.live_masks(R, seed=99)
    q = g.thr[: g.m].astype(np.float64) / 2**32
    kept = np.unpackbits(masks.view(np.uint8), axis=1).sum(axis=1)
    _sigma_check(int(kept.sum()), float(q.sum()) * R, float((q * (1 - q)).sum()) * R)
    indeg = np.bincount(g.col[: g.m], minlength=n)
    # every node with an in-arc expects exactly one kept in-arc per snapshot
    per_dst = np.bincount(g.col[: g.m], weights=kept, minlength=n)
    has = indeg > 0
    _sigma_check(float(per_dst[has].sum()), float(has.sum()) * R,
                 float((q * (1 - q)).sum()) * R)
    # in-degree-1 destinations keep their arc in every snapshot
    one = np.where(indeg[g.col[: g.m]] == 1)[0]
    assert np.all(kept[one] == R)


# --------------------------------------------------------- canonicalisation


def test_canonicalisation_drops_loops_and_repeats(oracle_mod):
    for seed in range(5):
        n, s, d = inputs.random_small(30, 400, seed, loops_and_dups=True)
        g = oracle.Graph(n, s, d, "uic", 0.5)
        want = brute.canonical_arcs(s, d)
        got = [(u, int(g.col[e])) for u in range(n) for e in range(g.rp[u], g.rp[u + 1])]
        assert got == want
        assert g.m == len(want)


# ------------------------------------------------------------- closed forms


MODES = [oracle.LITERAL, oracle.COVER, oracle.DU, oracle.CELF]


@pytest.mark.parametrize("mode", MODES)
def test_p0_every_node_reaches_itself_only(oracle_mod, mode):
    n, s, d = inputs.er_directed(60, 300, 8)
    g = oracle.Graph(n, s, d, "uic", 0.0)
    out = g.select(R=7, k=5, seed=1, mode=mode, want_init=(mode != oracle.LITERAL))
    assert list(out["seeds"]) == [0, 1, 2, 3, 4]
    assert list(out["gains"]) == [7] * 5
    if mode != oracle.LITERAL:
        assert np.all(out["s_init"] == 7)


@pytest.mark.parametrize("mode", MODES)
def test_p1_path(oracle_mod, mode):
    n, s, d = inputs.path_graph(12)
    R = 3
    g = oracle.Graph(n, s, d, "uic", 1.0)
    out = g.select(R=R, k=4, seed=5, mode=mode, want_init=(mode != oracle.LITERAL))
    if mode != oracle.LITERAL:
        assert list(out["s_init"]) == [R * (n - i) for i in range(n)]
    assert list(out["seeds"]) == [0, 1, 2, 3]
    assert list(out["gains"]) == [R * n, 0, 0, 0]


@pytest.mark.parametrize("mode", MODES)
def test_p1_out_star(oracle_mod, mode):
    n, s, d = inputs.out_star(20, centre=7)
    g = oracle.Graph(n, s, d, "uic", 1.0)
    out = g.select(R=5, k=4, seed=3, mode=mode)
    assert list(out["seeds"]) == [7, 0, 1, 2]
    assert list(out["gains"]) == [5 * 20, 0, 0, 0]


def test_spread_closed_forms(oracle_mod):
    """p = 1: the spread of a seed set is R times the nodes it reaches, and
    its snapshot-edge count R times their out-degree sum (path: a suffix;
    out-star: everything from the centre, the leaf alone otherwise)."""
    n, s, d = inputs.path_graph(12)
    g = oracle.Graph(n, s, d, "uic", 1.0)
    for S, reach in (([0], 12), ([5], 7), ([9, 3], 9), ([11], 1)):
        tot, ed = g.spread(6, 2, S, want_edges=True)
        assert tot == 6 * reach and ed == 6 * (reach - 1)
    n, s, d = inputs.out_star(20, centre=7)
    g = oracle.Graph(n, s, d, "uic", 1.0)
    assert g.spread(3, 1, [7], want_edges=True) == (3 * 20, 3 * 19)
    assert g.spread(3, 1, [4], want_edges=True) == (3, 0)
    assert g.spread(3, 1, [4, 7, 9], want_edges=True) == (3 * 20, 3 * 19)
    # p = 0: the seeds alone, and the out-degrees of the seeds are scanned
    g = oracle.Graph(n, s, d, "uic", 0.0)
    assert g.spread(5, 1, [7, 2], want_edges=True) == (10, 5 * 19)


def test_celf_evaluation_count_on_path(oracle_mod):
    """p = 1 path, lazy evaluation with the (bound desc, id asc) queue:
    round 0 takes node 0 straight from the initial gains (it covers
    everything).  In round 1 every other node's bound R(n - i) exceeds the
    true gain 0, so all n - 1 are evaluated before the lowest id (bound 0,
    fresh) is taken; in each later round the head is the lowest remaining
    id with a stale bound 0, evaluated once and taken: (n - 1) + (k - 2)
    evaluations."""
    n, s, d = inputs.path_graph(12)
    g = oracle.Graph(n, s, d, "uic", 1.0)
    out = g.select(R=3, k=4, seed=5, mode=oracle.CELF)
    assert out["evals"] == 11 + 2
    assert list(out["seeds"]) == [0, 1, 2, 3] and list(out["gains"]) == [36, 0, 0, 0]
    # an out-star: the centre first, then the 8 leaves (bound R each) are
    # all evaluated in round 1, one head evaluation in each later round
    n, s, d = inputs.out_star(9, centre=4)
    g = oracle.Graph(n, s, d, "uic", 1.0)
    out = g.select(R=2, k=4, seed=1, mode=oracle.CELF)
    assert list(out["seeds"]) == [4, 0, 1, 2] and list(out["gains"]) == [18, 0, 0, 0]
    assert out["evals"] == 8 + 2


def _subtree_sizes(n, parent_of):
    size = [1] * n
    for v in range(n - 1, 0, -1):  # parent < child
        size[parent_of[v]] += size[v]
    return size


def test_p1_out_tree(oracle_mod):
    n, s, d = inputs.out_tree(80, seed=4)
    parent_of = {int(c): int(p) for p, c in zip(s, d)}
    size = _subtree_sizes(n, parent_of)
    g = oracle.Graph(n, s, d, "wic")  # every node has in-degree <= 1: all arcs kept
    out = g.select(R=4, k=2, seed=9, mode=oracle.DU, want_init=True)
    assert list(out["s_init"]) == [4 * x for x in size]
    assert out["seeds"][0] == 0 and out["gains"][0] == 4 * n
    assert out["gains"][1] == 0 and out["seeds"][1] == 1


def test_p1_two_disjoint_trees(oracle_mod):
    n1, s1, d1 = inputs.out_tree(30, seed=1)
    n2, s2, d2 = inputs.out_tree(20, seed=2)
    s = np.concatenate([s2, s1 + n2])
    d = np.concatenate([d2, d1 + n2])
    g = oracle.Graph(n1 + n2, s, d, "uic", 1.0)
    for mode in MODES:
        out = g.select(R=3, k=3, seed=2, mode=mode)
        assert list(out["seeds"][:2]) == [n2, 0]
        assert list(out["gains"]) == [3 * n1, 3 * n2, 0]


def test_p1_connected_undirected(oracle_mod):
    n, s, d = inputs.chung_lu_undirected(40, 200, 2.5, 8.0, 6)
    # make it connected with a path through all nodes (both directions)
    p = np.arange(n - 1, dtype=np.int32)
    s = np.concatenate([s, p, p + 1])
    d = np.concatenate([d, p + 1, p])
    g = oracle.Graph(n, s, d, "uic", 1.0)
    out = g.select(R=6, k=5, seed=4, mode=oracle.DU, want_init=True)
    assert np.all(out["s_init"] == 6 * n)
    assert list(out["seeds"]) == [0, 1, 2, 3, 4]
    assert list(out["gains"]) == [6 * n, 0, 0, 0, 0]


# -------------------------------------------------------------- brute force


BRUTE_CASES = [
    (9, 18, "uic", 0.4, 1),
    (10, 25, "uic", 0.3, 2),
    (11, 22, "wic", 0.0, 3),
    (12, 30, "wic", 0.0, 4),
    (8, 20, "uic", 0.6, 5),
    (12, 16, "uic", 0.5, 6),
]


@pytest.mark.parametrize("n,m,model,p,gseed", BRUTE_CASES)
def test_greedy_matches_brute_force(oracle_mod, n, m, model, p, gseed):
    _, s, d = inputs.random_small(n, m, gseed, loops_and_dups=True)
    R, k, seed = 20, 4, 1000 + gseed
    b = brute.Brute(n, s, d, model, p, R, seed)
    bs, bg = b.greedy(k)
    g = oracle.Graph(n, s, d, model, p)
    for mode in MODES:
        out = g.select(R=R, k=k, seed=seed, mode=mode)
        assert list(out["seeds"]) == bs, mode
        assert list(out["gains"]) == bg, mode
    # f(S_k) >= (1 - 1/e) max_{|T|=k} f(T)  (Nemhauser et al.)
    opt = b.optimum(k)
    assert sum(bg) == b.f(bs)
    assert sum(bg) >= (1 - 1 / math.e) * opt
    # initial gains are the single-node spreads
    s_init = g.select(R=R, k=1, seed=seed, mode=oracle.DU, want_init=True)["s_init"]
    assert list(s_init) == [b.f([v]) for v in range(n)]


@pytest.mark.parametrize("model,p", [("uic", 0.3), ("wic", 0.0)])
def test_snapshot_mean_matches_exact_expectation(oracle_mod, model, p):
    """With R = 2^16 snapshots the mean of |R(G'_r, S)| lies within 5 sigma/sqrt(R)
    of the exact expected spread I(S), summed over all 2^m live-edge worlds."""
    n, s, d = inputs.random_small(7, 13, 11, loops_and_dups=False)
    R = 1 << 16
    g = oracle.Graph(n, s, d, model, p)
    assert g.m <= 16
    for S in ([0], [1, 4], [2, 3, 6]):
        mean, var = brute.exact_spread(n, s, d, model, p, S)
        est = Fraction(g.spread(R, seed=77, S=S), R)
        assert abs(float(est - mean)) <= 5 * math.sqrt(float(var)) / math.sqrt(R) + 1e-12


# ------------------------------------- linear threshold model (live-edge form)


LT_CASES = [(9, 20, 1), (10, 24, 2), (11, 18, 3), (12, 26, 4)]


@pytest.mark.parametrize("n,m,gseed", LT_CASES)
def test_lt_greedy_matches_brute_force(oracle_mod, n, m, gseed):
    """Live-edge linear threshold snapshots (one kept in-arc per node at
    most): every route of the oracle gives the brute-force greedy (own
    intervals, Warshall closure), within the Nemhauser bound."""
    _, s, d = inputs.random_small(n, m, gseed, loops_and_dups=True)
    R, k, seed = 24, 4, 700 + gseed
    b = brute.Brute(n, s, d, "lt", 0.0, R, seed)
    bs, bg = b.greedy(k)
    g = oracle.Graph(n, s, d, "lt")
    for mode in MODES:
        out = g.select(R=R, k=k, seed=seed, mode=mode)
        assert list(out["seeds"]) == bs, mode
        assert list(out["gains"]) == bg, mode
    assert sum(bg) >= (1 - 1 / math.e) * b.optimum(k)
    s_init = g.select(R=R, k=1, seed=seed, mode=oracle.DU, want_init=True)["s_init"]
    assert list(s_init) == [b.f([v]) for v in range(n)]


def test_lt_keeps_at_most_one_in_arc(oracle_mod):
    """Per snapshot every node keeps at most one in-arc, exactly one when its
    in-degree is a power of two (the intervals then tile 2^32), and each arc
    is kept with probability floor(2^32/d)/2^32 (within 6 sigma)."""
    n, s, d = inputs.chung_lu_undirected(2000, 8000, 2.5, 8.0, 5)
    g = oracle.Graph(n, s, d, "lt")
    R = 192
    masks = g.live_masks(R, seed=404)
    bits = np.unpackbits(masks.view(np.uint8), axis=1, bitorder="little")[:, :R]  # (m, R)
    col = g.col[: g.m]
    indeg = np.bincount(col, minlength=n)
    per_node = np.zeros((n, R), dtype=np.int64)
    np.add.at(per_node, col, bits.astype(np.int64))
    assert per_node.max() <= 1
    pow2 = (indeg > 0) & ((indeg & (indeg - 1)) == 0)
    assert np.all(per_node[pow2] == 1)
    q = ((1 << 32) // indeg[col]).astype(np.float64) / 2**32
    kept = bits.sum(axis=1)
    _sigma_check(int(kept.sum()), float(q.sum()) * R, float((q * (1 - q)).sum()) * R)


def test_lt_closed_forms(oracle_mod):
    """A directed path: every node has one in-arc, kept always, so
    s_i = R (n - i).  An in-star of 4 sources into c (in-degree 4, a power of
    two): in each snapshot exactly one source reaches c, so the sources'
    initial gains sum to 4R + R and c's is R."""
    n, s, d = inputs.path_graph(7)
    g = oracle.Graph(n, s, d, "lt")
    s_init = g.select(R=50, k=1, seed=3, mode=oracle.DU, want_init=True)["s_init"]
    assert list(s_init) == [50 * (n - i) for i in range(n)]
    g = oracle.Graph(5, [0, 1, 2, 3], [4, 4, 4, 4], "lt")
    for R, seed in ((64, 1), (100, 9), (333, 12345)):
        s_init, _ = g.init_gains(R, seed)
        assert int(s_init[:4].sum()) == 5 * R and int(s_init[4]) == R


def test_lt_snapshot_mean_matches_exact_expectation(oracle_mod):
    """R = 2^16 snapshots: the mean of |R(G'_r, S)| lies within 5 sigma/sqrt(R)
    of the exact linear-threshold spread, enumerated over every combination
    of per-node in-arc choices (Kempe et al.'s live-edge equivalence)."""
    n, s, d = inputs.random_small(6, 11, 17, loops_and_dups=False)
    g = oracle.Graph(n, s, d, "lt")
    R = 1 << 16
    for S in ([0], [1, 3], [2, 4, 5]):
        mean, var = brute.exact_spread_lt(n, s, d, S)
        est = Fraction(g.spread(R, seed=55, S=S), R)
        assert abs(float(est - mean)) <= 5 * math.sqrt(float(var)) / math.sqrt(R) + 1e-12


# ------------------------------------------- undirected variant (coupled coins)


COUPLED_CASES = [(9, 12, 0.4, 1), (10, 15, 0.3, 2), (12, 14, 0.5, 3), (8, 10, 0.6, 4)]


@pytest.mark.parametrize("n,m,p,gseed", COUPLED_CASES)
def test_coupled_greedy_matches_brute_force(oracle_mod, n, m, p, gseed):
    """One coin per undirected edge: every route of the oracle gives the
    brute-force greedy (own coupling, Warshall closure)."""
    _, s0, d0 = inputs.random_small(n, m, gseed)
    _, s, d = inputs.symmetric(n, s0, d0)
    R, k, seed = 24, 4, 500 + gseed
    b = brute.Brute(n, s, d, "uic_undirected", p, R, seed)
    bs, bg = b.greedy(k)
    g = oracle.Graph(n, s, d, "uic_undirected", p)
    for mode in MODES:
        out = g.select(R=R, k=k, seed=seed, mode=mode)
        assert list(out["seeds"]) == bs, mode
        assert list(out["gains"]) == bg, mode
    s_init = g.select(R=R, k=1, seed=seed, mode=oracle.DU, want_init=True)["s_init"]
    assert list(s_init) == [b.f([v]) for v in range(n)]
    # coupled snapshots are undirected: u reaches v iff v reaches u
    for reach in b.reach:
        for u in range(n):
            for v in range(n):
                assert bool(reach[u] >> v & 1) == bool(reach[v] >> u & 1)


def test_coupled_masks_pair_up(oracle_mod):
    n, s0, d0 = inputs.random_small(40, 120, 9)
    _, s, d = inputs.symmetric(n, s0, d0)
    g = oracle.Graph(n, s, d, "uic_undirected", 0.3)
    gu = oracle.Graph(n, s, d, "uic", 0.3)
    masks, masks_u = g.live_masks(130, 5), gu.live_masks(130, 5)
    rp, col = g.rp, g.col
    src_of = np.repeat(np.arange(n), np.diff(rp))
    index = {(int(u), int(v)): e for e, (u, v) in enumerate(zip(src_of, col[: g.m]))}
    differ = 0
    for e, (u, v) in enumerate(zip(src_of, col[: g.m])):
        r = index[(int(v), int(u))]
        assert np.array_equal(masks[e], masks[r])
        assert np.array_equal(masks[min(e, r)], masks_u[min(e, r)])  # the lower arc keeps its own coin
        differ += not np.array_equal(masks_u[e], masks_u[r])
    assert differ > 0  # uncoupled arcs of an edge disagree somewhere


def test_coupled_snapshot_mean_matches_exact_expectation(oracle_mod):
    """R = 2^16 coupled snapshots: the mean of |R(G'_r, S)| lies within 5
    sigma/sqrt(R) of the exact expectation over all 2^(m/2) edge worlds."""
    n, s0, d0 = inputs.random_small(7, 9, 13)
    _, s, d = inputs.symmetric(n, s0, d0)
    g = oracle.Graph(n, s, d, "uic_undirected", 0.4)
    assert g.m // 2 <= 16
    R = 1 << 16
    for S in ([0], [2, 5]):
        mean, var = brute.exact_spread(n, s, d, "uic_undirected", 0.4, S)
        est = Fraction(g.spread(R, seed=31, S=S), R)
        assert abs(float(est - mean)) <= 5 * math.sqrt(float(var)) / math.sqrt(R) + 1e-12


def test_coupled_rejects_asymmetric_graph(oracle_mod):
    n, s, d = inputs.path_graph(5)
    with pytest.raises(oracle.OracleError):
        oracle.Graph(n, s, d, "uic_undirected", 0.5)


# ----------------------------------------------------------------- invariants


@pytest.fixture(scope="module")
def medium_graphs(oracle_mod):
    n, s, d = inputs.chung_lu_undirected(2500, 9000, 2.5, 7.2, 21)
    return {
        "wic": oracle.Graph(n, s, d, "wic"),
        "uic": oracle.Graph(n, s, d, "uic", 0.05),
        "lt": oracle.Graph(n, s, d, "lt"),
    }


@pytest.mark.parametrize("model", ["wic", "uic", "lt"])
def test_du_matches_recompute_and_invariants(medium_graphs, model):
    g = medium_graphs[model]
    R, k, seed = 64, 15, 31
    du = g.select(R=R, k=k, seed=seed, mode=oracle.DU, want_init=True, want_hist=True)
    cv = g.select(R=R, k=k, seed=seed, mode=oracle.COVER)
    assert list(du["seeds"]) == list(cv["seeds"])
    assert list(du["gains"]) == list(cv["gains"])
    ce = g.select(R=R, k=k, seed=seed, mode=oracle.CELF)
    assert list(du["seeds"]) == list(ce["seeds"]) and list(du["gains"]) == list(ce["gains"])
    assert 0 < ce["evals"] < (k - 1) * g.n  # lazy: far fewer than recomputing every candidate
    gains = du["gains"]
    assert np.all(np.diff(gains) <= 0), "greedy gains of a submodular f are non-increasing"
    assert len(set(du["seeds"].tolist())) == k
    # sum of gains = f(S_k), by an independent multi-source BFS
    assert int(gains.sum()) == g.spread(R, seed, du["seeds"])
    # prefix spreads give each gain
    for i in range(1, k + 1, 4):
        assert int(gains[:i].sum()) == g.spread(R, seed, du["seeds"][:i])
    # initial gains equal on-demand reach sums; init counter equals theirs
    vs = np.arange(g.n, dtype=np.int32)
    sums, ed = g.reach_sums(R, seed, vs)
    assert np.array_equal(sums, du["s_init"])
    assert ed == int(du["counters"][0])
    # DU-maintained gains after round i are the marginal gains w.r.t. S_i
    rng = np.random.default_rng(3)
    for i in (0, 5, k - 1):
        S_i = du["seeds"][: i + 1]
        fS = g.spread(R, seed, S_i)
        for v in rng.choice(g.n, 6, replace=False):
            if v in S_i:
                continue
            assert du["s_hist"][i][v] == g.spread(R, seed, np.append(S_i, v)) - fS


def test_submodular_and_monotone(medium_graphs):
    g = medium_graphs["uic"]
    R, seed = 32, 8
    rng = np.random.default_rng(1)
    for _ in range(12):
        T = rng.choice(g.n, 10, replace=False)
        S = T[: rng.integers(0, 10)]
        v = int(rng.integers(0, g.n))
        while v in T:
            v = int(rng.integers(0, g.n))
        fS, fT = g.spread(R, seed, S), g.spread(R, seed, T)
        dS = g.spread(R, seed, np.append(S, v)) - fS
        dT = g.spread(R, seed, np.append(T, v)) - fT
        assert dS >= dT >= 0
        assert fT >= fS


def test_init_gains_split_over_snapshot_slices(medium_graphs):
    g = medium_graphs["wic"]
    full, e_full = g.init_gains(R=96, seed=4)
    a, ea = g.init_gains(R=96, seed=4, r0=0, r1=40)
    b, eb = g.init_gains(R=96, seed=4, r0=40, r1=96)
    assert np.array_equal(full, a + b) and e_full == ea + eb


def test_du_counters_against_definitions(oracle_mod):
    """Forward counter = sum over newly covered (u, r) of outdeg(u), i.e. the
    init-style count of the final seed set; reverse counter = sum over
    newly covered (w, r) and u reaching w of indeg(u) (brute force)."""
    n, s, d = inputs.random_small(10, 26, 9)
    R, k, seed = 16, 3, 5
    g = oracle.Graph(n, s, d, "uic", 0.45)
    out = g.select(R=R, k=k, seed=seed, mode=oracle.DU)
    b = brute.Brute(n, s, d, "uic", 0.45, R, seed)
    outdeg = np.diff(g.rp)
    indeg = np.bincount(g.col[: g.m], minlength=n)
    fwd = rev = 0
    for reach in b.reach:
        cov = 0
        for v in out["seeds"]:
            cov |= reach[int(v)]
        for w in range(n):
            if cov >> w & 1:
                fwd += int(outdeg[w])
                rev += sum(int(indeg[u]) for u in range(n) if reach[u] >> w & 1)
    init = sum(int(outdeg[x]) for reach in b.reach for v in range(n) for x in range(n) if reach[v] >> x & 1)
    assert list(map(int, out["counters"])) == [init, fwd, rev]


def test_literal_du_cover_agree_on_er_workload(oracle_mod):
    wl = inputs.workload("er2k_uic0.1")
    n, s, d = wl.graph()
    g = oracle.Graph(n, s, d, wl.model, wl.p)
    outs = [g.select(R=wl.R, k=wl.k, seed=wl.seed, mode=m) for m in MODES]
    for o in outs[1:]:
        assert list(o["seeds"]) == list(outs[0]["seeds"])
        assert list(o["gains"]) == list(outs[0]["gains"])
