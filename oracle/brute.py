"""Pure-Python brute force for tiny graphs (n <= 12, or m <= 16 arcs).

TEST INFRASTRUCTURE ONLY.  A second, independent route to the quantities
the C oracle computes, used to pin it: its own splitmix64, its own
canonicalisation, per-snapshot reachability as bitmask transitive closure
(no BFS), greedy by evaluating f over every candidate set, the optimum
over all k-subsets, and the exact expected spread by enumerating every
live-edge world with exact rational probabilities.

Paper: Cheng et al., "StaticGreedy" (CIKM'13).  f(S) = sum_r |R(G'_r, S)| is
the snapshot estimate of Section 3.1 (times R); greedy is Algorithm 1; the
(1 - 1/e) guarantee and the monotone / submodular definitions are those of
Section 3.2 (Nemhauser et al. 1978).
"""

from __future__ import annotations

import itertools
import math
from fractions import Fraction

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def canonical_arcs(src, dst):
    """Sorted distinct (u, v) arcs with u != v; index = canonical arc id."""
    return sorted({(int(u), int(v)) for u, v in zip(src, dst) if int(u) != int(v)})


def coin_ids(arcs, model):
    """The value each arc's coin hashes: its own index; for the undirected
    variant ("uic_undirected") the smaller index of the arc and its reverse;
    for the linear threshold model ("lt") the arc's destination (one draw
    per node decides which in-arc it keeps)."""
    if model == "lt":
        return [v for _, v in arcs]
    if model != "uic_undirected":
        return list(range(len(arcs)))
    index = {a: i for i, a in enumerate(arcs)}
    out = []
    for i, (u, v) in enumerate(arcs):
        if (v, u) not in index:
            raise ValueError("uic_undirected needs a symmetric graph")
        out.append(min(i, index[(v, u)]))
    return out


def intervals(n, arcs, model, p=0.0):
    """Kept interval [lo, hi) of each arc's 32-bit draw: [0, thr) for the
    cascades; for "lt", node v's in-arcs in order of source own consecutive
    intervals of width floor(2^32 / indeg(v)) (Kempe et al.'s live-edge
    linear threshold model with weights 1/indeg)."""
    if model != "lt":
        return [(0, t) for t in thresholds(n, arcs, model, p)]
    indeg = [0] * n
    for _, v in arcs:
        indeg[v] += 1
    seen = [0] * n
    out = []
    for _, v in arcs:  # canonical order: sources ascending
        w = (1 << 32) // indeg[v]
        out.append((seen[v] * w, (seen[v] + 1) * w))
        seen[v] += 1
    return out


def thresholds(n, arcs, model, p=0.0):
    """thr(e) in [0, 2^32]: floor(p 2^32) (UIC) or floor(2^32 / indeg(v)) (WIC)."""
    if model in ("uic", "uic_undirected"):
        t = math.floor(Fraction(p) * (1 << 32))
        return [t] * len(arcs)
    indeg = [0] * n
    for _, v in arcs:
        indeg[v] += 1
    return [(1 << 32) // indeg[v] for _, v in arcs]


def coin(seed, r, e, thr) -> bool:
    return (splitmix64((seed ^ (r << 40) ^ e) & MASK64) >> 32) < thr


def coin_range(seed, r, key, lo, hi) -> bool:
    h = splitmix64((seed ^ (r << 40) ^ key) & MASK64) >> 32
    return lo <= h < hi


def closure(n, live_arcs):
    """reach[v] bitmask (v included) by Warshall's transitive closure."""
    reach = [1 << v for v in range(n)]
    for u, v in live_arcs:
        reach[u] |= 1 << v
    for k in range(n):
        bk = 1 << k
        rk = reach[k]
        for i in range(n):
            if reach[i] & bk:
                reach[i] |= rk
    return reach


class Brute:
    """All snapshots of a tiny graph as reach bitmasks."""

    def __init__(self, n, src, dst, model, p, R, seed):
        self.n = n
        self.arcs = canonical_arcs(src, dst)
        iv = intervals(n, self.arcs, model, p)
        cid = coin_ids(self.arcs, model)
        self.R = R
        self.reach = []
        for r in range(R):
            live = [a for e, a in enumerate(self.arcs) if coin_range(seed, r, cid[e], *iv[e])]
            self.reach.append(closure(n, live))

    def f(self, S) -> int:
        tot = 0
        for reach in self.reach:
            cov = 0
            for v in S:
                cov |= reach[v]
            tot += bin(cov).count("1")
        return tot

    def greedy(self, k):
        """Algorithm 1 by direct evaluation of f; ties to the lowest id."""
        S, gains = [], []
        for _ in range(k):
            base = self.f(S)
            best, bestv = None, -1
            for v in range(self.n):
                if v in S:
                    continue
                val = self.f(S + [v])
                if best is None or val > best:
                    best, bestv = val, v
            S.append(bestv)
            gains.append(best - base)
        return S, gains

    def optimum(self, k) -> int:
        return max(self.f(list(T)) for T in itertools.combinations(range(self.n), k))


def exact_spread(n, src, dst, model, p, S):
    """Exact I(S) and Var(|R(S)|) over all 2^m live-edge worlds, with arc e
    kept with probability q_e = thr_e / 2^32 (the discretised probability the
    hash realises).  Returns (mean, variance) as Fractions."""
    arcs = canonical_arcs(src, dst)
    thr = thresholds(n, arcs, model, p)
    q = [Fraction(t, 1 << 32) for t in thr]
    cid = coin_ids(arcs, model)
    coins = sorted(set(cid))           # one independent coin per id (an edge, when coupled)
    slot = {c: i for i, c in enumerate(coins)}
    m = len(coins)
    mean = Fraction(0)
    second = Fraction(0)
    for world in range(1 << m):
        prob = Fraction(1)
        for i, c in enumerate(coins):
            prob *= q[c] if world >> i & 1 else 1 - q[c]
        live = [a for e, a in enumerate(arcs) if world >> slot[cid[e]] & 1]
        if prob == 0:
            continue
        reach = closure(n, live)
        cov = 0
        for v in S:
            cov |= reach[v]
        c = bin(cov).count("1")
        mean += prob * c
        second += prob * c * c
    return mean, second - mean * mean


def exact_spread_lt(n, src, dst, S):
    """Exact I(S) and Var(|R(S)|) under the live-edge linear threshold model
    with weights 1/indeg: every node independently keeps one of its d in-arcs,
    each with probability w/2^32 (w = floor(2^32/d), the discretised weight
    the hash realises), or none with the remaining probability; enumerates
    every combination of choices with exact rationals."""
    arcs = canonical_arcs(src, dst)
    ins = [[] for _ in range(n)]
    for u, v in arcs:
        ins[v].append(u)
    options = []
    for v in range(n):
        d = len(ins[v])
        if d == 0:
            options.append([(None, Fraction(1))])
            continue
        w = Fraction((1 << 32) // d, 1 << 32)
        opts = [(u, w) for u in ins[v]]
        rest = 1 - d * w
        if rest:
            opts.append((None, rest))
        options.append(opts)
    mean = Fraction(0)
    second = Fraction(0)
    for choice in itertools.product(*options):
        prob = Fraction(1)
        live = []
        for v, (u, q) in enumerate(choice):
            prob *= q
            if u is not None:
                live.append((u, v))
        reach = closure(n, live)
        cov = 0
        for v in S:
            cov |= reach[v]
        c = bin(cov).count("1")
        mean += prob * c
        second += prob * c * c
    return mean, second - mean * mean
