"""Writes oracle_regression.txt: the oracle's results on small seeded
workloads, a lock against unintended changes to its arithmetic.

These values are not pins to the paper (the oracle's own pins are in
test_oracle_pins.py); they record what the pinned oracle computes, so that
any later change to it shows up as a failing comparison and has to be
justified when this file is regenerated.  Calls only the oracle and the
seeded generators.  Run from the repository root:

    python tests/golden/make_oracle_regression.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1212_4779_gb300 import inputs  # noqa: E402

# (case, graph builder, model, p, R, k, hash seed)
CASES = [
    ("er2k_uic0.1", lambda: inputs.workload("er2k_uic0.1").graph(), "uic", 0.1, 100, 10, 1),
    ("cl15k_uic0.01", lambda: inputs.workload("cl15k_uic0.01").graph(), "uic", 0.01, 100, 50, 7),
    ("cl15k_wic", lambda: inputs.workload("cl15k_wic").graph(), "wic", 0.0, 100, 50, 7),
    ("er400_undirected0.2", lambda: inputs.symmetric(*inputs.er_directed(400, 1200, 12)), "uic_undirected",
     0.2, 64, 6, 3),
]
SPREAD = ("er2k_uic0.1", 1000, 77)  # case, fresh snapshots, hash seed


def compute():
    out = []
    seeds_of = {}
    for name, gen, model, p, R, k, seed in CASES:
        n, s, d = gen()
        g = oracle.Graph(n, s, d, model, p)
        du = g.select(R, k, seed, mode=oracle.DU)
        out.append((name, "seeds", [int(x) for x in du["seeds"]]))
        out.append((name, "gains", [int(x) for x in du["gains"]]))
        out.append((name, "counters", [int(x) for x in du["counters"]]))
        if model != "uic_undirected":
            celf = g.select(R, k, seed, mode=oracle.CELF)
            out.append((name, "celf_evals", [int(celf["evals"])]))
        seeds_of[name] = (g, du["seeds"])
    name, R, seed = SPREAD
    g, S = seeds_of[name]
    total, edges = g.spread(R, seed, S, want_edges=True)
    out.append((name, f"spread_R{R}_seed{seed}", [int(total), int(edges)]))
    return out


def main():
    lines = ["# Oracle results on small seeded workloads (written by make_oracle_regression.py).",
             "# case key values..."]
    for name, key, vals in compute():
        lines.append(" ".join([name, key] + [str(v) for v in vals]))
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
