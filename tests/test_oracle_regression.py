"""The oracle still computes what tests/golden/oracle_regression.txt
recorded (seeds, gains, the three snapshot-edge counters, CELF evaluation
counts, a spread).  The file is written by
tests/golden/make_oracle_regression.py from the oracle alone; a change to
the oracle's arithmetic fails here until the file is regenerated with the
change justified."""

import importlib.util
import os

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _recorded():
    rec = {}
    for line in open(os.path.join(GOLDEN, "oracle_regression.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, key, *vals = line.split()
        rec[(name, key)] = [int(v) for v in vals]
    return rec


def test_oracle_matches_its_recorded_results():
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(GOLDEN, "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rec = _recorded()
    got = {(name, key): vals for name, key, vals in mod.compute()}
    assert set(got) == set(rec)
    for k in sorted(rec):
        assert got[k] == rec[k], k
