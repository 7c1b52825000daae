"""The host graph builders (canonical CSR, CSC by a stable counting sort)
against numpy on random graphs with repeats, self-loops, unsorted and empty
rows, for several host thread counts (the results must not depend on it)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1212_4779_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("hgb") / "host_graph_build_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC, os.path.join(HERE, "host_graph_build_check.cpp"),
                    "-o", out], check=True)
    return out


def _random_csr(n, m, seed):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, n, m)
    # skewed destinations, some self-loops and repeats; rows left unsorted
    dst = np.minimum((rng.pareto(1.2, m) * 7).astype(np.int64), n - 1)
    dst = np.where(rng.random(m) < 0.01, src, dst)
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    return np.cumsum(rp), dst.astype(np.int32)


def _reference(n, rp, col):
    rows, cols = [], []
    for u in range(n):
        r = np.unique(col[rp[u]:rp[u + 1]])
        r = r[r != u]
        rows.append(np.full(r.size, u, dtype=np.int64))
        cols.append(r)
    src = np.concatenate(rows)
    dst = np.concatenate(cols).astype(np.int64)
    rpc = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rpc, src + 1, 1)
    rpc = np.cumsum(rpc)
    idx = np.argsort(dst, kind="stable")  # CSR order is (source, arc id)
    crp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(crp, dst + 1, 1)
    return rpc, dst, np.cumsum(crp), src[idx], idx


def _run(checker, tmp_path, n, rp, col, threads):
    inp, outp = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    with open(inp, "wb") as f:
        f.write(np.array([n, col.size], dtype=np.int64).tobytes())
        f.write(rp.astype(np.int64).tobytes())
        f.write(col.astype(np.int32).tobytes())
    subprocess.run([checker, inp, outp, str(threads)], check=True)
    raw = open(outp, "rb").read()
    mc = int(np.frombuffer(raw[:8], dtype=np.int64)[0])
    a = np.frombuffer(raw[8:], dtype=np.int32)
    rpc, a = a[:n + 1], a[n + 1:]
    colc, a = a[:mc], a[mc:]
    crp, a = a[:n + 1], a[n + 1:]
    cin = a[:2 * mc].reshape(mc, 2)
    return rpc, colc, crp, cin


@pytest.mark.parametrize("n,m,seed", [(5000, 1_200_000, 1), (7, 0, 2), (4099, 30_000, 3), (1, 5, 4)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_canonical_csr_and_stable_csc(checker, tmp_path, n, m, seed, threads):
    rp, col = _random_csr(n, m, seed)
    rpc, colc, crp, cin = _run(checker, tmp_path, n, rp, col, threads)
    ref_rp, ref_col, ref_crp, ref_src, ref_eid = _reference(n, rp, col)
    assert np.array_equal(rpc, ref_rp)
    assert np.array_equal(colc, ref_col)
    assert np.array_equal(crp, ref_crp)
    assert np.array_equal(cin[:, 0], ref_src)
    assert np.array_equal(cin[:, 1], ref_eid)
