"""Failure reporting, tested without a GPU fault.

sg_debug_inject_flags plants, into the next query, the device flags that a
failing device step leaves: a bounded wait that gave up (2) or a failed
consistency check (1, 8).  Every kind of call must report it.
- Synchronous calls return SG_ETIMEOUT / SG_EINTERNAL.
- Asynchronous calls leave seeds of -1 and gains of -flags.
- The server turns those outputs into the request's status.
Each test then checks that the next query on the same context is exact
again.  No kernel is made to wait, fault or trap."""

import time

import numpy as np
import pytest

import oracle
from paper_1212_4779_gb300 import inputs

pytestmark = pytest.mark.gpu

R, K, P, SEED = 100, 8, 0.1, 5


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1212_4779_gb300 import sg as _sg

    return _sg


@pytest.fixture(scope="module")
def case(sg):
    n, s, d = inputs.er_directed(600, 3000, 11)
    g = sg.Graph.from_coo(n, s, d)
    want = oracle.Graph(n, s, d, "uic", P).select(R, K, SEED, want_init=True)
    yield g, want
    sg.sg_debug_inject_flags(0)
    g.close()


def _exact(g, want):
    r = g.select(R, K, "uic", P, SEED)
    assert np.array_equal(r.seeds, want["seeds"])
    assert np.array_equal(r.gains, want["gains"])


@pytest.mark.parametrize("flags,status", [(2, "SG_ETIMEOUT"), (3, "SG_ETIMEOUT"), (1, "SG_EINTERNAL"),
                                          (8, "SG_EINTERNAL")])
def test_synchronous_select_returns_the_status(sg, case, flags, status):
    g, want = case
    sg.sg_debug_inject_flags(flags)
    with pytest.raises(sg.SGError) as e:
        g.select(R, K, "uic", P, SEED)  # pageable host outputs: returns after the stream
    assert e.value.status == getattr(sg, status)
    _exact(g, want)


def test_select_with_stats_returns_the_status(sg, case):
    g, want = case
    sg.sg_debug_inject_flags(2)
    with pytest.raises(sg.SGError) as e:
        g.select(R, K, "uic", P, SEED, stats=True)
    assert e.value.status == sg.SG_ETIMEOUT
    _exact(g, want)


def test_asynchronous_select_marks_its_outputs(sg, case):
    import torch

    g, want = case
    so = torch.zeros(K, dtype=torch.int32, device="cuda")
    go = torch.zeros(K, dtype=torch.int64, device="cuda")
    sg.sg_debug_inject_flags(2)
    sg.sg_select(g.handle, R, K, "uic", P, SEED, so, go)  # device outputs: returns once enqueued
    torch.cuda.synchronize()
    assert (so.cpu().numpy() == -1).all()
    assert (go.cpu().numpy() == -2).all()
    sg.sg_select(g.handle, R, K, "uic", P, SEED, so, go)
    torch.cuda.synchronize()
    assert np.array_equal(so.cpu().numpy(), want["seeds"])
    assert np.array_equal(go.cpu().numpy(), want["gains"])


def test_initial_gains_report_the_failure(sg, case):
    import torch

    g, want = case
    s = torch.zeros(g.n, dtype=torch.int64, device="cuda")
    sg.sg_debug_inject_flags(2)
    sg.sg_init_gains(g.handle, R, "uic", P, SEED, s)
    torch.cuda.synchronize()
    assert (s.cpu().numpy() == -2).all()
    sg.sg_debug_inject_flags(1)
    with pytest.raises(sg.SGError) as e:
        g.init_gains(R, "uic", P, SEED)
    assert e.value.status == sg.SG_EINTERNAL
    s_ok, _ = g.init_gains(R, "uic", P, SEED)
    assert np.array_equal(s_ok, want["s_init"])


def test_celf_returns_the_status(sg, case):
    g, want = case
    sg.sg_debug_inject_flags(2)
    with pytest.raises(sg.SGError) as e:
        g.select_celf(R, K, "uic", P, SEED)
    assert e.value.status == sg.SG_ETIMEOUT
    res, _ = g.select_celf(R, K, "uic", P, SEED)
    assert np.array_equal(res.seeds, want["seeds"])
    assert np.array_equal(res.gains, want["gains"])


def test_undirected_select_returns_the_status(sg):
    n, s, d = inputs.symmetric(*inputs.er_directed(400, 1200, 12))
    g = sg.Graph.from_coo(n, s, d)
    try:
        want = oracle.Graph(n, s, d, "uic_undirected", 0.2).select(64, 6, 3)
        sg.sg_debug_inject_flags(2)
        with pytest.raises(sg.SGError) as e:
            g.select(64, 6, "uic_undirected", 0.2, 3)
        assert e.value.status == sg.SG_ETIMEOUT
        r = g.select(64, 6, "uic_undirected", 0.2, 3)
        assert np.array_equal(r.seeds, want["seeds"])
        assert np.array_equal(r.gains, want["gains"])
    finally:
        g.close()


def _wait(sg, srv, rid):
    deadline = time.time() + 60
    while time.time() < deadline:
        done, seeds, gains, _ = sg.sg_server_poll(srv, rid, K)
        if done:
            return seeds, gains
        time.sleep(0.005)
    pytest.fail("request never finished")


def test_server_request_reports_the_status(sg, case):
    g, want = case
    srv = sg.sg_server_create(max_running=2, k_cap=16)
    try:
        sg.sg_debug_inject_flags(2)
        rid = sg.sg_server_submit(srv, g.handle, R, K, "uic", P, SEED)
        with pytest.raises(sg.SGError) as e:
            _wait(sg, srv, rid)
        assert e.value.status == sg.SG_ETIMEOUT
        rid = sg.sg_server_submit(srv, g.handle, R, K, "uic", P, SEED)
        seeds, gains = _wait(sg, srv, rid)
        assert np.array_equal(seeds, want["seeds"])
        assert np.array_equal(gains, want["gains"])
    finally:
        sg.sg_server_destroy(srv)


def test_real_bounded_wait_runs_out_and_reports_timeout(sg):
    """A real device wait running out, without a fault: every task is sent to
    the block-shared engines (tier limits of one key), whose idle warps poll
    the block's queue while one warp expands; with the wait budget cut to one
    poll they give up, set the wait flag and return.  The call reports
    SG_ETIMEOUT; with the default budget restored the next query on the same
    context is exact again (the engines clean their state on the way out)."""
    n, s, d = inputs.workload("cl15k_wic").graph()
    g = sg.Graph.from_coo(n, s, d)
    want = oracle.Graph(n, s, d, "wic").select(100, 10, 7)
    try:
        sg.sg_set_engine_limits(1, 1)
        sg.sg_debug_set_wait_limit(1)
        with pytest.raises(sg.SGError) as e:
            g.select(100, 10, "wic", 0.0, 7, stats=True)
        assert e.value.status == sg.SG_ETIMEOUT
        with pytest.raises(sg.SGError) as e:
            g.init_gains(100, "wic", 0.0, 7)
        assert e.value.status == sg.SG_ETIMEOUT
    finally:
        sg.sg_debug_set_wait_limit(0)
    try:
        r = g.select(100, 10, "wic", 0.0, 7, stats=True)  # still all in the block-shared engines
        assert r.stats["status_flags"] == 0
        assert np.array_equal(r.seeds, want["seeds"]) and np.array_equal(r.gains, want["gains"])
    finally:
        sg.sg_set_engine_limits(64, 2048)
    r = g.select(100, 10, "wic", 0.0, 7)
    assert np.array_equal(r.seeds, want["seeds"]) and np.array_equal(r.gains, want["gains"])
    g.close()
