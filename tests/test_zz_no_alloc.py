"""The allocation-free argmax entry point agrees with sg_select.

Callers that cannot allocate device memory where they need the argmax --
latency-bound serving loops that must not stall on an allocation, plug-ins
whose host framework owns all device memory -- use sg_argmax_noalloc, whose only
scratch is a statically sized device array shared by every call.  These
tests call it through the C ABI on two gain vectors in a row (the second
call sees the first call's leftover scratch) and compare with the seed and
gain that sg_select picks first on the same graph: integers, so equal."""

import ctypes

import numpy as np
import pytest

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


def _call(sg, s_dev, out_id, out_gain, stream):
    rc = sg.lib().sg_argmax_noalloc(ctypes.c_void_p(s_dev.data_ptr()), s_dev.numel(),
                                    ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out_id.data_ptr()),
                                    ctypes.c_void_p(out_gain.data_ptr()))
    assert rc == sg.SG_OK, sg.sg_last_error()


def test_noalloc_argmax_matches_select_twice_in_a_row(sg):
    import torch

    stream = torch.cuda.current_stream()
    out_id = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    out_gain = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    for name in ("cl15k_wic", "er2k_uic0.1"):
        wl = inputs.workload(name)
        n, s, d = wl.graph()
        g = sg.Graph.from_coo(n, s, d)
        s_dev = torch.zeros(n, dtype=torch.int64, device="cuda")
        sg.sg_init_gains(g.handle, wl.R, wl.model, wl.p, wl.seed, s_dev, stream=stream)
        _call(sg, s_dev, out_id, out_gain, stream)
        stream.synchronize()
        ref = g.select(wl.R, 1, wl.model, wl.p, wl.seed)
        assert int(out_id.item()) == int(ref.seeds[0])
        assert int(out_gain.item()) == int(ref.gains[0])
        g.close()


def test_noalloc_argmax_ties_exclusions_and_bounds(sg):
    import torch

    stream = torch.cuda.current_stream()
    out_id = torch.zeros(1, dtype=torch.int32, device="cuda")
    out_gain = torch.zeros(1, dtype=torch.int64, device="cuda")
    rng = np.random.default_rng(3)
    for n in (1, 255, 256, 257, 100_000, 3_000_000):
        host = rng.integers(0, 50, size=n).astype(np.int64)
        host[rng.random(n) < 0.3] = -(1 << 62)  # excluded entries, as sg_select marks seeds
        _call(sg, torch.from_numpy(host).cuda(), out_id, out_gain, stream)
        stream.synchronize()
        ok = host >= 0
        if ok.any():
            best = host[ok].max()
            assert int(out_gain.item()) == int(best)
            assert int(out_id.item()) == int(np.flatnonzero(host == best)[0])
        else:
            assert int(out_id.item()) == -1 and int(out_gain.item()) == -1
    L = sg.lib()
    assert L.sg_argmax_noalloc(ctypes.c_void_p(out_gain.data_ptr()), 0, None, ctypes.c_void_p(out_id.data_ptr()),
                               ctypes.c_void_p(out_gain.data_ptr())) == sg.SG_EINVAL
    assert L.sg_argmax_noalloc(None, 5, None, None, None) == sg.SG_EINVAL
