"""Failure detection on the GPU without a fault, trap or hang.

Each device-side wait of the kernels is bounded; when it runs out the kernel
records which wait gave up in the context's error word and returns.  The
self-test kernel makes each kind of wait run out on a flag that nothing sets;
the host then reads RR_ETIMEOUT, and the same context evaluates normally
afterwards.
"""
import time

import numpy as np
import pytest

from oracle import model as om
from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


@pytest.mark.parametrize("which,words", [(0, "staging copy"), (1, "work queue")])
def test_bounded_wait_runs_out_and_is_reported(rr, which, words):
    import torch
    wl = W.make_small("quadratic", npv=5, npt=700, seed=3)
    m = rr.model_for(wl)
    t0 = time.perf_counter()
    m.selftest_wait(which)
    with pytest.raises(rr.RRError) as ei:
        m.sync_status()
    assert ei.value.status == 6 and "RR_ETIMEOUT" in str(ei.value)
    assert words in str(ei.value)
    assert time.perf_counter() - t0 < 10.0          # bounded: about a second at most
    # the indicator is reset and the context still evaluates correctly
    m.sync_status()
    t, pb, p = rr.to_device(wl)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).double().cpu().numpy()
    torch.cuda.synchronize()
    ref = om.evaluate_workload(wl)
    assert np.abs(f - ref).max() <= 1e-6


def test_selftest_rejects_unknown_kind(rr):
    wl = W.make_small("quadratic", npv=1, npt=10, seed=3)
    m = rr.model_for(wl)
    with pytest.raises(rr.RRError):
        m.selftest_wait(7)
