"""rr_evaluate_noalloc: the same light curves as rr_evaluate, with no allocation.

Some callers cannot allocate device memory when they evaluate (for example
code running where CUDA allocation calls are not allowed, or an application
that has handed all device memory to its own allocator); this entry point
uses scratch memory that the library holds in a fixed array instead of a
caller-provided workspace.  The test calls it through the C ABI twice in a
row, on different inputs, the second batch smaller than the first (so the
second call runs over the first call's leftovers in the shared array), and
compares each result with rr_evaluate bitwise (the same kernels, on the
fixed array instead of a workspace); it also checks that a call changes
neither the device's free memory nor torch's allocated bytes.  The cases
cover the interpolated and direct models and a batch of 8 passbands.  It
sits in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


def _call_noalloc(rr, m, t, pb, p, wl, out, status):
    """rr_evaluate_noalloc through the C ABI (ctypes), on the current stream."""
    import torch
    ss = np.ascontiguousarray(wl.supersampling, np.int32)
    ex = np.ascontiguousarray(wl.exptime, np.float64)
    st = m.lib.rr_evaluate_noalloc(m._h, t.data_ptr(), pb.data_ptr(), t.numel(), p.data_ptr(), p.shape[0],
                                   ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.data_ptr(),
                                   status.data_ptr(), torch.cuda.current_stream().cuda_stream or None)
    return st


def _cases(kind):
    """Two batches for one model, the second smaller than the first (so that it runs over the
    first call's leftovers in the shared array)."""
    if kind == "interpolated":
        return [W.make_small("quadratic_tri", npv=40, npt=3000, seed=3, ss=(5,), exptime=(0.01,)),
                W.make_small("quadratic_tri", npv=7, npt=1100, seed=4)]
    if kind == "direct":
        return [W.make_small("quadratic", npv=30, npt=2500, seed=5, ss=(3,), exptime=(0.01,), direct=True),
                W.make_small("quadratic", npv=6, npt=900, seed=6, direct=True)]
    ss, ex = (1, 3, 5, 1, 3, 5, 1, 3), (0.0, 0.01, 0.02, 0.0, 0.01, 0.02, 0.0, 0.01)
    first = W.make_small("tabulated", npv=24, npt=4000, npb=8, seed=7, ss=ss, exptime=ex)
    second = W.make_small("tabulated", npv=5, npt=1500, npb=8, seed=8, ss=ss, exptime=ex)
    second.profiles = first.profiles      # one model: the first batch's profiles
    return [first, second]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("kind", ["interpolated", "direct", "8 passbands"])
def test_noalloc_matches_evaluate_on_two_calls_in_a_row(rr, kind, precision):
    """Bitwise the light curves of rr_evaluate (the same kernels on another scratch address), and
    no allocation: the device's free memory and torch's allocated bytes unchanged by each call."""
    import torch
    cases = _cases(kind)
    m = None
    for wl in cases:
        wl.precision = precision
        if m is None:
            m = rr.model_for(wl)
        t, pb, p = rr.to_device(wl)
        ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime)
        out = torch.full_like(ref, -7.0)
        status = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
        # the first call on the device looks up the array's address (and may load the module)
        assert _call_noalloc(rr, m, t, pb, p, wl, out, status) == 0, m.lib.rr_last_error(m._h)
        torch.cuda.synchronize()
        out.fill_(-7.0)
        status.fill_(-1)
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert _call_noalloc(rr, m, t, pb, p, wl, out, status) == 0, m.lib.rr_last_error(m._h)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        assert torch.all(status == 0)
        assert torch.equal(out, ref)
        assert (ref < 1).sum().item() > 50


def test_noalloc_rejects_batches_beyond_its_fixed_scratch(rr):
    import torch
    wl = W.make_small("quadratic", npv=2, npt=10)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    big = 200_000
    need = m.workspace_bytes(big, 10)
    assert need > (32 << 20)
    pbig = p[:1].repeat(big, 1).contiguous()
    out = torch.empty((big, 10), dtype=torch.float32, device=t.device)
    status = torch.empty(big, dtype=torch.int32, device=t.device)
    n0 = m.launch_count
    st = _call_noalloc(rr, m, t, pb, pbig, wl, out, status)
    assert st == 1
    assert b"scratch" in m.lib.rr_last_error(m._h)
    assert m.launch_count == n0
