"""rr_prepare + rr_evaluate_prepared / rr_evaluate_grad_prepared: one shared set-up
for a forward and an adjoint on the same batch, bitwise equal to the separate calls."""
import numpy as np
import pytest

from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    return _rr


CASES = [("quadratic_tri", 1, False, (1,), "mixed"), ("nonlinear", 1, False, (7,), "mixed"),
         ("quadratic", 3, True, (1, 5, 12), "mixed"), ("tabulated", 4, False, (1, 3, 1, 9), "mixed"),
         ("quadratic", 2, True, (1, 4), "fp64")]


@pytest.mark.parametrize("ld,npb,chromatic,ss,precision", CASES)
def test_prepared_equals_separate_calls(rr, ld, npb, chromatic, ss, precision):
    import torch
    wl = W.make_small(ld, npv=45, npt=2100, npb=npb, chromatic=chromatic, ss=ss,
                      exptime=tuple(0.02 for _ in ss), seed=5, precision=precision)
    wl.params[7, 2] = 0.5                      # a <= 1: invalid pv (NaN row, status bit)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st_ref = torch.empty(wl.npv, dtype=torch.int32, device=t.device)
    f_ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st_ref)
    gbar = torch.as_tensor(np.random.default_rng(1).normal(size=(wl.npv, wl.npt)), dtype=m.dtype, device=t.device)
    g_ref = m.evaluate_grad(t, p, gbar, pb, wl.supersampling, wl.exptime)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    ws = m.prepare(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st, prepared=ws)
    g = m.evaluate_grad(t, p, gbar, pb, wl.supersampling, wl.exptime, prepared=ws)
    torch.cuda.synchronize()
    assert torch.equal(st, st_ref) and st[7].item() != 0
    assert torch.equal(torch.nan_to_num(f, nan=-1.0), torch.nan_to_num(f_ref, nan=-1.0))
    assert torch.equal(torch.nan_to_num(g, nan=-1.0), torch.nan_to_num(g_ref, nan=-1.0))
    assert (f < 1).sum().item() > 100
    # the same workspace evaluated twice more gives the same again
    f2 = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, prepared=ws)
    assert torch.equal(torch.nan_to_num(f2, nan=-1.0), torch.nan_to_num(f_ref, nan=-1.0))


@pytest.mark.parametrize("ld,npb,chromatic,ss,precision", CASES)
def test_both_on_two_streams_equals_separate_calls(rr, ld, npb, chromatic, ss, precision):
    """rr_evaluate_both_prepared (the adjoint on the context's second stream beside the forward
    kernel): bitwise the separate prepared calls, status words included, and ordered on the
    caller's stream (a kernel enqueued after it sees both results)."""
    import torch
    wl = W.make_small(ld, npv=45, npt=2100, npb=npb, chromatic=chromatic, ss=ss,
                      exptime=tuple(0.02 for _ in ss), seed=6, precision=precision)
    wl.params[3, 2] = 0.5                      # a <= 1: invalid pv (NaN row, status bit)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    gbar = torch.as_tensor(np.random.default_rng(2).normal(size=(wl.npv, wl.npt)), dtype=m.dtype, device=t.device)
    st_ref = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    ws = m.prepare(t, p, pb, wl.supersampling, wl.exptime, pv_status=st_ref)
    f_ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st_ref, prepared=ws)
    g_ref = m.evaluate_grad(t, p, gbar, pb, wl.supersampling, wl.exptime, prepared=ws)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    ws2 = m.prepare(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    f, g = m.evaluate_both(t, p, gbar, ws2, pb, wl.supersampling, wl.exptime, pv_status=st)
    sums = torch.stack([torch.nan_to_num(f.double()).sum(), torch.nan_to_num(g).sum()])   # on the caller's stream
    torch.cuda.synchronize()
    assert torch.equal(st, st_ref) and st[3] != 0
    assert torch.equal(torch.nan_to_num(f, nan=-1.0), torch.nan_to_num(f_ref, nan=-1.0))
    assert torch.equal(torch.nan_to_num(g, nan=-1.0), torch.nan_to_num(g_ref, nan=-1.0))
    assert torch.equal(sums, torch.stack([torch.nan_to_num(f_ref.double()).sum(), torch.nan_to_num(g_ref).sum()]))


def test_prepared_autograd_and_small_workspace(rr):
    import torch
    wl = W.make_small("quadratic_tri", npv=12, npt=900, seed=9)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    pg = p.clone().requires_grad_(True)
    f = m.flux(t, pg, pb, wl.supersampling, wl.exptime)
    w = torch.linspace(-1, 1, wl.npt, device=t.device, dtype=torch.float32)
    (f * w).sum().backward()
    g_ref = m.evaluate_grad(t, p, (w.expand(wl.npv, -1)).contiguous(), pb, wl.supersampling, wl.exptime)
    assert torch.equal(pg.grad, g_ref)
    small = m.workspace(wl.npv, wl.npt, False)
    if small.numel() < m.workspace_bytes(wl.npv, wl.npt, True):
        with pytest.raises(rr.RRError, match="workspace too small"):
            m.prepare(t, p, pb, wl.supersampling, wl.exptime, workspace=small)
