"""Model.evaluate_host: host buffers in and out, pv chunks pipelined over copy and compute streams.

The results must be bitwise those of one device call on the whole batch (a
pv's flux and gradient do not depend on the other pvs of the launch)."""
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


@pytest.mark.parametrize("ld,npb,ss,chunk", [("quadratic_tri", 1, (1,), 16), ("nonlinear", 1, (5,), 7),
                                             ("tabulated", 3, (1, 4, 9), 32)])
def test_host_pipeline_matches_one_device_call(rr, ld, npb, ss, chunk):
    import torch
    wl = W.make_small(ld, npv=77, npt=2300, npb=npb, ss=ss, exptime=tuple(0.01 for _ in ss), seed=11)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu()
    gbar = np.random.default_rng(3).normal(size=(wl.npv, wl.npt)).astype(np.float32)
    gref = m.evaluate_grad(t, p, torch.as_tensor(gbar, device=t.device), pb, wl.supersampling, wl.exptime).cpu()
    # pageable numpy inputs, ragged last chunk
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, grad_flux=gbar,
                               chunk_pvs=chunk)
    assert torch.equal(f, ref)
    assert torch.equal(g, gref)
    assert not st.any()
    # forward only, pinned result buffers, one chunk
    out = torch.empty_like(ref).pin_memory()
    f2, g2, _ = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, out=out,
                                chunk_pvs=1000)
    assert g2 is None and f2.data_ptr() == out.data_ptr() and torch.equal(f2, ref)


def test_host_pipeline_status_and_empty(rr):
    wl = W.make_small("quadratic", npv=9, npt=300, seed=2)
    wl.params[4, 4] = 1.5                      # e outside [0, 1): NaN light curve + status bit
    m = rr.model_for(wl)
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, chunk_pvs=4)
    assert st[4] != 0 and np.isnan(f[4].numpy()).all()
    assert (st.numpy()[np.arange(9) != 4] == 0).all()
    f0, _, st0 = m.evaluate_host(wl.times, wl.params[:0], wl.pb_index, wl.supersampling, wl.exptime)
    assert f0.shape == (0, 300) and st0.shape == (0,)


def test_default_chunking_of_a_large_batch_matches_one_device_call(rr):
    """The default chunking (about eight chunks of at least 512 pvs) on a batch of several chunks."""
    import torch
    wl = W.make_small("quadratic_tri", npv=2100, npt=256, seed=29)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu()
    gbar = np.random.default_rng(7).normal(size=(wl.npv, wl.npt)).astype(np.float32)
    gref = m.evaluate_grad(t, p, torch.as_tensor(gbar, device=t.device), pb, wl.supersampling, wl.exptime).cpu()
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, grad_flux=gbar)
    assert torch.equal(f, ref)
    assert torch.equal(torch.nan_to_num(g, nan=-1.0), torch.nan_to_num(gref, nan=-1.0))
    f2, _, st2 = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime)
    assert torch.equal(f2, ref) and torch.equal(st2, st)
