"""Host buffers in and out (rr_evaluate_host, rr_enqueue_host).

The Python binding pins what it is given, so its calls take the in-place
path; the staged path is reached through the C ABI with numpy buffers.

Page-locked buffers are read and written in place by the kernels; any other
host memory goes through the staged path (pv chunks pipelined over copy and
compute streams).  Both must give bitwise the results of one device call on
the whole batch (a pv's flux and gradient do not depend on the other pvs of
the launch)."""
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
    # numpy inputs (the binding pins them: the in-place path, chunk_pvs unused)
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, grad_flux=gbar,
                               chunk_pvs=chunk)
    assert m.host_path == "in place"
    assert torch.equal(f, ref)
    assert torch.equal(g, gref)
    assert not st.any()
    # forward only, pinned result buffers
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
    """A batch of several default chunks (about eight chunks of at least 512 pvs): in place through
    the binding, and staged (pageable buffers through the C ABI, default chunking)."""
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
    g64 = gbar.astype(np.float32)
    flux = np.zeros((wl.npv, wl.npt), np.float32)
    gp = np.zeros((wl.npv, m.nparam))
    status = np.full(wl.npv, -1, np.int32)
    assert _c_host_call(m, wl, g64, flux, gp, status, 0) == 0
    assert m.host_path == "staged"
    assert torch.equal(torch.from_numpy(flux), ref)
    assert torch.equal(torch.nan_to_num(torch.from_numpy(gp), nan=-1.0), torch.nan_to_num(gref, nan=-1.0))


def _c_host_call(m, wl, gbar, flux, grad, status, chunk):
    """rr_evaluate_host through the C ABI on numpy (pageable) buffers: the staged path."""
    P = ctypes.c_void_p
    ss = np.ascontiguousarray(np.broadcast_to(np.asarray(wl.supersampling, np.int32), (m.npb,)))
    ex = np.ascontiguousarray(np.broadcast_to(np.asarray(wl.exptime, np.float64), (m.npb,)))
    t = np.ascontiguousarray(wl.times, np.float64)
    pb = np.ascontiguousarray(wl.pb_index, np.int32)
    p = np.ascontiguousarray(wl.params, np.float64)
    return m.lib.rr_evaluate_host(m._h, t.ctypes.data, pb.ctypes.data, wl.npt, p.ctypes.data, wl.npv,
                                  ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  None if gbar is None else gbar.ctypes.data, flux.ctypes.data,
                                  None if grad is None else grad.ctypes.data, P(status.ctypes.data), chunk)


@pytest.mark.parametrize("ld,npb,ss", [("quadratic_tri", 1, (1,)), ("tabulated", 3, (1, 4, 9))])
def test_in_place_and_staged_paths_agree_with_one_device_call(rr, ld, npb, ss):
    """Pinned buffers (in place: the kernels read the cotangent and write the light curves and
    gradient over the host link) and pageable numpy buffers (staged copies, ragged chunks) give
    bitwise the results of the device entry points."""
    import torch
    wl = W.make_small(ld, npv=61, npt=3001, npb=npb, ss=ss, exptime=tuple(0.01 for _ in ss), seed=13)
    wl.params[5, 4] = 1.5                      # e outside [0, 1): NaN light curve + status bit
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu()
    gbar = np.random.default_rng(5).normal(size=(wl.npv, wl.npt)).astype(np.float32)
    gref = m.evaluate_grad(t, p, torch.as_tensor(gbar, device=t.device), pb, wl.supersampling, wl.exptime).cpu()
    nan_eq = lambda a, b: torch.equal(torch.nan_to_num(a, nan=-9.0), torch.nan_to_num(b, nan=-9.0))  # noqa: E731
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, grad_flux=gbar)
    assert m.host_path == "in place"
    assert f.is_pinned() and nan_eq(f, ref) and nan_eq(g, gref)
    assert st[5] != 0 and (st.numpy()[np.arange(wl.npv) != 5] == 0).all()
    for grad in (False, True):
        flux = np.full((wl.npv, wl.npt), -3.0, np.float32)
        gp = np.zeros((wl.npv, m.nparam)) if grad else None
        status = np.full(wl.npv, -1, np.int32)
        assert _c_host_call(m, wl, gbar if grad else None, flux, gp, status, 13) == 0
        assert m.host_path == "staged"
        assert nan_eq(torch.from_numpy(flux), ref) and np.array_equal(status, st.numpy())
        if grad:
            assert nan_eq(torch.from_numpy(gp), gref)


@pytest.mark.parametrize("case", [dict(ld_model="quadratic", precision="fp64", ss=(3,), exptime=(0.01,)),
                                  dict(ld_model="nonlinear", direct=True, ss=(1,), exptime=(0.0,)),
                                  dict(ld_model="quadratic", npb=2, chromatic=True, ss=(1, 5), exptime=(0.0, 0.02)),
                                  dict(ld_model="tabulated", npb=2, ss=(1, 4), exptime=(0.0, 0.01), precision="fp64")],
                         ids=["fp64", "direct", "chromatic", "tabulated-fp64"])
def test_in_place_matches_device_call_across_forms(rr, case):
    """In place on pinned buffers for the FP64 kernels (which read each time through the read-only
    path), the direct model and chromatic radius ratios: bitwise the device entry points."""
    import torch
    precision = case.pop("precision", "mixed")
    wl = W.make_small(npv=23, npt=1703, seed=19, **case)
    wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu()
    gbar = np.random.default_rng(2).normal(size=(wl.npv, wl.npt)).astype(np.float32 if precision == "mixed" else np.float64)
    gref = m.evaluate_grad(t, p, torch.as_tensor(gbar, device=t.device), pb, wl.supersampling, wl.exptime).cpu()
    f, g, st = m.evaluate_host(wl.times, wl.params, wl.pb_index, wl.supersampling, wl.exptime, grad_flux=gbar)
    assert m.host_path == "in place"
    assert torch.equal(f, ref) and torch.equal(g, gref) and not st.any()


def test_enqueue_host_in_place_and_staged(rr):
    """rr_enqueue_host on pinned tensors (in place) and on pageable numpy buffers (staged copies)."""
    import torch
    wl = W.make_small("nonlinear", npv=19, npt=2222, ss=(3,), exptime=(0.02,), seed=17)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    ref = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu()
    gbar = np.random.default_rng(9).normal(size=(wl.npv, wl.npt)).astype(np.float32)
    gref = m.evaluate_grad(t, p, torch.as_tensor(gbar, device=t.device), pb, wl.supersampling, wl.exptime).cpu()
    scratch = torch.empty(m.request_bytes(wl.npv, wl.npt, True), dtype=torch.uint8, device=t.device)
    s = torch.cuda.Stream(device=t.device)
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).pin_memory()  # noqa: E731
    fo = torch.empty((wl.npv, wl.npt), dtype=torch.float32).pin_memory()
    go = torch.empty((wl.npv, m.nparam), dtype=torch.float64).pin_memory()
    so = torch.empty(wl.npv, dtype=torch.int32).pin_memory()
    m.enqueue_host(pin(wl.times, np.float64), pin(wl.params, np.float64), pin(wl.pb_index, np.int32),
                   wl.supersampling, wl.exptime, pin(gbar, np.float32), fo, go, so, scratch, s)
    s.synchronize()
    assert m.host_path == "in place"
    assert torch.equal(fo, ref) and torch.equal(go, gref) and not so.any()
    # pageable numpy buffers through the C ABI
    P = ctypes.c_void_p
    tt, pbb, pp = (np.ascontiguousarray(wl.times), np.ascontiguousarray(wl.pb_index, np.int32),
                   np.ascontiguousarray(wl.params))
    f2, g2, s2 = np.zeros((wl.npv, wl.npt), np.float32), np.zeros((wl.npv, m.nparam)), np.ones(wl.npv, np.int32)
    ss, ex = np.array([3], np.int32), np.array([0.02])
    st = m.lib.rr_enqueue_host(m._h, tt.ctypes.data, pbb.ctypes.data, wl.npt, pp.ctypes.data, wl.npv,
                               ss.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                               ex.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), gbar.ctypes.data, f2.ctypes.data,
                               g2.ctypes.data, P(s2.ctypes.data), scratch.data_ptr(), scratch.numel(), s.cuda_stream)
    assert st == 0 and m.host_path == "staged"
    s.synchronize()
    assert torch.equal(torch.from_numpy(f2), ref) and torch.equal(torch.from_numpy(g2), gref) and not s2.any()
