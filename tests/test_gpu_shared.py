"""Shared weights for transmission spectroscopy (Sect. 3.4) on the GPU, against the oracle.

Interpolated and direct models, FP64 and mixed forms: flux element by element
(1e-12 / 1e-6 absolute), status words exactly, and the adjoint with the
condition-scaled bounds of the other adjoint tests (the weights' k-derivative
is spread over every passband's radius ratio).
"""
import numpy as np
import pytest

from oracle import grad as og
from oracle import model as om
from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}
GRAD_RTOL = {"fp64": 1e-10, "mixed": 3e-5}


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


def _setup(wl):
    return om.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, wl.n_general, direct=wl.direct,
                    shared=True)


def _spread(wl, frac=0.03, seed=0):
    """Per-passband radius ratios within a few percent of each other (a transmission spectrum)."""
    rng = np.random.default_rng(seed)
    k = wl.params[:, 6].copy()
    for j in range(wl.npb):
        wl.params[:, 6 + j] = k * (1 + frac * rng.uniform(-1, 1, wl.npv))
    return wl


CASES = [
    dict(ld_model="quadratic", npb=3),
    dict(ld_model="quadratic", npb=2, ss=(3, 1), exptime=(0.01, 0.0), direct=True),
    dict(ld_model="tabulated", npb=2),
    dict(ld_model="tabulated", npb=3, direct=True, k_range=(0.1, 0.4)),
    dict(ld_model="nonlinear", npb=2, direct=True),
]


def _ids(c):
    return "-".join(str(v) for v in c.values())


def _make(case, npv, npt, seed):
    wl = W.make_small(npv=npv, npt=npt, seed=seed, span=6.0, chromatic=True, eccentric=True, shared_weights=True,
                      **case)
    return _spread(wl, seed=seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_shared_flux_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 17, 1501, 51)
    wl.precision = precision
    m = rr.model_for(wl)
    assert m.shared_weights
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert np.array_equal(st.cpu().numpy(), rst) and not rst.any()
    assert (ref < 1).sum() > 100
    assert np.abs(f - ref).max() <= TOL[precision]


@pytest.mark.parametrize("direct", [False, True])
def test_equal_radius_ratios_match_unshared_model(rr, direct):
    import torch
    wl = W.make_small("quadratic", npv=9, npt=700, npb=3, chromatic=True, seed=52, direct=direct)
    wl.params[:, 7] = wl.params[:, 6]
    wl.params[:, 8] = wl.params[:, 6]
    t, pb, p = rr.to_device(wl)
    out = []
    for sh in (False, True):
        wl.shared_weights = sh
        m = rr.model_for(wl)
        out.append(m.evaluate(t, p, pb, wl.supersampling, wl.exptime).cpu().numpy())
    torch.cuda.synchronize()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES[:4], ids=_ids)
def test_shared_adjoint_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 11, 1300, 53)
    wl.precision = precision
    gbar = np.random.default_rng(4).normal(size=(wl.npv, wl.npt))
    if precision == "mixed":
        gbar = gbar.astype(np.float32).astype(np.float64)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    gb = torch.as_tensor(gbar, dtype=m.dtype, device=t.device)
    g = m.evaluate_grad(t, p, gb, pb, wl.supersampling, wl.exptime).cpu().numpy()
    s = _setup(wl)
    ref = np.zeros(wl.params.shape)
    scale = np.zeros(wl.params.shape)
    for i in range(wl.npv):
        J = og.jacobian(s, wl.times, wl.pb_index, wl.params[i], wl.supersampling, wl.exptime)
        ref[i] = gbar[i] @ J
        scale[i] = np.abs(gbar[i]) @ np.abs(J)
    floor = 1e-3 * scale.max(axis=1, keepdims=True)
    err = np.abs(g - ref) / np.maximum(scale, np.maximum(floor, 1e-300))
    assert err.max() < GRAD_RTOL[precision], (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_transmission_workload_full_launch_sampled_rows(rr):
    """2,048 pvs x 8 channels x 2,500 times through the direct model with shared weights, as bench.py runs it."""
    import torch
    wl = W.make_ts()
    m = rr.model_for(wl)
    assert m.direct and m.shared_weights
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    torch.cuda.synchronize()
    f = f.double().cpu().numpy()
    assert not st.cpu().numpy().any()
    rows = np.random.default_rng(6).choice(wl.npv, 8, replace=False)
    sub = wl.subset(wl.npv)
    sub.params = wl.params[rows]
    ref = om.evaluate_workload(sub)
    assert np.abs(f[rows] - ref).max() <= 1e-6


def test_transmission_workload_full_launch_sampled_rows(rr):
    """The full transmission-spectroscopy launch the benchmark times (2,048 pvs x 8 channels x
    2,500 times, direct model, shared weights, mixed form): flux of sampled rows against the
    oracle at 1e-6, and every row valid."""
    import torch
    wl = W.make_ts()
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    assert f.shape == (2048, 20000) and not st.cpu().numpy().any()
    rows = np.random.default_rng(2).choice(2048, 5, replace=False)
    sub = wl.subset(2048)
    sub.params = wl.params[rows]
    ref = om.evaluate_workload(sub, _setup(sub))
    assert (ref < 1).sum() > 100
    assert np.abs(f[rows] - ref).max() <= 1e-6
