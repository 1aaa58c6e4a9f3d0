"""Power-2 limb-darkening laws (direct model) on the GPU, against the oracle.

Flux element by element (FP64 1e-12, mixed 1e-6), status words exactly, and
the adjoint with the condition-scaled bounds of the other adjoint tests.
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


CASES = [
    dict(ld_model="power2"),
    dict(ld_model="power2_pm"),
    dict(ld_model="power2", npb=3, ss=(1, 4, 9), exptime=(0.0, 0.01, 0.02)),
    dict(ld_model="power2_pm", npb=2, chromatic=True),
    dict(ld_model="power2", npb=2, chromatic=True, shared_weights=True),
]


def _ids(c):
    return "-".join(str(v) for v in c.values())


def _make(case, npv, npt, seed):
    return W.make_small(npv=npv, npt=npt, seed=seed, span=6.0, eccentric=True, direct=True, **case)


def _setup(wl):
    return om.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, direct=True, shared=wl.shared_weights)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_power2_flux_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 17, 1333, 81)
    wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert np.array_equal(st.cpu().numpy(), rst) and not rst.any()
    assert (ref < 1).sum() > 100
    assert np.abs(f - ref).max() <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_power2_invalid_exponent(rr, precision):
    import torch
    wl = _make(dict(ld_model="power2"), 3, 300, 82)
    wl.precision = precision
    wl.params[1, 8] = -0.5
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    assert list(st.cpu().numpy()) == [0, om.ST_LD_INVALID, 0] and np.all(np.isnan(f[1]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_power2_adjoint_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 11, 1300, 83)
    wl.precision = precision
    gbar = np.random.default_rng(6).normal(size=(wl.npv, wl.npt))
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
