"""Small-planet approximation (Sect. 3.4) on the GPU, against the oracle.

Batches mix pvs below and above the threshold; flux element by element (FP64
1e-12, mixed 1e-6), status words exactly, and the adjoint with the
condition-scaled bounds of the other adjoint tests.
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
                    shared=wl.shared_weights, k_small=wl.k_small)


CASES = [
    dict(ld_model="quadratic", k_range=(0.002, 0.08)),                 # below k0 and across the threshold
    dict(ld_model="quadratic_tri", k_range=(0.01, 0.08)),
    dict(ld_model="nonlinear", k_range=(0.01, 0.08), direct=True),
    dict(ld_model="tabulated", npb=3, k_range=(0.01, 0.08), ss=(1, 4, 9), exptime=(0.0, 0.01, 0.02)),
    dict(ld_model="logarithmic", k_range=(0.01, 0.08)),
    dict(ld_model="exponential", k_range=(0.01, 0.08)),
    dict(ld_model="general", n_general=3, k_range=(0.01, 0.08)),
    dict(ld_model="quadratic", npb=2, chromatic=True, k_range=(0.03, 0.07)),
]


def _ids(c):
    return "-".join(str(v) for v in c.values())


def _make(case, npv, npt, seed):
    wl = W.make_small(npv=npv, npt=npt, seed=seed, span=6.0, eccentric=True, **case)
    wl.k_small = 0.05
    return wl


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_small_planet_flux_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 19, 1401, 71)
    wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert np.array_equal(st.cpu().numpy(), rst) and not rst.any()
    ks = wl.params[:, 6:6 + (wl.npb if wl.chromatic else 1)]
    assert (ks < wl.k_small).any() and (ref < 1).sum() > 100
    assert np.abs(f - ref).max() <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_small_planet_status(rr, precision):
    import torch
    wl = _make(dict(ld_model="quadratic", k_range=(0.002, 0.004)), 4, 300, 72)
    wl.precision = precision
    wl.params[2, 6] = 0.0
    wl.params[3, 6] = 0.2        # above the threshold: needs the k table, inside it
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st).double().cpu().numpy()
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert list(st.cpu().numpy()) == list(rst) == [0, 0, om.ST_K_RANGE, 0]
    ok = [0, 1, 3]
    assert np.abs(f[ok] - ref[ok]).max() <= TOL[precision] and np.all(np.isnan(f[2]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3], CASES[7]], ids=_ids)
def test_small_planet_adjoint_matches_oracle(rr, case, precision):
    import torch
    wl = _make(case, 13, 1300, 73)
    wl.precision = precision
    gbar = np.random.default_rng(5).normal(size=(wl.npv, wl.npt))
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
