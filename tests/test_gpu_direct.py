"""Direct model (Sect. 3.1.2, weights for each exact k, interpolation in g only) on the GPU.

Flux against the FP64 oracle element by element (FP64 path 1e-12, mixed path
1e-6 absolute); status words exactly; the adjoint against the oracle's chain
rule with the condition-scaled bounds of the interpolated model's adjoint
tests (|g - ref| <= rtol S, S = sum_t |gbar_t J_tj|).
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
    return om.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, wl.n_general, direct=True)


def gpu_flux(rr, wl, precision):
    import torch
    wl.precision = precision
    m = rr.model_for(wl)
    assert m.direct
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    torch.cuda.synchronize()
    m.sync_status()
    return f.double().cpu().numpy(), st.cpu().numpy()


CASES = [
    dict(ld_model="quadratic", eccentric=False),
    dict(ld_model="quadratic", eccentric=True, k_range=(0.3, 0.7)),         # beyond a usual k table
    dict(ld_model="quadratic", eccentric=True, k_range=(0.001, 0.006)),     # small planets
    dict(ld_model="nonlinear", eccentric=True, k_range=(0.05, 0.45)),
    dict(ld_model="tabulated", eccentric=True, npb=3, ss=(1, 4, 9), exptime=(0.0, 0.01, 0.02)),
    dict(ld_model="tabulated", eccentric=True, npb=2, chromatic=True, k_range=(0.1, 0.5)),
    dict(ld_model="quadratic", eccentric=True, npb=2, chromatic=True, ss=(3, 1), exptime=(0.01, 0.0)),
    dict(ld_model="uniform", eccentric=True, k_range=(0.2, 0.9)),
    dict(ld_model="general", eccentric=True, n_general=3),
    dict(ld_model="exponential", eccentric=True, k_range=(0.05, 0.3)),
]


def _ids(c):
    return "-".join(str(v) for v in c.values())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=_ids)
def test_direct_flux_matches_oracle(rr, case, precision):
    wl = W.make_small(npv=21, npt=1333, seed=29, span=6.0, direct=True, **case)
    f, st = gpu_flux(rr, wl, precision)
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert np.array_equal(st, rst) and not st.any()
    assert (ref < 1).sum() > 100
    err = np.abs(f - ref).max()
    assert err <= TOL[precision], err
    # out of transit stays exactly 1
    assert np.all(f[ref == 1.0] == 1.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_direct_k_domain_and_status(rr, precision):
    wl = W.make_small("quadratic", npv=6, npt=400, seed=5, direct=True, k_range=(0.35, 0.6))
    wl.params[1, 6] = 0.0
    wl.params[2, 6] = 1.0
    wl.params[3, 6] = -0.1
    wl.params[4, 6] = np.nan
    f, st = gpu_flux(rr, wl, precision)
    ref, rst = om.evaluate_workload(wl, _setup(wl), return_status=True)
    assert np.array_equal(st, rst)
    assert list(st) == [0, om.ST_K_RANGE, om.ST_K_RANGE, om.ST_K_RANGE, om.ST_NONFINITE, 0]
    assert np.all(np.isnan(f[1:5]))
    assert np.abs(f[[0, 5]] - ref[[0, 5]]).max() <= TOL[precision]


def test_direct_agrees_with_interpolated_model_on_k_nodes(rr):
    """On a node of the k grid both models use the same weights (mixed path, within 1 ppm of each other)."""
    wl = W.make_small("quadratic", npv=8, npt=900, seed=12)
    g = wl.grid
    dk = (g["k1"] - g["k0"]) / (g["nk"] - 1)
    wl.params[:, 6] = g["k0"] + dk * np.arange(5, 5 + 8 * 3, 3)
    f_tab, _ = gpu_flux_any(rr, wl, direct=False)
    f_dir, _ = gpu_flux_any(rr, wl, direct=True)
    assert np.abs(f_tab - f_dir).max() <= 1e-6


def gpu_flux_any(rr, wl, direct):
    wl.direct = direct
    wl.precision = "mixed"
    import torch
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime)
    torch.cuda.synchronize()
    return f.double().cpu().numpy(), None


def test_direct_population_full_launch_sampled_rows(rr):
    """4096 pvs x 20000 times with k anywhere in (0.003, 0.5); sampled rows against the oracle."""
    wl = W.make_c3()
    wl.direct = True
    rng = np.random.default_rng(5)
    wl.params[:, 6] = np.exp(rng.uniform(np.log(0.003), np.log(0.5), wl.npv))
    f, st = gpu_flux(rr, wl, "mixed")
    assert f.shape == (4096, 20000) and not st.any()
    rows = rng.choice(4096, 16, replace=False)
    sub = wl.subset(4096)
    sub.params = wl.params[rows]
    ref = om.evaluate_workload(sub, _setup(sub))
    assert np.abs(f[rows] - ref).max() <= 1e-6
    assert np.all(f <= 1.0) and np.all(f > 0.0)


# ------------------------------------------------------------------ adjoint
def gpu_vjp(rr, wl, gbar, precision):
    import torch
    wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    gb = torch.as_tensor(gbar, dtype=m.dtype, device=t.device)
    g = m.evaluate_grad(t, p, gb, pb, wl.supersampling, wl.exptime)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def oracle_vjp(wl, gbar):
    s = _setup(wl)
    ref = np.zeros(wl.params.shape)
    scale = np.zeros(wl.params.shape)
    for p in range(wl.npv):
        J = og.jacobian(s, wl.times, wl.pb_index, wl.params[p], wl.supersampling, wl.exptime)
        ref[p] = gbar[p] @ J
        scale[p] = np.abs(gbar[p]) @ np.abs(J)
    return ref, scale


GRAD_CASES = [
    dict(ld_model="quadratic", eccentric=True),
    dict(ld_model="quadratic", eccentric=True, k_range=(0.3, 0.7)),
    dict(ld_model="quadratic", eccentric=True, k_range=(0.002, 0.008)),
    dict(ld_model="nonlinear", eccentric=True),
    dict(ld_model="tabulated", eccentric=True, npb=2, ss=(1, 4), exptime=(0.0, 0.01)),
    dict(ld_model="quadratic", eccentric=True, npb=2, chromatic=True, k_range=(0.1, 0.45)),
    dict(ld_model="uniform", eccentric=True, k_range=(0.2, 0.8)),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", GRAD_CASES, ids=_ids)
def test_direct_adjoint_matches_oracle_chain_rule(rr, case, precision):
    wl = W.make_small(npv=13, npt=1700, seed=31, span=6.0, direct=True, **case)
    gbar = np.random.default_rng(3).normal(size=(wl.npv, wl.npt))
    if precision == "mixed":
        gbar = gbar.astype(np.float32).astype(np.float64)
    g = gpu_vjp(rr, wl, gbar, precision)
    ref, scale = oracle_vjp(wl, gbar)
    floor = 1e-3 * scale.max(axis=1, keepdims=True)
    err = np.abs(g - ref) / np.maximum(scale, np.maximum(floor, 1e-300))
    assert err.max() < GRAD_RTOL[precision], (err.max(), np.unravel_index(err.argmax(), err.shape))
