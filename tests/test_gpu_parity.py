"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 path 1e-12 absolute flux; mixed path 1e-6 absolute flux
(1 ppm).  Integer outputs (status words) must match exactly.
"""
import json
import os

import numpy as np
import pytest

from oracle import ld as old
from oracle import model as om
from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


def gpu_flux(rr, wl, precision=None):
    import torch
    if precision:
        wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    torch.cuda.synchronize()
    m.sync_status()
    return f.double().cpu().numpy(), st.cpu().numpy()


def oracle_flux(wl):
    setup = om.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, wl.n_general)
    return om.evaluate_workload(wl, setup, return_status=True)


# ----------------------------------------------------------------- set-up tables
@pytest.mark.parametrize("ld_model", ["quadratic", "nonlinear", "tabulated", "linear", "general", "logarithmic",
                                      "exponential"])
def test_setup_tables_match_oracle(rr, ld_model):
    wl = W.make_small(ld_model, npv=1, npt=4, npb=2 if ld_model == "tabulated" else 1, seed=3,
                      n_general=3 if ld_model == "general" else 0)
    m = rr.model_for(wl)
    s = om.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, wl.n_general)
    np.testing.assert_allclose(m.read_table("ze"), s.ze, rtol=0, atol=2e-16)
    np.testing.assert_allclose(m.read_table("mu"), s.mu, rtol=0, atol=2e-16)
    w = m.read_table("weights").reshape(s.w.shape)
    # w multiplies the covered area a(1, k, c) in Eq. 5: compare covered areas per annulus
    # (FP64 round-off); w itself loses digits to cancellation in the lens areas at small k
    kk = s.k0 + s.dk * np.arange(s.nk)[:, None]
    atot = np.vectorize(lambda k, c: __import__("oracle").area.intersection_area(1.0, k, c))(
        kk, np.arange(s.ng)[None, :] * s.dg * (1 + kk))
    np.testing.assert_allclose(w * atot[..., None], s.w * atot[..., None], rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, s.w, rtol=0, atol=1e-12)
    nz = s.mu.size
    basis = m.read_table("basis").reshape(-1, nz)
    istar = m.read_table("istar")
    if ld_model == "tabulated":
        refb = np.stack([old.profile("tabulated", s.mu, table=tb) for tb in wl.profiles])
        refi = np.array([old.istar("tabulated", table=tb) for tb in wl.profiles])
    else:
        nc = old.ncoef(ld_model, wl.n_general)
        # basis c = I(coefficient vector e_c) - I(0): the law is affine in its coefficients
        zero = old.profile(ld_model, s.mu, (0.0,) * nc)
        refb = [zero] + [old.profile(ld_model, s.mu, tuple(np.eye(nc)[c])) - zero for c in range(nc)]
        refb = np.stack(refb)
        i0 = old.istar(ld_model, (0.0,) * nc)
        refi = np.array([i0] + [old.istar(ld_model, tuple(np.eye(nc)[c])) - i0 for c in range(nc)])
    np.testing.assert_allclose(basis, refb, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(istar, refi, rtol=1e-13, atol=1e-15)
    proj = m.read_table("proj").reshape(len(refb), s.nk, s.ng)
    # w carries ~1e-13 of FP64 round-off (lens-area differences): the projections carry it
    # scaled by the basis values (up to ~33 for the exponential law near the limb)
    np.testing.assert_allclose(proj, np.einsum("kgz,bz->bkg", s.w, refb), rtol=0,
                               atol=1e-13 * max(1.0, np.abs(refb).max()))


# ------------------------------------------------------------------- light curves
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c1_plain_method(rr, precision):
    wl = W.make_c1()
    f, st = gpu_flux(rr, wl, precision)
    ref, rst = oracle_flux(wl)
    assert list(st) == list(rst) == [0]
    assert np.abs(f - ref).max() <= TOL[precision]
    assert (ref < 1).sum() > 500


CASES = []
for _ld in ("uniform", "quadratic", "quadratic_tri", "nonlinear", "tabulated"):
    for _ecc in (False, True):
        CASES.append(dict(ld_model=_ld, eccentric=_ecc))
CASES += [dict(ld_model=_ld, eccentric=True) for _ld in ("linear", "logarithmic", "exponential")]
CASES += [
    dict(ld_model="general", eccentric=True, n_general=4),
    dict(ld_model="general", npb=2, n_general=2, ss=(1, 6), exptime=(0.0, 0.01)),
    dict(ld_model="quadratic", npb=3, chromatic=True, ss=(1, 4, 7), exptime=(0.0, 0.01, 0.02)),
    dict(ld_model="nonlinear", npb=2, ss=(5, 2), exptime=(0.02, 0.005)),
    dict(ld_model="tabulated", npb=4, ss=(1, 10, 30, 3), exptime=(0.001, 0.007, 0.021, 0.01)),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(str(v) for v in c.values()))
def test_small_cases_with_ragged_sizes(rr, case, precision):
    # 37 pvs (a ragged pv tile), 2,300 times (two full point tiles and a ragged one)
    wl = W.make_small(npv=37, npt=2300, seed=31, span=8.0, **case)
    f, st = gpu_flux(rr, wl, precision)
    ref, rst = oracle_flux(wl)
    np.testing.assert_array_equal(st, rst)
    assert np.abs(f - ref).max() <= TOL[precision], np.abs(f - ref).max()
    assert (ref < 1).sum() > 100


@pytest.mark.parametrize("npv,npt", [(1, 1), (1, 7), (2, 1024), (3, 1025), (33, 31), (5, 0), (0, 9)])
def test_edge_sizes(rr, npv, npt):
    wl = W.make_small("quadratic", npv=max(npv, 1), npt=max(npt, 1), seed=5, span=0.5)
    wl.params = wl.params[:npv]
    wl.times, wl.pb_index = wl.times[:npt], wl.pb_index[:npt]
    f, st = gpu_flux(rr, wl, "mixed")
    assert f.shape == (npv, npt)
    if npv and npt:
        ref, _ = oracle_flux(wl)
        assert np.abs(f - ref).max() <= 1e-6


def test_c2_eccentric_supersampled_full_size(rr):
    wl = W.make_c2()
    f, st = gpu_flux(rr, wl)
    ref, rst = oracle_flux(wl)
    assert st[0] == rst[0] == 0
    assert (ref < 1).sum() > 200
    assert np.abs(f - ref).max() <= 1e-6


def test_c3_population_full_launch_sampled_rows(rr):
    wl = W.make_c3()
    f, st = gpu_flux(rr, wl)
    assert f.shape == (4096, 20000) and not st.any()
    rows = np.random.default_rng(0).choice(4096, 24, replace=False)
    sub = wl.subset(4096)
    sub.params = wl.params[rows]
    ref, _ = oracle_flux(sub)
    assert np.abs(f[rows] - ref).max() <= 1e-6
    # every row: flux in (0, 1]; out of transit exactly 1 somewhere
    assert np.all(f <= 1.0) and np.all(f > 0.0) and np.all((f == 1.0).any(axis=1))


def test_c4_heterogeneous_full_launch_sampled_rows(rr):
    wl = W.make_c4()
    f, st = gpu_flux(rr, wl)
    assert f.shape == (2048, 60000) and not st.any()
    rows = np.random.default_rng(1).choice(2048, 6, replace=False)
    sub = wl.subset(2048)
    sub.params = wl.params[rows]
    ref, _ = oracle_flux(sub)
    assert np.abs(f[rows] - ref).max() <= 1e-6


def _sampled_rows(rr, wl, rows):
    """Evaluate the whole batch on the device; bring back only ``rows`` and the status words."""
    import torch
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    st = torch.full((wl.npv,), -1, dtype=torch.int32, device=t.device)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime, pv_status=st)
    torch.cuda.synchronize()
    m.sync_status()
    idx = torch.as_tensor(rows, device=f.device)
    out = f[idx].double().cpu().numpy(), st.cpu().numpy(), f.shape, int((f < 1).sum())
    del f
    torch.cuda.empty_cache()
    return out


def _rows_oracle(wl, rows):
    sub = wl.subset(len(rows))
    sub.params = wl.params[rows].copy()
    return oracle_flux(sub)[0]


@pytest.mark.parametrize("npv,npt", [(300_000, 640), (40_000, 60_000)])
def test_large_batches_sampled_rows(rr, npv, npt):
    """Large batches: 300,000 pvs (9,375 pv tiles on the grid) and 40,000 pvs x 60,000 times
    (2.4e9 flux elements, past 2^31, so the last rows sit beyond any 32-bit element offset).
    Sampled rows, the first and the last pv among them, against the oracle."""
    wl = W.make_small("quadratic_tri", npv=npv, npt=npt, seed=41, span=3.0, eccentric=False)
    rows = np.concatenate([[0, npv - 1], np.sort(np.random.default_rng(5).choice(npv - 1, 10, replace=False))])
    f, st, shape, n_in = _sampled_rows(rr, wl, rows)
    assert tuple(shape) == (npv, npt) and not st.any()
    assert np.abs(f - _rows_oracle(wl, rows)).max() <= TOL["mixed"]
    assert n_in > npv                      # every pv transits within the 3-day span


def test_out_of_transit_is_exactly_one(rr):
    wl = W.make_small("nonlinear", npv=16, npt=3000, seed=9, span=10.0)
    f, _ = gpu_flux(rr, wl, "mixed")
    T0, P = wl.params[:, 0:1], wl.params[:, 1:2]
    ph = ((wl.times[None, :] - T0) / P) % 1.0
    far = (ph > 0.25) & (ph < 0.75)
    assert np.all(f[far] == 1.0)


def test_invalid_parameter_vectors(rr):
    wl = W.make_small("quadratic_tri", npv=9, npt=500, seed=4)
    p = wl.params
    p[1, 6] = 0.31          # k > k1
    p[2, 4] = 1.2           # e >= 1
    p[3, 3] = -0.2          # b < 0
    p[4, 1] = -1.0          # P <= 0
    p[5, 2] = 0.5           # a <= 1
    p[6, 0] = np.inf        # non-finite
    p[7, 7] = 1.5           # q1 > 1
    for prec in ("fp64", "mixed"):
        f, st = gpu_flux(rr, wl, prec)
        ref, rst = oracle_flux(wl)
        np.testing.assert_array_equal(st, rst)
        assert np.all(np.isnan(f[1:8])) and np.all(np.isfinite(f[[0, 8]]))
        assert np.abs(f[[0, 8]] - ref[[0, 8]]).max() <= TOL[prec]


def test_paper_heterogeneous_example(rr):
    import torch
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_heterogeneous_example.json")
    g = json.load(open(path))
    for case in g["cases"].values():
        for prec in ("fp64", "mixed"):
            m = rr.Model("quadratic", npb=2, chromatic=case["chromatic"], precision=prec, grid=g["grid"]).build()
            dev = m.device
            f = m.evaluate(torch.tensor(g["times"], dtype=torch.float64, device=dev),
                           torch.tensor(case["params"], dtype=torch.float64, device=dev),
                           torch.tensor(g["pb_index"], dtype=torch.int32, device=dev), [1, 1], [0.0, 0.0])
            assert np.abs(f.double().cpu().numpy() - np.array(case["expected_flux"])).max() <= TOL[prec]


def test_argument_errors_are_reported_before_launch(rr):
    import torch
    wl = W.make_small("quadratic", npv=2, npt=100)
    m = rr.Model("quadratic")
    t, pb, p = rr.to_device(wl)
    with pytest.raises(rr.RRError, match="RR_ESTATE"):
        m.evaluate(t, p, pb)
    m.build()
    n0 = m.launch_count
    small = torch.empty(16, dtype=torch.uint8, device=t.device)
    with pytest.raises(rr.RRError, match="workspace"):
        m.evaluate(t, p, pb, workspace=small)
    with pytest.raises(rr.RRError, match="supersampling"):
        m.evaluate(t, p, pb, supersampling=[0])
    with pytest.raises(rr.RRError, match="exptime"):
        m.evaluate(t, p, pb, supersampling=[2], exptime=[-1.0])
    assert m.launch_count == n0
    with pytest.raises(rr.RRError, match="RR_ESTATE"):
        m.set_ld_profile(0, [0.0, 1.0], [0.5, 1.0])


def test_high_eccentricity_uses_fp64_kepler(rr):
    wl = W.make_small("quadratic", npv=4, npt=20000, seed=12, span=6.0)
    wl.params[:, 4] = [0.85, 0.9, 0.95, 0.82]
    wl.params[:, 2] = [40.0, 60.0, 120.0, 30.0]    # periastron outside the star
    f, st = gpu_flux(rr, wl, "mixed")
    ref, rst = oracle_flux(wl)
    np.testing.assert_array_equal(st, rst)
    assert np.abs(f - ref).max() <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grazing_and_missing_transits(rr, precision):
    """Impact parameters around 1 + k: the transit window must still contain every
    touching point, and orbits that never cross the disk give exactly 1."""
    wl = W.make_small("nonlinear", npv=48, npt=4000, seed=77, span=6.0)
    k = wl.params[:, 6]
    off = np.linspace(-0.02, 0.02, wl.npv)
    wl.params[:, 3] = np.clip((1 + k) * (1 + off), 0, None)    # b = (1 + k)(1 + off)
    f, st = gpu_flux(rr, wl, precision)
    ref, rst = oracle_flux(wl)
    np.testing.assert_array_equal(st, rst)
    assert np.abs(f - ref).max() <= TOL[precision]
    # pvs whose closest approach stays outside the disk: flux exactly 1 everywhere
    never = np.all(ref == 1.0, axis=1)
    assert never.any() and (~never).any()
    assert np.all(f[never] == 1.0)
