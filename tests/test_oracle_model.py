"""Pins for the oracle's whole model (Eq. 5, Sect. 3.1 interpolation, Sect. 4 supersampling)."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import exact, ld, model
from oracle.area import intersection_area
from paper_2009_08500_gb300 import workloads as W

COARSE = dict(zcut=0.5, nzin=12, nzlimb=18, ng=30, nk=6, k0=0.01, k1=0.3)


def _single(setup, k, z, coef=(), pb=0):
    """Eq. 5 for one planet position (in front of the star)."""
    _, istar, ldw = model.ld_weights(setup, k, coef, pb)
    return model.flux_from_distance(setup, np.atleast_1d(z), np.array([True]), k, ldw, istar)[0]


@pytest.mark.parametrize("g", [COARSE, W.GRID])
def test_uniform_disk_is_exact_for_any_grid(g):
    s = model.build(g, "uniform")
    rng = np.random.default_rng(0)
    for k in rng.uniform(g["k0"], g["k1"], 8):
        zs = rng.uniform(0, 1 + k, 50)
        _, istar, ldw = model.ld_weights(s, k, (), 0)
        f = model.flux_from_distance(s, zs, np.ones(50, bool), k, ldw, istar)
        np.testing.assert_allclose(f, 1 - intersection_area(1.0, k, zs) / np.pi, rtol=0, atol=2e-15)
        assert _single(s, k, 0.0) == pytest.approx(1 - k * k, abs=1e-15)


@pytest.mark.parametrize("k", [0.01, 0.05, 0.1, 0.25])
def test_quadratic_within_paper_error_level_of_exact_integral(k, grid):
    """Sect. 3.3 / Fig. 2-3: a few ppm at these resolutions, no asymptotic bias."""
    coef = (0.4, 0.25)
    s = model.build(grid, "quadratic")
    istar = ld.istar("quadratic", coef)
    I = lambda m: ld.profile("quadratic", m, coef)  # noqa: E731
    errs = []
    for g in np.linspace(0.0, 0.999, 60):
        z = g * (1 + k)
        errs.append(_single(s, k, z, coef) - exact.exact_flux(k, z, I, istar))
    errs = np.abs(errs)
    assert errs.max() < 9e-6          # Fig. 3 caption: max 9 ppm
    assert errs.mean() < 1e-6


@pytest.mark.parametrize("model_name,coef", [("nonlinear", (0.5, -0.2, 0.6, -0.25)), ("tabulated", ()),
                                             ("linear", (0.6,)), ("general", (0.35, 0.2, 0.05)),
                                             ("logarithmic", (0.5, 0.2)), ("exponential", (0.45, 0.03))])
def test_other_profiles_match_exact_integral(model_name, coef, grid):
    rng = np.random.Generator(np.random.PCG64(9))
    table = W.tabulated_profile(rng)
    s = model.build(grid, model_name, tables=[table], n_general=len(coef) if model_name == "general" else 0)
    I = lambda m: ld.profile(model_name, m, coef, table)  # noqa: E731
    istar = ld.istar(model_name, coef, table)
    for k in (0.05, 0.2):
        for g in (0.0, 0.4, 0.85, 0.97):
            z = g * (1 + k)
            assert _single(s, k, z, coef) == pytest.approx(exact.exact_flux(k, z, I, istar), abs=9e-6)


def test_against_pixel_integration_tiny_case(grid):
    """Brute-force 2-D integral of I over the covered pixels."""
    coef = (0.5, 0.2)
    s = model.build(grid, "quadratic")
    I = lambda m: ld.profile("quadratic", m, coef)  # noqa: E731
    istar = ld.istar("quadratic", coef)
    for k, z in [(0.1, 0.5), (0.2, 0.95)]:
        pix = 1 - exact.occulted_flux_pixels(k, z, I, n=3000) / istar
        assert _single(s, k, z, coef) == pytest.approx(pix, abs=4e-6)


def test_exact_radial_integral_reduces_to_area_for_uniform_disk():
    for k, z in [(0.1, 0.3), (0.1, 1.05), (0.3, 0.8)]:
        occ = exact.occulted_flux_radial(k, z, lambda r: 1.0)
        assert occ == pytest.approx(intersection_area(1.0, k, z), abs=1e-12)


def test_out_of_transit_and_behind_star_are_exactly_one(grid):
    wl = W.make_small("quadratic", npv=4, npt=400, seed=3)
    f, st = model.evaluate_workload(wl, return_status=True)
    assert not st.any()
    T0, P = wl.params[:, 0], wl.params[:, 1]
    # far from any conjunction: more than 0.2 of a period away
    ph = ((wl.times[None, :] - T0[:, None]) / P[:, None]) % 1.0
    far = (ph > 0.2) & (ph < 0.8)
    assert far.any() and np.all(f[far] == 1.0)
    assert np.all(f <= 1.0)


def test_supersampling_ss1_equals_plain_and_converges_to_exposure_mean(grid):
    wl = W.make_c1()
    s = model.build(grid, "quadratic")
    t = np.array([-0.07, -0.052, -0.03, 0.0, 0.049])
    plain = model.evaluate(s, t, np.zeros(5, int), wl.params, np.array([1]), np.array([0.0]))
    ss1 = model.evaluate(s, t, np.zeros(5, int), wl.params, np.array([1]), np.array([0.02]))
    np.testing.assert_array_equal(plain, ss1)
    ex = 0.02
    f = lambda tt: model.evaluate(s, np.array([tt]), np.zeros(1, int), wl.params, np.array([1]),  # noqa: E731
                                  np.array([0.0]))[0, 0]
    for ss in (64, 256):
        sup = model.evaluate(s, t, np.zeros(5, int), wl.params, np.array([ss]), np.array([ex]))[0]
        ref = np.array([quad(f, tt - ex / 2, tt + ex / 2, epsabs=1e-13, limit=200)[0] / ex for tt in t])
        assert np.abs(sup - ref).max() < (2e-6 if ss == 64 else 2e-7)
    # a constant (out-of-transit) stretch is unchanged by any supersampling
    far = model.evaluate(s, np.array([1.0, 1.2]), np.zeros(2, int), wl.params, np.array([30]), np.array([0.02]))
    assert np.all(far == 1.0)


def test_invalid_parameter_vectors_give_nan_and_status(grid):
    s = model.build(grid, "quadratic")
    good = [0.0, 3.0, 10.0, 0.3, 0.0, 0.0, 0.1, 0.4, 0.25]
    rows = np.array([good] * 8, float)
    rows[1, 6] = 0.4          # k > k1
    rows[2, 4] = 1.0          # e >= 1
    rows[3, 3] = -0.1         # b < 0
    rows[4, 1] = 0.0          # P <= 0
    rows[5, 2] = 0.9          # a <= 1
    rows[6, 7] = np.nan       # non-finite
    rows[7, 7:9] = (3.0, 3.0)  # I_star <= 0
    t = np.linspace(-0.1, 0.1, 7)
    f, st = model.evaluate(s, t, np.zeros(7, int), rows, np.array([1]), np.array([0.0]), return_status=True)
    assert st[0] == 0 and np.all(np.isfinite(f[0]))
    assert list(st[1:]) == [model.ST_K_RANGE, model.ST_E_RANGE, model.ST_B_RANGE, model.ST_P_RANGE,
                            model.ST_A_RANGE, model.ST_NONFINITE, model.ST_LD_INVALID]
    assert np.all(np.isnan(f[1:]))


def test_k_interpolation_is_linear_between_nodes(grid):
    s = model.build(grid, "quadratic")
    coef = (0.4, 0.25)
    ka, kb = s.k0 + 10 * s.dk, s.k0 + 11 * s.dk
    _, _, la = model.ld_weights(s, ka, coef, 0)
    _, _, lb = model.ld_weights(s, kb, coef, 0)
    _, _, lm = model.ld_weights(s, 0.3 * ka + 0.7 * kb, coef, 0)
    np.testing.assert_allclose(lm, 0.3 * la + 0.7 * lb, rtol=1e-12)
    # the end of the k range is usable and equals the last node
    _, _, le = model.ld_weights(s, s.k1, coef, 0)
    ldp = ld.profile("quadratic", s.mu, coef)
    np.testing.assert_allclose(le, s.w[-1] @ ldp, rtol=1e-13)
