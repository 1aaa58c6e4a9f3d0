"""Pins for the oracle's power-2 laws (Sect. 3.2.1): I = 1 - c (1 - mu^alpha) and its (h1, h2) form."""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import exact, grad, ld, model
from paper_2009_08500_gb300 import workloads as W


@pytest.mark.parametrize("law,coef", [("power2", (0.6, 0.7)), ("power2", (0.3, 2.5)), ("power2_pm", (0.7, 0.45))])
def test_istar_closed_form_matches_quadrature(law, coef):
    q, _ = quad(lambda m: m * ld.profile(law, np.array([m]), coef)[0], 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)
    assert ld.istar(law, coef) == pytest.approx(2 * np.pi * q, rel=1e-12)


def test_reductions_to_linear_and_quadratic():
    mu = np.linspace(0, 1, 101)
    np.testing.assert_allclose(ld.profile("power2", mu, (0.4, 1.0)), ld.profile("linear", mu, (0.4,)), atol=1e-15)
    # 1 - c (1 - mu^2) = 1 - 2c (1 - mu) + c (1 - mu)^2
    np.testing.assert_allclose(ld.profile("power2", mu, (0.3, 2.0)), ld.profile("quadratic", mu, (0.6, -0.3)),
                               atol=1e-15)
    assert ld.istar("power2", (0.3, 2.0)) == pytest.approx(ld.istar("quadratic", (0.6, -0.3)), rel=1e-15)


def test_h1_h2_are_the_profile_at_half_and_its_drop_to_the_limb():
    h1, h2 = 0.72, 0.41
    I = lambda m: ld.profile("power2_pm", np.array([m]), (h1, h2))[0]  # noqa: E731
    assert I(0.5) == pytest.approx(h1, abs=1e-15)
    assert I(0.5) - I(0.0) == pytest.approx(h2, abs=1e-15)


@pytest.mark.parametrize("law", ["power2", "power2_pm"])
def test_coefficient_partials_match_differences(law):
    from oracle.grad import _ld_partials
    mu = np.linspace(0.05, 1.0, 60)
    coef = np.array((0.6, 0.7) if law == "power2" else (0.7, 0.45))
    dp, di = _ld_partials(law, mu, coef, None)
    h = 1e-6
    for j in range(2):
        e = np.zeros(2)
        e[j] = h
        fd = (ld.profile(law, mu, coef + e) - ld.profile(law, mu, coef - e)) / (2 * h)
        np.testing.assert_allclose(dp[j], fd, rtol=1e-7, atol=1e-9)
        fdi = (ld.istar(law, coef + e) - ld.istar(law, coef - e)) / (2 * h)
        assert di[j] == pytest.approx(fdi, rel=1e-7)


@pytest.mark.parametrize("law,coef", [("power2", (0.6, 0.7)), ("power2_pm", (0.7, 0.45))])
def test_direct_model_within_paper_error_of_exact_integral(law, coef, grid):
    s = model.build(grid, law, direct=True)
    istar = ld.istar(law, coef)
    I = lambda m: ld.profile(law, m, coef)  # noqa: E731
    for k in (0.05, 0.15):
        _, _, ldw = model.ld_weights(s, k, coef, 0)
        for g in np.linspace(0.0, 0.98, 12):
            z = g * (1 + k)
            f = model.flux_from_distance(s, np.array([z]), np.array([True]), k, ldw, istar)[0]
            assert abs(f - exact.exact_flux(k, z, I, istar)) < 9e-6


def test_invalid_exponent_is_flagged(grid):
    wl = W.make_small("power2", npv=3, npt=100, seed=2, direct=True)
    wl.params[1, 8] = 0.0
    s = model.build(grid, "power2", direct=True)
    _, st = model.evaluate(s, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime, return_status=True)
    assert list(st) == [0, model.ST_LD_INVALID, 0]


@pytest.mark.parametrize("law", ["power2", "power2_pm"])
def test_power2_jacobian_matches_finite_differences(law):
    from tests.test_oracle_grad import _smooth_points
    wl = W.make_small(law, npv=2, npt=1500, seed=19, span=4.0, direct=True)
    s = model.build(wl.grid, law, direct=True)
    for p in range(wl.npv):
        row = wl.params[p].copy()
        steps = np.array([1e-6, 1e-7, 1e-6, 1e-6, 1e-6, 1e-6] + [1e-6] * (row.size - 6))
        J = grad.jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime)
        Jfd = grad.fd_jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime, steps)
        ok = _smooth_points(s, wl, row, steps)
        assert ok.sum() > 0.8 * wl.npt
        J, Jfd = J[ok], Jfd[ok]
        noise = 4 * np.finfo(float).eps * J.shape[0] / (2 * steps)
        assert np.all(np.abs(J.sum(0) - Jfd.sum(0)) <= 1e-5 * np.abs(Jfd.sum(0)) + noise)
        scale = np.maximum(np.abs(Jfd).max(0), 1e-12)
        assert np.all(np.abs(J - Jfd) / scale < 1e-4)
