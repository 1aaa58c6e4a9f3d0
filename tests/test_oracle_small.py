"""Pins for the oracle's small-planet approximation (Sect. 3.4) and the profile derivative it uses."""
import numpy as np
import pytest

from oracle import exact, grad, ld, model
from oracle.area import intersection_area
from paper_2009_08500_gb300 import workloads as W

LAWS = [("quadratic", (0.4, 0.25)), ("quadratic_tri", (0.36, 0.3)), ("nonlinear", (0.5, -0.2, 0.6, -0.25)),
        ("linear", (0.6,)), ("general", (0.35, 0.2, 0.05)), ("logarithmic", (0.5, 0.2)),
        ("exponential", (0.45, 0.03))]


@pytest.mark.parametrize("law,coef", LAWS)
def test_profile_derivative_matches_differences(law, coef):
    mu = np.linspace(0.02, 0.99, 300)
    h = 1e-6
    fd = (ld.profile(law, mu + h, coef) - ld.profile(law, mu - h, coef)) / (2 * h)
    np.testing.assert_allclose(ld.profile_dmu(law, mu, coef), fd, rtol=1e-7, atol=1e-7)


def test_tabulated_profile_derivative_is_the_segment_slope():
    rng = np.random.Generator(np.random.PCG64(3))
    table = W.tabulated_profile(rng, 50)
    tmu, tI = table
    mid = 0.5 * (tmu[:-1] + tmu[1:])
    np.testing.assert_allclose(ld.profile_dmu("tabulated", mid, table=table), np.diff(tI) / np.diff(tmu), rtol=1e-12)
    assert ld.profile_dmu("tabulated", np.array([1.0]), table=table)[0] == 0.0


def _flux_at(setup, k, z, coef):
    _, istar, ldw = model.ld_weights(setup, k, coef, 0)
    return model.flux_from_distance(setup, np.array([z]), np.array([True]), k, ldw, istar)[0]


def test_small_planet_error_is_fourth_order_in_k():
    """At the disk centre the mean brightness under a planet of radius k exceeds the central value by
    O(k^2), so the approximation's flux error against the exact integral scales as k^4."""
    coef = (0.4, 0.25)
    s = model.build(W.GRID, "quadratic", k_small=0.2)
    istar = ld.istar("quadratic", coef)
    I = lambda m: ld.profile("quadratic", m, coef)  # noqa: E731
    errs = []
    for k in (0.02, 0.04, 0.08):
        errs.append(abs(_flux_at(s, k, 0.0, coef) - exact.exact_flux(k, 0.0, I, istar)))
    assert errs[1] / errs[0] == pytest.approx(16, rel=0.1)
    assert errs[2] / errs[1] == pytest.approx(16, rel=0.1)


@pytest.mark.parametrize("law,coef", LAWS)
def test_small_planet_matches_exact_integral_for_small_k(law, coef):
    """On g nodes (no interpolation) a k = 0.004 planet is within 1e-9 of the exact integral inside the disk."""
    s = model.build(W.GRID, law, n_general=3 if law == "general" else 0, k_small=0.01)
    istar = ld.istar(law, coef)
    I = lambda m: ld.profile(law, m, coef)  # noqa: E731
    k = 0.004
    for i in (0, 40, 100, 150, 180):
        z = i * s.dg * (1 + k)
        assert abs(_flux_at(s, k, z, coef) - exact.exact_flux(k, z, I, istar)) < 1e-9


def test_small_planet_uniform_disk_is_exact():
    s = model.build(W.GRID, "uniform", k_small=0.1)
    k = 0.05
    zs = np.linspace(0, 1 + k, 51)[:-1]
    _, istar, ldw = model.ld_weights(s, k, (), 0)
    f = model.flux_from_distance(s, zs, np.ones(zs.size, bool), k, ldw, istar)
    np.testing.assert_allclose(f, 1 - intersection_area(1.0, k, zs) / np.pi, rtol=0, atol=2e-15)


def test_small_planet_nodes_and_limb_clamp():
    s = model.build(W.GRID, "quadratic", k_small=0.1)
    coef = (0.4, 0.25)
    _, _, ldw = model.ld_weights(s, 0.05, coef, 0)
    assert ldw[0] == 1.0                       # planet centred: I(mu = 1)
    mu_c, free, c = model.small_planet_mu(s, 0.05)
    assert np.all(mu_c >= s.mu[-1]) and not free[-1] and free[0]
    # beyond the limb the centre value is the outermost bin's
    assert ldw[-1] == pytest.approx(ld.profile("quadratic", s.mu[-1:], coef)[0], abs=1e-15)


def test_small_planet_status_and_k_table():
    """Below the threshold no k table is needed: k under k0 is valid; k <= 0 is not."""
    wl = W.make_small("quadratic", npv=3, npt=300, seed=9, k_range=(0.002, 0.004))
    s = model.build(wl.grid, "quadratic", k_small=0.01)
    wl.params[2, 6] = 0.0
    f, st = model.evaluate(s, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime, return_status=True)
    assert list(st) == [0, 0, model.ST_K_RANGE]
    assert np.all(np.isfinite(f[:2])) and np.all(np.isnan(f[2]))
    st_tab = model.evaluate(model.build(wl.grid, "quadratic"), wl.times, wl.pb_index, wl.params[:1],
                            wl.supersampling, wl.exptime, return_status=True)[1]
    assert st_tab[0] == model.ST_K_RANGE


@pytest.mark.parametrize("law", ["quadratic", "nonlinear", "tabulated"])
def test_small_planet_jacobian_matches_finite_differences(law):
    from tests.test_oracle_grad import _smooth_points
    wl = W.make_small(law, npv=2, npt=1500, seed=61, span=4.0, k_range=(0.02, 0.04))
    s = model.build(wl.grid, law, wl.npb, wl.chromatic, wl.profiles, k_small=0.05)
    for p in range(wl.npv):
        row = wl.params[p].copy()
        steps = np.array([1e-6, 1e-7, 1e-6, 1e-6, 1e-6, 1e-6] + [1e-6] * (row.size - 6))
        J = grad.jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime)
        Jfd = grad.fd_jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime, steps)
        ok = _smooth_points(s, wl, row, steps)
        # a small planet's ingress is short: keep central differences away from the contacts,
        # where the area's second derivative is unbounded
        from oracle import orbit
        z, _, _ = orbit.projected_distance(wl.times, *row[:6])
        k = row[6]
        ok &= (np.abs(z - (1 - k)) > 1e-3) & (np.abs(z - (1 + k)) > 1e-3)
        assert ok.sum() > 0.8 * wl.npt
        J, Jfd = J[ok], Jfd[ok]
        noise = 4 * np.finfo(float).eps * J.shape[0] / (2 * steps)
        assert np.all(np.abs(J.sum(0) - Jfd.sum(0)) <= 1e-5 * np.abs(Jfd.sum(0)) + noise)
        scale = np.maximum(np.abs(Jfd).max(0), 1e-12)
        assert np.all(np.abs(J - Jfd) / scale < 1e-4)
