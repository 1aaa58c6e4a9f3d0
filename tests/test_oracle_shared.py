"""Pins for the oracle's shared weights for transmission spectroscopy (Sect. 3.4).

One weight array, at the mean of a pv's per-passband radius ratios, serves
every passband; the area and g keep the passband's own k.
"""
import numpy as np
import pytest

from oracle import exact, grad, ld, model
from oracle.area import intersection_area
from paper_2009_08500_gb300 import workloads as W


def _wl(**kw):
    args = dict(ld_model="quadratic", npv=4, npt=900, npb=3, chromatic=True, seed=41, span=6.0)
    args.update(kw)
    return W.make_small(**args)


@pytest.mark.parametrize("direct", [False, True])
def test_equal_radius_ratios_reduce_to_per_passband_weights(direct):
    wl = _wl(direct=direct)
    wl.params[:, 7] = wl.params[:, 6]
    wl.params[:, 8] = wl.params[:, 6]
    s0 = model.build(wl.grid, wl.ld_model, wl.npb, True, direct=direct)
    s1 = model.build(wl.grid, wl.ld_model, wl.npb, True, direct=direct, shared=True)
    f0 = model.evaluate(s0, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime)
    f1 = model.evaluate(s1, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime)
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-15)


def test_uniform_disk_is_exact_with_shared_weights():
    """Every weight row sums to one, so a uniform disk gives 1 - a(z, k_pb) / pi whatever k the weights use."""
    s = model.build(W.GRID, "uniform", npb=3, chromatic=True, shared=True)
    ks = np.array([0.08, 0.1, 0.13])
    for pb, k in enumerate(ks):
        _, istar, ldw = model.ld_weights(s, model.weights_k(s, ks, k), (), pb)
        zs = np.linspace(0, 1 + k, 41)[:-1]
        f = model.flux_from_distance(s, zs, np.ones(zs.size, bool), k, ldw, istar)
        np.testing.assert_allclose(f, 1 - intersection_area(1.0, k, zs) / np.pi, rtol=0, atol=2e-15)


def test_weights_use_the_mean_radius_ratio_and_area_the_own():
    s = model.build(W.GRID, "quadratic", npb=2, chromatic=True, shared=True)
    ks = np.array([0.09, 0.11])
    assert model.weights_k(s, ks, 0.09) == pytest.approx(0.10, abs=1e-16)
    assert model.weights_k(model.build(W.GRID, "quadratic"), np.array([0.09]), 0.09) == 0.09


def test_sharing_error_is_first_order_in_the_spread_and_small_for_percent_level_spreads():
    """Sect. 3.4: per-passband variations of k change the weights little.  The flux change from
    sharing is linear in the spread, and a 1% spread adds less than 1e-3 of the transit depth
    to the model's error against the exact integral (about 5 ppm at k = 0.1)."""
    coef = (0.4, 0.25)
    istar = ld.istar("quadratic", coef)
    I = lambda m: ld.profile("quadratic", m, coef)  # noqa: E731
    s_sh = model.build(W.GRID, "quadratic", npb=2, chromatic=True, shared=True)
    s_pb = model.build(W.GRID, "quadratic", npb=2, chromatic=True)

    def flux(setup, ks, pb, z):
        _, _, ldw = model.ld_weights(setup, model.weights_k(setup, ks, ks[pb]), coef, pb)
        return model.flux_from_distance(setup, np.array([z]), np.array([True]), ks[pb], ldw, istar)[0]

    k0 = 0.1
    for g in np.linspace(0.05, 0.95, 10):
        z = g * (1 + k0)
        d1 = flux(s_sh, np.array([k0, k0 * 1.02]), 0, z) - flux(s_pb, np.array([k0, k0 * 1.02]), 0, z)
        d2 = flux(s_sh, np.array([k0, k0 * 1.04]), 0, z) - flux(s_pb, np.array([k0, k0 * 1.04]), 0, z)
        assert abs(d2 - 2 * d1) <= 0.1 * abs(d2) + 1e-9
        ks = np.array([k0 * 0.995, k0 * 1.005])
        ex = exact.exact_flux(ks[0], z, I, istar)
        # 1% spread: the sharing error stays below 1e-3 of the depth k^2 (taking k-bar for the
        # area as well would shift the depth by 1e-2 k^2)
        assert abs(flux(s_sh, ks, 0, z) - ex) < abs(flux(s_pb, ks, 0, z) - ex) + 1e-3 * k0 ** 2


@pytest.mark.parametrize("direct", [False, True])
def test_shared_jacobian_matches_finite_differences(direct):
    from tests.test_oracle_grad import _smooth_points
    wl = _wl(npv=2, npt=1400, npb=2, seed=43, direct=direct, k_range=(0.05, 0.2) if direct else (0.02, 0.25),
             shared_weights=True)
    s = model.build(wl.grid, wl.ld_model, wl.npb, True, direct=direct, shared=True)
    for p in range(wl.npv):
        row = wl.params[p].copy()
        if row[4] == 0.0:
            row[4] = 1e-4
        steps = np.array([1e-6, 1e-7, 1e-6, 1e-6, 1e-6, 1e-6] + [1e-6] * (row.size - 6))
        J = grad.jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime)
        Jfd = grad.fd_jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime, steps)
        ok = _smooth_points(s, wl, row, steps)
        # the k cell of the mean radius ratio moves too (table model): keep points whose stencil keeps it
        if not direct:
            for j in (6, 7):
                for sgn in (1, -1):
                    rr = row.copy()
                    rr[j] += sgn * steps[j]
                    if model.k_cell(s, rr[6:8].mean())[0] != model.k_cell(s, row[6:8].mean())[0]:
                        ok[:] = False
        assert ok.sum() > 0.8 * wl.npt
        J, Jfd = J[ok], Jfd[ok]
        noise = 4 * np.finfo(float).eps * J.shape[0] / (2 * steps)
        assert np.all(np.abs(J.sum(0) - Jfd.sum(0)) <= 1e-5 * np.abs(Jfd.sum(0)) + noise)
        scale = np.maximum(np.abs(Jfd).max(0), 1e-12)
        assert np.all(np.abs(J - Jfd) / scale < 1e-4)
        # the weights' k-derivative reaches the other passband's k column
        assert np.abs(J[wl.pb_index[ok] == 0, 7]).max() > 0
