"""Pins for the oracle's direct model (Sect. 3.1.2 without the interpolation in k)."""
import numpy as np
import pytest

from oracle import exact, grad, ld, model, weights
from oracle.area import intersection_area
from paper_2009_08500_gb300 import workloads as W


def _single(setup, k, z, coef=(), pb=0):
    _, istar, ldw = model.ld_weights(setup, k, coef, pb)
    return model.flux_from_distance(setup, np.atleast_1d(z), np.array([True]), k, ldw, istar)[0]


@pytest.mark.parametrize("k", [0.003, 0.1, 0.45, 0.8])
def test_lens_partials_against_50_digit_differences(k):
    """d a / d k and d a / d c against central differences of the arccos form at 50 digits."""
    mp = pytest.importorskip("mpmath")
    from oracle.exact import area_mp
    rng = np.random.default_rng(int(k * 1e4))
    rs = rng.uniform(0.05, 1.0, 12)
    cs = rng.uniform(0.0, 1.0 + k, 12)
    for r, c in zip(rs, cs):
        A, dk, dc = weights.lens_partials(np.array([r]), k, c)
        h = mp.mpf("1e-20")
        with mp.workdps(50):
            ref_k = (area_mp(r, mp.mpf(k) + h, c) - area_mp(r, mp.mpf(k) - h, c)) / (2 * h)
            ref_c = (area_mp(r, k, mp.mpf(c) + h) - area_mp(r, k, mp.mpf(c) - h)) / (2 * h)
        assert A[0] == pytest.approx(intersection_area(r, k, c), abs=1e-15)
        assert dk[0] == pytest.approx(float(ref_k), abs=1e-12), (r, c)
        assert dc[0] == pytest.approx(float(ref_c), abs=1e-12), (r, c)


def test_lens_partials_limits():
    k = 0.2
    # planet inside the disk: area pi k^2, d/dk = 2 pi k, d/dc = 0
    A, dk, dc = weights.lens_partials(np.array([0.9]), k, 0.3)
    assert (A[0], dk[0], dc[0]) == (pytest.approx(np.pi * k * k), pytest.approx(2 * np.pi * k), 0.0)
    # disk inside the planet: area pi r^2, no dependence on k or c
    A, dk, dc = weights.lens_partials(np.array([0.1]), k, 0.05)
    assert (A[0], dk[0], dc[0]) == (pytest.approx(np.pi * 0.01), 0.0, 0.0)
    # disjoint
    A, dk, dc = weights.lens_partials(np.array([0.5]), k, 0.8)
    assert (A[0], dk[0], dc[0]) == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("k", [0.004, 0.07, 0.35, 0.75])
def test_weight_derivative_matches_differences_and_sums_to_zero(k, grid):
    ze, _, _ = weights_grid(grid)
    h = 1e-6
    for g in (0.0, 0.2, 0.55, 0.8, 0.97, 1.0):
        dw = weights.weight_vector_dk(k, g, ze)
        fd = (weights.weight_vector(k + h, g * (1 + k + h), ze)
              - weights.weight_vector(k - h, g * (1 + k - h), ze)) / (2 * h)
        # rows sum to one for every k, so their k-derivative sums to zero
        assert abs(dw.sum()) < 1e-10 * max(1.0, np.abs(dw).max())
        # the area goes as d^(3/2) in the distance d of an edge from a contact, so a
        # difference across a contact is only O(sqrt(h)) accurate: skip those bins
        c = g * (1 + k)
        near = np.min(np.abs(ze[:, None] - np.array([c - k, c + k, k - c])[None, :]), axis=1) < 100 * h
        keep = ~(near[1:] | near[:-1])
        np.testing.assert_allclose(dw[keep], fd[keep], rtol=0, atol=2e-6 * max(1.0, np.abs(fd).max()))


def weights_grid(grid):
    from oracle import grid as G
    ze, zm, mu = G.create_z_grid(grid["zcut"], grid["nzin"], grid["nzlimb"])
    return ze, zm, mu


def test_direct_equals_table_on_k_nodes(grid):
    coef = (0.4, 0.25)
    st = model.build(grid, "quadratic")
    sd = model.build(grid, "quadratic", direct=True)
    for j in (0, 7, grid["nk"] - 1):
        k = grid["k0"] + j * st.dk
        _, _, lt = model.ld_weights(st, k, coef, 0)
        _, _, ldd = model.ld_weights(sd, k, coef, 0)
        np.testing.assert_allclose(ldd, lt, rtol=0, atol=1e-13)


@pytest.mark.parametrize("k", [0.002, 0.04, 0.33, 0.5, 0.8])
def test_direct_within_paper_error_level_of_exact_integral(k, grid):
    """The g-only interpolation keeps the few-ppm error of Sect. 3.3 up to k = 0.3; beyond the k
    table the error scales with the depth k^2 (worst near z = k, where the planet's rim crosses
    the star's centre and the mean brightness has a kink in g)."""
    coef = (0.4, 0.25)
    s = model.build(grid, "quadratic", direct=True)
    istar = ld.istar("quadratic", coef)
    I = lambda m: ld.profile("quadratic", m, coef)  # noqa: E731
    errs = [abs(_single(s, k, g * (1 + k), coef) - exact.exact_flux(k, g * (1 + k), I, istar))
            for g in np.linspace(0.0, 0.999, 40)]
    assert max(errs) < max(9e-6, 1.5e-4 * k * k)
    assert np.mean(errs) < 1e-6 * max(1.0, (k / 0.3) ** 2)


def test_direct_uniform_disk_is_exact():
    s = model.build(W.GRID, "uniform", direct=True)
    for k in (0.003, 0.4, 0.9):
        zs = np.linspace(0.0, 1 + k, 37)[:-1]
        _, istar, ldw = model.ld_weights(s, k, (), 0)
        f = model.flux_from_distance(s, zs, np.ones(zs.size, bool), k, ldw, istar)
        np.testing.assert_allclose(f, 1 - intersection_area(1.0, k, zs) / np.pi, rtol=0, atol=3e-15)


def test_direct_k_domain(grid):
    wl = W.make_small("quadratic", npv=4, npt=200, seed=3, direct=True, k_range=(0.35, 0.6))
    s = model.build(grid, "quadratic", direct=True)
    wl.params[1, 6] = 0.0
    wl.params[2, 6] = 1.0
    f, st = model.evaluate(s, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime, return_status=True)
    assert st[0] == 0 and st[3] == 0 and np.all(np.isfinite(f[[0, 3]]))
    assert st[1] == model.ST_K_RANGE and st[2] == model.ST_K_RANGE
    assert np.all(np.isnan(f[[1, 2]]))
    # the same k is out of range for the tabulated model
    st_tab = model.evaluate(model.build(grid, "quadratic"), wl.times, wl.pb_index, wl.params[:1],
                            wl.supersampling, wl.exptime, return_status=True)[1]
    assert st_tab[0] == model.ST_K_RANGE


def test_direct_jacobian_matches_finite_differences():
    from tests.test_oracle_grad import _smooth_points
    for case in (dict(ld_model="quadratic", eccentric=True, k_range=(0.32, 0.5)),
                 dict(ld_model="nonlinear", eccentric=True, k_range=(0.002, 0.01)),
                 dict(ld_model="quadratic", eccentric=True, npb=2, chromatic=True, k_range=(0.05, 0.2))):
        wl = W.make_small(npv=2, npt=1200, seed=23, span=4.0, direct=True, **case)
        s = model.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, direct=True)
        for p in range(wl.npv):
            row = wl.params[p].copy()
            if row[4] == 0.0:
                row[4] = 1e-4
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
