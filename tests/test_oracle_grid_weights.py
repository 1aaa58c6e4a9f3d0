"""Pins for the radial grid (Sect. 3.1.1) and the weight vectors (Sect. 2, 3.1)."""
import numpy as np
import pytest

from oracle import grid as G
from oracle import weights as Wt
from oracle.area import intersection_area


def test_grid_structure():
    ze, zm, mu = G.create_z_grid(0.7, 200, 300)
    assert ze.shape == (501,) and zm.shape == (500,) and mu.shape == (500,)
    assert ze[0] == 0.0 and ze[-1] == 1.0
    assert ze[200] == pytest.approx(0.7, abs=1e-15)
    assert np.all(np.diff(ze) > 0)
    # constant dz inside zcut
    np.testing.assert_allclose(np.diff(ze[:201]), 0.7 / 200, rtol=0, atol=1e-15)
    # constant dmu outside zcut
    mue = np.sqrt(1 - ze[200:] ** 2)
    # mu recovered from ze loses digits near the limb (1 - ze^2 cancels)
    np.testing.assert_allclose(np.diff(mue), -np.sqrt(1 - 0.49) / 300, rtol=0, atol=1e-13)
    np.testing.assert_allclose(zm, 0.5 * (ze[1:] + ze[:-1]), rtol=0, atol=0)
    np.testing.assert_allclose(mu ** 2 + zm ** 2, 1.0, atol=1e-15)


def test_grid_rejects_bad_arguments():
    with pytest.raises(ValueError):
        G.create_z_grid(1.0, 10, 10)
    with pytest.raises(ValueError):
        G.create_z_grid(0.5, 0, 10)


@pytest.fixture(scope="module")
def ze():
    return G.create_z_grid(0.7, 200, 300)[0]


@pytest.mark.parametrize("k", [0.005, 0.05, 0.1, 0.3])
def test_weight_rows_sum_to_one_and_are_nonnegative(ze, k):
    dg, w = Wt.calculate_weights(k, ze, 200)
    assert dg == pytest.approx(1 / 199)
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert w.min() >= -1e-13


def test_weight_support_is_the_covered_annuli(ze):
    k = 0.1
    for g in (0.0, 0.3, 0.8, 0.95):
        c = g * (1 + k)
        w = Wt.weight_vector(k, c, ze)
        lo, hi = c - k, c + k
        outside = (ze[1:] <= lo - 1e-12) | (ze[:-1] >= hi + 1e-12)
        assert np.all(w[outside] == 0.0)
        assert np.all(w[~outside] >= 0.0)


def test_weight_at_centre_is_annulus_area_over_planet_area(ze):
    # planet centred on the star: w_j = pi (ze_{j+1}^2 - ze_j^2) / (pi k^2) for annuli inside k
    k = 0.2
    w = Wt.weight_vector(k, 0.0, ze)
    inside = ze[1:] <= k
    np.testing.assert_allclose(w[inside], (ze[1:][inside] ** 2 - ze[:-1][inside] ** 2) / k ** 2,
                               rtol=1e-13)


def test_limit_node_g_equal_one(ze):
    w = Wt.weight_vector(0.1, 1.1, ze)
    assert w[-1] == 1.0 and np.count_nonzero(w) == 1


def test_weight_vector_by_pixel_counting(ze):
    # covered area of each annulus by brute force, for one planet position
    k, c = 0.15, 0.8
    n = 2500
    h = 2 * k / n
    xs = c - k + h * (np.arange(n) + 0.5)
    X, Y = np.meshgrid(xs, -k + h * (np.arange(n) + 0.5))
    r = np.hypot(X, Y)
    inside = ((X - c) ** 2 + Y * Y < k * k) & (r < 1)
    counts = np.histogram(r[inside], bins=ze)[0] * h * h
    w = Wt.weight_vector(k, c, ze)
    atot = intersection_area(1.0, k, c)
    assert np.abs(w * atot - counts).sum() < 2e-3 * atot


def test_3d_table_nodes(ze):
    dk, dg, w = Wt.calculate_weights_3d(5, 0.01, 0.05, ze, 20)
    assert dk == pytest.approx(0.01) and w.shape == (5, 20, 500)
    np.testing.assert_array_equal(w[2], Wt.calculate_weights(0.01 + 2 * dk, ze, 20)[1])
