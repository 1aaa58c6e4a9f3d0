"""Pins for the oracle's circle-circle intersection area (the a(c, k) of Eq. 5)."""
import numpy as np
import pytest

from oracle.area import intersection_area
from oracle.exact import area_mp


def test_disjoint_and_nested_limits():
    assert intersection_area(1.0, 0.1, 1.1) == 0.0
    assert intersection_area(1.0, 0.1, 2.0) == 0.0
    assert intersection_area(1.0, 0.1, 0.9) == pytest.approx(np.pi * 0.01, rel=0, abs=1e-16)
    assert intersection_area(1.0, 0.1, 0.0) == pytest.approx(np.pi * 0.01, rel=0, abs=1e-16)
    # planet larger than the star: the star is hidden completely
    assert intersection_area(1.0, 2.0, 0.5) == pytest.approx(np.pi, rel=0, abs=1e-15)
    # radius-0 circle
    assert intersection_area(0.0, 0.1, 0.05) == 0.0


def test_equal_unit_circles_closed_form():
    # two unit disks whose centres are one radius apart: 2 pi / 3 - sqrt(3) / 2
    assert intersection_area(1.0, 1.0, 1.0) == pytest.approx(2 * np.pi / 3 - np.sqrt(3) / 2, abs=1e-15)
    # centre of the planet on the limb, k = 1: same configuration
    # half-covered disk: r = k, circles through each other's centre is the case above;
    # a large planet whose edge passes through the stellar centre covers a lens with
    # the analytic value of a circular segment pair
    r, k, c = 1.0, 3.0, 3.0
    # chord through intersection points; compare with direct segment formula
    x = (c * c + r * r - k * k) / (2 * c)          # chord abscissa from the star centre
    seg_r = r * r * np.arccos(x / r) - x * np.sqrt(r * r - x * x)
    seg_k = k * k * np.arccos((c - x) / k) - (c - x) * np.sqrt(k * k - (c - x) ** 2)
    assert intersection_area(r, k, c) == pytest.approx(seg_r + seg_k, abs=1e-13)


def test_symmetric_in_the_two_radii():
    rng = np.random.default_rng(11)
    r = rng.uniform(0.05, 1.0, 200)
    k = rng.uniform(0.01, 0.5, 200)
    c = rng.uniform(0.0, 1.6, 200)
    np.testing.assert_allclose(intersection_area(r, k, c), intersection_area(k, r, c), rtol=0, atol=2e-16)


@pytest.mark.parametrize("k", [0.01, 0.1, 0.3, 0.7])
def test_against_50_digit_arccos_form_including_contacts(k):
    pytest.importorskip("mpmath")
    rng = np.random.default_rng(int(k * 1000))
    cs = list(rng.uniform(max(0.0, 1 - k), 1 + k, 40))
    # within a few ulp .. 1e-6 of both contact points
    for d in (1e-15, 1e-13, 1e-11, 1e-9, 1e-7, 1e-5):
        cs += [1 + k - d, 1 - k + d]
    for c in cs:
        got = intersection_area(1.0, k, c)
        ref = float(area_mp(1.0, k, c))
        assert abs(got - ref) <= 4e-16 * max(1.0, np.pi * k * k), (k, c, got, ref)


def test_against_pixel_count():
    # area by counting midpoints of a fine pixel grid over the planet's bounding box
    for (r, k, c) in [(1.0, 0.3, 0.9), (0.6, 0.2, 0.55), (1.0, 0.5, 1.2)]:
        n = 3000
        h = 2 * k / n
        xs = c - k + h * (np.arange(n) + 0.5)
        ys = -k + h * (np.arange(n) + 0.5)
        X, Y = np.meshgrid(xs, ys)
        cnt = np.count_nonzero((X * X + Y * Y < r * r) & ((X - c) ** 2 + Y * Y < k * k))
        assert intersection_area(r, k, c) == pytest.approx(cnt * h * h, rel=2e-4)


def test_derivative_in_distance_is_minus_chord():
    # d area / dc = -(length of the common chord) = -K / c; pins kappa_0, kappa_1 and K together
    for (r, k, c) in [(1.0, 0.1, 0.95), (0.8, 0.25, 0.7), (1.0, 0.2, 1.1)]:
        h = 1e-6
        fd = (intersection_area(r, k, c + h) - intersection_area(r, k, c - h)) / (2 * h)
        K = np.sqrt((r + k - c) * (c + r - k) * (c - r + k) * (c + r + k))
        assert fd == pytest.approx(-K / c, rel=1e-7)
