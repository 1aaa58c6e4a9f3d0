"""Pins against the analytic quadratic-law light curve of Mandel & Agol (2002).

The closed form (elliptic integrals, ``oracle/mandel_agol.py``) and the 1-D
radial quadrature of ``oracle/exact.py`` compute the same occulted flux by
independent routes; their agreement pins both.  The RoadRunner oracle is then
held to the paper's error level against the closed form on the C1 workload.
"""
import numpy as np
import pytest

from oracle import exact, mandel_agol as MA, model, orbit
from oracle.area import intersection_area
from paper_2009_08500_gb300 import workloads as W

# (p, z) pairs reaching every geometric case of the closed form: no overlap,
# partial overlaps with the planet's centre off and over the stellar disk, a
# planet wholly inside the disk (off and over the stellar centre), its rim
# through the centre (z = p), internal contact (z = 1 - p), a centred planet,
# p = z = 1/2, and planets larger than the star (partial and total eclipse).
CASES = sorted({(p, z) for p in (0.01, 0.1, 0.3, 0.5, 0.7, 1.0, 1.5)
                for z in (0.0, 0.5 * p, p, abs(1 - p), abs(1 - p) + 1e-3, 0.5, 0.9, 1.0, 1 + 0.5 * p,
                          1 + p - 1e-4, 1 + p)})
LAWS = [(0.4, 0.25), (0.1, 0.6), (1.0, 0.0), (0.8, -0.3), (0.0, 0.0)]


@pytest.mark.parametrize("g1,g2", LAWS)
def test_closed_form_matches_the_radial_quadrature(g1, g2):
    intensity = lambda mu: 1 - g1 * (1 - mu) - g2 * (1 - mu) ** 2  # noqa: E731
    istar = np.pi * (1 - g1 / 3 - g2 / 6)
    for p, z in CASES:
        ref = exact.exact_flux(p, z, intensity, istar) if z < 1 + p else 1.0
        assert MA.flux_quadratic(p, z, g1, g2) == pytest.approx(ref, abs=1e-10), (p, z)


def test_uniform_disk_and_total_eclipse():
    for p, z in CASES:
        expected = 1 - intersection_area(1.0, p, z) / np.pi if z < 1 + p else 1.0
        assert MA.flux_quadratic(p, z, 0.0, 0.0) == pytest.approx(expected, abs=1e-13), (p, z)
    for g1, g2 in LAWS:
        assert MA.flux_quadratic(1.5, 0.2, g1, g2) == pytest.approx(0.0, abs=1e-14)
        assert MA.flux_quadratic(1.0, 0.0, g1, g2) == pytest.approx(0.0, abs=1e-14)


def test_elliptic_integrals_against_their_definitions():
    from scipy.integrate import quad
    for k in (0.0, 0.3, 0.7, 0.95):
        s2 = lambda t: np.sin(t) ** 2  # noqa: E731
        K = quad(lambda t: 1 / np.sqrt(1 - k * k * s2(t)), 0, np.pi / 2, epsabs=1e-14)[0]
        E = quad(lambda t: np.sqrt(1 - k * k * s2(t)), 0, np.pi / 2, epsabs=1e-14)[0]
        assert MA.ellip_k(k) == pytest.approx(K, abs=1e-13)
        assert MA.ellip_e(k) == pytest.approx(E, abs=1e-13)
        for n in (-3.0, -0.5, 0.4):
            Pi = quad(lambda t: 1 / ((1 - n * s2(t)) * np.sqrt(1 - k * k * s2(t))), 0, np.pi / 2, epsabs=1e-14)[0]
            assert MA.ellip_pi(n, k) == pytest.approx(Pi, abs=1e-12)


def test_roadrunner_oracle_on_c1_within_the_paper_error_level():
    """Sect. 3.3, Fig. 2-3: a few ppm at most, well below 1 ppm on average."""
    wl = W.make_c1()
    flux = model.evaluate_workload(wl)[0]
    T0, P, a, b, e, w, k, u1, u2 = wl.params[0]
    z, front, ok = orbit.projected_distance(wl.times, T0, P, a, b, e, w)
    assert ok.all() and front.all()
    ref = np.array([MA.flux_quadratic(k, zi, u1, u2) for zi in z])
    err = np.abs(flux - ref)
    assert (ref < 1).sum() > 500          # the transit is well sampled
    assert err.max() < 5e-6
    assert err.mean() < 5e-7
