"""Exact references that do not use the RoadRunner discretisation.

* ``occulted_flux_radial`` -- the occluded integral of Eq. 1-2,
  int_{A_p} I dA, evaluated in one dimension thanks to radial symmetry
  (Sect. 2 cites the 1-D approach of Kreidberg 2015): on the circle of
  radius r about the stellar centre the planet covers the arc of
  half-angle theta(r) with cos theta = (r^2 + c^2 - k^2) / (2 r c), so
  int_{A_p} I dA = int_0^1 I(r) 2 theta(r) r dr.  Adaptive quadrature
  (scipy QUADPACK) with breakpoints where theta(r) has its square-root
  ends.  For quadratic limb darkening this is the quantity the analytic
  model of Mandel & Agol (2002) gives in closed form.
* ``occulted_flux_pixels`` -- brute-force 2-D midpoint-rule integration of
  I over the pixels covered by both disks.
* ``area_mp`` -- the textbook arccos lens area in 50-digit mpmath.
"""
import numpy as np


def _theta(r, k, c):
    if c == 0.0:
        return np.pi if r < k else 0.0
    x = (r * r + c * c - k * k) / (2.0 * r * c)
    return float(np.arccos(min(1.0, max(-1.0, x))))


def occulted_flux_radial(k: float, c: float, intensity_of_r, epsabs=1e-14, epsrel=1e-13):
    """int over the planet disk (clipped to the star) of I, as a 1-D radial integral."""
    from scipy.integrate import quad
    lo, hi = max(0.0, c - k), min(1.0, c + k)
    if hi <= lo:
        return 0.0
    cuts = sorted({lo, hi, *(x for x in (abs(c - k),) if lo < x < hi)})
    total = 0.0
    f = lambda r: intensity_of_r(r) * 2.0 * _theta(r, k, c) * r  # noqa: E731
    for a, b in zip(cuts[:-1], cuts[1:]):
        val, _ = quad(f, a, b, epsabs=epsabs, epsrel=epsrel, limit=2000)
        total += val
    return total


def exact_flux(k: float, c: float, intensity_of_mu, istar: float) -> float:
    """Normalised flux 1 - (occluded integral) / I_star for a planet in front of the star."""
    I_r = lambda r: intensity_of_mu(np.sqrt(max(0.0, 1.0 - r * r)))  # noqa: E731
    return 1.0 - occulted_flux_radial(k, c, I_r) / istar


def occulted_flux_pixels(k: float, c: float, intensity_of_mu, n: int = 2000, chunk: int = 250):
    """Midpoint-rule pixel sum of I over disk(0,1) intersected with disk((c,0),k)."""
    h = 2.0 * k / n
    xs = c - k + h * (np.arange(n) + 0.5)
    total = 0.0
    for j0 in range(0, n, chunk):
        ys = -k + h * (np.arange(j0, min(n, j0 + chunk)) + 0.5)
        X, Y = np.meshgrid(xs, ys, indexing="xy")
        r2 = X * X + Y * Y
        inside = (r2 < 1.0) & ((X - c) ** 2 + Y * Y < k * k)
        mu = np.sqrt(np.clip(1.0 - r2[inside], 0.0, 1.0))
        total += float(np.sum(intensity_of_mu(mu)))
    return total * h * h


def area_mp(r, k, c, dps: int = 50):
    """Textbook lens area with arccos, evaluated with ``dps`` decimal digits."""
    import mpmath as mp
    with mp.workdps(dps):
        r, k, c = mp.mpf(r), mp.mpf(k), mp.mpf(c)
        if c >= r + k:
            return mp.mpf(0)
        if c <= abs(r - k):
            return mp.pi * min(r, k) ** 2
        k0 = mp.acos((c * c + r * r - k * k) / (2 * c * r))
        k1 = mp.acos((c * c + k * k - r * r) / (2 * c * k))
        heron = (-c + r + k) * (c + r - k) * (c - r + k) * (c + r + k)
        return r * r * k0 + k * k * k1 - mp.sqrt(heron) / 2
