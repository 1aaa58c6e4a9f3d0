"""Analytic transit light curve for quadratic limb darkening (Mandel & Agol 2002).

Test infrastructure (like the rest of ``oracle/``): a second, independent
route to the quantity that ``exact.exact_flux`` integrates numerically, used
only to pin that quadrature and the RoadRunner oracle built on it.

Mandel & Agol (2002, ApJ 580, L171) give the flux of a star with
I(mu) = 1 - g1 (1 - mu) - g2 (1 - mu)^2 occulted by a dark disk of radius p
(stellar radii) at centre distance z in closed form.  Writing the law as
1 - c2 (1 - mu) - c4 (1 - mu^2) with c2 = g1 + 2 g2 and c4 = -g2,

    F = 1 - [ (1 - c2) lambda_e + c2 (lambda_d + 2/3 Theta(p - z)) - c4 eta_d ] / (4 Omega),
    4 Omega = 1 - c2 / 3 - c4 / 2,

where lambda_e is the occulted fraction of a uniform disk, and lambda_d and
eta_d the occulted parts of the disk integrals of mu and of 1 - mu^2, given
in that paper per geometric case (their Table 1) through complete elliptic
integrals of the first, second and third kind.  The elliptic integrals are
evaluated here from Carlson's symmetric forms (scipy.special.elliprf,
elliprd, elliprj):

    K(k)    = R_F(0, 1 - k^2, 1)
    E(k)    = R_F(0, 1 - k^2, 1) - k^2 / 3 R_D(0, 1 - k^2, 1)
    Pi(n,k) = R_F(0, 1 - k^2, 1) + n / 3 R_J(0, 1 - k^2, 1, 1 - n)

with Pi(n, k) = int_0^{pi/2} dtheta / ((1 - n sin^2 theta) sqrt(1 - k^2 sin^2 theta)).
"""
import numpy as np
from scipy.special import elliprd, elliprf, elliprj


def ellip_k(k):
    return float(elliprf(0.0, 1.0 - k * k, 1.0))


def ellip_e(k):
    m1 = 1.0 - k * k
    return float(elliprf(0.0, m1, 1.0) - k * k / 3.0 * elliprd(0.0, m1, 1.0))


def ellip_pi(n, k):
    m1 = 1.0 - k * k
    return float(elliprf(0.0, m1, 1.0) + n / 3.0 * elliprj(0.0, m1, 1.0, 1.0 - n))


def lambda_e(p, z):
    """Occulted fraction of a uniform stellar disk."""
    if z >= 1.0 + p:
        return 0.0
    if p >= 1.0 and z <= p - 1.0:
        return 1.0
    if z <= 1.0 - p:
        return p * p
    kap0 = np.arccos(np.clip((p * p + z * z - 1.0) / (2.0 * p * z), -1.0, 1.0))
    kap1 = np.arccos(np.clip((1.0 - p * p + z * z) / (2.0 * z), -1.0, 1.0))
    root = np.sqrt(max(0.0, 4.0 * z * z - (1.0 + z * z - p * p) ** 2))
    return float((p * p * kap0 + kap1 - 0.5 * root) / np.pi)


def _lambda1(p, z):
    a, b, q = (z - p) ** 2, (z + p) ** 2, p * p - z * z
    k = np.sqrt((1.0 - a) / (4.0 * z * p))
    t1 = ((1.0 - b) * (2.0 * b + a - 3.0) - 3.0 * q * (b - 2.0)) * ellip_k(k)
    t2 = 4.0 * p * z * (z * z + 7.0 * p * p - 4.0) * ellip_e(k)
    t3 = -3.0 * q / a * ellip_pi((a - 1.0) / a, k)
    return (t1 + t2 + t3) / (9.0 * np.pi * np.sqrt(p * z))


def _lambda2(p, z):
    a, b, q = (z - p) ** 2, (z + p) ** 2, p * p - z * z
    ki = np.sqrt(4.0 * z * p / (1.0 - a))
    t1 = (1.0 - 5.0 * z * z + p * p + q * q) * ellip_k(ki)
    t2 = (1.0 - a) * (z * z + 7.0 * p * p - 4.0) * ellip_e(ki)
    t3 = -3.0 * q / a * ellip_pi((a - b) / a, ki)
    return 2.0 / (9.0 * np.pi * np.sqrt(1.0 - a)) * (t1 + t2 + t3)


def _lambda3(p):
    k = 1.0 / (2.0 * p)
    return (1.0 / 3.0 + 16.0 * p / (9.0 * np.pi) * (2.0 * p * p - 1.0) * ellip_e(k)
            - (1.0 - 4.0 * p * p) * (3.0 - 8.0 * p * p) / (9.0 * np.pi * p) * ellip_k(k))


def _lambda4(p):
    k = 2.0 * p
    return 1.0 / 3.0 + 2.0 / (9.0 * np.pi) * (4.0 * (2.0 * p * p - 1.0) * ellip_e(k) + (1.0 - 4.0 * p * p) * ellip_k(k))


def _lambda5(p):
    return (2.0 / (3.0 * np.pi) * np.arccos(1.0 - 2.0 * p)
            - 4.0 / (9.0 * np.pi) * (3.0 + 2.0 * p - 8.0 * p * p) * np.sqrt(p * (1.0 - p))
            - (2.0 / 3.0 if p > 0.5 else 0.0))


def _lambda6(p):
    return -2.0 / 3.0 * (1.0 - p * p) ** 1.5


def _eta2(p, z):
    return 0.5 * p * p * (p * p + 2.0 * z * z)


def _eta1(p, z):
    a, b = (z - p) ** 2, (z + p) ** 2
    kap0 = np.arccos(np.clip((p * p + z * z - 1.0) / (2.0 * p * z), -1.0, 1.0))
    kap1 = np.arccos(np.clip((1.0 - p * p + z * z) / (2.0 * z), -1.0, 1.0))
    return (kap1 + 2.0 * _eta2(p, z) * kap0
            - 0.25 * (1.0 + 5.0 * p * p + z * z) * np.sqrt(max(0.0, (1.0 - a) * (b - 1.0)))) / (2.0 * np.pi)


def lambda_eta_d(p, z):
    """(lambda_d, eta_d) by the geometric cases of Mandel & Agol (2002), Table 1."""
    if z >= 1.0 + p:                                    # no overlap
        return 0.0, 0.0
    if p >= 1.0 and z <= p - 1.0:                       # the whole star covered
        return 0.0, 0.5
    if p == 0.5 and z == 0.5:
        return 1.0 / 3.0 - 4.0 / (9.0 * np.pi), 3.0 / 32.0
    if p < 1.0 and z == 1.0 - p:                        # internal contact (lambda_5 carries the p > 1/2 term)
        return _lambda5(p), _eta2(p, z)
    if z > 0.5 + abs(p - 0.5):                          # partial, planet centre outside the far chord
        return _lambda1(p, z), _eta1(p, z)
    if p > 0.5:
        if z == p:
            return _lambda3(p), _eta1(p, z)
        if abs(1.0 - p) <= z < p:                       # partial, planet over the stellar centre
            return _lambda1(p, z), _eta1(p, z)
    if z == 0.0:
        return _lambda6(p), _eta2(p, z)
    if p < 0.5 and z == p:
        return _lambda4(p), _eta2(p, z)
    return _lambda2(p, z), _eta2(p, z)                  # planet wholly inside the disk


def flux_quadratic(p, z, g1, g2):
    """Normalised flux of a star with quadratic limb darkening occulted by a disk of radius p at distance z."""
    p, z = float(p), abs(float(z))
    if p <= 0.0 or z >= 1.0 + p:
        return 1.0
    c2, c4 = g1 + 2.0 * g2, -g2
    le = lambda_e(p, z)
    ld, ed = lambda_eta_d(p, z)
    theta = 1.0 if p > z else 0.0
    return 1.0 - ((1.0 - c2) * le + c2 * (ld + 2.0 / 3.0 * theta) - c4 * ed) / (1.0 - c2 / 3.0 - c4 / 2.0)
