"""Keplerian orbit -> projected star-planet centre distance.

The paper names the orbit parameters (Sect. 4.1: zero epoch T0, period P,
scaled semi-major axis a, inclination, eccentricity e, argument of
periastron w; e and w default to 0) but prints no orbit equations.  This is
the textbook two-body form, in units of the stellar radius:

* mean motion n = 2 pi / P;
* mid-transit (conjunction) at true anomaly f0 = pi/2 - w, eccentric anomaly
  E0 = 2 atan2(sqrt(1-e) sin(f0/2), sqrt(1+e) cos(f0/2)), mean anomaly
  M0 = E0 - e sin E0, reached at t = T0;
* tau = t - T0 reduced to the nearest period (tau -= P round(tau/P)),
  M = M0 + n tau;
* Kepler's equation E - e sin E = M solved by Newton iteration;
* f = 2 atan2(sqrt(1+e) sin(E/2), sqrt(1-e) cos(E/2)), r = a (1 - e cos E);
* sky-plane position X = -r cos(w + f), Y = -r sin(w + f) cos i, and
  z = sqrt(X^2 + Y^2); the planet is in front of the star iff sin(w + f) > 0.

Reading: the library takes the impact parameter b instead of i, with
cos i = b / a (b is the nominal a cos i, without the eccentric factor).
"""
import numpy as np

KEPLER_MAX_ITER = 100
# Newton stops once a step is below this (relative); convergence is quadratic,
# so what remains after such a step is round-off.  FP64 round-off in the
# residual keeps steps near 1e-15 for e close to 1, hence not smaller.
KEPLER_TOL = 1e-13


def conjunction_anomalies(e, w):
    f0 = 0.5 * np.pi - w
    E0 = 2.0 * np.arctan2(np.sqrt(1.0 - e) * np.sin(0.5 * f0), np.sqrt(1.0 + e) * np.cos(0.5 * f0))
    M0 = E0 - e * np.sin(E0)
    return f0, E0, M0


def solve_kepler(M, e):
    """Eccentric anomaly E with E - e sin E = M; returns (E, converged)."""
    M = np.asarray(M, np.float64)
    E = M.copy()
    done = np.zeros(M.shape, bool)
    for _ in range(KEPLER_MAX_ITER):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = np.where(done, E, E - dE)
        done |= np.abs(dE) < KEPLER_TOL * np.maximum(1.0, np.abs(E))
        if done.all():
            break
    return E, done


def reduced_time(t, T0, P):
    tau = np.asarray(t, np.float64) - T0
    return tau - P * np.rint(tau / P)


def projected_distance(t, T0, P, a, b, e, w):
    """z(t) for one orbit; returns (z, in_front, converged) arrays shaped like t."""
    n = 2.0 * np.pi / P
    _, _, M0 = conjunction_anomalies(e, w)
    tau = reduced_time(t, T0, P)
    M = M0 + n * tau
    E, ok = solve_kepler(M, e)
    f = 2.0 * np.arctan2(np.sqrt(1.0 + e) * np.sin(0.5 * E), np.sqrt(1.0 - e) * np.cos(0.5 * E))
    r = a * (1.0 - e * np.cos(E))
    cos_i = b / a
    X = -r * np.cos(w + f)
    Y = -r * np.sin(w + f) * cos_i
    z = np.sqrt(X * X + Y * Y)
    return z, np.sin(w + f) > 0.0, ok
