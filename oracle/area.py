"""Circle-circle intersection area a(c, k) of Eq. 5.

The paper uses the area but does not print it; this is the textbook lens
area of two disks, radius r centred at the origin and radius k at distance
c:

* c >= r + k            : 0 (disjoint)
* c <= |r - k|          : pi min(r, k)^2 (one inside the other)
* otherwise             : r^2 kappa_0 + k^2 kappa_1 - K / 2

where kappa_0 (kappa_1) is the half-angle subtended at the centre of the
r (k) circle by the chord through the two intersection points, and
K / 2 = 2 * (area of the triangle with sides r, k, c).  Heron's formula
gives K = sqrt((r + k - c)(c + r - k)(c - r + k)(c + r + k)).  The angles
are taken as atan2(K, c^2 + r^2 - k^2) and atan2(K, c^2 + k^2 - r^2), which
equal the textbook arccos((c^2 + r^2 - k^2) / (2 c r)) and
arccos((c^2 + k^2 - r^2) / (2 c k)) exactly (sin kappa_0 = K / (2 c r)),
but keep full relative accuracy near the contact points where the arccos
argument approaches +-1.
"""
import numpy as np


def intersection_area(r, k, c):
    """Area common to disk(0, r) and disk(c, k); all arguments broadcast."""
    r, k, c = np.broadcast_arrays(np.asarray(r, np.float64), np.asarray(k, np.float64),
                                  np.asarray(c, np.float64))
    out = np.zeros(np.broadcast(r, k, c).shape)
    disjoint = c >= r + k
    nested = (~disjoint) & (c <= np.abs(r - k))
    lens = ~(disjoint | nested)
    m = np.minimum(r, k)
    out[nested] = np.pi * m[nested] ** 2
    rr, kk, cc = r[lens], k[lens], c[lens]
    heron = (rr + kk - cc) * (cc + rr - kk) * (cc - rr + kk) * (cc + rr + kk)
    K = np.sqrt(np.maximum(heron, 0.0))
    kappa0 = np.arctan2(K, cc * cc + rr * rr - kk * kk)
    kappa1 = np.arctan2(K, cc * cc + kk * kk - rr * rr)
    out[lens] = rr * rr * kappa0 + kk * kk * kappa1 - 0.5 * K
    return out if out.ndim else float(out)
