"""Radial discretisation of the stellar disk (Sect. 3.1.1).

The disk radius [0, 1] is cut at z_cut.  Inside, the annulus edges are
spaced uniformly in z (nzin annuli); outside, uniformly in mu = sqrt(1 - z^2)
(nzlimb annuli), so the limb, where the brightness changes fastest, is
sampled densely.  Returned: edges ze (nz + 1), bin "means" zm (nz), and
mu at zm, with nz = nzin + nzlimb.

Reading: the paper calls zm the bin means without defining them; the
arithmetic midpoint in z of each bin is used for both regions.
"""
import numpy as np


def create_z_grid(zcut: float, nzin: int, nzlimb: int):
    if not (0.0 < zcut < 1.0) or nzin < 1 or nzlimb < 1:
        raise ValueError("need 0 < zcut < 1, nzin >= 1, nzlimb >= 1")
    ze_inner = np.array([j * zcut / nzin for j in range(nzin + 1)], dtype=np.float64)
    mu_cut = np.sqrt(1.0 - zcut * zcut)
    mu_outer = np.array([mu_cut * (1.0 - m / nzlimb) for m in range(1, nzlimb + 1)])
    ze_outer = np.sqrt(1.0 - mu_outer * mu_outer)
    ze = np.concatenate([ze_inner, ze_outer])
    zm = 0.5 * (ze[:-1] + ze[1:])
    mu = np.sqrt(1.0 - zm * zm)
    return ze, zm, mu
