"""Weight vectors w on the (k, g) grid (Sect. 2 below Eq. 4; Sect. 3.1, 3.1.2).

For a planet of radius ratio k at centre distance c, weight j is the area of
annulus j (between edges ze[j] and ze[j+1]) covered by the planet divided by
the total covered area:

    w_j = [a(ze[j+1], k, c) - a(ze[j], k, c)] / a(1, k, c)

Weights are tabulated against the grazing value g = c / (1 + k), g in [0, 1]
(Sect. 3.1), and -- for the interpolated model -- against k on [k0, k1]
(Sect. 3.1.2), giving w[nk][ng][nz].

Readings: g nodes are g_i = i dg with dg = 1 / (ng - 1), so that g = 0 and
g = 1 are nodes and the interpolation of Sect. 3.1.1 never reads past the
last node for g < 1; k nodes are k_m = k0 + m dk with dk = (k1 - k0) / (nk - 1).
At g = 1 the planet only touches the limb and the covered area is zero; the
weight vector there is taken as its limit, all weight in the outermost
annulus.  That node never contributes to a flux (g >= 1 is out of transit).
"""
import numpy as np

from .area import intersection_area


def weight_vector(k: float, c: float, ze: np.ndarray) -> np.ndarray:
    nz = len(ze) - 1
    a_tot = intersection_area(1.0, k, c)
    if c >= 1.0 + k or a_tot <= 0.0:
        w = np.zeros(nz)
        w[-1] = 1.0
        return w
    a_edges = intersection_area(ze, k, c)
    return (a_edges[1:] - a_edges[:-1]) / a_tot


def calculate_weights(k: float, ze: np.ndarray, ng: int):
    """Weight table in g for one k (the direct model): returns dg, w[ng][nz]."""
    dg = 1.0 / (ng - 1)
    w = np.stack([weight_vector(k, (i * dg) * (1.0 + k), ze) for i in range(ng)])
    return dg, w


def calculate_weights_3d(nk: int, k0: float, k1: float, ze: np.ndarray, ng: int):
    """Weight table in (k, g): returns dk, dg, w[nk][ng][nz]."""
    dk = (k1 - k0) / (nk - 1)
    tables = []
    dg = None
    for m in range(nk):
        dg, w = calculate_weights(k0 + m * dk, ze, ng)
        tables.append(w)
    return dk, dg, np.stack(tables)
