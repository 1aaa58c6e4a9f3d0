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


def lens_partials(r, k, c):
    """a(r, k, c) with its partials d a / d k and d a / d c (arrays r).

    Overlap of the radius-r disk and the planet: d a / d k is the arc of the
    planet's rim inside the disk, 2 k kappa_1, and d a / d c is minus the
    common chord, -K / c (K = sqrt of Heron's product); both vanish for
    disjoint circles, and for nested ones d a / d k = 2 pi k when the planet
    is the inner circle."""
    r = np.asarray(r, np.float64)
    A = np.zeros_like(r)
    dk = np.zeros_like(r)
    dc = np.zeros_like(r)
    nested = c <= np.abs(r - k)
    inner = nested & (k < r)
    A[nested] = np.pi * np.minimum(r[nested], k) ** 2
    dk[inner] = 2.0 * np.pi * k
    lens = ~nested & (c < r + k)
    rr = r[lens]
    heron = ((rr + k) - c) * (c + (rr - k)) * (c - (rr - k)) * (c + (rr + k))
    K = np.sqrt(np.maximum(heron, 0.0))
    kap0 = np.arctan2(K, c * c + (rr * rr - k * k))
    kap1 = np.arctan2(K, c * c + (k * k - rr * rr))
    A[lens] = rr * rr * kap0 + k * k * kap1 - 0.5 * K
    dk[lens] = 2.0 * k * kap1
    dc[lens] = -K / c
    return A, dk, dc


def weight_vector_dk(k: float, g: float, ze: np.ndarray) -> np.ndarray:
    """d w / d k at fixed g (c = g (1 + k)) of weight_vector(k, c, ze); 0 at g = 1."""
    c = g * (1.0 + k)
    nz = len(ze) - 1
    a_tot, dtot_k, dtot_c = lens_partials(np.array([1.0]), k, c)
    if c >= 1.0 + k or a_tot[0] <= 0.0:
        return np.zeros(nz)
    a, ak, ac = lens_partials(ze, k, c)
    da = ak + ac * g                      # along c = g (1 + k)
    dtot = dtot_k[0] + dtot_c[0] * g
    w = (a[1:] - a[:-1]) / a_tot[0]
    return (da[1:] - da[:-1]) / a_tot[0] - w * dtot / a_tot[0]


def calculate_weights(k: float, ze: np.ndarray, ng: int, with_dk: bool = False):
    """Weight table in g for one k (the direct model, Sect. 3.1.2): returns dg, w[ng][nz]
    (and d w / d k at fixed g with `with_dk`)."""
    dg = 1.0 / (ng - 1)
    w = np.stack([weight_vector(k, (i * dg) * (1.0 + k), ze) for i in range(ng)])
    if not with_dk:
        return dg, w
    return dg, w, np.stack([weight_vector_dk(k, i * dg, ze) for i in range(ng)])


def calculate_weights_3d(nk: int, k0: float, k1: float, ze: np.ndarray, ng: int):
    """Weight table in (k, g): returns dk, dg, w[nk][ng][nz]."""
    dk = (k1 - k0) / (nk - 1)
    tables = []
    dg = None
    for m in range(nk):
        dg, w = calculate_weights(k0 + m * dk, ze, ng)
        tables.append(w)
    return dk, dg, np.stack(tables)
