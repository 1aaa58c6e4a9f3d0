"""Batched RoadRunner light curves: Eq. 5 with interpolation in (k, g).

Follows the model evaluation of Sect. 3.1.1 and its interpolated variant of
Sect. 3.1.2, step by step, for each parameter vector and passband:

    ldp   = ldmodel(mu, ldpar)                       (LD profile at bin means)
    x     = (k - k0) / dk ; ik = floor(x) ; ak = x - ik
    ldw   = (1 - ak) dot(w[ik], ldp) + ak dot(w[ik+1], ldp)
    for every distance c:
        g  = c / (1 + k) ; i = floor(g / dg) ; a = g / dg - i
        ip = (1 - a) ldw[i] + a ldw[i+1]             (mean occluded brightness)
        ap = area(1, k, c)                           (occluded area)
        f  = (I_star - ip ap) / I_star               (Eq. 5)

Direct model (Sect. 3.1.2, the interpolation in k left out): ldw =
dot(w(k), ldp) with the weights computed for the vector's own k on the g
grid (``weights.calculate_weights``); k may then be anywhere in (0, 1).

Small-planet approximation (Sect. 3.4): below the radius ratio k_small the
weighted average ldw[i] of every g node is replaced by the profile at the
planet's centre, I(mu_i) with mu_i = sqrt(1 - min(c_i, 1)^2), c_i = g_i (1 + k),
clamped below to the outermost bin mean (the grid's limb resolution; keeps
laws that diverge at mu = 0 finite); such pvs need no k table.

Transmission spectroscopy (Sect. 3.4): with shared weights and one k per
passband, ldw of every passband is computed at the mean of the pv's radius
ratios; the area and g = c / (1 + k) use the passband's own k.

Points where the planet is behind the star or g >= 1 have f = 1 exactly.
Exposure supersampling (Sect. 4.1): each point is the mean of f over ss
sub-exposures.  Reading (placement unstated): midpoint rule,
t_s = t + exptime ((s + 1/2) / ss - 1/2), s = 0 .. ss-1.

Heterogeneous series (Sect. 4.2): every point carries a passband index; k is
one value or one per passband (chromatic); LD coefficients are per passband.

Readings: ik is clamped to nk - 2 (so k = k1 uses ak = 1) and i to ng - 2;
a value exactly on a node takes the lower cell.  Parameter vectors outside
the tabulated k range or the orbit's domain give a NaN light curve and a
nonzero status word (bits below); the paper is silent on invalid input.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache
from typing import List, Optional, Sequence

import numpy as np

from . import grid as _grid
from . import ld as _ld
from . import orbit as _orbit
from . import weights as _weights
from .area import intersection_area

# per parameter-vector status bits
ST_K_RANGE = 1
ST_E_RANGE = 2
ST_B_RANGE = 4
ST_P_RANGE = 8
ST_NONFINITE = 16
ST_LD_INVALID = 32
ST_A_RANGE = 64
ST_KEPLER = 128


@dataclass
class Setup:
    ze: np.ndarray
    zm: np.ndarray
    mu: np.ndarray
    w: np.ndarray          # (nk, ng, nz)
    dk: float
    dg: float
    k0: float
    k1: float
    nk: int
    ng: int
    ld_model: str
    npb: int
    chromatic: bool
    tables: Optional[List[tuple]]
    n_general: int = 0      # coefficients of the general law
    direct: bool = False    # direct model: weights for each exact k, interpolation in g only (Sect. 3.1.2)
    shared: bool = False    # transmission spectroscopy: one weight array at the mean k of the passbands
    k_small: float = 0.0    # small-planet approximation below this radius ratio (0 = off)

    @property
    def nldc(self) -> int:
        return _ld.ncoef(self.ld_model, self.n_general)

    @property
    def nparam(self) -> int:
        return 6 + (self.npb if self.chromatic else 1) + self.npb * self.nldc


@lru_cache(maxsize=8)
def _tables(zcut, nzin, nzlimb, ng, nk, k0, k1):
    ze, zm, mu = _grid.create_z_grid(zcut, nzin, nzlimb)
    dk, dg, w = _weights.calculate_weights_3d(nk, k0, k1, ze, ng)
    for arr in (ze, zm, mu, w):
        arr.setflags(write=False)
    return ze, zm, mu, dk, dg, w


def build(grid: dict, ld_model: str, npb: int = 1, chromatic: bool = False,
          tables: Optional[Sequence[tuple]] = None, n_general: int = 0, direct: bool = False,
          shared: bool = False, k_small: float = 0.0) -> Setup:
    """Model initialisation: radial grid, mu at the bin means and the (k, g) weight table
    (the direct model computes its weights per call for each k instead)."""
    ze, zm, mu, dk, dg, w = _tables(grid["zcut"], grid["nzin"], grid["nzlimb"], grid["ng"],
                                    grid["nk"], grid["k0"], grid["k1"])
    return Setup(ze, zm, mu, w, dk, dg, grid["k0"], grid["k1"], grid["nk"], grid["ng"],
                 ld_model, npb, chromatic, list(tables) if tables is not None else None, n_general, direct,
                 shared, k_small)


def unpack(setup: Setup, row: np.ndarray):
    T0, P, a, b, e, w = (float(x) for x in row[:6])
    nkp = setup.npb if setup.chromatic else 1
    ks = np.asarray(row[6:6 + nkp], np.float64)
    ldc = np.asarray(row[6 + nkp:], np.float64).reshape(setup.npb, setup.nldc)
    return T0, P, a, b, e, w, ks, ldc


def pv_status(setup: Setup, row: np.ndarray) -> int:
    T0, P, a, b, e, w, ks, ldc = unpack(setup, row)
    st = 0
    if not np.all(np.isfinite(row)):
        return ST_NONFINITE
    # every radius ratio in (0, 1); the interpolated model also needs the weights' radius ratio
    # (own, or the mean with shared weights) inside the k table, unless the small-planet
    # approximation replaces the weights
    if np.any(ks <= 0.0) or np.any(ks >= 1.0):
        st |= ST_K_RANGE
    elif not setup.direct:
        for k in ks:
            kw = weights_k(setup, ks, float(k))
            if kw >= setup.k_small and not (setup.k0 <= kw <= setup.k1):
                st |= ST_K_RANGE
    if not (0.0 <= e < 1.0):
        st |= ST_E_RANGE
    if not (P > 0.0):
        st |= ST_P_RANGE
    if not (a > 1.0):
        st |= ST_A_RANGE
    if not (0.0 <= b <= a):
        st |= ST_B_RANGE
    for pb in range(setup.npb):
        c = ldc[pb]
        if setup.ld_model == "quadratic_tri" and not (0.0 <= c[0] <= 1.0 and 0.0 <= c[1] <= 1.0):
            st |= ST_LD_INVALID
        elif setup.ld_model == "power2" and not (c[1] > 0.0):
            st |= ST_LD_INVALID
        elif setup.ld_model == "power2_pm" and not (c[1] > 0.0 and 1.0 - c[0] > 0.0):
            st |= ST_LD_INVALID          # needs h2 > 0 and c > h2, so that alpha > 0
        elif not (_ld.istar(setup.ld_model, c, _table(setup, pb)) > 0.0):
            st |= ST_LD_INVALID
    return st


def _table(setup: Setup, pb: int):
    return setup.tables[pb] if setup.ld_model == "tabulated" else None


def k_cell(setup: Setup, k: float):
    x = (k - setup.k0) / setup.dk
    ik = min(int(np.floor(x)), setup.nk - 2)
    return ik, x - ik


def small_planet_mu(setup: Setup, k: float):
    """mu under the planet's centre at every g node, c_i = g_i (1 + k) (mu = 0 beyond the limb),
    clamped below to the outermost bin mean; and whether each node is unclamped."""
    c = np.arange(setup.ng) * setup.dg * (1.0 + k)
    mu = np.sqrt(1.0 - np.minimum(c, 1.0) ** 2)
    free = (c < 1.0) & (mu > setup.mu[-1])
    return np.where(free, mu, setup.mu[-1]), free, c


def ld_weights(setup: Setup, k: float, coef, pb: int):
    """Per-passband profile weights: ldp, I_star and the k-interpolated ldw[ng].

    Small-planet approximation (Sect. 3.4): for k < k_small the weighted average at every g
    node is replaced by the profile at the planet's centre, I(mu(c_i)) (``small_planet_mu``)."""
    table = _table(setup, pb)
    ldp = _ld.profile(setup.ld_model, setup.mu, coef, table)
    istar = _ld.istar(setup.ld_model, coef, table)
    if k < setup.k_small:
        mu_c, _, _ = small_planet_mu(setup, k)
        return ldp, istar, _ld.profile(setup.ld_model, mu_c, coef, table)
    if setup.direct:
        _, w = _weights.calculate_weights(k, setup.ze, setup.ng)
        return ldp, istar, w @ ldp
    ik, ak = k_cell(setup, k)
    ldw = (1.0 - ak) * np.dot(setup.w[ik], ldp) + ak * np.dot(setup.w[ik + 1], ldp)
    return ldp, istar, ldw


def weights_k(setup: Setup, ks, k: float) -> float:
    """Radius ratio the passband's weights are computed at: its own k, or with shared weights
    (Sect. 3.4, transmission spectroscopy) the mean of the pv's per-passband radius ratios;
    the area and g = z / (1 + k) keep the passband's own k."""
    return float(np.mean(ks)) if (setup.shared and setup.chromatic) else k


def g_cell(setup: Setup, g):
    x = g / setup.dg
    i = np.minimum(np.floor(x).astype(np.int64), setup.ng - 2)
    return i, x - i


def flux_from_distance(setup: Setup, z, in_front, k, ldw, istar):
    """Eq. 5 for an array of distances; 1 where behind the star or g >= 1."""
    z = np.asarray(z, np.float64)
    f = np.ones_like(z)
    g = z / (1.0 + k)
    m = in_front & (g < 1.0)
    if np.any(m):
        i, a = g_cell(setup, g[m])
        ip = (1.0 - a) * ldw[i] + a * ldw[i + 1]
        ap = intersection_area(1.0, k, z[m])
        f[m] = (istar - ip * ap) / istar
    return f


def sample_times(t, exptime: float, ss: int, s: int):
    return t + exptime * ((s + 0.5) / ss - 0.5)


def evaluate(setup: Setup, times, pb_index, params, supersampling, exptime, return_status=False):
    """Flux (npv, npt) for every parameter vector (rows of ``params``)."""
    times = np.asarray(times, np.float64)
    pb_index = np.asarray(pb_index, np.int64)
    params = np.atleast_2d(np.asarray(params, np.float64))
    npv, npt = params.shape[0], times.shape[0]
    flux = np.empty((npv, npt))
    status = np.zeros(npv, np.int64)
    for p in range(npv):
        row = params[p]
        st = pv_status(setup, row)
        if st:
            flux[p] = np.nan
            status[p] = st
            continue
        T0, P, a, b, e, w, ks, ldc = unpack(setup, row)
        for pb in range(setup.npb):
            idx = np.nonzero(pb_index == pb)[0]
            if idx.size == 0:
                continue
            k = ks[pb] if setup.chromatic else ks[0]
            _, istar, ldw = ld_weights(setup, weights_k(setup, ks, k), ldc[pb], pb)
            ss = int(supersampling[pb])
            acc = np.zeros(idx.size)
            bad = np.zeros(idx.size, bool)
            for s in range(ss):
                ts = sample_times(times[idx], float(exptime[pb]), ss, s)
                z, front, ok = _orbit.projected_distance(ts, T0, P, a, b, e, w)
                acc += flux_from_distance(setup, z, front, k, ldw, istar)
                bad |= ~ok
            out = acc / ss
            if bad.any():
                out[bad] = np.nan
                status[p] |= ST_KEPLER
            flux[p, idx] = out
    return (flux, status) if return_status else flux


def evaluate_workload(wl, setup: Optional[Setup] = None, return_status=False):
    """Oracle flux for a :class:`paper_2009_08500_gb300.workloads.Workload`-shaped object."""
    if setup is None:
        setup = build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, getattr(wl, "n_general", 0),
                      getattr(wl, "direct", False), getattr(wl, "shared_weights", False),
                      getattr(wl, "k_small", 0.0))
    return evaluate(setup, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime,
                    return_status=return_status)
