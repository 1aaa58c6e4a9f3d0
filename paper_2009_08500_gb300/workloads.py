"""Seeded synthetic inputs shaped like the RoadRunner paper's workloads.

This module only draws random numbers and lays them out; it evaluates no
part of the transit model.  Both the CUDA path (bench, GPU tests) and the
FP64 oracle (CPU tests) take their inputs from here, so the two sides always
see identical arrays.

Parameter rows follow the library's layout (one row per parameter vector):

    [T0, P, a, b, e, w, k_0 .. k_{nk-1}, ldc_0 .. ldc_{npb*nldc-1}]

T0 and P in days, a and b in stellar radii (b = a cos i, the nominal impact
parameter), e the eccentricity, w the argument of periastron in radians, k
the radius ratio (one value, or one per passband when ``chromatic``), ldc
the limb-darkening coefficients per passband.

Workload sizes follow the paper's use cases (Sect. 4 and 5): a plain single
light curve, a supersampled eccentric light curve, an MCMC-style population
of parameter vectors, a heterogeneous multi-passband time series, and a
stream of requests from many concurrent fits.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MINUTE = 1.0 / 1440.0

#: limb-darkening model names and their coefficient counts per passband (the
#: general law takes 1 to 4, given as ``n_general``)
LD_NCOEF = {"uniform": 0, "quadratic": 2, "quadratic_tri": 2, "nonlinear": 4, "tabulated": 0,
            "linear": 1, "logarithmic": 2, "exponential": 2, "power2": 2, "power2_pm": 2}


def ld_ncoef(ld_model: str, n_general: int = 0) -> int:
    if ld_model == "general":
        if not 1 <= n_general <= 4:
            raise ValueError("the general law takes 1 to 4 coefficients")
        return n_general
    return LD_NCOEF[ld_model]

#: grid settings used by every workload (radial grid of 500 annuli, k grid 0.005-0.3)
GRID = dict(zcut=0.7, nzin=200, nzlimb=300, ng=200, nk=60, k0=0.005, k1=0.3)


@dataclass
class Workload:
    name: str
    times: np.ndarray            # (npt,) float64, days
    pb_index: np.ndarray         # (npt,) int32
    params: np.ndarray           # (npv, nparam) float64
    supersampling: np.ndarray    # (npb,) int32
    exptime: np.ndarray          # (npb,) float64, days
    ld_model: str
    npb: int
    chromatic: bool
    precision: str               # "mixed" or "fp64"
    profiles: Optional[List[tuple]] = None   # per passband (mu, I) for tabulated LD
    grid: dict = field(default_factory=lambda: dict(GRID))
    n_general: int = 0                       # coefficients of the general law
    direct: bool = False                     # direct model: per-k weights, no k grid
    shared_weights: bool = False             # one weight array at the mean k of the passbands
    k_small: float = 0.0                     # small-planet approximation below this k (0 = off)

    @property
    def npv(self) -> int:
        return int(self.params.shape[0])

    @property
    def npt(self) -> int:
        return int(self.times.shape[0])

    @property
    def nparam(self) -> int:
        return int(self.params.shape[1])

    def samples_per_pv(self) -> int:
        """Number of exposure sub-samples one parameter vector evaluates."""
        return int(self.supersampling[self.pb_index].sum())

    def subset(self, npv: int, npt: Optional[int] = None) -> "Workload":
        """First ``npv`` parameter vectors (and optionally the first ``npt`` times)."""
        sl = slice(None) if npt is None else slice(0, npt)
        return Workload(self.name, self.times[sl].copy(), self.pb_index[sl].copy(),
                        self.params[:npv].copy(), self.supersampling.copy(), self.exptime.copy(),
                        self.ld_model, self.npb, self.chromatic, self.precision,
                        self.profiles, dict(self.grid), self.n_general, self.direct, self.shared_weights,
                        self.k_small)


def nparam_for(ld_model: str, npb: int, chromatic: bool, n_general: int = 0) -> int:
    return 6 + (npb if chromatic else 1) + npb * ld_ncoef(ld_model, n_general)


def monotone_bernstein_coefficients(rng: np.random.Generator, degree: int, lo: float, hi: float):
    """Ascending Bernstein coefficients beta_0 <= ... <= beta_degree = 1, beta_0 ~ U(lo, hi).

    A Bernstein polynomial with non-negative ascending coefficients is
    non-negative and non-decreasing on [0, 1]; it is used to synthesise
    physically valid (positive, limb-darkened) stellar profiles.
    """
    b0 = rng.uniform(lo, hi)
    mid = np.sort(rng.uniform(b0, 1.0, size=degree - 1))
    return np.concatenate([[b0], mid, [1.0]])


def bernstein_eval(beta: np.ndarray, x: np.ndarray) -> np.ndarray:
    from math import comb
    n = len(beta) - 1
    x = np.asarray(x, dtype=np.float64)
    return sum(beta[m] * comb(n, m) * x ** m * (1.0 - x) ** (n - m) for m in range(n + 1))


def bernstein_to_power(beta: np.ndarray) -> np.ndarray:
    """Power-basis coefficients p_j (sum_j p_j x^j) of a Bernstein polynomial."""
    from math import comb
    n = len(beta) - 1
    p = np.zeros(n + 1)
    for m in range(n + 1):
        for j in range(m, n + 1):
            p[j] += beta[m] * comb(n, m) * comb(n - m, j - m) * (-1.0) ** (j - m)
    return p


def nonlinear_coefficients(rng: np.random.Generator) -> np.ndarray:
    """Four-coefficient ("nonlinear") LD coefficients from the physical region.

    The profile is drawn as a degree-4 Bernstein polynomial in s = sqrt(mu)
    with ascending coefficients ending at 1, so it is positive, increases
    towards the disk centre and equals 1 there.  Written in powers of s it
    is p_0 + c_1 s + c_2 s^2 + c_3 s^3 + c_4 s^4 with p_0 = 1 - sum c_n,
    which is exactly the four-coefficient law's form; c_1..c_4 are returned.
    """
    beta = monotone_bernstein_coefficients(rng, 4, 0.05, 0.6)
    p = bernstein_to_power(beta)
    return p[1:].copy()


def _eccentric_orbit(rng, n, a, min_periastron):
    e = np.empty(n)
    w = np.empty(n)
    for i in range(n):
        while True:
            ei = rng.uniform(0.0, 0.5)
            if a[i] * (1.0 - ei) > min_periastron[i]:
                break
        e[i] = ei
        w[i] = rng.uniform(0.0, 2.0 * np.pi)
    return e, w


def make_c1(seed: int = 0) -> Workload:
    """Plain method, FP64: one circular orbit, quadratic LD, 2,000 times over +-0.15 d."""
    times = np.linspace(-0.15, 0.15, 2000)
    params = np.array([[0.0, 3.0, 10.0, 0.3, 0.0, 0.0, 0.1, 0.4, 0.25]])
    return Workload("c1_plain_fp64", times, np.zeros(2000, np.int32), params,
                    np.array([1], np.int32), np.array([0.0]), "quadratic", 1, False, "fp64")


def make_c2(seed: int = 1) -> Workload:
    """Single eccentric light curve: nonlinear LD, 27 d at 2-min cadence, 2-min exposures, ss=10."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P, a, b, k = 5.0, 15.0, 0.4, 0.1
    start = 2459000.5
    t0 = start + rng.uniform(0.0, P)
    e, w = _eccentric_orbit(rng, 1, np.array([a]), np.array([2.0]))
    ldc = nonlinear_coefficients(rng)
    npt = 19440
    times = start + 2.0 * MINUTE * np.arange(npt)
    params = np.array([[t0, P, a, b, e[0], w[0], k, *ldc]])
    return Workload("c2_eccentric_ss10", times, np.zeros(npt, np.int32), params,
                    np.array([10], np.int32), np.array([2.0 * MINUTE]), "nonlinear", 1, False, "mixed")


def _population(rng, npv):
    k = rng.uniform(0.01, 0.25, npv)
    a = rng.uniform(3.0, 30.0, npv)
    b = rng.uniform(0.0, 1.0 + k)
    P = rng.uniform(1.0, 10.0, npv)
    e, w = _eccentric_orbit(rng, npv, a, 1.0 + k + 0.5)
    t0 = rng.uniform(0.0, P)
    return t0, P, a, b, e, w, k


def make_c3(seed: int = 2, npv: int = 4096, npt: int = 20000, q1_min: float = 0.0) -> Workload:
    """MCMC-like population: 4,096 parameter vectors, Kipping (q1, q2), 20,000 times over 5 transits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t0, P, a, b, e, w, k = _population(rng, npv)
    q1 = rng.uniform(q1_min, 1.0, npv)
    q2 = rng.uniform(0.0, 1.0, npv)
    times = np.sort(rng.uniform(0.0, 5 * 5.5, npt))
    params = np.stack([t0, P, a, b, e, w, k, q1, q2], axis=1)
    return Workload("c3_population_4096x20000", times, np.zeros(npt, np.int32), params,
                    np.array([1], np.int32), np.array([0.0]), "quadratic_tri", 1, False, "mixed")


def tabulated_profile(rng: np.random.Generator, n: int = 500):
    """A smooth, positive, limb-darkened profile I(mu) on a uniform mu grid of n points."""
    beta = monotone_bernstein_coefficients(rng, 6, 0.05, 0.4)
    mu = np.linspace(0.0, 1.0, n)
    return mu, bernstein_eval(beta, mu)


def make_c4(seed: int = 3, npv: int = 2048, per_pb: int = 7500) -> Workload:
    """Heterogeneous series: 8 passbands with tabulated profiles, mixed cadence and supersampling."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t0, P, a, b, e, w, k = _population(rng, npv)
    npb = 8
    cycle = [(2.0 * MINUTE, 1), (10.0 * MINUTE, 10), (30.0 * MINUTE, 30)]
    exptime = np.array([cycle[j % 3][0] for j in range(npb)])
    ss = np.array([cycle[j % 3][1] for j in range(npb)], np.int32)
    profiles = [tabulated_profile(rng) for _ in range(npb)]
    t = np.concatenate([exptime[j] * np.arange(per_pb) for j in range(npb)])
    pb = np.concatenate([np.full(per_pb, j, np.int32) for j in range(npb)])
    order = np.argsort(t, kind="stable")
    params = np.stack([t0, P, a, b, e, w, k], axis=1)
    return Workload("c4_heterogeneous_2048x60000", t[order], pb[order], params, ss, exptime,
                    "tabulated", npb, False, "mixed", profiles)


def make_ts(seed: int = 5, npv: int = 2048, npb: int = 8, per_pb: int = 2500) -> Workload:
    """Transmission spectroscopy: the population of the population workload observed
    simultaneously in npb spectroscopic channels (every time stamp once per channel), a radius
    ratio per channel within 3% of the pv's mean, quadratic LD per channel; evaluated with the
    direct model and one shared weight array per pv (Sect. 3.4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t0, P, a, b, e, w, k = _population(rng, npv)
    ks = k[:, None] * (1.0 + 0.03 * rng.uniform(-1.0, 1.0, (npv, npb)))
    u1 = rng.uniform(0.1, 0.5, (npv, npb))
    u2 = rng.uniform(0.0, 0.3, (npv, npb))
    base = np.sort(rng.uniform(0.0, 5 * 5.5, per_pb))
    times = np.repeat(base, npb)
    pb_index = np.tile(np.arange(npb, dtype=np.int32), per_pb)
    ldc = np.stack([u1, u2], axis=2).reshape(npv, 2 * npb)
    params = np.concatenate([np.stack([t0, P, a, b, e, w], axis=1), ks, ldc], axis=1)
    return Workload(f"ts_transmission_{npv}x{npb}x{per_pb}", times, pb_index, params,
                    np.ones(npb, np.int32), np.zeros(npb), "quadratic", npb, True, "mixed",
                    direct=True, shared_weights=True)


def make_small(ld_model: str = "quadratic", npv: int = 3, npt: int = 257, npb: int = 1,
               chromatic: bool = False, ss=(1,), exptime=(0.0,), seed: int = 7,
               eccentric: bool = True, precision: str = "mixed", span: float = 6.0,
               n_general: int = 0, direct: bool = False, k_range=(0.02, 0.25),
               shared_weights: bool = False) -> Workload:
    """Small seeded case for parity tests: a few pvs, a ragged number of times."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.uniform(k_range[0], k_range[1], npv)
    a = rng.uniform(3.0, 12.0, npv)
    b = rng.uniform(0.0, 1.0 + k) * 0.9
    P = rng.uniform(1.0, 3.0, npv)
    if eccentric:
        e, w = _eccentric_orbit(rng, npv, a, 1.0 + k + 0.5)
    else:
        e, w = np.zeros(npv), np.zeros(npv)
    t0 = rng.uniform(0.0, P)
    times = np.sort(rng.uniform(0.0, span, npt))
    pb_index = rng.integers(0, npb, npt).astype(np.int32)
    cols = [t0, P, a, b, e, w]
    if chromatic:
        lo, hi = (1e-3, 0.95) if direct else (0.006, 0.29)
        cols += [np.clip(k * rng.uniform(0.95, 1.05), lo, hi) for _ in range(npb)]
    else:
        cols += [k]
    profiles = None
    for _ in range(npb):
        if ld_model == "quadratic":
            cols += [rng.uniform(0.1, 0.5, npv), rng.uniform(0.0, 0.3, npv)]
        elif ld_model == "quadratic_tri":
            cols += [rng.uniform(0.05, 1.0, npv), rng.uniform(0.0, 1.0, npv)]
        elif ld_model == "nonlinear":
            c = np.stack([nonlinear_coefficients(rng) for _ in range(npv)])
            cols += [c[:, 0], c[:, 1], c[:, 2], c[:, 3]]
        elif ld_model == "linear":
            cols += [rng.uniform(0.1, 0.9, npv)]
        elif ld_model == "general":
            # positive, limb-darkened profiles: 1 - sum c_n >= 0.1 at the limb
            c = np.stack([rng.uniform(0.2, 0.6, npv)] +
                         [rng.uniform(0.0, 0.2, npv) / n for n in range(2, n_general + 1)], axis=1)
            c *= np.minimum(1.0, 0.9 / c.sum(axis=1))[:, None]
            cols += [c[:, j] for j in range(n_general)]
        elif ld_model == "logarithmic":
            cols += [rng.uniform(0.2, 0.7, npv), rng.uniform(0.0, 0.3, npv)]
        elif ld_model == "exponential":
            cols += [rng.uniform(0.3, 0.6, npv), rng.uniform(0.0, 0.05, npv)]
        elif ld_model == "power2":
            cols += [rng.uniform(0.4, 0.8, npv), rng.uniform(0.4, 1.2, npv)]
        elif ld_model == "power2_pm":
            cols += [rng.uniform(0.6, 0.8, npv), rng.uniform(0.3, 0.55, npv)]
    if ld_model == "tabulated":
        profiles = [tabulated_profile(rng) for _ in range(npb)]
    params = (np.stack(cols, axis=1) if npv > 0
              else np.zeros((0, nparam_for(ld_model, npb, chromatic, n_general))))
    ss_arr = np.array([ss[j % len(ss)] for j in range(npb)], np.int32)
    ex_arr = np.array([exptime[j % len(exptime)] for j in range(npb)], np.float64)
    return Workload(f"small_{ld_model}", times, pb_index, params, ss_arr, ex_arr, ld_model, npb,
                    chromatic, precision, profiles, n_general=n_general, direct=direct,
                    shared_weights=shared_weights)


@dataclass
class Request:
    """One evaluation request of the serving workload."""
    fit: int
    arrival: float              # seconds from stream start
    workload: Workload
    grad: bool


def make_c5_fits(seed: int = 4, nfits: int = 64):
    """Per-fit static description: LD model and orbit family for each of the concurrent fits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    models = ["quadratic", "nonlinear", "tabulated"]
    return [dict(ld_model=models[int(rng.integers(0, 3))], eccentric=bool(i % 2),
                 seed=int(rng.integers(0, 2**31))) for i in range(nfits)]


def make_c5_stream(rate_hz: float, duration_s: float, seed: int = 4, nfits: int = 64,
                   npv_max: int = 4096, npt_max: int = 200_000, npt_min: int = 500):
    """Poisson request stream from ``nfits`` concurrent fits (log-uniform npv and npt, fwd:grad 3:1)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    fits = make_c5_fits(seed, nfits)
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        f = int(rng.integers(0, nfits))
        npv = int(np.exp(rng.uniform(0.0, np.log(npv_max))))
        npt = int(np.exp(rng.uniform(np.log(npt_min), np.log(npt_max))))
        spec = fits[f]
        wl = make_small(spec["ld_model"], npv=max(npv, 1), npt=npt, seed=int(rng.integers(0, 2**31)),
                        eccentric=spec["eccentric"], span=max(2.0, npt / 720.0))
        # every request of one fit shares that fit's LD profile (resident on the device)
        if spec["ld_model"] == "tabulated":
            wl.profiles = [tabulated_profile(np.random.Generator(np.random.PCG64(spec["seed"])))]
        reqs.append(Request(f, t, wl, bool(rng.uniform() < 0.25)))
    return fits, reqs
