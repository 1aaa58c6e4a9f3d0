"""Limb-darkening profiles and the stellar disk integral (Sect. 3.2; Eq. 2-4).

Each law gives the surface brightness I(mu), mu = sqrt(1 - z^2) in [0, 1].
The normalisation I_star = 2 pi int_0^1 z I(z) dz (Eq. 2 and 4) equals
2 pi int_0^1 mu I(mu) dmu.  Named laws are integrated in closed form
(Sect. 3.2.1 says the named models are integrated analytically); the
tabulated profile (the "custom" profile of Sect. 3.2.2, sampled on a
mu grid) is linearly interpolated, held constant outside the table, and
its I_star is the exact integral of that piecewise-linear function.

Laws (coefficients per passband):
  uniform        I = 1
  quadratic      I = 1 - u1 (1 - mu) - u2 (1 - mu)^2
  quadratic_tri  quadratic with u1 = 2 sqrt(q1) q2, u2 = sqrt(q1) (1 - 2 q2)
                 (Kipping's triangular parametrisation, footnote of Sect. 3.2.1)
  nonlinear      I = 1 - sum_{n=1..4} c_n (1 - mu^(n/2))
  linear         I = 1 - u (1 - mu)
  general        I = 1 - sum_{n=1..N} c_n (1 - mu)^n            (N = 1..4)
  logarithmic    I = 1 - u1 (1 - mu) - u2 mu ln mu
  exponential    I = 1 - u1 (1 - mu) - u2 / (1 - exp(mu))
  power2         I = 1 - c (1 - mu^alpha)                      (c, alpha > 0)
  power2_pm      power2 with h1 = I(1/2) = 1 - c (1 - 2^-alpha), h2 = I(1/2) - I(0) = c 2^-alpha,
                 i.e. c = 1 - h1 + h2, alpha = log2(c / h2)
(the laws named in Sect. 3.2.1, written in their usual forms; all but the
power-2 laws are affine in their coefficients).  Closed-form disk integrals:
  linear       pi (1 - u/3)
  general      pi (1 - sum_n 2 c_n / ((n+1)(n+2)))     [int_0^1 mu (1-mu)^n dmu = 1/((n+1)(n+2))]
  logarithmic  pi (1 - u1/3 + 2 u2/9)                   [int_0^1 mu^2 ln mu dmu = -1/9]
  exponential  pi (1 - u1/3) + 2 pi u2 C,  C = int_0^1 mu / (e^mu - 1) dmu
               = pi^2/6 - Li2(1/e) + ln(1 - 1/e)       [expand 1/(e^mu - 1) = sum_k e^(-k mu)]
  power2       pi (1 - c alpha / (alpha + 2))           [int_0^1 mu^(1+alpha) dmu = 1/(alpha+2)]
"""
import numpy as np
from scipy.special import spence

NCOEF = {"uniform": 0, "quadratic": 2, "quadratic_tri": 2, "nonlinear": 4, "tabulated": 0,
         "linear": 1, "logarithmic": 2, "exponential": 2, "power2": 2, "power2_pm": 2}

#: int_0^1 mu / (e^mu - 1) dmu; scipy's spence(z) is Li2(1 - z)
EXP_C = np.pi ** 2 / 6.0 - spence(1.0 - np.exp(-1.0)) + np.log(1.0 - np.exp(-1.0))


def ncoef(model: str, n_general: int = 0) -> int:
    """Coefficients per passband of a law (the general law takes n_general = 1..4)."""
    if model == "general":
        if not 1 <= n_general <= 4:
            raise ValueError("the general law takes 1 to 4 coefficients")
        return n_general
    return NCOEF[model]


def kipping_to_quadratic(q1, q2):
    sq = np.sqrt(q1)
    return 2.0 * sq * q2, sq * (1.0 - 2.0 * q2)


def pm_to_power2(h1, h2):
    """(h1, h2) of the power-2 law to (c, alpha)."""
    c = 1.0 - h1 + h2
    return c, np.log2(c / h2)


def power2_coef(model: str, coef):
    return pm_to_power2(*coef) if model == "power2_pm" else tuple(coef)


def profile(model: str, mu, coef=(), table=None):
    """I(mu) for the named law (coefficients ``coef``) or the tabulated profile ``table``."""
    mu = np.asarray(mu, np.float64)
    if model == "uniform":
        return np.ones_like(mu)
    if model == "quadratic":
        u1, u2 = coef
        return 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
    if model == "quadratic_tri":
        u1, u2 = kipping_to_quadratic(*coef)
        return 1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
    if model == "nonlinear":
        c1, c2, c3, c4 = coef
        return (1.0 - c1 * (1.0 - mu ** 0.5) - c2 * (1.0 - mu) - c3 * (1.0 - mu ** 1.5)
                - c4 * (1.0 - mu ** 2))
    if model == "tabulated":
        tmu, tI = table
        return np.interp(mu, tmu, tI)
    if model == "linear":
        (u,) = coef
        return 1.0 - u * (1.0 - mu)
    if model == "general":
        return 1.0 - sum(c * (1.0 - mu) ** (n + 1) for n, c in enumerate(coef))
    if model == "logarithmic":
        u1, u2 = coef
        mlm = np.where(mu > 0.0, mu * np.log(np.where(mu > 0.0, mu, 1.0)), 0.0)
        return 1.0 - u1 * (1.0 - mu) - u2 * mlm
    if model == "exponential":
        u1, u2 = coef
        return 1.0 - u1 * (1.0 - mu) - u2 / (1.0 - np.exp(mu))
    if model in ("power2", "power2_pm"):
        c, alpha = power2_coef(model, coef)
        return 1.0 - c * (1.0 - mu ** alpha)
    raise ValueError(f"unknown LD model {model!r}")


def profile_dmu(model: str, mu, coef=(), table=None):
    """dI/dmu of ``profile`` (mu > 0); for a table, the slope of the segment holding mu
    (0 outside the nodes, the right-hand segment on a node)."""
    mu = np.asarray(mu, np.float64)
    if model == "uniform":
        return np.zeros_like(mu)
    if model in ("quadratic", "quadratic_tri"):
        u1, u2 = kipping_to_quadratic(*coef) if model == "quadratic_tri" else coef
        return u1 + 2.0 * u2 * (1.0 - mu)
    if model == "nonlinear":
        c1, c2, c3, c4 = coef
        return 0.5 * c1 * mu ** -0.5 + c2 + 1.5 * c3 * mu ** 0.5 + 2.0 * c4 * mu
    if model == "tabulated":
        tmu, tI = (np.asarray(x, np.float64) for x in table)
        i = np.clip(np.searchsorted(tmu, mu, side="right") - 1, 0, tmu.size - 2)
        slope = (tI[i + 1] - tI[i]) / (tmu[i + 1] - tmu[i])
        return np.where((mu >= tmu[0]) & (mu < tmu[-1]), slope, 0.0)
    if model == "linear":
        (u,) = coef
        return np.full_like(mu, u)
    if model == "general":
        return sum((n + 1) * c * (1.0 - mu) ** n for n, c in enumerate(coef))
    if model == "logarithmic":
        u1, u2 = coef
        return u1 - u2 * (np.log(mu) + 1.0)
    if model == "exponential":
        u1, u2 = coef
        em = np.exp(mu)
        return u1 - u2 * em / (1.0 - em) ** 2
    if model in ("power2", "power2_pm"):
        c, alpha = power2_coef(model, coef)
        return c * alpha * mu ** (alpha - 1.0)
    raise ValueError(f"unknown LD model {model!r}")


def istar(model: str, coef=(), table=None) -> float:
    """I_star = 2 pi int_0^1 mu I(mu) dmu."""
    if model == "uniform":
        return np.pi
    if model in ("quadratic", "quadratic_tri"):
        u1, u2 = coef if model == "quadratic" else kipping_to_quadratic(*coef)
        return np.pi * (1.0 - u1 / 3.0 - u2 / 6.0)
    if model == "nonlinear":
        c1, c2, c3, c4 = coef
        return np.pi * (1.0 - c1 / 5.0 - c2 / 3.0 - 3.0 * c3 / 7.0 - c4 / 2.0)
    if model == "tabulated":
        tmu, tI = (np.asarray(x, np.float64) for x in table)
        # constant below the first and above the last node
        s = 0.5 * tI[0] * tmu[0] ** 2 + 0.5 * tI[-1] * (1.0 - tmu[-1] ** 2)
        # int_{m0}^{m1} mu (linear I) dmu = h/6 [I0 (2 m0 + m1) + I1 (m0 + 2 m1)]
        m0, m1, i0, i1 = tmu[:-1], tmu[1:], tI[:-1], tI[1:]
        s += np.sum((m1 - m0) / 6.0 * (i0 * (2.0 * m0 + m1) + i1 * (m0 + 2.0 * m1)))
        return 2.0 * np.pi * s
    if model == "linear":
        (u,) = coef
        return np.pi * (1.0 - u / 3.0)
    if model == "general":
        return np.pi * (1.0 - sum(2.0 * c / ((n + 2.0) * (n + 3.0)) for n, c in enumerate(coef)))
    if model == "logarithmic":
        u1, u2 = coef
        return np.pi * (1.0 - u1 / 3.0 + 2.0 * u2 / 9.0)
    if model == "exponential":
        u1, u2 = coef
        return np.pi * (1.0 - u1 / 3.0) + 2.0 * np.pi * u2 * EXP_C
    if model in ("power2", "power2_pm"):
        c, alpha = power2_coef(model, coef)
        return np.pi * (1.0 - c * alpha / (alpha + 2.0))
    raise ValueError(f"unknown LD model {model!r}")
