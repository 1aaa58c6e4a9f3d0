"""Pins for the LD laws / disk integral (Sect. 3.2, Eq. 2-4) and the Keplerian orbit."""
import numpy as np
import pytest
from scipy.integrate import quad, solve_ivp

from oracle import ld
from oracle import orbit as O

LAWS = [("uniform", ()), ("quadratic", (0.4, 0.25)), ("quadratic_tri", (0.36, 0.3)),
        ("nonlinear", (0.5, -0.2, 0.6, -0.25))]


@pytest.mark.parametrize("model,coef", LAWS)
def test_istar_closed_form_matches_quadrature(model, coef):
    ref = 2 * np.pi * quad(lambda m: m * ld.profile(model, m, coef), 0, 1, epsabs=1e-14, epsrel=1e-13)[0]
    assert ld.istar(model, coef) == pytest.approx(ref, rel=1e-12)


def test_istar_is_also_the_z_integral_of_eq2():
    # Eq. 2 integrates over z; the laws are functions of mu = sqrt(1 - z^2)
    coef = (0.3, 0.1, 0.2, 0.05)
    ref = 2 * np.pi * quad(lambda z: z * ld.profile("nonlinear", np.sqrt(1 - z * z), coef), 0, 1,
                           epsabs=1e-13, limit=200)[0]
    assert ld.istar("nonlinear", coef) == pytest.approx(ref, rel=1e-9)


def test_law_values_at_centre_and_limb():
    assert ld.profile("quadratic", 1.0, (0.4, 0.25)) == 1.0
    assert ld.profile("quadratic", 0.0, (0.4, 0.25)) == pytest.approx(1 - 0.4 - 0.25)
    assert ld.profile("nonlinear", 0.0, (0.1, 0.2, 0.3, 0.1)) == pytest.approx(0.3)
    assert ld.profile("nonlinear", 0.25, (1.0, 0.0, 0.0, 0.0)) == pytest.approx(0.5)


def test_kipping_map_round_trip():
    rng = np.random.default_rng(3)
    q1, q2 = rng.uniform(0, 1, 100), rng.uniform(0, 1, 100)
    u1, u2 = ld.kipping_to_quadratic(q1, q2)
    np.testing.assert_allclose((u1 + u2) ** 2, q1, atol=1e-14)
    m = q1 > 1e-6
    np.testing.assert_allclose(u1[m] / (2 * (u1[m] + u2[m])), q2[m], atol=1e-12)


def test_tabulated_profile_and_istar():
    rng = np.random.default_rng(5)
    tmu = np.concatenate([[0.05], np.sort(rng.uniform(0.05, 0.95, 30)), [0.95]])
    tI = np.sort(rng.uniform(0.2, 1.0, tmu.size))
    f = lambda m: np.interp(m, tmu, tI)  # noqa: E731
    ref = 2 * np.pi * quad(lambda m: m * f(m), 0, 1, points=list(tmu), limit=500, epsabs=1e-14)[0]
    assert ld.istar("tabulated", table=(tmu, tI)) == pytest.approx(ref, rel=1e-12)
    # a table sampling a linear law reproduces that law and its closed-form I_star
    mu = np.linspace(0, 1, 11)
    lin = 1 - 0.6 * (1 - mu)
    assert ld.istar("tabulated", table=(mu, lin)) == pytest.approx(ld.istar("quadratic", (0.6, 0.0)), rel=1e-14)
    np.testing.assert_allclose(ld.profile("tabulated", [0.33, 0.71], table=(mu, lin)),
                               ld.profile("quadratic", np.array([0.33, 0.71]), (0.6, 0.0)), rtol=1e-15)


def test_circular_orbit_closed_forms():
    a, b, P, T0 = 10.0, 0.3, 3.0, 0.7
    z, front, ok = O.projected_distance(np.array([T0, T0 + P, T0 - 5 * P]), T0, P, a, b, 0.0, 0.0)
    np.testing.assert_allclose(z, b, atol=1e-13)
    assert front.all() and ok.all()
    tau = np.linspace(-0.4, 0.4, 41)
    z1 = O.projected_distance(T0 + tau, T0, P, a, b, 0.0, 1.3)[0]
    z2 = O.projected_distance(T0 - tau, T0, P, a, b, 0.0, 1.3)[0]
    np.testing.assert_allclose(z1, z2, atol=1e-12)
    phi = 2 * np.pi * tau / P
    np.testing.assert_allclose(z1, np.sqrt(a * a * np.sin(phi) ** 2 + b * b * np.cos(phi) ** 2), atol=1e-12)
    # half a period later the planet is behind the star
    assert not O.projected_distance(np.array([T0 + P / 2 + 0.01]), T0, P, a, b, 0.0, 0.0)[1][0]


@pytest.mark.parametrize("e,w", [(0.3, 0.4), (0.5, 4.0), (0.1, 2.5), (0.7, 5.5)])
def test_eccentric_conjunction_distance(e, w):
    a, b, P, T0 = 12.0, 0.5, 4.0, 1.1
    z, front, ok = O.projected_distance(np.array([T0, T0 + 3 * P]), T0, P, a, b, e, w)
    np.testing.assert_allclose(z, b * (1 - e * e) / (1 + e * np.sin(w)), rtol=1e-12)
    assert front.all() and ok.all()


def test_kepler_residual_and_period():
    rng = np.random.default_rng(1)
    M = rng.uniform(-np.pi, np.pi, 500)
    for e in (0.0, 0.2, 0.6, 0.9):
        E, ok = O.solve_kepler(M, e)
        assert ok.all()
        np.testing.assert_allclose(E - e * np.sin(E), M, atol=2e-15)
    t = rng.uniform(-5, 5, 50)
    args = (0.3, 2.5, 8.0, 0.4, 0.35, 1.0)
    np.testing.assert_allclose(O.projected_distance(t, *args)[0], O.projected_distance(t + 2.5, *args)[0],
                               atol=1e-11)


def test_small_eccentricity_approaches_circular():
    t = np.linspace(-0.3, 0.3, 31)
    zc = O.projected_distance(t, 0.0, 3.0, 10.0, 0.3, 0.0, 0.0)[0]
    ze = O.projected_distance(t, 0.0, 3.0, 10.0, 0.3, 1e-9, 0.8)[0]
    np.testing.assert_allclose(ze, zc, atol=1e-7)


@pytest.mark.parametrize("e,w", [(0.0, 0.0), (0.4, 1.0), (0.6, 3.9)])
def test_orbit_against_two_body_integration(e, w):
    """Integrate Newton's two-body equations from the conjunction state and project."""
    a, b, P, T0 = 9.0, 0.45, 3.3, 0.25
    GM = 4 * np.pi ** 2 * a ** 3 / P ** 2
    f0 = np.pi / 2 - w
    p = a * (1 - e * e)
    r0 = p / (1 + e * np.cos(f0))
    u0 = w + f0                                  # angle from the sky X axis direction
    vr = np.sqrt(GM / p) * e * np.sin(f0)        # radial and tangential velocity
    vt = np.sqrt(GM / p) * (1 + e * np.cos(f0))
    y0 = [r0 * np.cos(u0), r0 * np.sin(u0),
          vr * np.cos(u0) - vt * np.sin(u0), vr * np.sin(u0) + vt * np.cos(u0)]

    def rhs(_, s):
        x, y, vx, vy = s
        r3 = (x * x + y * y) ** 1.5
        return [vx, vy, -GM * x / r3, -GM * y / r3]

    ts = np.linspace(0.0, 1.3 * P, 60)
    for sign in (1.0, -1.0):
        sol = solve_ivp(rhs, (0, sign * ts[-1]), y0, t_eval=sign * ts, rtol=1e-12, atol=1e-12, method="DOP853")
        X, Y = -sol.y[0], -sol.y[1] * (b / a)
        z, front, _ = O.projected_distance(T0 + sol.t, T0, P, a, b, e, w)
        np.testing.assert_allclose(z, np.hypot(X, Y), rtol=1e-7, atol=1e-7)
        np.testing.assert_array_equal(front, sol.y[1] > 0)


# ---- the remaining named laws (linear, general, logarithmic, exponential) ----
MORE_LAWS = [("linear", (0.55,)), ("general", (0.4,)), ("general", (0.35, 0.2, 0.05)),
             ("general", (0.3, 0.1, 0.05, 0.02)), ("logarithmic", (0.5, 0.2)), ("exponential", (0.45, 0.03))]


@pytest.mark.parametrize("model,coef", MORE_LAWS)
def test_more_laws_istar_closed_form_matches_quadrature(model, coef):
    # mu I(mu) is finite at mu = 0 for every law (the exponential law's 1/mu term included)
    f = lambda m: m * ld.profile(model, m, coef) if m > 0 else (coef[1] if model == "exponential" else 0.0)  # noqa: E731
    ref = 2 * np.pi * quad(f, 0, 1, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    assert ld.istar(model, coef) == pytest.approx(ref, rel=1e-11)


def test_exponential_constant_against_quadrature():
    ref = quad(lambda m: m / np.expm1(m) if m > 0 else 1.0, 0, 1, epsabs=1e-15, epsrel=1e-14)[0]
    assert ld.EXP_C == pytest.approx(ref, rel=1e-14)
    assert ld.EXP_C == pytest.approx(0.7775046341122, rel=1e-12)


def test_more_laws_reduce_to_known_ones():
    mu = np.linspace(0.0, 1.0, 101)
    q = (0.4, 0.25)
    # general with two coefficients is the quadratic law; with one, the linear law
    assert np.allclose(ld.profile("general", mu, q), ld.profile("quadratic", mu, q), atol=1e-15)
    assert ld.istar("general", q) == pytest.approx(ld.istar("quadratic", q), rel=1e-15)
    assert np.allclose(ld.profile("general", mu, (0.3,)), ld.profile("linear", mu, (0.3,)), atol=1e-15)
    # linear is the quadratic law without its second term
    assert np.allclose(ld.profile("linear", mu, (0.3,)), ld.profile("quadratic", mu, (0.3, 0.0)), atol=1e-15)
    assert ld.istar("linear", (0.3,)) == pytest.approx(ld.istar("quadratic", (0.3, 0.0)), rel=1e-15)
    # logarithmic and exponential laws with a zero second coefficient are the linear law
    for m in ("logarithmic", "exponential"):
        assert np.allclose(ld.profile(m, mu[1:], (0.3, 0.0)), ld.profile("linear", mu[1:], (0.3,)), atol=1e-15)
        assert ld.istar(m, (0.3, 0.0)) == pytest.approx(ld.istar("linear", (0.3,)), rel=1e-15)
    # the logarithmic term vanishes at the centre and the limb, the laws give 1 at the centre
    for m, c in MORE_LAWS:
        if m != "exponential":
            assert ld.profile(m, 1.0, c) == pytest.approx(1.0, abs=1e-15)
    assert ld.profile("logarithmic", 0.0, (0.5, 0.2)) == pytest.approx(0.5)
