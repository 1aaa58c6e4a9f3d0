"""Exact flux (radial integral, no grid) and the automatic grid choice, on the GPU.

rr_exact_flux against the oracle's adaptive quadrature of the same integral;
rr_choose_grid's grid checked independently with the oracle's model against
the oracle's exact integral at planet positions the search never saw.
"""
import numpy as np
import pytest

from oracle import exact, ld
from oracle import model as om
from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


LAWS = [("quadratic", (0.4, 0.25)), ("nonlinear", (0.5, -0.2, 0.6, -0.25)), ("logarithmic", (0.5, 0.2)),
        ("exponential", (0.45, 0.03)), ("quadratic_tri", (0.36, 0.3)), ("tabulated", ())]


@pytest.mark.parametrize("law,coef", LAWS)
def test_exact_flux_matches_oracle_quadrature(rr, law, coef):
    import torch
    rng = np.random.Generator(np.random.PCG64(5))
    table = W.tabulated_profile(rng)
    m = rr.Model(law, precision="fp64", direct=True)
    if law == "tabulated":
        m.set_ld_profile(0, *table)
    m.build()
    zs, ks = [], []
    for k in (0.005, 0.05, 0.2, 0.6, 0.9):
        for z in (0.0, 0.3 * k, 0.5, 1 - k - 1e-9, 1 - k + 1e-9, 1.0, 1 + 0.5 * k, 1 + k - 1e-9, 1 + k + 0.1):
            zs.append(z)
            ks.append(k)
    out = m.exact_flux(torch.tensor(zs, dtype=torch.float64), torch.tensor(ks, dtype=torch.float64),
                       coef).cpu().numpy()
    istar = ld.istar(law, coef, table)
    I = lambda mu: ld.profile(law, mu, coef, table)  # noqa: E731
    ref = np.array([exact.exact_flux(k, z, I, istar) if z < 1 + k else 1.0 for z, k in zip(zs, ks)])
    # FP64 round-off for laws polynomial in mu; the mu^(1/2), mu ln mu and 1/(1 - e^mu) terms are not
    # smooth at the limb and a table has a kink at each node (a fixed rule resolves them less well)
    tol = {"nonlinear": 1e-10, "logarithmic": 1e-10, "exponential": 1e-10, "tabulated": 1e-8}.get(law, 1e-12)
    assert np.abs(out - ref).max() < tol, np.abs(out - ref).max()


@pytest.mark.parametrize("target", [1e-5, 1e-6])
def test_chosen_grid_meets_the_target_on_unseen_positions(rr, target):
    coef = (0.4, 0.25)
    ks = [0.01, 0.1, 0.3]
    got = rr.choose_grid("quadratic", ks, coef, target=target)
    assert got["met"] and got["max_error"] <= target
    grid = dict(zcut=got["zcut"], nzin=got["nzin"], nzlimb=got["nzlimb"], ng=got["ng"], nk=2, k0=0.005, k1=0.3)
    s = om.build(grid, "quadratic", direct=True)
    istar = ld.istar("quadratic", coef)
    I = lambda mu: ld.profile("quadratic", mu, coef)  # noqa: E731
    rng = np.random.default_rng(11)
    worst = 0.0
    for k in ks:
        _, _, ldw = om.ld_weights(s, k, coef, 0)
        for g in rng.uniform(0, 0.999, 60):
            z = g * (1 + k)
            f = om.flux_from_distance(s, np.array([z]), np.array([True]), k, ldw, istar)[0]
            worst = max(worst, abs(f - exact.exact_flux(k, z, I, istar)))
    # unseen positions: within the target up to the search's sampling of the worst case
    assert worst <= 1.5 * target, (worst, got)


def test_tighter_target_costs_more_and_tabulated_law_works(rr):
    coef = (0.4, 0.25)
    loose = rr.choose_grid("quadratic", [0.1], coef, target=1e-4)
    tight = rr.choose_grid("quadratic", [0.1], coef, target=1e-6)
    cost = lambda g: (g["nzin"] + g["nzlimb"]) * g["ng"]  # noqa: E731
    assert loose["met"] and tight["met"] and cost(loose) < cost(tight)
    rng = np.random.Generator(np.random.PCG64(8))
    tab = rr.choose_grid("tabulated", [0.05, 0.2], target=1e-5, profile=W.tabulated_profile(rng))
    assert tab["met"] and tab["max_error"] <= 1e-5
