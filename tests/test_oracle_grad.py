"""Pins for the oracle gradient: chain rule vs central finite differences of the model."""
import numpy as np
import pytest

from oracle import grad, model
from paper_2009_08500_gb300 import workloads as W

from gradcheck import smooth_points as _smooth_points


CASES = [
    dict(ld_model="quadratic", eccentric=False),
    dict(ld_model="quadratic", eccentric=True),
    dict(ld_model="quadratic_tri", eccentric=True),
    dict(ld_model="nonlinear", eccentric=True),
    dict(ld_model="tabulated", eccentric=True, npb=2, ss=(1, 5), exptime=(0.0, 0.01)),
    dict(ld_model="quadratic", eccentric=True, npb=2, chromatic=True),
    dict(ld_model="linear", eccentric=True),
    dict(ld_model="general", eccentric=True, n_general=3),
    dict(ld_model="logarithmic", eccentric=True),
    dict(ld_model="exponential", eccentric=False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{v}" for v in c.values()))
def test_chain_rule_matches_finite_differences(case):
    wl = W.make_small(npv=2, npt=1500, seed=21, span=4.0, **case)
    s = model.build(wl.grid, wl.ld_model, wl.npb, wl.chromatic, wl.profiles, wl.n_general)
    rng = np.random.default_rng(4)
    for p in range(wl.npv):
        row = wl.params[p].copy()
        if row[4] == 0.0:
            row[4] = 1e-4      # the orbit is defined for e >= 0 only: keep the stencil inside
        steps = np.array([1e-6, 1e-7, 1e-6, 1e-6, 1e-6, 1e-6] + [1e-6] * (row.size - 6))
        J = grad.jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime)
        Jfd = grad.fd_jacobian(s, wl.times, wl.pb_index, row, wl.supersampling, wl.exptime, steps)
        ok = _smooth_points(s, wl, row, steps)
        assert ok.sum() > 0.9 * wl.npt
        J, Jfd = J[ok], Jfd[ok]
        gbar = rng.normal(size=J.shape[0])
        v, vfd = gbar @ J, gbar @ Jfd
        # central differences carry ~eps / h of round-off per point
        noise = 4 * np.finfo(float).eps * np.abs(gbar).sum() / (2 * steps)
        assert np.all(np.abs(v - vfd) <= 1e-5 * np.maximum(np.abs(vfd), 1e-5 * np.abs(vfd).max()) + noise)
        # plain sums too (no random cancellation), and every element against its column scale
        noise = 4 * np.finfo(float).eps * J.shape[0] / (2 * steps)
        assert np.all(np.abs(J.sum(0) - Jfd.sum(0)) <= 1e-5 * np.abs(Jfd.sum(0)) + noise)
        scale = np.maximum(np.abs(Jfd).max(0), 1e-12)
        assert np.all(np.abs(J - Jfd) / scale < 1e-4)


def test_gradient_is_zero_out_of_transit():
    wl = W.make_small("quadratic", npv=1, npt=300, seed=5)
    s = model.build(wl.grid, "quadratic")
    J = grad.jacobian(s, wl.times, wl.pb_index, wl.params[0], wl.supersampling, wl.exptime)
    f = model.evaluate_workload(wl, s)[0]
    assert np.all(J[f == 1.0] == 0.0)
    assert np.any(J[f < 1.0] != 0.0)


def test_vjp_shape_and_linearity():
    wl = W.make_small("quadratic_tri", npv=3, npt=200, seed=8)
    s = model.build(wl.grid, wl.ld_model)
    gb = np.random.default_rng(1).normal(size=(3, 200))
    v1 = grad.vjp(s, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime, gb)
    v2 = grad.vjp(s, wl.times, wl.pb_index, wl.params, wl.supersampling, wl.exptime, 2.0 * gb)
    assert v1.shape == (3, 9)
    np.testing.assert_allclose(v2, 2.0 * v1, rtol=1e-14)


def test_chain_rule_matches_central_differences_on_population_rows():
    """The bar the GPU adjoint is held to (1e-5 relative on sign-weighted columns) holds, far
    tighter (1e-6; the differences' truncation error near the contact points is a few 1e-7),
    between the oracle's chain rule and central differences of the oracle model, on
    population-workload pvs over the full time grid."""
    full = W.make_c3(q1_min=1e-3)
    s = model.build(full.grid, full.ld_model)
    steps = np.array([1e-6, 1e-7, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6])
    checked = 0
    for p in np.arange(11, 4096, 331)[:12]:
        row = full.params[p]
        J = grad.jacobian(s, full.times, full.pb_index, row, full.supersampling, full.exptime)
        Jfd = grad.fd_jacobian(s, full.times, full.pb_index, row, full.supersampling, full.exptime, steps)
        ok = _smooth_points(s, full, row, steps)
        c = np.sign(Jfd) * ok[:, None]
        ref = (c * Jfd).sum(0)
        if not np.any(ref):
            continue
        got = (c * J).sum(0)
        noise = 4 * np.finfo(float).eps * np.abs(c).sum(0) / (2 * steps)
        scale = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max())
        assert np.all(np.abs(got - ref) <= 1e-6 * scale + noise), (np.abs(got - ref) / scale).max()
        checked += 1
    assert checked >= 6
