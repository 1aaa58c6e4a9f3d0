"""Pins for the oracle gradient: chain rule vs central finite differences of the model."""
import numpy as np
import pytest

from oracle import grad, model
from paper_2009_08500_gb300 import workloads as W


def _smooth_points(s, wl, row, steps):
    """Points whose finite-difference stencil crosses no kink of the model.

    The model is piecewise smooth: the g and k interpolants are linear per
    cell, and the area has unbounded second derivative at the contact points
    (g = 1 and z = 1 - k).  Central differences are only compared where every
    sub-exposure stays in one smooth piece for every perturbed parameter.
    """
    from oracle import orbit
    ok = np.ones(wl.npt, bool)
    nkp = wl.npb if wl.chromatic else 1

    def state(r):
        T0, P, a, b, e, w = r[:6]
        out = []
        for pb in range(wl.npb):
            k = r[6 + (pb if wl.chromatic else 0)]
            ik, _ = model.k_cell(s, k)
            ss, ex = int(wl.supersampling[pb]), float(wl.exptime[pb])
            sts = []
            for j in range(ss):
                z, fr, _ = orbit.projected_distance(model.sample_times(wl.times, ex, ss, j), T0, P, a, b, e, w)
                g = z / (1 + k)
                inside = fr & (g < 1)
                cell = np.where(inside, np.minimum(np.floor(g / s.dg), s.ng - 2), -1)
                sts.append(np.stack([inside, cell, z <= 1 - k, np.full(z.shape, ik)]))
            out.append((wl.pb_index == pb, np.stack(sts)))
        return out

    for j in range(row.size):
        rp, rm = row.copy(), row.copy()
        rp[j] += steps[j]
        rm[j] -= steps[j]
        for (mp, sp), (_, sm) in zip(state(rp), state(rm)):
            same = np.all(sp == sm, axis=(0, 1))
            ok &= ~mp | same
    del nkp
    return ok


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
