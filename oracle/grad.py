"""Gradient of the batched light curve w.r.t. every parameter.

Two independent routes:

* ``jacobian`` -- the chain rule through the steps of ``model`` and
  ``orbit`` (textbook Keplerian form), written out term by term:
    f = 1 - ip ap / I_star,   ip = lerp_g(ldw),  ap = area(1, k, z),
    ldw = (1 - ak) w[ik].ldp + ak w[ik+1].ldp,   g = z / (1 + k),
  (the direct model: ldw = w(k).ldp with d w / d k from the lens-area
  partials, ``weights.weight_vector_dk``),
  with the derivative of the piecewise-linear interpolants taken inside the
  cell that holds the point (the lower cell on a node, as ``model``
  evaluates), d area / dz = -(chord length) and d area / dk = 2 k kappa_1
  (arc of the planet's rim inside the star), and z(T0, P, a, b, e, w)
  differentiated through Kepler's equation.
* ``fd_jacobian`` -- central finite differences of ``model.evaluate``.

``vjp`` contracts a cotangent over the times: out[pv] = sum_t gbar[pv, t] J[pv, t, :].
"""
import numpy as np

from . import ld as _ld
from . import orbit as _orbit
from . import weights as _weights
from .model import (Setup, _table, g_cell, k_cell, pv_status, sample_times, unpack, evaluate, weights_k,
                    small_planet_mu)


def _area_and_partials(k, z):
    """area(1, k, z), d/dz, d/dk for arrays z (planet in front, g < 1)."""
    A = np.zeros_like(z)
    dAdz = np.zeros_like(z)
    dAdk = np.zeros_like(z)
    nested = z <= abs(1.0 - k)
    if k < 1.0:
        A[nested] = np.pi * k * k
        dAdk[nested] = 2.0 * np.pi * k
    else:
        A[nested] = np.pi
    lens = ~nested
    zz = z[lens]
    heron = (1.0 + k - zz) * (zz + 1.0 - k) * (zz - 1.0 + k) * (zz + 1.0 + k)
    K = np.sqrt(np.maximum(heron, 0.0))
    kap0 = np.arctan2(K, zz * zz + 1.0 - k * k)
    kap1 = np.arctan2(K, zz * zz + k * k - 1.0)
    A[lens] = kap0 + k * k * kap1 - 0.5 * K
    dAdz[lens] = -K / zz
    dAdk[lens] = 2.0 * k * kap1
    return A, dAdz, dAdk


def _orbit_partials(t, T0, P, a, b, e, w):
    """z and dz/d(T0, P, a, b, e, w) (shape (6, n)) plus the in-front mask."""
    n = 2.0 * np.pi / P
    f0, E0, M0 = _orbit.conjunction_anomalies(e, w)
    tau_raw = np.asarray(t, np.float64) - T0
    m = np.rint(tau_raw / P)
    tau = tau_raw - P * m
    M = M0 + n * tau
    E, ok = _orbit.solve_kepler(M, e)
    se = np.sqrt(1.0 - e * e)
    f = 2.0 * np.arctan2(np.sqrt(1.0 + e) * np.sin(0.5 * E), np.sqrt(1.0 - e) * np.cos(0.5 * E))
    den = 1.0 - e * np.cos(E)
    r = a * den
    u = w + f
    ci = b / a
    X = -r * np.cos(u)
    Y = -r * np.sin(u) * ci
    z = np.sqrt(X * X + Y * Y)

    den0 = 1.0 - e * np.cos(E0)
    dM0_dw = -den0 * den0 / se
    dM0_de = -den0 * np.sin(E0) / (1.0 - e * e) - np.sin(E0)
    # dM / d(T0, P, a, b, e, w)
    dM = [np.full_like(M, -n), -n * (tau + m * P) / P, np.zeros_like(M), np.zeros_like(M),
          np.full_like(M, dM0_de), np.full_like(M, dM0_dw)]
    dfdE = se / den
    dz = np.zeros((6,) + z.shape)
    for j in range(6):
        dE = (dM[j] + (np.sin(E) if j == 4 else 0.0)) / den
        du = dfdE * dE + (np.sin(f) / (1.0 - e * e) if j == 4 else 0.0) + (1.0 if j == 5 else 0.0)
        dr = a * e * np.sin(E) * dE
        if j == 2:
            dr = dr + den
        if j == 4:
            dr = dr - a * np.cos(E)
        dci = -b / (a * a) if j == 2 else (1.0 / a if j == 3 else 0.0)
        dX = -dr * np.cos(u) + r * np.sin(u) * du
        dY = -ci * (dr * np.sin(u) + r * np.cos(u) * du) - r * np.sin(u) * dci
        with np.errstate(invalid="ignore", divide="ignore"):
            dz[j] = (X * dX + Y * dY) / z
    return z, dz, np.sin(u) > 0.0, ok


def _ld_partials(model, mu, coef, table):
    """d ldp / d coef (nc, nz) and d I_star / d coef (nc,)."""
    if model == "quadratic":
        return np.stack([-(1.0 - mu), -(1.0 - mu) ** 2]), np.array([-np.pi / 3.0, -np.pi / 6.0])
    if model == "quadratic_tri":
        q1, q2 = coef
        sq = np.sqrt(q1)
        # u1 = 2 sqrt(q1) q2, u2 = sqrt(q1) (1 - 2 q2)
        J = np.array([[q2 / sq, 2.0 * sq], [(1.0 - 2.0 * q2) / (2.0 * sq), -2.0 * sq]])
        dp_u = np.stack([-(1.0 - mu), -(1.0 - mu) ** 2])
        di_u = np.array([-np.pi / 3.0, -np.pi / 6.0])
        return J.T @ dp_u, J.T @ di_u
    if model == "nonlinear":
        dp = np.stack([-(1.0 - mu ** (nn / 2.0)) for nn in (1, 2, 3, 4)])
        di = np.array([-np.pi * nn / (nn + 4.0) for nn in (1, 2, 3, 4)])
        return dp, di
    # the remaining named laws are affine in their coefficients: the partials are
    # the laws' terms and their disk integrals
    if model == "linear":
        return np.stack([-(1.0 - mu)]), np.array([-np.pi / 3.0])
    if model == "general":
        n = len(coef)
        dp = np.stack([-(1.0 - mu) ** (j + 1) for j in range(n)])
        di = np.array([-2.0 * np.pi / ((j + 2.0) * (j + 3.0)) for j in range(n)])
        return dp, di
    if model == "logarithmic":
        mlm = np.where(mu > 0.0, mu * np.log(np.where(mu > 0.0, mu, 1.0)), 0.0)
        return np.stack([-(1.0 - mu), -mlm]), np.array([-np.pi / 3.0, 2.0 * np.pi / 9.0])
    if model == "exponential":
        return (np.stack([-(1.0 - mu), -1.0 / (1.0 - np.exp(mu))]),
                np.array([-np.pi / 3.0, 2.0 * np.pi * _ld.EXP_C]))
    if model in ("power2", "power2_pm"):
        # I = 1 - c (1 - mu^a), I_star = pi (1 - c a / (a + 2)): not affine in a
        c, a = _ld.power2_coef(model, coef)
        ma = mu ** a
        dp = np.stack([-(1.0 - ma), c * ma * np.log(mu)])
        di = np.array([-np.pi * a / (a + 2.0), -2.0 * np.pi * c / (a + 2.0) ** 2])
        if model == "power2_pm":
            # c = 1 - h1 + h2, a = log2(c / h2): chain rule to (h1, h2)
            h2 = coef[1]
            J = np.array([[-1.0, 1.0], [-1.0 / (c * np.log(2.0)), (1.0 / c - 1.0 / h2) / np.log(2.0)]])
            dp, di = J.T @ dp, J.T @ di
        return dp, di
    return np.zeros((0, mu.size)), np.zeros(0)


def jacobian(setup: Setup, times, pb_index, row, supersampling, exptime):
    """d flux[t] / d row[j] for one parameter vector: shape (npt, nparam)."""
    times = np.asarray(times, np.float64)
    pb_index = np.asarray(pb_index, np.int64)
    J = np.zeros((times.size, setup.nparam))
    if pv_status(setup, row):
        J[:] = np.nan
        return J
    T0, P, a, b, e, w, ks, ldc = unpack(setup, row)
    nkp = setup.npb if setup.chromatic else 1
    nldc = setup.nldc
    for pb in range(setup.npb):
        idx = np.nonzero(pb_index == pb)[0]
        if idx.size == 0:
            continue
        kcol = 6 + (pb if setup.chromatic else 0)
        lcol = 6 + nkp + pb * nldc
        k = ks[pb] if setup.chromatic else ks[0]
        kw = weights_k(setup, ks, k)          # the weights' radius ratio (shared: mean over passbands)
        shared = setup.shared and setup.chromatic
        table = _table(setup, pb)
        ldp = _ld.profile(setup.ld_model, setup.mu, ldc[pb], table)
        istar = _ld.istar(setup.ld_model, ldc[pb], table)
        dldp, distar = _ld_partials(setup.ld_model, setup.mu, ldc[pb], table)
        if kw < setup.k_small:
            # small-planet approximation: ldw_i = I(mu(c_i)), c_i = g_i (1 + k), mu = sqrt(1 - c^2)
            mu_c, free, cc = small_planet_mu(setup, kw)
            ldw = _ld.profile(setup.ld_model, mu_c, ldc[pb], table)
            g_nodes = np.arange(setup.ng) * setup.dg
            dmu_dk = np.where(free, -cc * g_nodes / mu_c, 0.0)
            dldw_dk = _ld.profile_dmu(setup.ld_model, mu_c, ldc[pb], table) * dmu_dk
            dldp_c, _ = _ld_partials(setup.ld_model, mu_c, ldc[pb], table)
            dldw_dc = [dldp_c[c] for c in range(dldp_c.shape[0])]
        elif setup.direct:
            # weights for this exact k and their k-derivative at fixed g (Sect. 3.1.2)
            _, wk, wdk = _weights.calculate_weights(kw, setup.ze, setup.ng, with_dk=True)
            ldw = wk @ ldp
            dldw_dk = wdk @ ldp
            dldw_dc = [wk @ dldp[c] for c in range(dldp.shape[0])]
        else:
            ik, ak = k_cell(setup, kw)
            row_lo, row_hi = np.dot(setup.w[ik], ldp), np.dot(setup.w[ik + 1], ldp)
            ldw = (1.0 - ak) * row_lo + ak * row_hi
            dldw_dk = (row_hi - row_lo) / setup.dk
            dldw_dc = [(1.0 - ak) * np.dot(setup.w[ik], dldp[c]) + ak * np.dot(setup.w[ik + 1], dldp[c])
                       for c in range(dldp.shape[0])]
        ss = int(supersampling[pb])
        acc = np.zeros((idx.size, setup.nparam))
        for s in range(ss):
            ts = sample_times(times[idx], float(exptime[pb]), ss, s)
            z, dz, front, _ = _orbit_partials(ts, T0, P, a, b, e, w)
            g = z / (1.0 + k)
            msk = front & (g < 1.0)
            if not np.any(msk):
                continue
            zz, gg = z[msk], g[msk]
            i, al = g_cell(setup, gg)
            ip = (1.0 - al) * ldw[i] + al * ldw[i + 1]
            dip_dg = (ldw[i + 1] - ldw[i]) / setup.dg
            dip_dk_tab = (1.0 - al) * dldw_dk[i] + al * dldw_dk[i + 1]
            A, dA_dz, dA_dk = _area_and_partials(k, zz)
            # f = 1 - ip A / I_star
            df_dz = -(dip_dg / (1.0 + k) * A + ip * dA_dz) / istar
            df_dk_own = -((-dip_dg * zz / (1.0 + k) ** 2) * A + ip * dA_dk) / istar
            df_dk_row = -(dip_dk_tab * A) / istar     # through the weights' radius ratio
            sub = np.zeros((zz.size, setup.nparam))
            for j in range(6):
                sub[:, j] = df_dz * dz[j][msk]
            sub[:, kcol] += df_dk_own
            if shared:
                # d kw / d k_j = 1 / nkp for every passband's radius ratio
                for j in range(nkp):
                    sub[:, 6 + j] += df_dk_row / nkp
            else:
                sub[:, kcol] += df_dk_row
            for c in range(len(dldw_dc)):
                dip_dc = (1.0 - al) * dldw_dc[c][i] + al * dldw_dc[c][i + 1]
                sub[:, lcol + c] = -(dip_dc * A) / istar + ip * A * distar[c] / istar ** 2
            acc[np.nonzero(msk)[0]] += sub
        J[idx] = acc / ss
    return J


def vjp(setup: Setup, times, pb_index, params, supersampling, exptime, gbar):
    params = np.atleast_2d(params)
    out = np.zeros(params.shape)
    for p in range(params.shape[0]):
        out[p] = np.asarray(gbar[p]) @ jacobian(setup, times, pb_index, params[p], supersampling, exptime)
    return out


DEFAULT_STEPS = (1e-6, 1e-7, 1e-5, 1e-6, 1e-6, 1e-6)  # T0, P, a, b, e, w


def fd_jacobian(setup: Setup, times, pb_index, row, supersampling, exptime, steps=None):
    """Central differences of the model, one column per parameter."""
    row = np.asarray(row, np.float64)
    J = np.zeros((np.asarray(times).size, row.size))
    for j in range(row.size):
        h = (steps[j] if steps is not None else
             (DEFAULT_STEPS[j] if j < 6 else 1e-6))
        rp, rm = row.copy(), row.copy()
        rp[j] += h
        rm[j] -= h
        hh = rp[j] - rm[j]
        fp = evaluate(setup, times, pb_index, rp[None], supersampling, exptime)[0]
        fm = evaluate(setup, times, pb_index, rm[None], supersampling, exptime)[0]
        J[:, j] = (fp - fm) / hh
    return J
