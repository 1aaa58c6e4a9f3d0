"""Helpers of the gradient checks (CPU pins and GPU parity): which points a
central-difference stencil may be compared at, and the relative-error
formula with its floor."""
import numpy as np

from oracle import model


def gradient_rel(g, ref):
    """|g - ref| / max(|ref|, 1e-6 max_theta |ref|) per component (last axis = parameters)."""
    ref = np.asarray(ref, np.float64)
    floor = 1e-6 * np.abs(ref).max(axis=-1, keepdims=True)
    return np.abs(np.asarray(g) - ref) / np.maximum(np.abs(ref), np.maximum(floor, 1e-300))


def smooth_points(s, wl, row, steps):
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


