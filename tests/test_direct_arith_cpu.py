"""The FP32 arithmetic of the direct model's weight kernel, restated in numpy float32.

The constants are read from the kernel source, so these tests pin what the
kernel evaluates: the fitted arctangent polynomial and the small-angle series
of the circular segment, and the lens-area formula built from them, against
numpy's FP64 arctangent and sine and the oracle's lens area.  (numpy float32
stands in for the device: fused multiply-adds are formed in FP64 and rounded
once, which is within an ulp of the device's.)
"""
import os
import re

import numpy as np
import pytest

from oracle.area import intersection_area

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2009_08500_gb300", "csrc")
SOURCES = [os.path.join(CSRC, f) for f in ("rr_setup.cu", "rr_device.cuh")]
f32 = np.float32


def _function_body(name):
    src = next(t for t in (open(f).read() for f in SOURCES) if "__forceinline__ float " + name + "(" in t)
    i = src.index(name + "(")
    j = src.index("{", i)
    depth, k = 0, j
    while True:
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                return src[j:k]
        k += 1


def _fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _atan_coefficients():
    body = _function_body("atan2_upper")
    first = re.search(r"float p = ([-0-9.e+]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, u, ([-0-9.e+]+)f\);", body)
    return [f32(float(first))] + [f32(float(x)) for x in rest]


def atan2_upper(y, x):
    cf = _atan_coefficients()
    y, x = f32(y), f32(x)
    ax = abs(x)
    mx, mn = max(y, ax), min(y, ax)
    t = f32(mn / mx) if mx > 1e-30 else f32(0)
    u = f32(t * t)
    p = cf[0]
    for c in cf[1:]:
        p = _fma(p, u, c)
    a = f32(t * p)
    if y > ax:
        a = f32(f32(np.pi / 2) - a)
    if x < 0:
        a = f32(f32(np.pi) - a)
    return a


def seg_phi_small(x):
    body = _function_body("seg_phi_small")
    first = re.search(r"float p = -1\.0f / ([0-9.]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, t2, (-?)1\.0f / ([0-9.]+)f\);", body)
    cf = [f32(-1.0 / float(first))] + [f32((-1.0 if s else 1.0) / float(d)) for s, d in rest]
    cf.append(f32(1.0))
    t = f32(2 * f32(x))
    t2 = f32(t * t)
    p = cf[0]
    for c in cf[1:]:
        p = _fma(p, t2, c)
    return f32(f32(f32(t * t2) * f32(1.0 / 12.0)) * p)


def test_arctangent_polynomial_within_two_ulp():
    cf = _atan_coefficients()
    assert len(cf) == 9 and cf[-1] == 1.0
    t = np.linspace(0, 1, 100001, dtype=f32)
    u = (t * t).astype(f32)
    p = np.full_like(t, cf[0])
    for c in cf[1:]:
        p = (p.astype(np.float64) * u + c).astype(f32)
    got = (t * p).astype(f32)
    ref = np.arctan(t.astype(np.float64))
    ulp = np.abs(got - ref)[1:] / np.spacing(ref[1:].astype(f32))
    assert ulp.max() < 1.5


def lawson_arctangent_fit(nodes=2000, rounds=1000):
    """Coefficients c8 .. c1, 1 of P(u), atan(t) ~ t P(t^2), minimising the largest relative error
    over [0, 1]: least squares on Chebyshev nodes, each node's weight multiplied by its error
    every round (Lawson's iteration, which converges to the minimax solution)."""
    k = np.arange(nodes)
    t = 0.5 * (1.0 - np.cos(np.pi * (k + 0.5) / nodes))
    u, at = t * t, np.arctan(t)
    A = np.stack([t * u ** j / at for j in range(1, 9)], axis=1)    # relative error = A c - b
    b = 1.0 - t / at
    w = np.full(nodes, 1.0 / nodes)
    for _ in range(rounds):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], b * sw, rcond=None)
        e = A @ c - b
        w = w * np.abs(e)
        w /= w.sum()
    return np.concatenate([c[::-1], [1.0]]), np.abs(e).max()


def test_arctangent_coefficients_are_the_minimax_fit():
    """The kernel's coefficients are the FP64 minimax fit of the relative error, rounded to FP32."""
    cf = np.array(_atan_coefficients(), np.float64)
    fit, err = lawson_arctangent_fit()
    assert err < 1.7e-8
    assert np.all(np.abs(cf - fit) <= 2 * np.spacing(np.abs(fit).astype(f32)))
    # the converged fit: more rounds or nodes change nothing at FP32 precision
    fit2, _ = lawson_arctangent_fit(nodes=3000, rounds=2000)
    assert np.all(np.abs(fit2 - fit) <= np.spacing(np.abs(fit).astype(f32)))


def test_upper_half_plane_folding_matches_atan2():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(20000):
        y = f32(abs(rng.normal()) * 10 ** rng.uniform(-6, 1))
        x = f32(rng.normal() * 10 ** rng.uniform(-6, 1))
        got = atan2_upper(y, x)
        ref = np.arctan2(np.float64(y), np.float64(x))
        worst = max(worst, abs(got - ref) / np.spacing(f32(ref)))
    assert worst < 4.5
    assert atan2_upper(0.0, 1.0) == 0.0
    assert atan2_upper(1.0, 0.0) == pytest.approx(np.pi / 2, abs=2e-7)
    assert atan2_upper(0.0, -1.0) == pytest.approx(np.pi, abs=3e-7)


def test_segment_series_matches_x_minus_sin_cos():
    for x in np.linspace(1e-4, 0.75, 400):
        ref = x - np.sin(x) * np.cos(x)
        assert abs(seg_phi_small(x) - ref) <= 4 * np.spacing(f32(ref))


def lens32(r, k, c):
    """The kernel's FP32 lens area (segment form), restated."""
    r, k, c = f32(r), f32(k), f32(c)

    def s3(x, y, z):
        s = f32(x + y)
        bb = f32(s - x)
        e = f32(f32(x - f32(s - bb)) + f32(y - bb))
        return f32(f32(s - z) + e)
    if c >= 2 * k:      # r - c is exact for every edge that reaches the lens
        dr = f32(r - c)
        p1, p2, s2 = f32(k + dr), f32(k - dr), f32(f32(c + r) - k)
    else:
        p1, p2, s2 = s3(r, k, c), s3(c, k, r), s3(c, r, k)
    if p1 <= 0:
        return f32(0)
    if p2 <= 0:
        return f32(f32(np.pi) * k * k)
    if s2 <= 0:
        return f32(f32(np.pi) * r * r)
    inv_c = f32(f32(1) / c)
    inv4c2 = f32(f32(0.25) * inv_c * inv_c)
    P = f32(f32(p1 * p2) * f32(f32(r + k + c) * s2))
    K = f32(P * f32(1 / np.sqrt(np.float64(P)))) if P > 1e-30 else f32(0)
    drk = f32(r - k)
    c2 = f32(c * c)
    x0 = _fma(drk, r + k, c2) if abs(drk) < abs(f32(c - k)) else _fma(c - k, c + k, f32(r * r))
    x1 = _fma(-drk, r + k, c2) if abs(drk) < abs(f32(c - r)) else _fma(c - r, c + r, f32(k * k))
    k0, k1 = atan2_upper(K, x0), atan2_upper(K, x1)
    q = f32(K * inv4c2)
    s0 = f32(f32(r * r) * seg_phi_small(k0)) if k0 < 0.75 else _fma(f32(r * r), k0, -f32(q * x0))
    s1 = f32(f32(k * k) * seg_phi_small(k1)) if k1 < 0.75 else _fma(f32(k * k), k1, -f32(q * x1))
    return f32(s0 + s1)


@pytest.mark.parametrize("k", [0.001, 0.01, 0.1, 0.3, 0.7])
def test_fp32_lens_area_few_ulp_relative(k):
    """Relative error of a few ulp everywhere in the lens region, including k << r and the contacts."""
    rng = np.random.default_rng(int(k * 1e4))
    worst = 0.0
    for _ in range(1500):
        r = rng.uniform(0.01, 1.0)
        lo, hi = abs(r - k), r + k
        c = lo + (hi - lo) * rng.choice([rng.uniform(), rng.uniform(0, 1e-4), 1 - rng.uniform(0, 1e-4)])
        ref = intersection_area(float(f32(r)), float(f32(k)), float(f32(c)))
        if ref <= 0:
            continue
        worst = max(worst, abs(float(lens32(r, k, c)) - ref) / ref / np.finfo(f32).eps)
    assert worst < 16
