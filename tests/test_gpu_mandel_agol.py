"""GPU light curves against the analytic quadratic-law model of Mandel & Agol (2002), on the same inputs.

The library approximates the occulted flux (Sect. 3); on the plain-method
workload (one circular orbit, quadratic law, the default grids) both of its
forms must stay within the paper's error level of the closed form
(Sect. 3.3: a few ppm at most, well below 1 ppm on average)."""
import numpy as np
import pytest

from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c1_within_the_paper_error_level_of_the_closed_form(precision):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    special = pytest.importorskip("scipy.special")
    if not all(hasattr(special, f) for f in ("elliprf", "elliprd", "elliprj")):
        pytest.skip("scipy without Carlson elliptic integrals")
    from oracle import mandel_agol as MA
    from oracle import orbit
    from paper_2009_08500_gb300 import rr

    wl = W.make_c1()
    wl.precision = precision
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    f = m.evaluate(t, p, pb, wl.supersampling, wl.exptime).double().cpu().numpy()[0]
    T0, P, a, b, e, w, k, u1, u2 = wl.params[0]
    z, front, ok = orbit.projected_distance(wl.times, T0, P, a, b, e, w)
    ref = np.array([MA.flux_quadratic(k, zi, u1, u2) for zi in z])
    err = np.abs(f - ref)
    assert (ref < 1).sum() > 500
    assert err.max() < 5e-6
    assert err.mean() < 5e-7
