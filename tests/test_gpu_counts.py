"""The kernels' counting form (the work units of the roofline): the same results as the plain
form, and a count of in-transit samples that matches the oracle's orbit sample by sample."""
import numpy as np
import pytest

from oracle import model as om
from oracle import orbit as oorb
from paper_2009_08500_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2009_08500_gb300 import rr as _rr
    _rr.load_library()
    return _rr


def oracle_in_transit(wl):
    """Samples (pv, time, sub-exposure) with the planet in front and g = z / (1 + k) < 1."""
    n = 0
    for row in wl.params:
        T0, P, a, b, e, w, k = row[:7]
        for pb in range(wl.npb):
            sel = wl.pb_index == pb
            ss, ex = int(wl.supersampling[pb]), float(wl.exptime[pb])
            for s in range(ss):
                z, front, _ = oorb.projected_distance(om.sample_times(wl.times[sel], ex, ss, s), T0, P, a, b, e, w)
                n += int(np.sum(front & (z / (1.0 + k) < 1.0)))
    return n


@pytest.mark.parametrize("ss", [(1,), (4,)])
def test_counting_form_same_results_and_in_transit_count(rr, ss):
    import torch
    wl = W.make_small("quadratic_tri", npv=24, npt=3000, seed=5, ss=ss, exptime=(0.01,), span=6.0)
    m = rr.model_for(wl)
    t, pb, p = rr.to_device(wl)
    gbar = torch.randn((wl.npv, wl.npt), device=t.device, generator=torch.Generator(device=t.device).manual_seed(3))
    f0 = m.evaluate(t, p, pb, wl.supersampling, wl.exptime)
    g0 = m.evaluate_grad(t, p, gbar, pb, wl.supersampling, wl.exptime)
    m.count_read("flux", reset=True)
    m.count_samples(True)
    f1 = m.evaluate(t, p, pb, wl.supersampling, wl.exptime)
    g1 = m.evaluate_grad(t, p, gbar, pb, wl.supersampling, wl.exptime)
    m.count_samples(False)
    cf, cg = m.count_read("flux"), m.count_read("grad")
    m.count_read("flux", reset=True)
    assert torch.equal(f0, f1) and torch.equal(g0, g1)
    for c in (cf, cg):
        assert c["transit"] <= c["orbit"] <= c["samples"] and c["cand"] * ss[0] == c["samples"]
        assert c["newton"] >= c["orbit"] - c["circular"] and 0 < c["lens"] < c["transit"]
    # the adjoint skips times whose cotangent is zero: none here, so the front parts agree
    assert cf["samples"] == cg["samples"] and cf["transit"] == cg["transit"]
    assert cg["refined"] > 0 and cf["refined"] == 0
    # FP32 and FP64 may disagree on samples within rounding of a contact point
    assert abs(cf["transit"] - oracle_in_transit(wl)) <= 2
