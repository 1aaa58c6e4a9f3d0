"""The paper's worked heterogeneous example (Sect. 4.2) through the oracle."""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import ld, model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_heterogeneous_example.json")


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_passband_mapping_of_the_dummy_example(golden):
    # lcids map exposures to light curves, pbids map light curves to passbands
    assert golden["pb_index"] == [golden["pbids"][i] for i in golden["lcids"]] == [0, 0, 1, 1, 1, 0]


@pytest.mark.parametrize("name", ["achromatic", "chromatic", "two_parameter_sets"])
def test_oracle_reproduces_stored_values_and_structure(golden, name):
    case = golden["cases"][name]
    setup = model.build(golden["grid"], "quadratic", npb=2, chromatic=case["chromatic"])
    flux = model.evaluate(setup, np.array(golden["times"]), np.array(golden["pb_index"]),
                          np.array(case["params"]), np.array([1, 1]), np.array([0.0, 0.0]))
    np.testing.assert_allclose(flux, case["expected_flux"], rtol=0, atol=1e-14)
    assert flux.shape == (len(case["params"]), 6)
    pb = np.array(golden["pb_index"])
    if name != "two_parameter_sets":
        # every exposure sits at mid-transit (t0 = 0, p = 1): the flux depends only on the passband
        for b in (0, 1):
            assert np.ptp(flux[0, pb == b]) == 0.0
        # mid-transit depth against the exact centred-planet integral 2 pi int_0^k I r dr
        row = case["params"][0]
        for b in (0, 1):
            k = row[6 + (b if case["chromatic"] else 0)]
            u = row[6 + (2 if case["chromatic"] else 1) + 2 * b: 8 + (2 if case["chromatic"] else 1) + 2 * b]
            occ = quad(lambda r: ld.profile("quadratic", np.sqrt(1 - r * r), u) * 2 * np.pi * r, 0, k,
                       epsabs=1e-15)[0]
            assert flux[0, pb == b][0] == pytest.approx(1 - occ / ld.istar("quadratic", u), abs=2e-6)
    else:
        # the periods differ from 1 d, so only the first exposure is in transit
        assert np.all(flux[:, 1:] == 1.0) and np.all(flux[:, 0] < 1.0)
