"""Write the stored expected values under tests/golden/ (calls only the oracle).

paper_heterogeneous_example.json: the dummy heterogeneous time series of
Sect. 4.2 (six exposures in three light curves observed in two passbands)
and its three example evaluations -- achromatic radius ratio, chromatic
radius ratio, and two parameter sets at once -- with the inputs exactly as
printed there.  The LD law is not named in that example; its four
coefficients per parameter set (two passbands x two coefficients) are read
as the quadratic law.  The inclination i is converted to the library's
impact parameter b = a cos i.  The expected fluxes are the oracle's.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import model  # noqa: E402

GRID = dict(zcut=0.7, nzin=200, nzlimb=300, ng=200, nk=60, k0=0.005, k1=0.3)


def main():
    times = [0.0, 1.0, 2.0, 3.0, 4.0, 5.0]
    lcids = [0, 0, 1, 1, 1, 2]
    pbids = [0, 1, 0]
    pb_index = [pbids[i] for i in lcids]
    pi = np.pi
    cases = {
        "achromatic": dict(k=[[0.10]], ldc=[[0.2, 0.1, 0.5, 0.1]], t0=[0.0], p=[1.0], a=[3.0], i=[0.5 * pi]),
        "chromatic": dict(k=[[0.10, 0.11]], ldc=[[0.2, 0.1, 0.5, 0.1]], t0=[0.0], p=[1.0], a=[3.0], i=[0.5 * pi]),
        "two_parameter_sets": dict(k=[[0.10, 0.12], [0.11, 0.13]],
                                   ldc=[[0.2, 0.1, 0.5, 0.1], [0.4, 0.2, 0.6, 0.2]],
                                   t0=[0.0, 0.01], p=[1.1, 1.2], a=[3.0, 2.9], i=[0.5 * pi, 0.49 * pi]),
    }
    out = dict(citation="Sect. 4.2 heterogeneous light curves: dummy example and its evaluate calls",
               times=times, lcids=lcids, pbids=pbids, pb_index=pb_index, ld_model="quadratic",
               grid=GRID, cases={})
    for name, c in cases.items():
        chrom = len(c["k"][0]) > 1
        rows = []
        for j in range(len(c["t0"])):
            a = c["a"][j]
            b = a * np.cos(c["i"][j])
            rows.append([c["t0"][j], c["p"][j], a, b, 0.0, 0.0, *c["k"][j], *c["ldc"][j]])
        setup = model.build(GRID, "quadratic", npb=2, chromatic=chrom)
        flux = model.evaluate(setup, np.array(times), np.array(pb_index), np.array(rows),
                              np.array([1, 1]), np.array([0.0, 0.0]))
        out["cases"][name] = dict(inputs=c, chromatic=chrom, params=rows, expected_flux=flux.tolist())
    with open(os.path.join(HERE, "paper_heterogeneous_example.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
