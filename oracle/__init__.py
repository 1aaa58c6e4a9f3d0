"""Plain, slow FP64 CPU oracle for the RoadRunner transit model (Parviainen 2020).

TEST INFRASTRUCTURE ONLY.  The only code allowed to import, call or execute
anything here is ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The library in
``paper_2009_08500_gb300`` never imports this package, and this package
imports nothing from the library: the two share no code.  Inputs come from
``paper_2009_08500_gb300.workloads`` (random draws only) or from the tests.

What each module follows (sections and equations of the paper):

* ``grid``      -- radial discretisation, Sect. 3.1.1 (two regions split at
                   z_cut: constant dz inside, constant dmu outside).
* ``area``      -- circle-circle intersection area a(c, k) of Eq. 5.
* ``weights``   -- weight vectors w (occluded annulus area / occluded area,
                   Sect. 2 below Eq. 4) tabulated on the (k, g) grid,
                   Sect. 3.1 and 3.1.2.
* ``ld``        -- limb-darkening laws of Sect. 3.2.1 and the tabulated
                   (numerical) profile of Sect. 3.2.2; the disk integral
                   I_star = 2 pi int_0^1 z I(z) dz of Eq. 2.
* ``orbit``     -- time -> projected star-planet distance for a Keplerian
                   orbit (parameters named in Sect. 4.1; the paper gives no
                   orbit equations, so this is the textbook two-body form).
* ``model``     -- the model evaluation of Sect. 3.1.1 / 3.1.2 (Eq. 5 with
                   interpolation in g and k) and exposure supersampling
                   (Sect. 4.1), for batches of parameter vectors (Sect. 4.1,
                   4.2).
* ``grad``      -- gradient of the batched flux w.r.t. every parameter, by
                   the chain rule through ``orbit`` and ``model``, and by
                   central finite differences.
* ``exact``     -- references that are not RoadRunner: the occulted flux as
                   an exact 1-D radial integral (Sect. 2, Eq. 1-2), 2-D
                   pixel integration over the stellar disk, and a 50-digit
                   mpmath intersection area.
* ``mandel_agol`` -- the analytic quadratic-law light curve of Mandel & Agol
                   (2002) in closed form (elliptic integrals): a second,
                   independent route to what ``exact`` integrates.

Pins (tests/test_oracle_*.py, CPU only) tie every function to something
other than itself: closed forms, the exact integral within the paper's
stated error level (Sect. 3.3, Fig. 2 and 3 captions), brute force on tiny
inputs, and orbit invariants.

Parity unpinned: the two readings the paper cannot decide -- the bin "mean"
of ``grid.create_z_grid`` taken as the z-midpoint, and the g / k node
placement of ``weights`` -- are pinned only through the whole-model error
bound against the exact integral, not individually.
"""
from . import grid, area, weights, ld, orbit, model, grad, exact  # noqa: F401
