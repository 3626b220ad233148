"""Plain, slow, FP64 CPU oracle for the cavity-radiation hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or
calls this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It shares no code with the CUDA library: it is written directly from the paper
(Baburin, Ballani, Peterson, Knezevic, "Hierarchical Block Low-rank
Approximation of Cavity Radiation"), in numpy float64, with no blocking, fusion
or reordering beyond what each definition states.

Modules
-------
geometry    facets (centroid, unit normal, area) of a triangle mesh, §3.1
viewfactor  view-factor entries, Eq. (10) with the 1-point centroid rule;
            composite quadrature used only by the pins
htree       Algorithm 1 (cluster tree), Eq. (28) admissibility, Algorithm 2
aca         cross approximation, Eq. (30), with full and partial pivoting and
            the stopping rule of Eq. (31)
hmatrix     block low-rank matrix built from the above, its matvec (§5.2)
radiosity   reflection matrix Eq. (11), direct solve, facet flux Eq. (12)
hlu         hierarchical LU of the reflection matrix with rank truncation
            (§5.1) and its forward / backward substitution (§5.2)

Pins (see ``tests/test_oracle_*.py``): closed-form parallel and perpendicular
plate view factors, the sphere identity, the two-grey-planes flux Eq. (5),
closed-cavity and uniform-temperature identities, energy conservation,
brute-force tree invariants and a hand-derived 1-D block structure, exact
rank-r ACA recovery and the cross identity of Eq. (30), the H-LU as the
unique LU of C without truncation, its error following eps_rel with it.
"""

SIGMA_SB = 5.670374419e-8
"""Stefan-Boltzmann constant (CODATA 2018), W m^-2 K^-4.

The paper prints 5.669e-9 next to Eq. (4); the exponent is a typo (the
physical constant is 5.67e-8).  Every call takes sigma as a parameter.
"""
