"""Plain FP64 CPU oracle for the IIM Poisson solver (test infrastructure only).

This package is the reference the CUDA path is checked against.  It is slow
on purpose: numpy for vector work, LAPACK QR / dense solves as library steps,
Python loops over control points.  It shares no code with the CUDA library
and must never be imported by the product path; only ``tests/``, the smoke
check and the bench's CPU-baseline leg use it.

Layout
  geometry.py  level sets (closed-form bodies, polar Fourier curves, level sets given
               at the grid's nodes), grid-line crossings, normals, curvature (Sec. 2.1)
  stencils.py  centred second-derivative coefficients, sigma_max     (Sec. 2.5, Tab. 1)
  fits.py      least-squares interpolants, ghost / Neumann / jump rows (Sec. 2.1-2.2)
  operator.py  the (n,k) IIM operator L_Omega and data term           (Sec. 2.3, Eq. 12)
  sw.py        Shortley-Weller operators and 1D formulas              (Sec. 3.1, Eqs. 18-21)
  mg.py        geometric multigrid V- and W-cycles                   (Sec. 3.3)
  fgmres.py    right-preconditioned flexible GMRES(m) (Sec. 4.1) and
               left-preconditioned GMRES(m)                          (Sec. 3.2)
  dense.py     dense assembly of the operator for brute-force checks
  problem.py   glue: build everything for one problem, solve it

Parity-unpinned readings (no printed value pins them; only the invariants in
tests/ do): the half-ellipse semi-axes of the least-squares region, the
outer-box closure, the coarsest-grid size rule, the degree of the spherical
harmonic of the perturbed sphere, the degree-5 interpolant of a level set given on
the grid (pinned by polynomial exactness and by reproducing the closed-form quadrics,
tests/test_oracle_geometry_input.py).  The cell-centred transfer weights are pinned
by multilinear exactness (tests/test_oracle_transfers.py); the 2D/3D Shortley-Weller
assembly and the smoother's colours by tests/test_oracle_sw_assembly.py.
"""
