"""Oracle: a plain, slow, FP64 CPU restatement of the GMRES(s)-smoothed multigrid
inversion of the complex-stretched-grid (CSG) Helmholtz preconditioner and of the
outer flexible GMRES solve (Reps, Vanroose, bin Zubair, arXiv:1012.5379).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_1012_5379_gb300``) never imports, links or runs anything here,
and this package imports nothing from the product: the two share no code.

Every function cites the passage of the paper it follows (section, equation, lemma,
table).  Where the paper is silent or garbled, the reading taken is stated in the
docstring.  Arithmetic is complex128 throughout; NumPy array operations and a few
LAPACK calls (``numpy.linalg.solve`` / ``lstsq``) serve as library primitives.

Parity status per function (what pins it, see ``tests/test_oracle_pins.py``):

* ``spacings`` / ``coefficients_1d`` / ``apply_operator``: pinned (quadrature-built
  node coordinates + Lagrange second-difference matrix, closed-form Dirichlet
  eigenpairs, e^{-2i theta} rotation identity, exactness on complex quadratics).
* ``complex_map(ecs_sides="high")`` (one-sided layers, Benchmark 3 of Sec. 5): pinned by
  its closed-form end point and end intervals, exactness on a complex quadratic, and
  the model's bound-state energy at nu = 7 against an ODE shooting solve
  (``tests/test_oracle_gaussian.py``, which also holds Tables 4-5 as a soft band).
* ``restrict_fw`` / ``prolong``: pinned (P = 2^d R^T, exactness on linear fields).
* ``gmres_sweep``: pinned (brute-force Krylov least squares, residual monotonicity).
* ``coarse_solve``: pinned (independently assembled matrix times solution).
* ``vcycle``: pinned as a whole cycle by a dense brute-force restatement that shares
  only the paper's reading with it (each level's matrix from quadrature nodes and
  Lagrange weights, transfers as Kronecker products of the 1D full weighting and its
  doubled transpose, phi sampled at the coincident coarse nodes, every GMRES(s) step
  by brute-force Krylov least squares; 2D and 3D, constant and sampled phi, several
  V(nu1, nu2) and s); as a stationary iteration converging to the direct solve and by
  the paper's contraction bound (soft); and by its exactness on s eigenvectors.  The
  paper prints no cycle output to compare with.
* ``fgmres``: pinned (sparse direct solve, manufactured solution, every residual
  estimate of a run with a fixed linear preconditioner against the brute-force
  minimum over the Krylov space, plain and restarted; paper Table 2 iteration counts
  as a soft band).
* ``polysmoother`` (the third-degree polynomial smoother of Sec. 4): pinned by the
  paper's Fig. ex1 (which phi maps the spectrum inside the unit circle), the critical
  angle of Fig. critical_parameters and the stability of Fig. hierarchy_spectrum_smoother;
  its V-cycle ``vcycle_poly`` is linear and pinned as a cycle by its error propagator
  (the two-grid recursion with p(M) in Taylor form on both sides, dense matrices on
  tiny grids) and as a stationary iteration converging to the direct solve.
"""
from .helmholtz import (  # noqa: F401
    Level,
    build_hierarchy,
    coarse_solve,
    coefficients_1d,
    complex_map,
    fgmres,
    gmres_sweep,
    level_sizes,
    prolong,
    restrict_fw,
    spacings,
    apply_operator,
    vcycle,
)
