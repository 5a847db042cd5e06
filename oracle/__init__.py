"""FP64 CPU oracle for IGA collocation + fast-diagonalization (FD) preconditioned GMRES.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run this
package.  The CUDA path never imports it and shares no code with it; the only
module both sides use is ``workload`` (seeded inputs, no method arithmetic).

What it is: a plain, slow, obviously-correct restatement of Tani, "A preconditioning
strategy for linear systems arising from nonsymmetric schemes in isogeometric
analysis" (arXiv:1705.04384), in numpy/scipy FP64:

* ``bspline``     -- open knot vectors (Sec. 2.1), Cox--de Boor basis and derivatives,
                     Greville abscissae (eq. greville, Sec. 2.2).
* ``geometry``    -- single-patch maps F (Sec. 2.1) and the pull-back of -Laplace
                     (the general collocation operator the paper omits, Sec. 2.2;
                     derived in the docstring of ``geometry.pullback_coefficients``).
* ``collocation`` -- 1D collocation factors (eq. univariatecolloc), the assembled
                     sparse collocation matrix A_C (eq. collocation / collocationsystem)
                     and the preconditioner P_C (eq. colloc2D / colloc3D, Sec. 3).
* ``fd``          -- generalized eigendecomposition (eq. eigendecomposition, Remark 1)
                     and the FD solve (eq. FD2D / FD3D, Sec. 4).
* ``gmres``       -- unrestarted right-preconditioned GMRES (Saad--Schultz, cited in
                     Sec. 3) with modified Gram--Schmidt and Givens rotations, plus the
                     flexible variant used for a variable preconditioner.
* ``bicgstab``    -- right-preconditioned BiCGStab (van der Vorst 1992), the solver of
                     Sec. 5, with the paper's half-iteration counting.
* ``wq``          -- the weighted-quadrature Galerkin discretization (Sec. 2.3, eq.
                     WQapprox, eq. Q, eq. wq2D / wq3D): univariate rules exact on the
                     spline space, the assembled A_wq, the exact Galerkin A_G, the
                     Galerkin right-hand side and P_wq (symmetric FD of Sec. 4).
* convection--diffusion (Sec. 3.2) with a constant wind: ``geometry.wind_coefficients``,
  the ``wind`` arguments of ``collocation`` and ``fd.FD``.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, library routines, invariants or brute force; none is
"parity unpinned".
"""

from . import bspline, geometry, collocation, fd, gmres, bicgstab, wq  # noqa: F401
