"""Plain FP64 CPU oracle for the two-grid GMsFEM-preconditioned mixed Darcy solver.

TEST INFRASTRUCTURE ONLY. This package is a slow, literal restatement of the
method of Yang, Fu & Chung, "A two-grid preconditioner with an adaptive coarse
space for flow simulations in highly heterogeneous media" (arXiv 1807.07220),
written with numpy/scipy sparse matrices in the paper's own saddle-point form:

* ``fine``        -- Section 2: two-scale grid, RT0/P0 matrices A_h, B_h, F_h
                     (eqs. matrixform, fine_system), restriction to
                     subdomains, and the sparse direct solve of the full
                     saddle-point system.
* ``preprocess``  -- Section 3: coarse RT0 solve plus per-block zero-flux
                     Neumann corrections giving B_h vbar_h = F_h
                     (eq. subproblem), and the reduced right-hand side
                     (eq. reduced_fine_system).
* ``coarse``      -- Section 4: snapshot space (eq. snapshot_eqn), local
                     spectral problem (eqs. spectral_1, spectral_eqn) solved
                     by the package's own cyclic Jacobi eigensolver, basis
                     selection; plus the MsFEM (eq. msfem) and RT0 comparator
                     coarse spaces.
* ``learned``     -- the learned coarse basis: face input map, labels from
                     the spectral problems of Section 4.2, the subspace loss,
                     a perceptron with its backward pass and Adam, and the
                     Rayleigh-Ritz selection on predicted flux profiles.
* ``impes``       -- Section 6.2: two-phase flow by IMPES, total mobility
                     and fractional flow (eqs. mobility, fraction) and the
                     upstream-weighted saturation update (eq.
                     DisSatEq_Implicit) evaluated explicitly with a CFL step.
* ``twogrid``     -- Section 5: smoother (eq. smooth), coarse correction
                     (eq. coarsepre), multiplicative two-grid cycle, PCG with
                     the stopping rule of Section 6 and a Lanczos estimate of
                     the condition number, and Steps 1-4 of the algorithm.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path and must never be used as a fallback for it.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force, library routines or the paper's printed
worked example (kappa == 1 row of Model 1), except where a docstring says
"parity unpinned".
"""

from .fine import Grid, assemble, solve_direct, boundary_lift, curl_matrix  # noqa: F401
from .coarse import jacobi_eigh, build_coarse_space  # noqa: F401
from .twogrid import TwoGridSolver  # noqa: F401
