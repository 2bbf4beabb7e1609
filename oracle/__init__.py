"""FP64 CPU oracle for the pressure-correction Poisson solve on the Jacobi-transformed shell.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (``paper_2305_17875_gb300``) and imports nothing
from it.

Every function is plain numpy / scipy in float64 and follows the paper:

* ``grid``      - mapping (Section 2), radial clustering (Eq. stretching) and the
                  five-step face metric (Section 3.2, Eqs. jacobi/skewness), also
                  with exact derivatives at the face centres (the analytic option);
                  sectors between colatitude walls, or the full sphere with the
                  shell cut of Sections 3.5 and 3.7 (``full_sphere``).
* ``operator``  - the conservative discretisation of d_p(G_pq d_q phi)
                  (Section 3.3, Eqs. PC_8, PC_term1-3), assembled as a sparse matrix.
* ``mg``        - geometric multigrid on that operator (the paper's own solver is
                  HYPRE SMG, Section 3.6; the cycle here is this library's design,
                  restated plainly so every GPU step has a CPU twin).
* ``direct``    - bordered sparse direct solve of the same system (tiny grids).
* ``mms``       - manufactured solutions with closed-form Laplacians (pins only).
* ``pc``        - the steps either side of the solve: right side of Eq. PC_6 and
                  the correction of Eq. PC_7 on a staggered velocity (Section 3.6).
* ``tridiag``   - the Thomas algorithm and its periodic variant (Section 3.5,
                  Eqs. FIBRE_TA1-TA2, FIBRE_TAP1-TAP8); ``mg`` uses it for the
                  radial-line Gauss-Seidel smoother.
* ``adi``       - the ADI-CN implicit viscous sweeps of Section 3.4 (Eqs.
                  solve_2 to solve_4) on a cell-centred field.
* ``smg``       - semi-coarsening multigrid with zebra plane relaxation (the
                  solver class of Section 3.6): coarsening along zeta only, the
                  (eta, xi) planes solved exactly or by a 2-D cycle of eta
                  semi-coarsening and periodic-Thomas xi-line relaxation.

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
multigrid convergence factors (``mg`` and ``smg``), which the paper does not
give (parity unpinned: convergence factor only; the converged answer is pinned
by the direct solve).
"""

from .grid import (Shell, shell, full_sphere, face_metrics, cell_volume, vertex,
                   analytic_face_metrics)
from .operator import assemble, apply_rows
from . import mg, direct, smg

__all__ = [
    "Shell", "shell", "full_sphere", "face_metrics", "cell_volume", "vertex",
    "analytic_face_metrics", "assemble", "apply_rows", "mg", "direct", "smg",
]
