"""Bordered sparse direct solve of the discrete Poisson problem (oracle; test infrastructure only).

The unique discrete answer of Eq. PC_6 on the shell: A x = b with the gauge
sum_c |J^{-1}|_c x_c = 0, obtained from the bordered system

    [ A    1 ] [ x   ]   [ b ]
    [ J^T  0 ] [ lam ] = [ 0 ]

by scipy's SuperLU.  Only for tiny grids (fill-in grows fast in 3-D)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def bordered_solve(A, b, w):
    n = A.shape[0]
    one = sp.csr_matrix(np.ones((n, 1)))
    B = sp.bmat([[A, one], [sp.csr_matrix(np.asarray(w, dtype=np.float64).reshape(1, n)), None]],
                format="csc")
    rhs = np.concatenate([np.asarray(b, dtype=np.float64).ravel(), [0.0]])
    sol = spla.spsolve(B, rhs)
    return sol[:n], sol[n]
