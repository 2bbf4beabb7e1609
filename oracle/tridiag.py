"""Tridiagonal line solves (oracle; test infrastructure only).

Section 3.5 (the solver of the implicit sweeps): the Thomas algorithm for
A psi = g with A tridiagonal (Eqs. FIBRE_TA1 and FIBRE_TA2: forward sweep that
eliminates the sub-diagonal, then back substitution), and its periodic variant
(Eqs. FIBRE_TAP1 to FIBRE_TAP8: split off the last unknown, solve two
tridiagonal systems with the leading block, recover the last unknown from the
last equation, combine).

Coefficient convention (the paper's): in row m, ``a[m]`` multiplies psi_{m-1},
``b[m]`` psi_m and ``c[m]`` psi_{m+1}.  For the plain system a[0] and c[n-1]
are not used; for the periodic system they are the corner entries (psi_{-1}
is psi_{n-1} and psi_n is psi_0).

Every array has the position along the line on axis 0; any further axes
index independent lines, which are solved together (elementwise over those
axes, no reordering within a line).
"""
from __future__ import annotations

import numpy as np


def thomas(a, b, c, g):
    """Solve the tridiagonal systems (Eqs. FIBRE_TA1, FIBRE_TA2).

    Forward sweep: b'_0 = b_0, g'_0 = g_0 and, for m >= 1,
    b'_m = b_m - a_m b'^{-1}_{m-1} c_{m-1}, g'_m = g_m - a_m b'^{-1}_{m-1} g'_{m-1}.
    Back substitution: psi_{n-1} = g'_{n-1}/b'_{n-1},
    psi_m = (g'_m - c_m psi_{m+1}) / b'_m."""
    a, b, c, g = (np.asarray(v, dtype=np.float64) for v in (a, b, c, g))
    n = b.shape[0]
    bp = np.empty_like(b)
    gp = np.empty(np.broadcast_shapes(b.shape, g.shape))
    bp[0] = b[0]
    gp[0] = g[0]
    for m in range(1, n):
        w = a[m] / bp[m - 1]
        bp[m] = b[m] - w * c[m - 1]
        gp[m] = g[m] - w * gp[m - 1]
    psi = np.empty_like(gp)
    psi[n - 1] = gp[n - 1] / bp[n - 1]
    for m in range(n - 2, -1, -1):
        psi[m] = (gp[m] - c[m] * psi[m + 1]) / bp[m]
    return psi


def thomas_periodic(a, b, c, g):
    """Solve the cyclic tridiagonal systems (Eqs. FIBRE_TAP1 to FIBRE_TAP8).

    With A_c the leading (n-1) x (n-1) tridiagonal block, psi1 = A_c^{-1} g[:n-1]
    and psi2 = A_c^{-1} (-a_0, 0, ..., 0, -c_{n-2}) (Eqs. TAP5, TAP6); the last
    unknown follows from the last equation (Eq. TAP8),
    psi_{n-1} = (g_{n-1} - c_{n-1} psi1_0 - a_{n-1} psi1_{n-2})
                / (b_{n-1} + c_{n-1} psi2_0 + a_{n-1} psi2_{n-2}),
    and psi = psi1 + psi2 psi_{n-1} on the leading block (Eq. TAP4)."""
    a, b, c, g = (np.asarray(v, dtype=np.float64) for v in (a, b, c, g))
    n = b.shape[0]
    if n < 3:
        raise ValueError("a periodic line needs at least 3 unknowns")
    g = np.broadcast_to(g, np.broadcast_shapes(b.shape, g.shape))
    e = np.zeros_like(g[: n - 1])
    e[0] = -a[0]
    e[n - 2] = e[n - 2] - c[n - 2]
    psi1 = thomas(a[: n - 1], b[: n - 1], c[: n - 1], g[: n - 1])
    psi2 = thomas(a[: n - 1], b[: n - 1], c[: n - 1], e)
    last = (g[n - 1] - c[n - 1] * psi1[0] - a[n - 1] * psi1[n - 2]) / (
        b[n - 1] + c[n - 1] * psi2[0] + a[n - 1] * psi2[n - 2])
    psi = np.empty_like(g)
    psi[: n - 1] = psi1 + psi2 * last
    psi[n - 1] = last
    return psi
