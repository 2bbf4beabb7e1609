"""ADI-CN implicit viscous sweeps (oracle; test infrastructure only).

Section 3.4 (Eqs. solve_1 to solve_4): the diagonal viscous terms
d_p(G_pp d_p u) are marched implicitly one direction at a time, each split in
two equal Crank-Nicolson halves, the other directions' diagonal terms being
explicit in the first sweep.  With kappa = (h / 2) sqrt(Pr / Ra) (h the
RKW3 sub-step) and L_p u the discrete diagonal term of direction p (Eq.
PC_term1; the flux form of Section 3.3):

  zeta (solve_2):  J u*   - kappa L_zeta u*  = J u^n + s + kappa L_zeta u^n
                                              + 2 kappa (L_eta + L_xi) u^n
  eta  (solve_3):  J u**  - kappa L_eta u**  = J u*   - kappa L_eta u^n
  xi   (solve_4):  J u*** - kappa L_xi u***  = J u**  - kappa L_xi u^n

J is the cell's |J^{-1}| and s the caller's explicit terms (beta h times the
advection, cross-diffusion, pressure and buoyancy terms), both volume
integrated like L.  Each sweep is a set of tridiagonal systems along the grid
lines of its direction, solved with ``tridiag.thomas`` (zeta, eta) and
``tridiag.thomas_periodic`` (xi, periodic).

Readings where the paper is silent (the paper's domain has no colatitude
walls, its no-slip radial walls are stated for the DNS only):
* Every value is cell-centred ([nr][nth][nph], like the pressure).
* A wall carries either zero flux ("flux0") or a given value ("value") at
  the wall face, half a cell from the centre: the wall-face flux is then
  2 G_pp(wall face) (u_w - u_c) in the outward sense.
* Longitude is periodic.
"""
from __future__ import annotations

import numpy as np

from .grid import shell
from .tridiag import thomas, thomas_periodic

FLUX0, VALUE = "flux0", "value"


def walls(radius=(VALUE, 0.0, 0.0), colatitude=(VALUE, 0.0, 0.0)):
    """Wall conditions: per pair (kind, value at the lower wall, value at the
    upper wall); the default is no-slip (u = 0) everywhere."""
    return {1: radius, 0: colatitude}


def _axis(d):
    return {0: 1, 1: 0, 2: 2}[d]        # paper direction -> array axis of [nr][nth][nph]


def face_G(sh, fm, d):
    """G_dd on every d-normal face, wall planes included, indexed by the array
    axes (face m along the axis lies below cell m)."""
    g = fm[f"G{d}"][..., d]
    if d == 0:
        return g                                     # [nr][nth + 1][nph]
    if d == 1:
        return g                                     # [nr + 1][nth][nph]
    return g                                         # [nr][nth][nph], face k below cell k


def apply_diag(sh, fm, u, d, bc):
    """(L_d u)_c = F(c + 1/2) - F(c - 1/2), F = G_dd (u_up - u_down) on interior
    faces; on a wall face 2 G_dd (u_w - u_c) outward ("value"), 0 ("flux0")."""
    sh = shell(sh)
    u = np.asarray(u, dtype=np.float64).reshape(sh.shape)
    ax = _axis(d)
    G = face_G(sh, fm, d)
    if d == 2:
        F = G * (u - np.roll(u, 1, axis=2))          # face k: between k-1 and k
        return np.roll(F, -1, axis=2) - F
    n = u.shape[ax]
    um = np.moveaxis(u, ax, 0)
    Gm = np.moveaxis(G, ax, 0)
    F = np.zeros((n + 1,) + um.shape[1:])
    F[1:n] = Gm[1:n] * (um[1:] - um[:-1])
    kind, lo, hi = bc[d]
    if kind == VALUE:
        F[0] = 2.0 * Gm[0] * (um[0] - lo)
        F[n] = 2.0 * Gm[n] * (hi - um[n - 1])
    return np.moveaxis(F[1:] - F[:-1], 0, ax)


def line_system(sh, fm, d, kappa, bc):
    """(a, b, c, w) of (J - kappa L_d) along the d-lines, position on the array
    axis: a, c couple the neighbours, b the cell, w the right-side term of the
    wall values (2 kappa G_w u_w)."""
    sh = shell(sh)
    ax = _axis(d)
    G = np.moveaxis(face_G(sh, fm, d), ax, 0)
    J = np.moveaxis(np.asarray(fm["J"]).reshape(sh.shape), ax, 0)
    n = J.shape[0]
    if d == 2:
        lo = G
        hi = np.roll(G, -1, axis=0)
        return -kappa * lo, J + kappa * (lo + hi), -kappa * hi, np.zeros_like(J)
    lo = G[:n].copy()
    hi = G[1:].copy()
    a = -kappa * lo
    c = -kappa * hi
    a[0] = 0.0
    c[n - 1] = 0.0
    kind, wl, wh = bc[d]
    glo, ghi = lo.copy(), hi.copy()
    w = np.zeros_like(J)
    if kind == VALUE:
        glo[0] = 2.0 * lo[0]
        ghi[n - 1] = 2.0 * hi[n - 1]
        w[0] += 2.0 * kappa * lo[0] * wl
        w[n - 1] += 2.0 * kappa * hi[n - 1] * wh
    else:
        glo[0] = 0.0
        ghi[n - 1] = 0.0
    b = J + kappa * (glo + ghi)
    return a, b, c, w


def sweep(sh, fm, d, kappa, rhs, bc):
    """Solve (J - kappa L_d) u = rhs along every d-line (Thomas; periodic
    Thomas in longitude)."""
    sh = shell(sh)
    ax = _axis(d)
    a, b, c, w = line_system(sh, fm, d, kappa, bc)
    g = np.moveaxis(np.asarray(rhs, dtype=np.float64).reshape(sh.shape), ax, 0) + w
    psi = (thomas_periodic if d == 2 else thomas)(a, b, c, g)
    return np.moveaxis(psi, 0, ax)


def substep(sh, fm, un, kappa, bc, src=None):
    """One ADI-CN sub-step (Eqs. solve_2, solve_3, solve_4): returns u***."""
    sh = shell(sh)
    un = np.asarray(un, dtype=np.float64).reshape(sh.shape)
    J = np.asarray(fm["J"]).reshape(sh.shape)
    L = [apply_diag(sh, fm, un, d, bc) for d in range(3)]
    r1 = J * un + kappa * L[0] + 2.0 * kappa * (L[1] + L[2])
    if src is not None:
        r1 = r1 + np.asarray(src).reshape(sh.shape)
    u1 = sweep(sh, fm, 0, kappa, r1, bc)
    u2 = sweep(sh, fm, 1, kappa, J * u1 - kappa * L[1], bc)
    return sweep(sh, fm, 2, kappa, J * u2 - kappa * L[2], bc)
