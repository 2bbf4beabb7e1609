"""The steps either side of the pressure solve (oracle; test infrastructure only).

Section 3.6: the right side of Eq. PC_6, d_j(C_ji u***_i), and the correction
of Eq. PC_7, u = u*** - (1/J^{-1}) d_j(C_ji h dP), written for a staggered
velocity: the Cartesian components of the intermediate velocity live at the
face centres, and both steps use the face metric of Section 3.2 (C and
|J^{-1}| of the face, Eq. skewness).

Layout: ``u[d]`` holds (u_1, u_2, u_3) at every d-normal face, shape
face_shape(d) + (3,), with face_shape as in ``grid.face_metrics`` (both wall
planes included; d in zeta, eta, xi order).  Wall faces carry no flux: they
are left out of the divergence and left unchanged by the correction.

Readings where the paper is silent:
* The contravariant flux through a d-face is U_d = sum_a C_da u_a with the
  face's own C; the divergence is the flux balance of the cell,
  D(U)_c = sum_d U_d(c + 1/2 e_d) - U_d(c - 1/2 e_d) (the discrete d_j of
  PC_6 with unit computational spacing, volume-integrated like b).
* The correction uses at each face the gradient of the operator's flux
  (Eqs. PC_term1-3): the normal difference, and for the 19-point operator the
  averaged tangential differences (mirror ghosts at walls, wrap in
  longitude, across the pole on the full sphere with the shell cut); the
  7-point operator keeps the normal difference only.  Then
  U_d(new) = U_d - F_d(h dP) face by face, with F_d the operator's face
  flux, so D(U_new) = D(U***) - A (h dP): the corrected field's divergence is
  the solver's residual.
"""
from __future__ import annotations

import numpy as np

from .grid import shell


def face_shapes(sh):
    sh = shell(sh)
    return [(sh.nr, sh.nth + 1, sh.nph), (sh.nr + 1, sh.nth, sh.nph), (sh.nr, sh.nth, sh.nph)]


def _interior(sh, d):
    """Mask of the non-wall faces normal to d."""
    m = np.ones(face_shapes(sh)[d], dtype=bool)
    if d == 0:
        m[:, 0, :] = m[:, -1, :] = False
    elif d == 1:
        m[0, :, :] = m[-1, :, :] = False
    return m


def contravariant_flux(sh, fm, u, d):
    """U_d = sum_a C_da u_a at every d-face (zero on the walls)."""
    U = np.einsum("...a,...a->...", fm[f"C{d}"][..., d, :], u[d])
    return np.where(_interior(sh, d), U, 0.0)


def divergence(sh, fm, u):
    """D(U)_c, shape [nr][nth][nph] (volume-integrated, like b of Eq. PC_6)."""
    sh = shell(sh)
    U0, U1, U2 = (contravariant_flux(sh, fm, u, d) for d in range(3))
    D = (U0[:, 1:, :] - U0[:, :-1, :]) + (U1[1:, :, :] - U1[:-1, :, :])
    D = D + (np.roll(U2, -1, axis=2) - U2)       # xi plane k is the face between k-1 and k
    return D


def rhs(sh, fm, u):
    """The pointwise right side f = D(U)/|J^{-1}| to hand to the solver; its
    solution is x = h dP."""
    return divergence(sh, fm, u) / fm["J"]


def _cell(x, j, i, k):
    return x[j, i, k]


def face_gradient(sh, x, d, stencil):
    """Gradient components (zeta, eta, xi) of x at every interior d-face, shape
    face_shape(d) + (3,): the normal difference x_U - x_L and, for 19 points,
    the averaged tangential differences [(x_{L+q} + x_{U+q}) - (x_{L-q} + x_{U-q})] / 4."""
    sh = shell(sh)
    n = (sh.nth, sh.nr, sh.nph)                  # extent per paper direction
    xr = np.asarray(x).reshape(sh.shape)
    fj, fi, fk = np.meshgrid(*[np.arange(s) for s in face_shapes(sh)[d]], indexing="ij")
    # L and U cells of each face, (i, j, k) paper order; wall faces clamped (masked later)
    if d == 0:
        U = (np.clip(fi, 0, sh.nth - 1), fj, fk)
        L = (np.clip(fi - 1, 0, sh.nth - 1), fj, fk)
    elif d == 1:
        U = (fi, np.clip(fj, 0, sh.nr - 1), fk)
        L = (fi, np.clip(fj - 1, 0, sh.nr - 1), fk)
    else:
        U = (fi, fj, fk)
        L = (fi, fj, np.mod(fk - 1, sh.nph))

    def X(c):
        return xr[c[1], c[0], c[2]]

    def shift(c, q, s):
        v = list(c)
        if q == 2:
            v[q] = np.mod(c[q] + s, n[q])
        else:
            v[q] = np.clip(c[q] + s, 0, n[q] - 1)
            if q == 0 and sh.cut:               # across a pole: same row, longitude + nph/2
                across = (c[0] + s < 0) | (c[0] + s > n[0] - 1)
                v[2] = np.where(across, np.mod(c[2] + n[2] // 2, n[2]), c[2])
        return tuple(v)

    g = np.zeros(face_shapes(sh)[d] + (3,))
    g[..., d] = X(U) - X(L)
    if stencil == 19:
        for q in range(3):
            if q == d:
                continue
            g[..., q] = ((X(shift(L, q, 1)) + X(shift(U, q, 1))) - (X(shift(L, q, -1)) + X(shift(U, q, -1)))) / 4.0
    return np.where(_interior(sh, d)[..., None], g, 0.0)


def project(sh, fm, x, u, stencil):
    """Eq. PC_7 on the faces: u_a -= (1/|J^{-1}|_face) sum_j C_ja grad_j x at
    every interior face (x = h dP); returns the corrected face velocities."""
    out = []
    for d in range(3):
        g = face_gradient(sh, x, d, stencil)
        with np.errstate(divide="ignore", invalid="ignore"):     # zero-area pole faces: masked
            corr = np.einsum("...ja,...j->...a", fm[f"C{d}"], g) / fm[f"det{d}"][..., None]
        out.append(np.where(_interior(sh, d)[..., None], u[d] - corr, u[d]))
    return out
