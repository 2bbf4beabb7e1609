"""Conservative discretisation of d_p(G_pq d_q phi) (oracle; test infrastructure only).

Section 3.3, Eqs. PC_8 and PC_term1-3: with unit computational spacing, the
flux through the face between cell L and its upper neighbour U = L + e_p is

    F = G_pp (x_U - x_L)
        + sum_{q != p} G_pq / 2 * [ (x_{L+e_q} + x_{U+e_q}) / 2 - (x_{L-e_q} + x_{U-e_q}) / 2 ]

with G the row p of the metric at that face, and (A x)_c = sum_p F(c+1/2 e_p) - F(c-1/2 e_p).

Readings where the paper is silent (boundary conditions of the pressure
correction are not stated):
* longitude (xi) is periodic (Section 3.7);
* radial and colatitude walls carry zero total flux (u.n = 0 makes the
  projection of Eq. PC_7 leave the wall velocity unchanged);
* a tangential difference that would reach one cell outside a wall uses the
  mirror ghost x_ghost = x_adjacent (zero normal derivative);
* the 7-point stencil (orthogonal mappings) keeps only the G_pp terms.
These choices make A 1 = 0 and 1^T A = 0 exactly.

Full sphere with the shell cut (Sections 3.5 and 3.7): a zeta line leaving
the grid through a pole re-enters at the same colatitude row, longitude
k + nph/2, so the cell one beyond row 0 (or row nth - 1) is that row's cell
across the pole.  The pole faces have zero area (no flux, see ``grid``); the
cut therefore enters only through the tangential differences of the cross
terms, where it replaces the mirror ghost.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .grid import shell, face_jacobian, metric_from_jacobian

PERIODIC = (False, False, True)   # zeta, eta, xi


def _flat(sh_shape, i, j, k):
    nr, nth, nph = sh_shape
    return (j * nth + i) * nph + k


def _shift(idx, q, s, n, cut=False):
    """Neighbour index along direction q (paper order, 0-based; |s| = 1):
    wrap in xi, mirror-clamp at the radial and colatitude walls, or across a
    pole of the shell cut (same zeta row, longitude + nph/2)."""
    out = list(idx)
    v = idx[q] + s
    if PERIODIC[q]:
        v = np.mod(v, n[q])
    elif q == 0 and cut:
        across = (v < 0) | (v > n[0] - 1)
        out[2] = np.where(across, np.mod(idx[2] + n[2] // 2, n[2]), idx[2])
        v = np.clip(v, 0, n[q] - 1)
    else:
        v = np.clip(v, 0, n[q] - 1)
    out[q] = v
    return tuple(out)


def _face_row(fm, d, L, n):
    """Row d of G at the face between L and L + e_d (face arrays are [j][i][k])."""
    i, j, k = L
    G = fm[f"G{d}"]
    if d == 0:
        return G[j, i + 1, k]
    if d == 1:
        return G[j + 1, i, k]
    return G[j, i, np.mod(k + 1, n[2])]


def _face_terms(d, L, U, g, n, stencil, cut=False):
    """(column cells, weights) whose weighted sum is the flux through the face."""
    terms = [(U, g[..., d]), (L, -g[..., d])]
    if stencil == 19:
        for q in range(3):
            if q == d:
                continue
            w = 0.25 * g[..., q]
            terms += [(_shift(L, q, +1, n, cut), w), (_shift(U, q, +1, n, cut), w),
                      (_shift(L, q, -1, n, cut), -w), (_shift(U, q, -1, n, cut), -w)]
    return terms


def assemble(sh, fm, stencil: int = 19, shape=None, cut=None):
    """Sparse A (CSR, N x N, cells ordered [j][i][k]) from the face G rows ``fm``.

    ``shape`` = (nr, nth, nph) and ``cut`` default to the shell's; coarse
    multigrid levels pass their own shape with aggregated face rows."""
    if cut is None:
        cut = shell(sh).cut if sh is not None else False
    if shape is None:
        shape = shell(sh).shape
    nr, nth, nph = shape
    n = (nth, nr, nph)                       # paper order zeta, eta, xi
    N = nr * nth * nph
    rows, cols, vals = [], [], []
    for d in range(3):
        ranges = [np.arange(nth), np.arange(nr), np.arange(nph)]
        if not PERIODIC[d]:
            ranges[d] = np.arange(n[d] - 1)  # interior faces only: walls carry no flux
        if len(ranges[d]) == 0:
            continue
        L = tuple(a.ravel() for a in np.meshgrid(*ranges, indexing="ij"))
        U = _shift(L, d, +1, n)
        g = _face_row(fm, d, L, n)
        fL = _flat(shape, *L)
        fU = _flat(shape, *U)
        for cell, w in _face_terms(d, L, U, g, n, stencil, cut):
            fc = _flat(shape, *cell)
            rows += [fL, fU]
            cols += [fc, fc]
            vals += [w, -w]                  # row L gets +F, row U gets -F
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


def apply_rows(sh, x, cells, stencil: int = 19):
    """(A x) at selected cells, computing each face metric on demand from the
    mapping (no full-grid arrays); ``cells`` = (j, i, k) integer arrays.
    Used for sampled checks on grids too large to assemble."""
    sh = shell(sh)
    n = (sh.nth, sh.nr, sh.nph)
    xr = np.asarray(x).reshape(sh.shape)
    j, i, k = (np.asarray(c, dtype=np.int64) for c in cells)
    c = (i, j, k)
    out = np.zeros(i.shape, dtype=np.float64)
    for d in range(3):
        for side in (+1, -1):
            # face between L and U = L + e_d; the cell is L (side +1) or U (side -1)
            if side == +1:
                L = c
                U = tuple(np.mod(a + 1, n[q]) if (q == d and PERIODIC[q]) else (a + 1 if q == d else a)
                          for q, a in enumerate(c))
            else:
                U = c
                L = tuple(np.mod(a - 1, n[q]) if (q == d and PERIODIC[q]) else (a - 1 if q == d else a)
                          for q, a in enumerate(c))
            inside = np.ones(i.shape, dtype=bool)
            if not PERIODIC[d]:
                inside = (L[d] >= 0) & (U[d] <= n[d] - 1)
            Ls = tuple(np.where(inside, a, 0) for a in L)
            Us = tuple(np.where(inside, a, 0) for a in U)
            # face corner vertex: plane U_d along d, L's indices elsewhere
            corner = list(Ls)
            corner[d] = Us[d] if not PERIODIC[d] else np.mod(Ls[d] + 1, n[d])
            with np.errstate(divide="ignore", invalid="ignore"):   # pole faces: masked
                _, G, _ = metric_from_jacobian(face_jacobian(sh, d, *corner))
            g = G[..., d, :]
            F = np.zeros(i.shape)
            for cell, w in _face_terms(d, Ls, Us, g, n, stencil, sh.cut):
                F = F + w * xr[cell[1], cell[0], cell[2]]
            out += np.where(inside, side * F, 0.0)
    return out
