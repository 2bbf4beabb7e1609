"""Geometric multigrid for A x = b on the shell (oracle; test infrastructure only).

The paper solves Eq. PC_6 with HYPRE's semi-coarsening multigrid
(Section 3.6); the hierarchy, transfers and smoothers below are this library's
own cell-centred design, written out plainly so every GPU step has a CPU twin:

* coarse face metric by aggregation: a coarse face is tiled by fine faces,
  G^c_pq = (sum of fine G_pq over the tiling faces) / c_q, c_q in {1, 2} the
  coarsening factor along q (keeps the stencil pattern, A 1 = 0 and 1^T A = 0);
* coarsening policy: a direction may halve while its cell count is even and
  >= 4 (longitude additionally stays even); with the ``semi`` policy only the
  directions whose mean diagonal coefficient is >= SEMI_RATIO = 0.7 of the
  strongest are halved (semi-coarsening toward isotropy, the idea behind SMG);
* restriction: sum over children (b is volume integrated);
* prolongation: cell-centred trilinear (3/4, 1/4 per halved direction),
  mirror at walls, wrap in longitude; on the full sphere with the shell cut
  the colatitude partner beyond a pole is the coarse cell of the same row at
  longitude k + nph/2 (interpolation across the polar axis);
* smoothers: multicolour Gauss-Seidel (7-point: red/black by (i+j+k) mod 2;
  19-point: four colours ((i+j) mod 2) + 2((j+k) mod 2), swept 0..3), or
  weighted Jacobi (omega 6/7 for 7-point, 4/5 for 19-point), diagonal = diag(A),
  or radial-line Gauss-Seidel: every radial line (fixed colatitude and
  longitude index) is one block, solved exactly with the Thomas algorithm of
  Section 3.5 (``tridiag.thomas``) on its tridiagonal part of A; lines are
  coloured so that no two lines of a colour are coupled (7-point: zebra by
  (i+k) mod 2; 19-point: four colours (i mod 2) + 2 (k mod 2)), swept in
  colour order;
  or longitude-line Gauss-Seidel: every longitude line (fixed radius and
  colatitude index, periodic) is one block, solved with the periodic Thomas
  algorithm of Section 3.5 (``tridiag.thomas_periodic``) on the cyclic
  tridiagonal part of A on the line (couplings inside the line beyond it,
  the shell cut's, taken from the current iterate); colours 7-point
  (i+j) mod 2, 19-point (i mod 2) + 2 (j mod 2); a level with fewer than
  four longitudes is swept by point Gauss-Seidel instead;
  or alternating lines: one radial-line sweep, then one longitude-line sweep,
  per smoothing step (radial clustering and thin shells make the radial
  couplings strong, the poles the longitude ones);
* coarsest level: dense bordered solve [A 1; 1^T 0][e; lam] = [r; 0];
* V(nu1, nu2) cycle, iterated from x0 until ||b - A x||_2 / ||b||_2 <= tol;
* gauge: the J-weighted mean of x is removed at the end (discrete volume
  average of Eq. volumeavg).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np
import scipy.sparse as sp

from .grid import shell, face_metrics
from .operator import assemble
from .tridiag import thomas, thomas_periodic

SEMI, FULL = 0, 1
GS, JACOBI, LINE, XLINE, ALT = 0, 1, 2, 3, 4
SEMI_RATIO = 0.7


@dataclass
class Level:
    shape: tuple          # (nr, nth, nph)
    fm: dict              # face rows G0, G1, G2 (and J on the fine level)
    stencil: int
    A: sp.csr_matrix = None
    D: np.ndarray = None
    factors: tuple = None  # (c_zeta, c_eta, c_xi) to the next level, or None
    colours: list = field(default_factory=list)
    colour_rows: list = field(default_factory=list)   # A restricted to each colour's rows
    lines: list = None     # per line colour: (cells [nr][m], rows of A, lower, diag, upper)
    xlines: list = None    # per longitude-line colour: (cells [nph][m], rows of A, a, b, c)
    cut: bool = False      # full sphere: zeta lines joined through the poles

    @property
    def n(self):
        return int(np.prod(self.shape))


def colour_of(shape, stencil):
    """Colour index of every cell, [j][i][k] order."""
    nr, nth, nph = shape
    j, i, k = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nph), indexing="ij")
    if stencil == 7:
        return ((i + j + k) & 1).ravel()
    return (((i + j) & 1) + 2 * ((j + k) & 1)).ravel()


def line_colour_of(shape, stencil):
    """Colour of the radial line through every cell, [j][i][k] order."""
    nr, nth, nph = shape
    j, i, k = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nph), indexing="ij")
    if stencil == 7:
        return ((i + k) & 1).ravel()
    return ((i & 1) + 2 * (k & 1)).ravel()


def line_systems(lv):
    """For each line colour: the cells of its radial lines as an [nr][m] array
    (m lines, j on axis 0), the rows of A for those cells, and the tridiagonal
    part of A on each line: lower[j] = A(c_j, c_{j-1}), diag[j] = A(c_j, c_j),
    upper[j] = A(c_j, c_{j+1}) (zero past the walls)."""
    if lv.lines is None:
        nr = lv.shape[0]
        col = line_colour_of(lv.shape, lv.stencil)
        A = lv.A.tocsr()
        lv.lines = []
        for c in range(2 if lv.stencil == 7 else 4):
            cells = np.nonzero(col == c)[0].reshape(nr, -1)
            diag = np.asarray(A[cells.ravel(), cells.ravel()]).reshape(cells.shape)
            lower = np.zeros(cells.shape)
            upper = np.zeros(cells.shape)
            if nr > 1:
                lower[1:] = np.asarray(A[cells[1:].ravel(), cells[:-1].ravel()]).reshape(nr - 1, -1)
                upper[:-1] = np.asarray(A[cells[:-1].ravel(), cells[1:].ravel()]).reshape(nr - 1, -1)
            lv.lines.append((cells, A[cells.ravel()], lower, diag, upper))
    return lv.lines


def xline_colour_of(shape, stencil):
    """Colour of the longitude line through every cell, [j][i][k] order."""
    nr, nth, nph = shape
    j, i, k = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nph), indexing="ij")
    if stencil == 7:
        return ((i + j) & 1).ravel()
    return ((i & 1) + 2 * (j & 1)).ravel()


def xline_systems(lv):
    """For each longitude-line colour: the cells of its lines as an [nph][m]
    array (m lines, k on axis 0), the rows of A for those cells, and the
    cyclic tridiagonal part of A on each line: a[k] = A(c_k, c_{k-1}),
    b[k] = A(c_k, c_k), c[k] = A(c_k, c_{k+1}), indices wrapping."""
    if lv.xlines is None:
        nph = lv.shape[2]
        col = xline_colour_of(lv.shape, lv.stencil)
        A = lv.A.tocsr()
        lv.xlines = []
        for c in range(2 if lv.stencil == 7 else 4):
            sel = np.nonzero(col == c)[0]
            if sel.size == 0:
                continue
            cells = sel.reshape(-1, nph).T                       # [nph][m]
            flat = cells.ravel()
            km = np.roll(cells, 1, axis=0).ravel()
            kp = np.roll(cells, -1, axis=0).ravel()
            a = np.asarray(A[flat, km]).reshape(cells.shape)
            b = np.asarray(A[flat, flat]).reshape(cells.shape)
            cc = np.asarray(A[flat, kp]).reshape(cells.shape)
            lv.xlines.append((cells, A[flat], a, b, cc))
    return lv.xlines


def make_level(shape, fm, stencil, cut=False):
    lv = Level(shape=tuple(shape), fm=fm, stencil=stencil, cut=cut)
    lv.A = assemble(None, fm, stencil=stencil, shape=lv.shape, cut=cut)
    lv.D = lv.A.diagonal().copy()
    col = colour_of(lv.shape, stencil)
    ncol = 2 if stencil == 7 else 4
    lv.colours = [np.nonzero(col == c)[0] for c in range(ncol)]
    lv.colour_rows = [lv.A[idx] for idx in lv.colours]
    return lv


def mean_diagonal_coefficients(shape, fm):
    """Mean G_pp over the faces that carry flux, per direction (zeta, eta, xi)."""
    nr, nth, nph = shape
    m0 = fm["G0"][:, 1:nth, :, 0].mean() if nth > 1 else 0.0
    m1 = fm["G1"][1:nr, :, :, 1].mean() if nr > 1 else 0.0
    m2 = fm["G2"][..., 2].mean()
    return (m0, m1, m2)


def plan_factors(shape, fm, policy):
    """Coarsening factors (c_zeta, c_eta, c_xi) for the next level, or None."""
    nr, nth, nph = shape
    n = (nth, nr, nph)
    can = [d for d in range(3)
           if n[d] % 2 == 0 and n[d] >= 4 and (d != 2 or n[d] % 4 == 0)]
    if not can:
        return None
    if policy == FULL:
        chosen = can
    else:
        m = mean_diagonal_coefficients(shape, fm)
        top = max(m[d] for d in can)
        chosen = [d for d in can if m[d] >= SEMI_RATIO * top]
    return tuple(2 if d in chosen else 1 for d in range(3))


def coarsen_faces(shape, fm, c):
    """Aggregate fine face rows onto the coarse faces they tile."""
    nr, nth, nph = shape
    cz, ce, cx = c
    ncr, nct, ncp = nr // ce, nth // cz, nph // cx
    div = np.array([cz, ce, cx], dtype=np.float64)
    G0 = fm["G0"][:, ::cz, :, :]                                  # planes 0, cz, .., nth
    G0 = G0.reshape(ncr, ce, nct + 1, ncp, cx, 3).sum(axis=(1, 4)) / div
    G1 = fm["G1"][::ce, :, :, :]                                  # planes 0, ce, .., nr
    G1 = G1.reshape(ncr + 1, nct, cz, ncp, cx, 3).sum(axis=(2, 4)) / div
    G2 = fm["G2"][:, :, ::cx, :]                                  # planes 0, cx, .. (periodic)
    G2 = G2.reshape(ncr, ce, nct, cz, ncp, 3).sum(axis=(1, 3)) / div
    return (ncr, nct, ncp), {"G0": G0, "G1": G1, "G2": G2}


def build_hierarchy(fine_shape, fm, stencil=19, policy=SEMI, max_levels=16, coarse_max=512,
                    cut=False):
    levels = [make_level(fine_shape, fm, stencil, cut)]
    while len(levels) < max_levels and levels[-1].n > coarse_max:
        c = plan_factors(levels[-1].shape, levels[-1].fm, policy)
        if c is None:
            break
        levels[-1].factors = c
        shp, cfm = coarsen_faces(levels[-1].shape, levels[-1].fm, c)
        levels.append(make_level(shp, cfm, stencil, cut))
    return levels


# ---------------------------------------------------------------- transfers
def _restrict_1d(nc, c):
    if c == 1:
        return sp.identity(nc, format="csr")
    rows = np.repeat(np.arange(nc), 2)
    cols = np.arange(2 * nc)
    return sp.csr_matrix((np.ones(2 * nc), (rows, cols)), shape=(nc, 2 * nc))


def _prolong_1d(nc, c, periodic):
    if c == 1:
        return sp.identity(nc, format="csr")
    rows, cols, vals = [], [], []
    for C in range(nc):
        for s, nb in ((0, C - 1), (1, C + 1)):
            f = 2 * C + s
            if periodic:
                nb %= nc
            elif nb < 0 or nb >= nc:
                nb = C                     # mirror ghost at a wall
            rows += [f, f]
            cols += [C, nb]
            vals += [0.75, 0.25]
    return sp.coo_matrix((vals, (rows, cols)), shape=(2 * nc, nc)).tocsr()


def _prolong_sphere_plane(nct, ncp, cz, cx):
    """Prolongation on one (theta, phi) plane of a cut shell, [i][k] order: as
    the Kronecker product of the 1-D rules, except that a colatitude partner
    beyond a pole is the coarse cell of the same row at longitude + ncp/2."""
    nth, nph = nct * cz, ncp * cx
    rows, cols, vals = [], [], []
    for i in range(nth):
        if cz == 1:
            th = [(i, 1.0, 0)]
        else:
            C, s = divmod(i, 2)
            nb = C - 1 if s == 0 else C + 1
            th = [(C, 0.75, 0), (nb, 0.25, 0) if 0 <= nb < nct else (C, 0.25, ncp // 2)]
        for k in range(nph):
            if cx == 1:
                ph = [(k, 1.0)]
            else:
                C, s = divmod(k, 2)
                ph = [(C, 0.75), (((C - 1) if s == 0 else (C + 1)) % ncp, 0.25)]
            for ic, wt, turn in th:
                for kc, wp in ph:
                    rows.append(i * nph + k)
                    cols.append(ic * ncp + (kc + turn) % ncp)
                    vals.append(wt * wp)
    return sp.coo_matrix((vals, (rows, cols)), shape=(nth * nph, nct * ncp)).tocsr()


def transfer_matrices(fine_shape, c, cut=False):
    """(R, P): children sum and trilinear prolongation between a level and the
    next one, as Kronecker products over the [j][i][k] axes."""
    nr, nth, nph = fine_shape
    cz, ce, cx = c
    R = sp.kron(_restrict_1d(nr // ce, ce),
                sp.kron(_restrict_1d(nth // cz, cz), _restrict_1d(nph // cx, cx))).tocsr()
    if cut:
        plane = _prolong_sphere_plane(nth // cz, nph // cx, cz, cx)
    else:
        plane = sp.kron(_prolong_1d(nth // cz, cz, False), _prolong_1d(nph // cx, cx, True))
    P = sp.kron(_prolong_1d(nr // ce, ce, False), plane).tocsr()
    return R, P


# ---------------------------------------------------------------- level operations
def residual(lv, x, b):
    return b - lv.A @ x


def smooth(lv, x, b, sweeps, kind=GS):
    """``sweeps`` smoothing sweeps on A x = b, in place order of the colours."""
    x = np.array(x, dtype=np.float64, copy=True)
    if kind == GS:
        for _ in range(sweeps):
            for idx, rows in zip(lv.colours, lv.colour_rows):
                x[idx] += (b[idx] - rows @ x) / lv.D[idx]
    elif kind in (LINE, XLINE, ALT):
        for _ in range(sweeps):
            if kind in (LINE, ALT):
                for cells, rows, lower, diag, upper in line_systems(lv):
                    r = (b[cells.ravel()] - rows @ x).reshape(cells.shape)
                    x[cells.ravel()] += thomas(lower, diag, upper, r).ravel()
            if kind in (XLINE, ALT):
                if lv.shape[2] < 4:
                    x = smooth(lv, x, b, 1, GS)
                    continue
                for cells, rows, a, bb, c in xline_systems(lv):
                    r = (b[cells.ravel()] - rows @ x).reshape(cells.shape)
                    x[cells.ravel()] += thomas_periodic(a, bb, c, r).ravel()
    else:
        w = 6.0 / 7.0 if lv.stencil == 7 else 4.0 / 5.0
        for _ in range(sweeps):
            x = x + w * (b - lv.A @ x) / lv.D
    return x


def coarse_solve(lv, r):
    """Dense bordered solve on the coarsest level: [A 1; 1^T 0][e; lam] = [r; 0]."""
    n = lv.n
    B = np.zeros((n + 1, n + 1))
    B[:n, :n] = lv.A.toarray()
    B[:n, n] = 1.0
    B[n, :n] = 1.0
    rhs = np.concatenate([r, [0.0]])
    return np.linalg.solve(B, rhs)[:n]


class Hierarchy:
    def __init__(self, levels):
        self.levels = levels
        self.transfers = [transfer_matrices(lv.shape, lv.factors, lv.cut) if lv.factors else None
                          for lv in levels]

    def vcycle(self, l, x, b, nu1=2, nu2=2, kind=GS):
        lv = self.levels[l]
        if l == len(self.levels) - 1:
            return coarse_solve(lv, b)
        R, P = self.transfers[l]
        x = smooth(lv, x, b, nu1, kind)
        rc = R @ residual(lv, x, b)
        ec = self.vcycle(l + 1, np.zeros(rc.shape), rc, nu1, nu2, kind)
        x = x + P @ ec
        return smooth(lv, x, b, nu2, kind)


# ---------------------------------------------------------------- the solve
def prepare_rhs(J, f):
    """b = |J^{-1}| (f - mean_J f): the volume-integrated right side of Eq. PC_6,
    made compatible (sum b = 0) by removing the J-weighted mean."""
    J = np.asarray(J, dtype=np.float64).ravel()
    f = np.asarray(f, dtype=np.float64).ravel()
    mean = (J * f).sum() / J.sum()
    return J * (f - mean), mean


def gauge(J, x):
    """Remove the J-weighted mean of x (null space of A is the constants)."""
    J = np.asarray(J, dtype=np.float64).ravel()
    return x - (J * x).sum() / J.sum()


def default_stencil(sh):
    return 7 if shell(sh).mapping == 0 else 19


def setup(sh, stencil=None, policy=SEMI, max_levels=16, coarse_max=512, fm=None):
    sh = shell(sh)
    if stencil is None:
        stencil = default_stencil(sh)
    if fm is None:
        fm = face_metrics(sh)
    levels = build_hierarchy(sh.shape, fm, stencil, policy, max_levels, coarse_max, sh.cut)
    return Hierarchy(levels), fm


def solve(sh, f, tol=1e-10, stencil=None, policy=SEMI, nu1=2, nu2=2, kind=GS,
          max_levels=16, coarse_max=512, max_iters=200, x0=None, hier=None, fm=None):
    """FP64 multigrid solve of (1/J) d_i(J g^ij d_j p) = f on the shell.

    Returns (x, info); x has zero J-weighted mean, info holds ``iters``,
    ``rel_res`` (final), ``hist`` (per-iteration relative residuals),
    ``removed_mean`` and ``levels``."""
    sh = shell(sh)
    if hier is None:
        hier, fm = setup(sh, stencil, policy, max_levels, coarse_max, fm)
    J = fm["J"].ravel()
    b, mean = prepare_rhs(J, f)
    A = hier.levels[0].A
    x = np.zeros(sh.n) if x0 is None else np.array(x0, dtype=np.float64).ravel().copy()
    bn = np.linalg.norm(b)
    bn = bn if bn > 0 else 1.0
    hist = []
    it = 0
    while True:
        rel = np.linalg.norm(b - A @ x) / bn
        hist.append(rel)
        if rel <= tol or it >= max_iters:
            break
        x = hier.vcycle(0, x, b, nu1, nu2, kind)
        it += 1
    x = gauge(J, x)
    return x, {"iters": it, "rel_res": hist[-1], "hist": hist, "removed_mean": mean,
               "levels": len(hier.levels), "converged": hist[-1] <= tol}
