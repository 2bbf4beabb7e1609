"""Semi-coarsening multigrid with plane relaxation (oracle; test infrastructure only).

The paper solves Eq. PC_6 with a semi-coarsening multigrid (Section 3.6);
this module is this library's own plain statement of that solver class on the
shell, not a restatement of any library's code:

* the grid is coarsened along one direction only, the colatitude zeta, by
  two, until one plane is left (or the row count is odd); the coarse face
  metric is the aggregation of ``mg.coarsen_faces`` with factors (2, 1, 1);
* the smoother is zebra plane relaxation: every (eta, xi) plane (fixed zeta
  row i, all radii and longitudes) is one block of a block Gauss-Seidel
  sweep, x_P += A_PP^{-1} (b - A x)_P, planes with i even first, then odd.
  Both stencils couple a plane with its two neighbours only, so the planes of
  one parity are independent;
* restriction sums the two children, prolongation is linear in zeta
  (3/4, 1/4), mirrored at a colatitude wall, across the polar axis on the
  full sphere (``mg.transfer_matrices``);
* the coarsest level (one plane, or an odd row count) is solved by the
  bordered direct solve of ``direct``.

Reading (the paper names the solver class only): zeta is the coarsening
direction because every strong coupling of the shell lies inside the
(eta, xi) planes: the radial clustering of Eq. stretching and thin shells
strengthen eta, the poles strengthen xi (G_xixi grows like 1/sin(theta)),
and the shell cut joins cells of the same zeta row (k and k + nph/2), so the
plane solves take the cut couplings in whole.

The plane solve is either exact (sparse LU of A_PP: the definition of plane
relaxation) or ``plane_cycles`` cycles of the same construction one dimension
down: each plane is coarsened along eta, relaxed by zebra xi-lines (rows of
fixed j, even first), each line solved with the periodic Thomas algorithm of
Section 3.5 (``tridiag.thomas_periodic``) on the tridiagonal part of A on the
line, the rest of the plane's couplings (19-point diagonals, the cut) taken
from the current iterate.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .grid import shell, face_metrics
from .mg import coarsen_faces, transfer_matrices, prepare_rhs, gauge, default_stencil
from .operator import assemble
from .direct import bordered_solve
from .tridiag import thomas_periodic

EXACT = 0          # plane solve: sparse LU of the plane block


class Level:
    """One level: shape (nr, nth, nph), face rows, A, plane blocks."""

    def __init__(self, shape, fm, stencil, cut):
        self.shape = tuple(shape)
        self.fm = fm
        self.stencil = stencil
        self.cut = cut
        self.A = assemble(None, fm, stencil=stencil, shape=self.shape, cut=cut).tocsr()
        nr, nth, nph = self.shape
        idx = np.arange(self.n).reshape(nr, nth, nph)
        # cells of plane i in [j][k] order, and the rows of A for them
        self.planes = [idx[:, i, :].ravel() for i in range(nth)]
        self.rows = [self.A[c] for c in self.planes]
        self._lu = {}
        self._plane2d = {}

    @property
    def n(self):
        return int(np.prod(self.shape))

    def plane_block(self, i):
        c = self.planes[i]
        return self.rows[i][:, c].tocsc()

    def plane_lu(self, i):
        if i not in self._lu:
            self._lu[i] = spla.splu(self.plane_block(i))
        return self._lu[i]

    def plane_hierarchy(self, i):
        if i not in self._plane2d:
            nr, _, nph = self.shape
            self._plane2d[i] = PlaneHierarchy(self.plane_block(i).tocsr(), nr, nph)
        return self._plane2d[i]


# ---------------------------------------------------------------- the 2-D plane cycle
def _coarsen_rows_2d(B, nr, nph):
    """Coarse plane operator B_c = R B P: R sums the two eta children, P is
    the linear prolongation along eta.  For the eta couplings this is the
    fine coefficient over the coarsening factor 2 (as the face aggregation of
    the 3-D levels); the xi couplings of the two children add up."""
    R = sp.kron(_children(nr // 2), sp.identity(nph)).tocsr()
    P = sp.kron(_prolong_eta(nr // 2), sp.identity(nph)).tocsr()
    return (R @ B @ P).tocsr(), R, P


def _children(nc):
    rows = np.repeat(np.arange(nc), 2)
    return sp.csr_matrix((np.ones(2 * nc), (rows, np.arange(2 * nc))), shape=(nc, 2 * nc))


def _prolong_eta(nc):
    """Linear prolongation along eta (3/4, 1/4), mirrored at the walls."""
    rows, cols, vals = [], [], []
    for C in range(nc):
        for s, nb in ((0, C - 1), (1, C + 1)):
            nb = min(max(nb, 0), nc - 1)
            rows += [2 * C + s] * 2
            cols += [C, nb]
            vals += [0.75, 0.25]
    return sp.coo_matrix((vals, (rows, cols)), shape=(2 * nc, nc)).tocsr()


class PlaneHierarchy:
    """Semi-coarsening along eta for one (eta, xi) plane block B (cells [j][k]),
    relaxed by zebra xi-lines with the periodic Thomas algorithm."""

    def __init__(self, B, nr, nph):
        self.levels = []
        while True:
            lines = self._line_parts(B, nr, nph)
            self.levels.append((B, nr, nph, lines))
            if nr % 2 or nr < 2:
                break
            Bc, R, P = _coarsen_rows_2d(B, nr, nph)
            self.levels[-1] = self.levels[-1] + (R, P)
            B, nr = Bc, nr // 2
        self.coarse = spla.splu(B.tocsc())

    @staticmethod
    def _line_parts(B, nr, nph):
        """Per parity of j: the xi-lines' cells as an [nph][m] array (m lines,
        position k on axis 0), the rows of B for them, and the cyclic
        tridiagonal part of B on each line: a couples k to k - 1, c to k + 1
        (wrapping), b the cell itself."""
        parts = []
        for parity in (0, 1):
            js = np.arange(parity, nr, 2)
            if js.size == 0:
                continue
            cells = (js[None, :] * nph + np.arange(nph)[:, None])      # [nph][m]
            flat = cells.ravel()
            km = np.roll(cells, 1, axis=0).ravel()
            kp = np.roll(cells, -1, axis=0).ravel()
            b = np.asarray(B[flat, flat]).reshape(cells.shape)
            a = np.asarray(B[flat, km]).reshape(cells.shape)
            c = np.asarray(B[flat, kp]).reshape(cells.shape)
            parts.append((cells, B[flat], a, b, c))
        return parts

    def relax(self, l, x, r):
        """Zebra xi-line relaxation: lines of even j, then odd j."""
        for cells, rows, a, b, c in self.levels[l][3]:
            flat = cells.ravel()
            res = (r[flat] - rows @ x).reshape(cells.shape)
            x[flat] += thomas_periodic(a, b, c, res).ravel()
        return x

    def cycle(self, l, x, r):
        if l == len(self.levels) - 1:
            return self.coarse.solve(r)
        B, nr, nph, lines, R, P = self.levels[l]
        x = self.relax(l, x, r)
        ec = self.cycle(l + 1, np.zeros(R.shape[0]), R @ (r - B @ x))
        x = x + P @ ec
        return self.relax(l, x, r)


# ---------------------------------------------------------------- the 3-D solver
class Hierarchy:
    def __init__(self, fine_shape, fm, stencil, cut, coarse_max_planes=1):
        self.levels = [Level(fine_shape, fm, stencil, cut)]
        self.transfers = []
        while True:
            nr, nth, nph = self.levels[-1].shape
            if nth % 2 or nth <= coarse_max_planes:
                break
            shp, cfm = coarsen_faces(self.levels[-1].shape, self.levels[-1].fm, (2, 1, 1))
            self.transfers.append(transfer_matrices(self.levels[-1].shape, (2, 1, 1), cut))
            self.levels.append(Level(shp, cfm, stencil, cut))

    def relax(self, lv, x, b, plane_cycles=EXACT):
        """One zebra sweep of plane relaxation (even rows, then odd rows)."""
        nth = lv.shape[1]
        for parity in (0, 1):
            for i in range(parity, nth, 2):
                c = lv.planes[i]
                r = b[c] - lv.rows[i] @ x
                if plane_cycles == EXACT:
                    x[c] += lv.plane_lu(i).solve(r)
                else:
                    ph = lv.plane_hierarchy(i)
                    e = np.zeros(c.size)
                    for _ in range(plane_cycles):
                        e = ph.cycle(0, e, r)
                    x[c] += e
        return x

    def vcycle(self, l, x, b, nu1=1, nu2=1, plane_cycles=EXACT):
        lv = self.levels[l]
        if l == len(self.levels) - 1:
            return bordered_solve(lv.A, b, np.ones(lv.n))[0]
        R, P = self.transfers[l]
        x = np.array(x, dtype=np.float64, copy=True)
        for _ in range(nu1):
            x = self.relax(lv, x, b, plane_cycles)
        rc = R @ (b - lv.A @ x)
        x = x + P @ self.vcycle(l + 1, np.zeros(rc.shape), rc, nu1, nu2, plane_cycles)
        for _ in range(nu2):
            x = self.relax(lv, x, b, plane_cycles)
        return x


def setup(sh, stencil=None, fm=None):
    sh = shell(sh)
    if stencil is None:
        stencil = default_stencil(sh)
    if fm is None:
        fm = face_metrics(sh)
    return Hierarchy(sh.shape, fm, stencil, sh.cut), fm


def solve(sh, f, tol=1e-10, stencil=None, nu1=1, nu2=1, plane_cycles=EXACT,
          max_iters=100, hier=None, fm=None):
    """Semi-coarsening multigrid solve of (1/J) d_i(J g^ij d_j p) = f; returns
    (x, info) like ``mg.solve`` (zero J-weighted mean; iters, rel_res, hist)."""
    sh = shell(sh)
    if hier is None:
        hier, fm = setup(sh, stencil, fm)
    J = fm["J"].ravel()
    b, mean = prepare_rhs(J, f)
    A = hier.levels[0].A
    x = np.zeros(sh.n)
    bn = np.linalg.norm(b) or 1.0
    hist = []
    it = 0
    while True:
        rel = np.linalg.norm(b - A @ x) / bn
        hist.append(rel)
        if rel <= tol or it >= max_iters:
            break
        x = hier.vcycle(0, x, b, nu1, nu2, plane_cycles)
        it += 1
    x = gauge(J, x)
    return x, {"iters": it, "rel_res": hist[-1], "hist": hist, "removed_mean": mean,
               "levels": len(hier.levels), "converged": hist[-1] <= tol}
