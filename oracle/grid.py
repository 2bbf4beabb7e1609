"""Shell grid, mapping and the five-step face metric (oracle; test infrastructure only).

Notation follows the paper: computational directions 1 = zeta (colatitude theta,
integer index i), 2 = eta (radius, index j), 3 = xi (longitude phi, index k);
the computational cell has unit side (Section 3.1).  Arrays are stored with
shape [j][i][k] (radius slowest, longitude fastest).  Inside this module the
directions are numbered 0, 1, 2 for zeta, eta, xi.

Readings where the paper is silent:
* radial vertices follow Eq. stretching, mapped affinely from [-1/2, 1/2] to
  [r_in, r_out]; a zero stretching factor means uniform spacing (the limit);
* the paper writes out the metric stencil for the zeta-normal face only
  (Section 3.2, step 1); the eta- and xi-normal faces use the same stencil with
  the axes permuted;
* ghost vertices one plane outside the domain (needed by the normal
  derivative at wall faces) come from evaluating the analytic mapping there.

Full sphere with the shell cut (Section 3.5 "Handling shell cut", Section
3.7): with ``cut`` the colatitude runs over [0, pi] and a zeta grid line
continues through either pole into the line at longitude k + nph/2.  The
mapping evaluated at theta < 0 or theta > pi is already the point across the
pole (sin changes sign where cos(phi + pi) = -cos(phi)), so the vertex
stencil needs no special case.  Readings (the paper gives no pole metric):
* the zeta faces at theta = 0 and theta = pi have all four corners on the
  polar axis, hence zero area; the determinant of Section 3.2 vanishes there
  and the face carries no flux: its G row, C and determinant are zero.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict
import numpy as np

SPHERE, OBLATE, TRIAXIAL = 0, 1, 2


@dataclass(frozen=True)
class Shell:
    """Grid description: cells per direction and the mapping parameters."""
    nr: int
    nth: int
    nph: int
    r_in: float = 1.0
    r_out: float = 2.0
    th0: float = np.pi / 6
    th1: float = 5 * np.pi / 6
    mapping: int = SPHERE      # 0 sphere, 1 oblate, 2 triaxial
    flattening: float = 0.0    # x1 scaled by (1 - flattening)
    e2: float = 0.0            # x2 scaled by (1 + e2)
    stretch: float = 0.0       # rx_2 of Eq. stretching; 0 = uniform
    cut: bool = False          # full sphere, zeta lines joined through the poles

    def __post_init__(self):
        # Section 3.2's normal derivative at a longitude face differences the
        # vertex planes one cell to either side; with two cells around the
        # circle both are the same plane and the face determinant is zero.
        if self.nph < 4 or self.nph % 2:
            raise ValueError("nph must be even and >= 4")
        if self.cut and (self.th0 != 0.0 or self.th1 != np.pi):
            raise ValueError("the shell cut needs the full colatitude range [0, pi]")

    @property
    def shape(self):
        return (self.nr, self.nth, self.nph)

    @property
    def n(self):
        return self.nr * self.nth * self.nph

    def as_dict(self):
        return asdict(self)


def full_sphere(nr, nth, nph, **kw) -> Shell:
    """A shell over the whole sphere, theta in [0, pi], with the shell cut."""
    return Shell(nr, nth, nph, th0=0.0, th1=np.pi, cut=True, **kw)


def shell(d) -> Shell:
    """Accept a Shell, or a dict with Shell's field names."""
    if isinstance(d, Shell):
        return d
    keys = Shell.__dataclass_fields__.keys()
    return Shell(**{k: v for k, v in dict(d).items() if k in keys})


def _scales(sh: Shell):
    if sh.mapping == SPHERE:
        return 0.0, 0.0
    if sh.mapping == OBLATE:
        return sh.flattening, 0.0
    return sh.flattening, sh.e2


# ---------------------------------------------------------------- 1-D coordinates
def stretch_unit(jv, n, rx):
    """Eq. stretching, Section 3.7: s = tanh(rx((j-1)/n - 1/2)) / (2 tanh(rx/2)).

    ``jv`` is the 0-based vertex index (the paper's j - 1); it may be
    fractional (cell centres) or lie outside [0, n] (ghost vertices)."""
    t = np.asarray(jv, dtype=np.float64) / n - 0.5
    if rx == 0:
        return t
    return np.tanh(rx * t) / (2.0 * np.tanh(rx / 2.0))


def d_stretch_unit(jv, n, rx):
    """Derivative of ``stretch_unit`` with respect to the index (analytic)."""
    t = np.asarray(jv, dtype=np.float64) / n - 0.5
    if rx == 0:
        return np.full_like(t, 1.0 / n)
    return rx / (n * np.cosh(rx * t) ** 2 * 2.0 * np.tanh(rx / 2.0))


def radius(sh: Shell, jv):
    return sh.r_in + (sh.r_out - sh.r_in) * (stretch_unit(jv, sh.nr, sh.stretch) + 0.5)


def colatitude(sh: Shell, iv):
    return sh.th0 + (sh.th1 - sh.th0) * np.asarray(iv, dtype=np.float64) / sh.nth


def longitude(sh: Shell, kv):
    return 2.0 * np.pi * np.asarray(kv, dtype=np.float64) / sh.nph


def vertex(sh: Shell, i, j, k):
    """Cartesian position of computational point (i, j, k) (Section 2 mapping:
    x1 along the polar axis, x2 = r sin(theta) cos(phi), x3 = r sin(theta) sin(phi)),
    with the polar axis scaled by (1 - flattening) and x2 by (1 + e2)."""
    fl, e2 = _scales(sh)
    rho = radius(sh, j)
    th = colatitude(sh, i)
    ph = longitude(sh, k)
    x1 = (1.0 - fl) * rho * np.cos(th)
    x2 = (1.0 + e2) * rho * np.sin(th) * np.cos(ph)
    x3 = rho * np.sin(th) * np.sin(ph)
    return np.stack(np.broadcast_arrays(x1, x2, x3), axis=-1)


# ---------------------------------------------------------------- Section 3.2, step 1
def face_jacobian(sh: Shell, d: int, i, j, k):
    """J^{-1} = [dx_a/dzeta_p] at the face normal to direction d whose lowest
    corner is vertex (i, j, k) (Section 3.2 step 1, Eq. jacobi).

    The normal derivative is 0.125 x (sum of the 4 face-corner vertices one plane
    above - the same 4 one plane below); each tangential derivative is
    0.5 x (sum over the face's two edges of the vertex difference along that edge).
    Returns M with M[..., a, p] = dx_a/dzeta_p."""
    e = np.eye(3, dtype=np.int64)
    t1, t2 = [a for a in range(3) if a != d]
    base = (np.asarray(i), np.asarray(j), np.asarray(k))

    def V(off):
        return vertex(sh, base[0] + off[0], base[1] + off[1], base[2] + off[2])

    cols = [None, None, None]
    acc = 0.0
    for a in (0, 1):
        for b in (0, 1):
            t = a * e[t1] + b * e[t2]
            acc = acc + V(t + e[d]) - V(t - e[d])
    cols[d] = 0.125 * acc
    cols[t1] = 0.5 * ((V(e[t1]) - V(0 * e[t1])) + (V(e[t1] + e[t2]) - V(e[t2])))
    cols[t2] = 0.5 * ((V(e[t2]) - V(0 * e[t2])) + (V(e[t1] + e[t2]) - V(e[t1])))
    return np.stack(cols, axis=-1)


# ---------------------------------------------------------------- steps 2, 4, 5
def metric_from_jacobian(M):
    """Steps 2, 4 and 5 of Section 3.2 for a stack of J^{-1} matrices.

    det = |J^{-1}|; the inverse J = [dzeta_p/dx_a] = cof(J^{-1})^T / det;
    G_pq = |J^{-1}| sum_a J_pa J_qa and C_pq = |J^{-1}| J_pq (Eq. skewness).
    Returns (|det|, G, C)."""
    m = M
    cof = np.empty_like(m)
    cof[..., 0, 0] = m[..., 1, 1] * m[..., 2, 2] - m[..., 1, 2] * m[..., 2, 1]
    cof[..., 0, 1] = -(m[..., 1, 0] * m[..., 2, 2] - m[..., 1, 2] * m[..., 2, 0])
    cof[..., 0, 2] = m[..., 1, 0] * m[..., 2, 1] - m[..., 1, 1] * m[..., 2, 0]
    cof[..., 1, 0] = -(m[..., 0, 1] * m[..., 2, 2] - m[..., 0, 2] * m[..., 2, 1])
    cof[..., 1, 1] = m[..., 0, 0] * m[..., 2, 2] - m[..., 0, 2] * m[..., 2, 0]
    cof[..., 1, 2] = -(m[..., 0, 0] * m[..., 2, 1] - m[..., 0, 1] * m[..., 2, 0])
    cof[..., 2, 0] = m[..., 0, 1] * m[..., 1, 2] - m[..., 0, 2] * m[..., 1, 1]
    cof[..., 2, 1] = -(m[..., 0, 0] * m[..., 1, 2] - m[..., 0, 2] * m[..., 1, 0])
    cof[..., 2, 2] = m[..., 0, 0] * m[..., 1, 1] - m[..., 0, 1] * m[..., 1, 0]
    det = (m[..., 0, 0] * cof[..., 0, 0] + m[..., 0, 1] * cof[..., 0, 1]
           + m[..., 0, 2] * cof[..., 0, 2])
    Jinv_T = cof / det[..., None, None]          # [a, p] = J[p, a]
    J = np.swapaxes(Jinv_T, -1, -2)              # J[p, a] = dzeta_p / dx_a
    adet = np.abs(det)
    G = adet[..., None, None] * np.einsum("...pa,...qa->...pq", J, J)
    C = adet[..., None, None] * J
    return adet, G, C


def _face_index_grids(sh: Shell, d: int, jslice=None):
    """Vertex-index grids (i, j, k) of every face normal to d, in [j][i][k] order.

    zeta faces: planes i = 0..nth   -> shape (nr, nth+1, nph)
    eta faces:  planes j = 0..nr    -> shape (nr+1, nth, nph)
    xi faces:   planes k = 0..nph-1 -> shape (nr, nth, nph); plane k is the
                face between cells k-1 (mod nph) and k (periodic)."""
    nj = sh.nr + 1 if d == 1 else sh.nr
    ni = sh.nth + 1 if d == 0 else sh.nth
    js = np.arange(nj) if jslice is None else np.arange(nj)[jslice]
    jj, ii, kk = np.meshgrid(js, np.arange(ni), np.arange(sh.nph), indexing="ij")
    return ii, jj, kk


def _zero_pole_faces(sh: Shell, out: dict):
    """Zero-area zeta faces at the poles of a cut shell: no flux, no area."""
    if not sh.cut:
        return
    for key in ("G0", "det0", "C0"):
        if key in out:
            out[key][:, 0] = 0.0
            out[key][:, sh.nth] = 0.0


def face_metrics(sh, chunk_cells: int = 1 << 20, with_C: bool = False):
    """The five-step metric of Section 3.2 on every face of the grid.

    Returns a dict with, for each direction d in (0 zeta, 1 eta, 2 xi):
      ``G{d}``   - row d of G at every d-normal face, shape face_shape + (3,)
                   (entries ordered zeta, eta, xi);
      ``det{d}`` - |J^{-1}| at every d-normal face;
    and ``J`` - the cell-centre |J^{-1}| of step 3, shape [nr][nth][nph]."""
    sh = shell(sh)
    out = {}
    for d in range(3):
        nj = sh.nr + 1 if d == 1 else sh.nr
        per_plane = (sh.nth + (d == 0)) * sh.nph
        step = max(1, chunk_cells // max(per_plane, 1))
        Gs, dets, Cs = [], [], []
        for j0 in range(0, nj, step):
            ii, jj, kk = _face_index_grids(sh, d, slice(j0, min(nj, j0 + step)))
            M = face_jacobian(sh, d, ii, jj, kk)
            with np.errstate(divide="ignore", invalid="ignore"):   # pole faces, zeroed below
                adet, G, C = metric_from_jacobian(M)
            Gs.append(G[..., d, :])
            dets.append(adet)
            if with_C:
                Cs.append(C)
        out[f"G{d}"] = np.concatenate(Gs, axis=0)
        out[f"det{d}"] = np.concatenate(dets, axis=0)
        if with_C:
            out[f"C{d}"] = np.concatenate(Cs, axis=0)
    _zero_pole_faces(sh, out)
    out["J"] = cell_volume(sh, out)
    return out


def cell_volume(sh, fm):
    """Step 3 of Section 3.2: cell |J^{-1}| = mean of the six face determinants."""
    sh = shell(sh)
    d0, d1, d2 = fm["det0"], fm["det1"], fm["det2"]
    return (d0[:, :-1, :] + d0[:, 1:, :] + d1[:-1] + d1[1:]
            + d2 + np.roll(d2, -1, axis=2)) / 6.0


# ---------------------------------------------------------------- analytic metric
def analytic_jacobian(sh: Shell, iv, jv, kv):
    """Exact dx_a/dzeta_p at fractional computational point (iv, jv, kv)."""
    fl, e2 = _scales(sh)
    rho = radius(sh, jv)
    drho = (sh.r_out - sh.r_in) * d_stretch_unit(jv, sh.nr, sh.stretch)
    th = colatitude(sh, iv)
    dth = (sh.th1 - sh.th0) / sh.nth
    ph = longitude(sh, kv)
    dph = 2.0 * np.pi / sh.nph
    ct, st, cp, sp = np.cos(th), np.sin(th), np.cos(ph), np.sin(ph)
    rho, drho, ct, st, cp, sp = np.broadcast_arrays(rho, drho, ct, st, cp, sp)
    M = np.empty(rho.shape + (3, 3))
    # p = zeta (theta)
    M[..., 0, 0] = -(1 - fl) * rho * st * dth
    M[..., 1, 0] = (1 + e2) * rho * ct * cp * dth
    M[..., 2, 0] = rho * ct * sp * dth
    # p = eta (radius)
    M[..., 0, 1] = (1 - fl) * ct * drho
    M[..., 1, 1] = (1 + e2) * st * cp * drho
    M[..., 2, 1] = st * sp * drho
    # p = xi (phi)
    M[..., 0, 2] = 0.0
    M[..., 1, 2] = -(1 + e2) * rho * st * sp * dph
    M[..., 2, 2] = rho * st * cp * dph
    return M


def analytic_face_metrics(sh):
    """G rows and |J^{-1}| from exact derivatives at face centres (metric pins)."""
    sh = shell(sh)
    out = {}
    for d in range(3):
        ii, jj, kk = _face_index_grids(sh, d)
        c = [ii.astype(float), jj.astype(float), kk.astype(float)]
        for a in range(3):
            if a != d:
                c[a] = c[a] + 0.5
        M = analytic_jacobian(sh, c[0], c[1], c[2])
        with np.errstate(divide="ignore", invalid="ignore"):
            adet, G, _ = metric_from_jacobian(M)
        out[f"G{d}"] = G[..., d, :]
        out[f"det{d}"] = adet
    _zero_pole_faces(sh, out)
    return out


def face_metrics_analytic(sh):
    """The metric with exact derivatives at the face centres instead of the
    differences of Section 3.2 step 1 (steps 2 to 5 unchanged): G rows and
    |J^{-1}| of every face, and the cell |J^{-1}| as the mean of the six face
    determinants (step 3), in the layout of ``face_metrics``."""
    out = analytic_face_metrics(sh)
    out["J"] = cell_volume(sh, out)
    return out


def cell_centres(sh):
    """(rho, theta, phi) at cell centres = computational midpoints, mapped."""
    sh = shell(sh)
    jj, ii, kk = np.meshgrid(np.arange(sh.nr) + 0.5, np.arange(sh.nth) + 0.5,
                             np.arange(sh.nph) + 0.5, indexing="ij")
    return radius(sh, jj), colatitude(sh, ii), longitude(sh, kk)


def shell_volume(sh):
    """Exact volume of the mapped shell sector (closed form, used as a pin):
    (r_out^3 - r_in^3)/3 x (cos th0 - cos th1) x 2 pi x (1 - fl)(1 + e2)."""
    sh = shell(sh)
    fl, e2 = _scales(sh)
    return ((sh.r_out ** 3 - sh.r_in ** 3) / 3.0 * (np.cos(sh.th0) - np.cos(sh.th1))
            * 2.0 * np.pi * (1 - fl) * (1 + e2))


def cell_volume_at(sh, cells):
    """Step 3 of Section 3.2 at selected cells (j, i, k), computing the six face
    determinants on demand (for sampled checks on grids too large to hold)."""
    sh = shell(sh)
    j, i, k = (np.asarray(c, dtype=np.int64) for c in cells)
    total = np.zeros(i.shape)
    for d in range(3):
        lo = [i, j, k]
        hi = [i, j, k]
        hi[d] = hi[d] + 1
        if d == 2:
            hi[2] = np.mod(hi[2], sh.nph)
        for corner in (lo, hi):
            with np.errstate(divide="ignore", invalid="ignore"):
                adet, _, _ = metric_from_jacobian(face_jacobian(sh, d, *corner))
            if d == 0 and sh.cut:
                adet = np.where((corner[0] == 0) | (corner[0] == sh.nth), 0.0, adet)
            total += adet
    return total / 6.0
