"""Seeded synthetic workloads for the shell Poisson solve.

This module holds only input generation: grid descriptions and right-hand
sides evaluated at cell-centre *computational* coordinates (no mapping, metric
or operator arithmetic).  Tests, ``bench.py`` and the oracle harness all draw
their inputs from here, so the oracle and the CUDA library always receive the
same float64 buffers.

Workloads (sizes and distributions follow the paper's shells: radius ratio,
colatitude band pi/6..5pi/6 without the poles, periodic longitude, tanh wall
clustering of Eq. stretching):

* ``single_sphere_32``      - 32 x 32 x 64 sphere, r in [1, 2], uniform; RHS =
  closed-form spherical Laplacian of p* = cos(pi(r-1)) cos(3 theta) sin(2 phi)
  plus N(0, 1e-3) noise (seed 0); plain FP64 multigrid, 4 levels, V(2,2).
* ``single_sphere_128``     - 128 x 128 x 256 sphere, tanh stretching 2.0;
  RHS = 16 random Legendre x cosine modes (seed 0).
* ``single_oblate_256``     - 256 x 256 x 512 oblate shell (flattening 0.1),
  r in [1, 1/0.6], 19-point stencil; same RHS family (seed 0).
* ``batch_64``              - 64 shells, nr in {32, 64, 96, 128}, nth = nr,
  nph = 2 nr, radius ratio U[0.35, 0.8], flattening U[0, 0.15]; RHS seed 1000+s.
* ``serve_stream``          - request stream: nr log-uniform in [32, 192]
  snapped to the multigrid-friendly sizes 2^a x {1, 3, 5}, flattening
  U[0, 0.15], tol in {1e-6, 1e-8, 1e-10}, Poisson arrivals.
"""
from __future__ import annotations

import math
import numpy as np
from numpy.polynomial import legendre

PI = math.pi


def grid_desc(nr, nth=None, nph=None, r_in=1.0, r_out=2.0, th0=PI / 6, th1=5 * PI / 6,
              mapping=0, flattening=0.0, e2=0.0, stretch=0.0, cut=False):
    """Grid description dict (the C field names).  ``cut`` makes it the full
    sphere with the shell cut (th0 = 0, th1 = pi)."""
    nth = nr if nth is None else nth
    nph = 2 * nr if nph is None else nph
    if cut:
        th0, th1 = 0.0, PI
    return dict(nr=int(nr), nth=int(nth), nph=int(nph), r_in=float(r_in), r_out=float(r_out),
                th0=float(th0), th1=float(th1), mapping=int(mapping),
                flattening=float(flattening), e2=float(e2), stretch=float(stretch), cut=int(bool(cut)))


def _centres(g):
    """Computational cell-centre coordinates in [0, 1] (radius, colatitude) and
    longitude in [0, 2 pi), arrays of shape [nr][nth][nph]."""
    rh = (np.arange(g["nr"]) + 0.5) / g["nr"]
    th = (np.arange(g["nth"]) + 0.5) / g["nth"]
    ph = 2 * PI * (np.arange(g["nph"]) + 0.5) / g["nph"]
    return np.meshgrid(rh, th, ph, indexing="ij")


def rhs_pstar(g, seed=0, noise=1e-3):
    """Closed-form spherical Laplacian of p* = cos(pi(r-1)) cos(3 theta) sin(2 phi)
    at the centres of a *uniform* sphere grid, plus i.i.d. N(0, noise^2)."""
    if g["mapping"] != 0 or g["stretch"] != 0.0:
        raise ValueError("rhs_pstar is defined on the uniform sphere")
    rh, thh, ph = _centres(g)
    r = g["r_in"] + (g["r_out"] - g["r_in"]) * rh
    th = g["th0"] + (g["th1"] - g["th0"]) * thh
    R = np.cos(PI * (r - 1))
    dR = -PI * np.sin(PI * (r - 1))
    d2R = -PI ** 2 * np.cos(PI * (r - 1))
    T = np.cos(3 * th)
    lapT = -3 * np.cos(th) / np.sin(th) * np.sin(3 * th) - 9 * np.cos(3 * th)
    P = np.sin(2 * ph)
    f = ((d2R + 2 / r * dR) * T * P + R / r ** 2 * lapT * P
         - 4 * R * T * P / (r ** 2 * np.sin(th) ** 2))
    if noise:
        f = f + np.random.default_rng(seed).normal(0.0, noise, size=f.shape)
    return np.ascontiguousarray(f, dtype=np.float64)


def rhs_modes(g, seed=0, n_modes=16):
    """Smooth random field: sum of ``n_modes`` modes
    a P_n(2 r_hat - 1) cos(pi k theta_hat) cos(l phi + psi), a ~ N(0,1),
    n, k in {0..4}, l in {0..8}, psi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    rh, thh, ph = _centres(g)
    x = 2 * rh[:, 0, 0] - 1
    f = np.zeros(rh.shape)
    for _ in range(n_modes):
        a = rng.normal()
        n = int(rng.integers(0, 5))
        k = int(rng.integers(0, 5))
        l = int(rng.integers(0, 9))
        psi = rng.uniform(0, 2 * PI)
        c = np.zeros(n + 1)
        c[n] = 1.0
        Pr = legendre.legval(x, c)[:, None, None]
        f += a * Pr * np.cos(PI * k * thh[:1, :, :1]) * np.cos(l * ph[:1, :1, :] + psi)
    return np.ascontiguousarray(f, dtype=np.float64)


SINGLE = {
    "single_sphere_32": dict(grid=grid_desc(32), rhs=("pstar", 0), tol=1e-10,
                             precision="fp64", max_levels=4, coarsen="full"),
    "single_sphere_128": dict(grid=grid_desc(128, stretch=2.0), rhs=("modes", 0), tol=1e-10,
                              precision="fp32"),
    "single_oblate_256": dict(grid=grid_desc(256, r_out=1 / 0.6, mapping=1, flattening=0.1),
                              rhs=("modes", 0), tol=1e-10, precision="fp32"),
    # a thin shell (radius ratio 1.05, tanh clustering 2): radial coupling
    # dominates by ~10^3; the case the radial-line smoother is for
    "single_thin_128": dict(grid=grid_desc(128, r_out=1.05, stretch=2.0), rhs=("modes", 0), tol=1e-10,
                            precision="fp32"),
    # the whole sphere with the shell cut (theta in [0, pi]): the paper's own
    # domain; longitude coupling grows like 1/sin^2(theta) toward the poles
    "single_full_sphere_128": dict(grid=grid_desc(128, stretch=2.0, cut=True), rhs=("modes", 0), tol=1e-10,
                                   precision="fp32"),
    # the oblate whole sphere (19 points, the cross terms across the poles;
    # point smoothing stalls at the poles, so many V-cycles)
    "single_full_oblate_64": dict(grid=grid_desc(64, r_out=1 / 0.6, mapping=1, flattening=0.1, cut=True),
                                  rhs=("modes", 0), tol=1e-10, precision="fp32", max_iters=1000),
}


def rhs_for(g, rhs):
    kind, seed = rhs
    if kind == "pstar":
        return rhs_pstar(g, seed)
    return rhs_modes(g, seed)


def single(name, scale=1):
    """Grid + RHS of a named single-solve workload; ``scale`` > 1 shrinks every
    dimension by that factor (parity-test sizes)."""
    w = dict(SINGLE[name])
    g = dict(w["grid"])
    if scale != 1:
        g.update(nr=g["nr"] // scale, nth=g["nth"] // scale, nph=g["nph"] // scale)
    w["grid"] = g
    w["f"] = rhs_for(g, w["rhs"])
    return w


def batch_shells(n=64, seed=0, sizes=(32, 64, 96, 128)):
    """Grids and RHS of the uneven batch: nr in ``sizes``, radius ratio
    U[0.35, 0.8] (r_in = 1, r_out = 1/ratio), flattening U[0, 0.15]."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        nr = int(rng.choice(sizes))
        ratio = float(rng.uniform(0.35, 0.8))
        fl = float(rng.uniform(0.0, 0.15))
        g = grid_desc(nr, r_out=1.0 / ratio, mapping=1, flattening=fl)
        out.append(dict(grid=g, f=None, seed=1000 + s))
    return out


def batch_rhs(item):
    return rhs_modes(item["grid"], item["seed"])


FRIENDLY = sorted({m * 2 ** a for m in (1, 3, 5) for a in range(3, 9)
                   if 32 <= m * 2 ** a <= 192})


def snap_friendly(nr):
    """Nearest (in log) size of the form 2^a x {1, 3, 5}: the coarsest multigrid
    level of such a grid stays small enough for a dense direct solve."""
    return min(FRIENDLY, key=lambda s: abs(math.log(s) - math.log(nr)))


def serve_stream(n=10000, rate=100.0, seed=0, ratio=0.5):
    """Requests with Poisson arrival times (seconds), log-uniform size,
    flattening U[0, 0.15] and tolerance in {1e-6, 1e-8, 1e-10}."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for q in range(n):
        nr = snap_friendly(math.exp(rng.uniform(math.log(32), math.log(192))))
        fl = float(rng.uniform(0.0, 0.15))
        tol = float(rng.choice([1e-6, 1e-8, 1e-10]))
        g = grid_desc(nr, r_out=1.0 / ratio, mapping=1, flattening=fl)
        out.append(dict(grid=g, tol=tol, t_arrive=float(t[q]), seed=2000 + q))
    return out
