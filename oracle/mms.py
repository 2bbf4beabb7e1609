"""Manufactured solutions with closed-form Laplacians (oracle pins; test infrastructure only).

The continuous operator behind Eq. PC_8 is the Laplacian written in the
curvilinear coordinates, (1/sqrt g) d_a (sqrt g g^{ab} d_b p).  It is
coordinate invariant, so it is derived here symbolically (sympy) in the
physical coordinates (rho, theta, phi) of the mapping, independently of the
paper's discrete metric:

* ``cosine``  - p = cos(pi rho_hat) cos(2 pi theta_hat) sin(2 phi): zero normal
  derivative at every wall of the orthogonal (spherical) mapping;
* ``bump``    - p = sin^2(pi rho_hat) sin^2(pi theta_hat) sin(2 phi): its whole
  gradient vanishes on the walls, so the wall flux is zero for any metric;
* ``conductive`` - p = a / r + b (Eq. conductive profile), exactly harmonic on
  the sphere; used in interior cells only (its wall flux is not zero);
* ``polar``   - p = sin^2(pi rho_hat) (cos theta + sin theta cos phi
  + sin^2 theta sin 2 phi): degree-one and degree-two surface harmonics, smooth
  through both poles (for the full sphere with the shell cut), whole gradient
  zero on the radial walls.

rho_hat = (rho - r_in)/(r_out - r_in), theta_hat = (theta - th0)/(th1 - th0).
"""
from __future__ import annotations

import functools
import numpy as np
import sympy as sy

from .grid import shell, cell_centres, _scales


@functools.lru_cache(maxsize=32)
def _lambdas(kind, fl, e2, r_in, r_out, th0, th1):
    rho, th, ph = sy.symbols("rho theta phi", real=True)
    X = sy.Matrix([(1 - fl) * rho * sy.cos(th),
                   (1 + e2) * rho * sy.sin(th) * sy.cos(ph),
                   rho * sy.sin(th) * sy.sin(ph)])
    u = [rho, th, ph]
    Jm = X.jacobian(u)                      # Jm[a, b] = dX_a / du_b
    g = (Jm.T * Jm)                         # covariant metric g_ab
    detg = sy.simplify(g.det()) if (fl == 0 and e2 == 0) else g.det()
    sqrtg = sy.sqrt(detg)
    ginv = g.adjugate() / detg              # contravariant g^{ab}
    rh = (rho - r_in) / (r_out - r_in)
    thh = (th - th0) / (th1 - th0)
    if kind == "cosine":
        p = sy.cos(sy.pi * rh) * sy.cos(2 * sy.pi * thh) * sy.sin(2 * ph)
    elif kind == "bump":
        p = sy.sin(sy.pi * rh) ** 2 * sy.sin(sy.pi * thh) ** 2 * sy.sin(2 * ph)
    elif kind == "conductive":
        p = 1 / rho + sy.Rational(1, 3)
    elif kind == "polar":
        p = sy.sin(sy.pi * rh) ** 2 * (sy.cos(th) + sy.sin(th) * sy.cos(ph)
                                       + sy.sin(th) ** 2 * sy.sin(2 * ph))
    else:
        raise ValueError(kind)
    grad = [sy.diff(p, v) for v in u]
    lap = 0
    for a in range(3):
        flux = sum(ginv[a, b] * grad[b] for b in range(3))
        lap += sy.diff(sqrtg * flux, u[a])
    lap = lap / sqrtg
    fp = sy.lambdify((rho, th, ph), p, "numpy")
    fl_ = sy.lambdify((rho, th, ph), lap, "numpy")
    return fp, fl_


def manufactured(sh, kind):
    """(p, Laplacian p) at the cell centres, [j][i][k] order."""
    sh = shell(sh)
    fl, e2 = _scales(sh)
    fp, flap = _lambdas(kind, float(fl), float(e2), float(sh.r_in), float(sh.r_out),
                        float(sh.th0), float(sh.th1))
    rho, th, ph = cell_centres(sh)
    p = np.broadcast_to(fp(rho, th, ph), rho.shape).astype(np.float64)
    lap = np.broadcast_to(flap(rho, th, ph), rho.shape).astype(np.float64)
    return p, lap
