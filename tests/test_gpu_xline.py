"""Longitude-line and alternating-line smoothers on the GPU against the oracle.

Every longitude line is solved on the cyclic tridiagonal part of its block
by the periodic Thomas algorithm (Section 3.5), one thread per line; the
alternating smoother sweeps radial lines, then longitude lines.  Grids: 7
and 19 points, ragged sizes, odd colatitude and radius counts (colours of
unequal size), the smallest longitude ring (a level with two longitudes takes
a point sweep), walled sectors and the full sphere.  Tolerances as in the
radial-line tests: FP64 1e-12, FP32 1e-5, FP16 coefficients 2e-3 of the
largest value, widened to eps * cond of the line blocks.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, mg as omg

pytestmark = pytest.mark.gpu

XLINE, ALT = 3, 4
XGRIDS = {
    "sphere_ragged": W.grid_desc(7, 9, 12, stretch=2.0),
    "triaxial_odd": W.grid_desc(5, 7, 12, mapping=2, flattening=0.1, e2=0.05, stretch=1.0),
    "oblate_nph4": W.grid_desc(6, 6, 4, r_out=1 / 0.6, mapping=1, flattening=0.1),
    "sphere_cut": W.grid_desc(6, 8, 16, stretch=1.0, cut=True),
}
TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3}
EPS = {0: 2.2e-16, 1: 6e-8, 2: 6e-8}


def _cyclic_cond(lv):
    worst = 1.0
    if lv.shape[2] >= 4:
        for cells, _, a, b, c in omg.xline_systems(lv):
            n = cells.shape[0]
            for l in range(cells.shape[1]):
                M = np.diag(b[:, l])
                for k in range(n):
                    M[k, (k - 1) % n] += a[k, l]
                    M[k, (k + 1) % n] += c[k, l]
                worst = max(worst, np.linalg.cond(M))
    for cells, _, lower, diag, upper in omg.line_systems(lv):
        for l in range(cells.shape[1]):
            M = np.diag(diag[:, l]) + np.diag(lower[1:, l], -1) + np.diag(upper[:-1, l], 1)
            worst = max(worst, np.linalg.cond(M))
    return worst


def _dev(a, prec):
    import torch
    dt = torch.float64 if prec == 0 else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda:0", dtype=dt)


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64).ravel()


def _st(g):
    return 7 if g["mapping"] == 0 else 19


@pytest.mark.parametrize("kind", [XLINE, ALT])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(XGRIDS))
def test_line_sweeps_match_oracle(lib, name, prec, kind):
    g = XGRIDS[name]
    h = lib.mg_setup(g, dict(precision=prec, smoother=kind, coarse_max=16))
    hier, fm = omg.setup(g, _st(g), coarse_max=16)
    rng = np.random.default_rng(41)
    for l, lv in enumerate(hier.levels[:-1]):
        x0 = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        xd, bd = _dev(x0, prec), _dev(b, prec)
        lib.mg_smooth(h, l, prec, xd, bd, 2, kind)
        ref = omg.smooth(lv, _np(_dev(x0, prec)), _np(bd), 2, kind)
        tol = max(TOL[prec], EPS[prec] * _cyclic_cond(lv))
        np.testing.assert_allclose(_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                   err_msg=f"level {l} shape {lv.shape}")


@pytest.mark.parametrize("chunks", [False, True])
@pytest.mark.parametrize("kind", [XLINE, ALT])
@pytest.mark.parametrize("name", list(XGRIDS))
def test_fp64_iterates_match_oracle(lib, name, kind, chunks, monkeypatch):
    """Plain FP64 multigrid through the batched engine with the line smoothers
    (one thread per line, or MG_XLINE_CHUNKS=1: several threads per line):
    iterates and residual histories after 1 and 3 V-cycles."""
    import torch
    if chunks:
        monkeypatch.setenv("MG_XLINE_CHUNKS", "1")
    g = XGRIDS[name]
    n = grid.shell(g).n
    f = np.random.default_rng(42).standard_normal(n)
    for iters in (1, 3):
        h = lib.mg_setup(g, dict(precision=0, smoother=kind, coarse_max=16, max_iters=iters))
        hier, fm = omg.setup(g, _st(g), coarse_max=16)
        fd = _dev(f, 0)
        xd = torch.zeros_like(fd)
        rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
        xo, info = omg.solve(g, f, tol=1e-300, hier=hier, fm=fm, kind=kind, max_iters=iters)
        assert rep["iters"] == info["iters"] == iters
        np.testing.assert_allclose(_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
        # FP64 evaluation of b - A x rounds at about eps * cond(A) of ||b||:
        # an absolute floor in relative-residual units beside the relative check
        np.testing.assert_allclose(rep["res_hist"], info["hist"], rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("prec", [0, 1])
def test_alternating_lines_solve_the_full_sphere(lib, prec):
    """Full sphere, 32 x 32 x 64: alternating lines reach 1e-12 in the
    oracle's iteration count (FP64) and agree with the oracle's solution."""
    import torch
    g = W.grid_desc(32, 32, 64, stretch=1.0, cut=True)
    f = W.rhs_modes(g, seed=5)
    h = lib.mg_setup(g, dict(precision=prec, smoother=ALT))
    hier, fm = omg.setup(g, 7)
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    xo, info = omg.solve(g, f.ravel(), tol=1e-12, hier=hier, fm=fm, kind=omg.ALT)
    assert rep["rel_res"] <= 1e-12 and info["converged"]
    if prec == 0:
        assert rep["iters"] == info["iters"]
    assert rep["iters"] <= 14
    assert np.abs(_np(xd) - xo).max() <= 1e-9 * np.abs(xo).max()


def test_mixed_smoothers_in_one_batch(lib):
    """A batch of handles with point, radial-line and alternating smoothers
    gives each shell the bits of its lone solve."""
    import torch
    g = XGRIDS["sphere_ragged"]
    f = _dev(W.rhs_modes(g, seed=6), 0)
    hs, xs = [], []
    for kind in (0, 2, ALT, XLINE):
        hs.append(lib.mg_setup(g, dict(precision=1, smoother=kind)))
        xs.append(torch.zeros_like(f))
    lib.mg_solve_batch(hs, [f] * 4, xs, [1e-10] * 4)
    for h, x in zip(hs, xs):
        lone = torch.zeros_like(f)
        lib.mg_solve(h, f, lone, tol=1e-10)
        assert torch.equal(lone, x)
