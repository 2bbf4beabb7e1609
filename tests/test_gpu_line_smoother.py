"""The radial-line Gauss-Seidel smoother on the GPU against the oracle.

Every radial line is solved exactly on its tridiagonal block (Thomas
algorithm, Section 3.5); the GPU splits a line into chunks of rows whose
recurrences are composed through shared memory, so grids with more radial
cells than one chunk (several chunks per line) are included, with ragged
chunk lengths, odd colatitude counts (19-point colours of unequal size) and
the smallest longitude ring.  Tolerances as in the other parity tests: FP64
1e-12, FP32 1e-5, FP16 coefficients 2e-3 of the largest value.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, mg as omg

pytestmark = pytest.mark.gpu

LINE = 2
LGRIDS = {
    # 40 radial cells: four chunks of 10 rows (37: the last one holds 7)
    "sphere_tall": W.grid_desc(40, 6, 8, r_out=4.0, stretch=1.0),
    # 256 radial cells: sixteen chunks of 16 rows, two chunks per warp
    "sphere_256": W.grid_desc(256, 8, 16, r_out=20.0, stretch=1.0),
    "sphere_ragged": W.grid_desc(13, 10, 12, stretch=2.0),
    "triaxial_tall": W.grid_desc(37, 7, 8, r_out=4.0, mapping=2, flattening=0.1, e2=0.05, stretch=1.0),
    "oblate_nph4": W.grid_desc(12, 6, 4, r_out=1 / 0.6, mapping=1, flattening=0.1),
}
TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3}
EPS = {0: 2.2e-16, 1: 6e-8, 2: 6e-8}


def _line_cond(lv):
    """Largest condition number of the level's radial-line blocks: a line
    solve in working precision eps is good to about cond * eps."""
    worst = 1.0
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


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(LGRIDS))
def test_line_sweeps_match_oracle(lib, name, prec):
    g = LGRIDS[name]
    h = lib.mg_setup(g, dict(precision=prec, smoother=LINE, coarse_max=32))
    hier, fm = omg.setup(g, _st(g), coarse_max=32)
    rng = np.random.default_rng(31)
    for l, lv in enumerate(hier.levels[:2]):
        x0 = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        xd, bd = _dev(x0, prec), _dev(b, prec)
        lib.mg_smooth(h, l, prec, xd, bd, 2, LINE)
        ref = omg.smooth(lv, _np(_dev(x0, prec)), _np(bd), 2, omg.LINE)
        tol = max(TOL[prec], EPS[prec] * _line_cond(lv))
        np.testing.assert_allclose(_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                   err_msg=f"level {l}")


def test_line_sweep_on_a_gauss_seidel_handle(lib):
    """mg_smooth kind 2 on a handle set up for point Gauss-Seidel factors the
    line blocks on first use."""
    g = LGRIDS["sphere_ragged"]
    h = lib.mg_setup(g, dict(precision=1))
    hier, _ = omg.setup(g, 7)
    lv = hier.levels[0]
    rng = np.random.default_rng(32)
    x0, b = rng.standard_normal(lv.n), rng.standard_normal(lv.n)
    xd, bd = _dev(x0, 1), _dev(b, 1)
    lib.mg_smooth(h, 0, 1, xd, bd, 1, LINE)
    ref = omg.smooth(lv, _np(_dev(x0, 1)), _np(bd), 1, omg.LINE)
    np.testing.assert_allclose(_np(xd), ref, rtol=0, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("iters", [1, 3])
@pytest.mark.parametrize("name", list(LGRIDS))
def test_fp64_line_smoothed_iterates_match_oracle(lib, name, iters):
    """Plain FP64 multigrid with the radial-line smoother through the batched
    engine: iterate and residual history after k V-cycles."""
    import torch
    g = LGRIDS[name]
    n = grid.shell(g).n
    f = np.random.default_rng(33).standard_normal(n)
    h = lib.mg_setup(g, dict(precision=0, smoother=LINE, coarse_max=16, max_iters=iters))
    hier, fm = omg.setup(g, _st(g), coarse_max=16)
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
    xo, info = omg.solve(g, f, tol=1e-300, hier=hier, fm=fm, max_iters=iters, kind=omg.LINE)
    assert rep["iters"] == info["iters"] == iters
    np.testing.assert_allclose(_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    # the line smoother contracts by ~1e-3 per cycle: by the third cycle the
    # relative residual nears the FP64 rounding floor of ||A|| ||x|| eps
    np.testing.assert_allclose(rep["res_hist"][:iters + 1], info["hist"], rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("wl,scale", [("single_sphere_128", 4), ("single_oblate_256", 8)])
def test_line_smoothed_solves_match_oracle(lib, wl, scale, prec):
    import torch
    w = W.single(wl, scale)
    g, f = w["grid"], w["f"]
    h = lib.mg_setup(g, dict(precision=prec, smoother=LINE))
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    assert rep["status"] == "MG_OK" and rep["rel_res"] <= 1e-12
    xo, info = omg.solve(g, f.ravel(), tol=1e-12, kind=omg.LINE, max_iters=400)
    assert info["converged"]
    err = np.abs(_np(xd) - xo).max() / np.abs(xo).max()
    assert err <= 1e-9, err


def test_thin_shell_iteration_counts(lib):
    """Radius 1 to 1.05, stretched, full coarsening: point Gauss-Seidel stalls,
    radial lines converge; the FP64 iteration counts are the oracle's."""
    import torch
    g = W.grid_desc(16, 16, 32, r_in=1.0, r_out=1.05, stretch=2.0)
    f = np.random.default_rng(0).standard_normal(grid.shell(g).n)
    its = {}
    for kind in (0, LINE):
        h = lib.mg_setup(g, dict(precision=0, smoother=kind, coarsen=1, max_iters=60))
        fd = _dev(f, 0)
        xd = torch.zeros_like(fd)
        rep = lib.mg_solve(h, fd, xd, tol=1e-10, allow=(lib.MG_OK, lib.MG_ENOCONV))
        _, info = omg.solve(g, f, tol=1e-10, policy=omg.FULL, kind=kind, max_iters=60)
        assert rep["iters"] == info["iters"]
        its[kind] = rep["iters"]
    assert its[0] == 60 and its[LINE] <= 10, its


def test_batched_line_solves_equal_lone_solves(lib):
    import torch
    shells = [W.grid_desc(16, stretch=2.0), W.grid_desc(24, 12, 16, r_out=1 / 0.6, mapping=1, flattening=0.1),
              W.grid_desc(12, 8, 8, mapping=2, flattening=0.05, e2=0.05)]
    fs = [W.rhs_modes(g, seed=40 + s) for s, g in enumerate(shells)]
    opts = dict(precision=1, smoother=LINE)
    hs = [lib.mg_setup(g, opts) for g in shells]
    fd = [_dev(f, 0) for f in fs]
    xs = [torch.zeros_like(f) for f in fd]
    reps = lib.mg_solve_batch(hs, fd, xs, [1e-10] * 3)
    for g, f, x, rep in zip(shells, fd, xs, reps):
        h = lib.mg_setup(g, opts)
        xl = torch.zeros_like(f)
        rl = lib.mg_solve(h, f, xl, tol=1e-10)
        assert rep["iters"] == rl["iters"]
        assert torch.equal(x, xl)


def test_mixed_smoothers_in_one_batch(lib):
    """Point and radial-line Gauss-Seidel handles solved together (one launch
    per level operation for each smoother): each equals its lone solve."""
    import torch
    shells = [W.grid_desc(16, stretch=2.0), W.grid_desc(12, 8, 16, mapping=2, flattening=0.05, e2=0.05),
              W.grid_desc(16, 16, 32, r_out=1.05, stretch=2.0), W.grid_desc(8, stretch=1.0)]
    smoothers = [0, LINE, LINE, 0]
    fs = [_dev(W.rhs_modes(g, seed=60 + s), 0) for s, g in enumerate(shells)]
    hs = [lib.mg_setup(g, dict(precision=1, smoother=sm)) for g, sm in zip(shells, smoothers)]
    xs = [torch.zeros_like(f) for f in fs]
    reps = lib.mg_solve_batch(hs, fs, xs, [1e-10] * len(hs))
    for g, sm, f, x, rep in zip(shells, smoothers, fs, xs, reps):
        xl = torch.zeros_like(f)
        rl = lib.mg_solve(lib.mg_setup(g, dict(precision=1, smoother=sm)), f, xl, tol=1e-10)
        assert rep["iters"] == rl["iters"] and torch.equal(x, xl)


def test_too_many_radial_cells_is_rejected(lib):
    with pytest.raises(lib.MGError) as e:
        lib.mg_setup(W.grid_desc(520, 4, 8), dict(precision=1, smoother=LINE))
    assert e.value.status == lib.MG_EINVAL
