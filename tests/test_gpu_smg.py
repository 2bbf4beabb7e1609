"""The semi-coarsening multigrid with zebra plane relaxation (Section 3.6's
solver class, reading 27) on the GPU against the oracle's (oracle/smg.py).

The hierarchy halves the colatitude only, down to one plane (the dense
bordered solve, or, for a plane beyond it, the point-smoothed semi-coarsening
of the other solvers below it); every (radius, longitude) plane is relaxed as
one block,
even colatitude rows first, each plane solved by 2-D V(1,1) cycles (radius
semi-coarsening with R B P coarse operators, zebra longitude lines by the
periodic Thomas algorithm of Section 3.5).  Checked: one and two zebra
sweeps on every level against the oracle's, FP64 iterates and residual
histories after 1 and 3 V(1,1) cycles, solves against the oracle's solution
(walled sectors and the full sphere), and the combinations that are not
built are refused.  Tolerances: FP64 1e-12, FP32 1e-5 of the largest
value, widened to eps * cond of the plane blocks (the GPU and the oracle
solve the same systems in another rounding order).
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, smg

pytestmark = pytest.mark.gpu

PLANE = 5
GRIDS = {
    "sphere_stretched": W.grid_desc(8, 8, 16, stretch=1.0),
    "sphere_ragged_rows": W.grid_desc(4, 12, 8),               # 12 -> 6 -> 3 colatitude rows
    "full_sphere": W.grid_desc(4, 8, 8, cut=True),
    "thin_shell": W.grid_desc(8, 8, 16, r_out=1.05, stretch=2.0),
}


def _torch():
    import torch
    return torch, torch.device("cuda:0")


def _dev(a, prec):
    torch, dev = _torch()
    dt = torch.float64 if prec == 0 else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dt)


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64).ravel()


def _plane_cond(lv):
    """Largest condition number of the level's plane blocks: the GPU and the
    oracle take the same steps in another rounding order, so their results
    differ by up to eps * cond of the blocks solved."""
    return max(np.linalg.cond(lv.plane_block(i).toarray()) for i in range(lv.shape[1]))


def _handle(lib, g, prec, cycles=1, **kw):
    return lib.mg_setup(g, dict(precision=prec, smoother=PLANE, nu1=1, nu2=1, plane_cycles=cycles, **kw))


@pytest.mark.parametrize("cycles", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(GRIDS))
def test_plane_sweeps_match_oracle(lib, name, prec, cycles):
    g = GRIDS[name]
    sh = grid.shell(g)
    hier, fm = smg.setup(sh, 7)
    h = _handle(lib, g, prec, cycles)
    assert lib.mg_get_level_info(h, 0)["levels"] == len(hier.levels)
    rng = np.random.default_rng(31)
    for l, lv in enumerate(hier.levels[:-1]):
        tol = max(1e-12 if prec == 0 else 1e-5, (2.2e-16 if prec == 0 else 6e-8) * _plane_cond(lv))
        li = lib.mg_get_level_info(h, l)
        assert (li["nr"], li["nth"], li["nph"]) == lv.shape
        x0 = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        for sweeps in (1, 2):
            xd, bd = _dev(x0, prec), _dev(b, prec)
            lib.mg_smooth(h, l, prec, xd, bd, sweeps, PLANE)
            ref = _np(_dev(x0, prec))
            for _ in range(sweeps):
                ref = hier.relax(lv, ref, _np(bd), plane_cycles=cycles)
            np.testing.assert_allclose(_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                       err_msg=f"level {l} {lv.shape} sweeps {sweeps}")
    h.close()


@pytest.mark.parametrize("name", list(GRIDS))
def test_smg_fp64_iterates_match_oracle(lib, name):
    """Plain FP64 V(1,1) cycles through the batched engine: the iterate and
    the residual history after 1 and 3 cycles."""
    import torch
    g = GRIDS[name]
    sh = grid.shell(g)
    f = np.random.default_rng(32).standard_normal(sh.n)
    hier, fm = smg.setup(sh, 7)
    for iters in (1, 3):
        h = _handle(lib, g, 0, max_iters=iters)
        fd = _dev(f, 0)
        xd = torch.zeros_like(fd)
        rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
        xo, info = smg.solve(sh, f, tol=1e-300, hier=hier, fm=fm, max_iters=iters, plane_cycles=1)
        assert rep["iters"] == info["iters"] == iters
        np.testing.assert_allclose(_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
        np.testing.assert_allclose(rep["res_hist"][:iters + 1], info["hist"], rtol=1e-9, atol=1e-13)
        h.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["sphere_stretched", "full_sphere", "thin_shell"])
def test_smg_solve_matches_oracle(lib, name, prec):
    """Solves to 1e-12 against the oracle's (the thin shell to 1e-11: its FP64
    residual floor, eps * cond, lies near 2e-12): the solution within 1e-9 of
    its largest value, and (FP64) the oracle's iteration count."""
    import torch
    g = GRIDS[name]
    tol = 1e-11 if name == "thin_shell" else 1e-12
    sh = grid.shell(g)
    f = W.rhs_modes(g, seed=5).ravel()
    hier, fm = smg.setup(sh, 7)
    xo, info = smg.solve(sh, f, tol=tol, hier=hier, fm=fm, plane_cycles=1, max_iters=200)
    assert info["converged"]
    h = _handle(lib, g, prec, max_iters=200)
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=tol)
    assert rep["rel_res"] <= tol
    err = np.abs(_np(xd) - xo).max() / np.abs(xo).max()
    assert err <= 1e-9, err
    if prec == 0:
        assert rep["iters"] == info["iters"]
    h.close()


def test_smg_full_sphere_converges_where_point_smoothing_stalls(lib):
    """Full sphere 16 x 16 x 32: plane relaxation reaches 1e-10 in a few
    V(1,1) cycles (the oracle's count), point Gauss-Seidel multigrid needs far
    more V(2,2) cycles."""
    import torch
    g = W.grid_desc(16, cut=True)
    sh = grid.shell(g)
    f = W.rhs_modes(g, seed=6).ravel()
    _, info = smg.solve(sh, f, tol=1e-10, plane_cycles=1, stencil=7)
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(_handle(lib, g, 1, max_iters=100), fd, xd, tol=1e-10)
    assert rep["iters"] <= info["iters"] + 1
    xd.zero_()
    rep_gs = lib.mg_solve(lib.mg_setup(g, dict(precision=1, max_iters=200)), fd, xd, tol=1e-10)
    assert rep_gs["iters"] > 2 * rep["iters"]


@pytest.mark.parametrize("prec", [0, 1])
def test_smg_with_a_large_coarsest_plane(lib, prec):
    """32 x 32 x 128: the one plane the colatitude coarsening ends on (32 x
    128 = 4096 cells) is beyond the dense solve, so the hierarchy continues
    below it with the point-smoothed semi-coarsening of the other solvers;
    the solution still matches the oracle's SMG (whose coarsest plane is a
    sparse direct solve) within 1e-9 at 1e-12."""
    import torch
    g = W.grid_desc(32, 32, 128, stretch=1.0)
    sh = grid.shell(g)
    f = W.rhs_modes(g, seed=8).ravel()
    xo, info = smg.solve(sh, f, tol=1e-12, plane_cycles=1, stencil=7, max_iters=200)
    assert info["converged"]
    h = _handle(lib, g, prec, max_iters=200)
    assert lib.mg_get_level_info(h, 0)["levels"] > info["levels"]
    fd = _dev(f, 0)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    assert rep["rel_res"] <= 1e-12
    assert rep["iters"] <= info["iters"] + 3
    err = np.abs(_np(xd) - xo).max() / np.abs(xo).max()
    assert err <= 1e-9, err
    h.close()


def test_plane_smoother_refuses_what_is_not_built(lib):
    for g, why in ((W.grid_desc(8, mapping=1, flattening=0.1, r_out=1 / 0.6), "7-point"),
                   (W.grid_desc(6, 8, 16), "power of two")):
        with pytest.raises(lib.MGError) as e:
            _handle(lib, g, 1)
        assert e.value.status == lib.MG_EINVAL
        assert why in str(e.value)
