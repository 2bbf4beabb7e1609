"""The full sphere with the shell cut (Sections 3.5 and 3.7) on the GPU
against the oracle: the 7-point operator (the sphere mapping) and the
19-point one (oblate shells, and the sphere with 19 points).

The pole faces carry no flux (zero area), so the 7-point operator, smoothers
and residuals are the walled ones with th0 = 0, th1 = pi; the cut enters the
multigrid through the prolongation, whose colatitude partner for the first
and last coarse rows lies across the pole.  With 19 points the cut also
enters the cross terms: a colatitude difference beyond the first or last row
takes the cell across the pole (same row, longitude + nph/2) instead of the
mirror, and the cells of one colour that couple across the pole are updated
as one step (the oracle's colour update).  Checked: the hierarchy, face rows
and cell volumes, every level operation, FP64 V-cycles (also through the
coarse tail), batched iterates and residual histories, solves against the
oracle's solution, the ADI sub-step and the pressure-correction steps; and
the combinations that are not built are refused.  Tolerances as in the
walled parity tests.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adi, grid, mg as omg, pc

pytestmark = pytest.mark.gpu

SPHERES = {
    "cut_8": W.grid_desc(8, 8, 16, cut=True),
    "cut_stretched_ragged": W.grid_desc(6, 10, 20, stretch=2.0, cut=True),
    "cut_nph8": W.grid_desc(4, 8, 8, cut=True),
}
TOL = {0: 1e-12, 1: 1e-5}


def _torch():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a, dtype):
    torch, dev = _torch()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64).ravel()


def vtype(prec):
    torch, _ = _torch()
    return torch.float64 if prec == 0 else torch.float32


def make(lib, g, prec, **opts):
    h = lib.mg_setup(g, dict(precision=prec, **opts))
    hier, fm = omg.setup(g, 7, policy=opts.get("coarsen", 0), max_levels=opts.get("max_levels", 16),
                         coarse_max=opts.get("coarse_max", 512))
    return h, hier, fm


@pytest.mark.parametrize("name", list(SPHERES))
def test_cut_hierarchy_metric_and_volumes(lib, name):
    torch, dev = _torch()
    g = SPHERES[name]
    h, hier, fm = make(lib, g, 0, coarse_max=32)
    assert hier.levels[0].cut
    assert lib.mg_get_level_info(h, 0)["levels"] == len(hier.levels)
    for l, lv in enumerate(hier.levels):
        li = lib.mg_get_level_info(h, l)
        assert (li["nr"], li["nth"], li["nph"]) == lv.shape
        nr, nth, nph = lv.shape
        G0 = lv.fm["G0"][:, :nth, :, 0].copy()     # lower faces; the north pole face is zero
        G1 = lv.fm["G1"][:nr, :, :, 1].copy()
        G1[0] = 0
        rows = [G0, G1, lv.fm["G2"][..., 2]]
        buf = torch.empty(lv.n, dtype=torch.float64, device=dev)
        for d in range(3):
            lib.mg_get_metric(h, l, 4 * d, buf)
            np.testing.assert_allclose(to_np(buf), rows[d].ravel(), rtol=0, atol=1e-12 * np.abs(rows[d]).max(),
                                       err_msg=f"level {l} G[{d}][{d}]")
    buf = torch.empty(grid.shell(g).n, dtype=torch.float64, device=dev)
    lib.mg_get_metric(h, 0, 9, buf)
    np.testing.assert_allclose(to_np(buf), fm["J"].ravel(), rtol=1e-12)


def _scale(A, x):
    return float((abs(A) @ np.abs(x)).max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(SPHERES))
def test_cut_level_operations(lib, name, prec):
    g = SPHERES[name]
    h, hier, fm = make(lib, g, prec, coarse_max=32)
    rng = np.random.default_rng(31)
    for l, lv in enumerate(hier.levels):
        x = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        xd, yd = to_dev(x, vtype(prec)), to_dev(np.zeros(lv.n), vtype(prec))
        lib.mg_apply(h, l, prec, xd, yd)
        np.testing.assert_allclose(to_np(yd), lv.A @ to_np(xd), rtol=0, atol=TOL[prec] * _scale(lv.A, x),
                                   err_msg=f"apply, level {l}")
        xd, bd = to_dev(x, vtype(prec)), to_dev(b, vtype(prec))
        lib.mg_smooth(h, l, prec, xd, bd, 1, 0)
        ref = omg.smooth(lv, to_np(to_dev(x, vtype(prec))), to_np(bd), 1, omg.GS)
        np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=TOL[prec] * np.abs(ref).max(),
                                   err_msg=f"smooth, level {l}")
        if lv.factors is None:
            continue
        R, P = hier.transfers[l]
        nc = hier.levels[l + 1].n
        ec = rng.standard_normal(nc)
        ecd = to_dev(ec, vtype(prec))
        xd = to_dev(x, vtype(prec))
        xx = to_np(xd)
        lib.mg_prolong_add(h, l, prec, ecd, xd)
        np.testing.assert_allclose(to_np(xd), xx + P @ to_np(ecd), rtol=0,
                                   atol=(1e-15 if prec == 0 else 1e-6) * 4, err_msg=f"prolong, level {l}")


@pytest.mark.parametrize("tail", [False, True])
@pytest.mark.parametrize("name", list(SPHERES))
def test_cut_fp64_vcycle(lib, name, tail, monkeypatch):
    if tail:
        monkeypatch.setenv("MG_TAIL", "1")
    g = SPHERES[name]
    h, hier, fm = make(lib, g, 0, coarse_max=32)
    rng = np.random.default_rng(32)
    n = grid.shell(g).n
    x0 = rng.standard_normal(n)
    b, _ = omg.prepare_rhs(fm["J"], rng.standard_normal(n))
    xd, bd = to_dev(x0, vtype(0)), to_dev(b, vtype(0))
    lib.mg_vcycle(h, 0, xd, bd)
    ref = hier.vcycle(0, x0, b)
    np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("iters", [1, 3])
@pytest.mark.parametrize("name", list(SPHERES))
def test_cut_batched_iterates(lib, name, iters):
    torch, _ = _torch()
    g = SPHERES[name]
    n = grid.shell(g).n
    f = np.random.default_rng(33).standard_normal(n)
    h, hier, fm = make(lib, g, 0, coarse_max=16, max_iters=iters)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
    xo, info = omg.solve(g, f, tol=1e-300, hier=hier, fm=fm, max_iters=iters)
    assert rep["iters"] == info["iters"] == iters
    np.testing.assert_allclose(to_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    np.testing.assert_allclose(rep["res_hist"], info["hist"], rtol=1e-9, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_cut_solve_matches_oracle(lib, prec):
    torch, _ = _torch()
    g = W.grid_desc(16, 16, 32, stretch=1.0, cut=True)
    f = W.rhs_modes(g, seed=4)
    h, hier, fm = make(lib, g, prec)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    xo, info = omg.solve(g, f.ravel(), tol=1e-12, hier=hier, fm=fm, max_iters=400)
    assert rep["rel_res"] <= 1e-12 and info["converged"]
    assert np.abs(to_np(xd) - xo).max() <= 1e-9 * np.abs(xo).max()


def test_cut_refuses_what_is_not_built(lib):
    oblate = W.grid_desc(8, 8, 16, mapping=1, flattening=0.1, r_out=1 / 0.6, cut=True)
    for g, o, why in ((W.grid_desc(8, 8, 16, mapping=2, flattening=0.1, e2=0.05, cut=True), {}, "axisymmetric"),
                      (oblate, dict(smoother=2), "point smoothers"),
                      (oblate, dict(smoother=5), "point smoothers")):
        with pytest.raises(lib.MGError) as e:
            lib.mg_setup(g, dict(precision=1, **o))
        assert why in str(e.value)
    bad = W.grid_desc(8, 8, 16)
    bad["cut"] = 1                       # cut with a sector's colatitude range
    with pytest.raises(lib.MGError):
        lib.mg_setup(bad, dict(precision=1))


def _dev64(a):
    torch, dev = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


@pytest.mark.parametrize("name", ["cut_8", "cut_stretched_ragged"])
def test_cut_adi_substep(lib, name):
    """Colatitude wall values are ignored at the poles (zero-area faces): the
    sub-step equals the oracle's with the pole faces' G = 0."""
    torch, dev = _torch()
    g = SPHERES[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh)
    h = lib.mg_setup(g, dict(precision=1))
    rng = np.random.default_rng(34)
    un = rng.standard_normal(sh.shape)
    src = 0.1 * rng.standard_normal(sh.shape) * fm["J"]
    kappa = 1.0 / (np.abs(fm["G1"][..., 1]).max() / fm["J"].min())
    u = torch.empty(sh.shape, dtype=torch.float64, device=dev)
    wg = dict(radius=1, colatitude=1, v_r_in=0.3, v_r_out=-0.2, v_th0=0.5, v_th1=0.1)
    lib.mg_adi_substep(h, kappa, _dev64(un), u, src=_dev64(src), walls=wg)
    want = adi.substep(sh, fm, un, kappa, adi.walls((adi.VALUE, 0.3, -0.2), (adi.VALUE, 0.5, 0.1)), src=src)
    np.testing.assert_allclose(u.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_cut_pressure_correction_steps(lib):
    torch, dev = _torch()
    from test_gpu_pc import to_gpu_layout, from_gpu_layout
    g = SPHERES["cut_8"]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    h = lib.mg_setup(g, dict(precision=0))
    rng = np.random.default_rng(35)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    x = rng.standard_normal(sh.n)
    ud = torch.from_numpy(to_gpu_layout(sh, u)).to(dev)
    fd = torch.empty(sh.n, dtype=torch.float64, device=dev)
    lib.mg_pc_rhs(h, ud, fd)
    ref = pc.rhs(sh, fm, u).ravel()
    np.testing.assert_allclose(fd.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    lib.mg_pc_correct(h, torch.from_numpy(x).to(dev), ud)
    got = from_gpu_layout(sh, ud.cpu().numpy(), u)
    want = pc.project(sh, fm, x, u, 7)
    for d in range(3):
        np.testing.assert_allclose(got[d], want[d], rtol=0, atol=1e-12 * np.abs(want[d]).max())


# ---------------------------------------------------------------- 19 points
# nph / 2 even: cells of one colour couple across the pole (the colour pass
# reads their values from the copy of the pole rows); nph / 2 = 7: they do not.
SPHERES19 = {
    "oblate_cut_8": W.grid_desc(8, 8, 16, mapping=1, flattening=0.1, r_out=1 / 0.6, cut=True),
    "oblate_cut_ragged": W.grid_desc(6, 10, 20, mapping=1, flattening=0.1, r_out=1 / 0.6, stretch=1.5,
                                     cut=True),
    "oblate_cut_half7": W.grid_desc(4, 8, 14, mapping=1, flattening=0.1, r_out=1 / 0.6, cut=True),
    "sphere19_cut": W.grid_desc(6, 8, 16, stretch=1.0, cut=True),
}


def make19(lib, g, prec, **opts):
    h = lib.mg_setup(g, dict(precision=prec, stencil=19, **opts))
    hier, fm = omg.setup(g, 19, policy=opts.get("coarsen", 0), max_levels=opts.get("max_levels", 16),
                         coarse_max=opts.get("coarse_max", 512))
    return h, hier, fm


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(SPHERES19))
def test_cut19_level_operations(lib, name, prec):
    """Operator, one and two Gauss-Seidel sweeps, Jacobi, residual and
    restriction, prolongation, on every level."""
    torch, dev = _torch()
    g = SPHERES19[name]
    h, hier, fm = make19(lib, g, prec, coarse_max=32)
    assert lib.mg_get_level_info(h, 0)["levels"] == len(hier.levels)
    rng = np.random.default_rng(41)
    tol = {0: 1e-12, 1: 1e-5, 2: 3e-3}[prec]
    for l, lv in enumerate(hier.levels):
        li = lib.mg_get_level_info(h, l)
        assert (li["nr"], li["nth"], li["nph"]) == lv.shape
        x = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        A = lv.A
        if prec == 2:   # FP16 coefficients: compare with the operator of the FP32 cycle's own arithmetic
            continue
        xd, yd = to_dev(x, vtype(prec)), to_dev(np.zeros(lv.n), vtype(prec))
        lib.mg_apply(h, l, prec, xd, yd)
        np.testing.assert_allclose(to_np(yd), A @ to_np(xd), rtol=0, atol=tol * _scale(A, x),
                                   err_msg=f"apply, level {l}")
        for sweeps in (1, 2):
            xd, bd = to_dev(x, vtype(prec)), to_dev(b, vtype(prec))
            lib.mg_smooth(h, l, prec, xd, bd, sweeps, 0)
            ref = omg.smooth(lv, to_np(to_dev(x, vtype(prec))), to_np(bd), sweeps, omg.GS)
            np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                       err_msg=f"Gauss-Seidel {sweeps}, level {l}")
        xd, bd = to_dev(x, vtype(prec)), to_dev(b, vtype(prec))
        lib.mg_smooth(h, l, prec, xd, bd, 1, 1)
        ref = omg.smooth(lv, to_np(to_dev(x, vtype(prec))), to_np(bd), 1, omg.JACOBI)
        np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                   err_msg=f"Jacobi, level {l}")
        if lv.factors is None:
            continue
        R, P = hier.transfers[l]
        nc = hier.levels[l + 1].n
        xd, bd = to_dev(x, vtype(prec)), to_dev(b, vtype(prec))
        rc = to_dev(np.zeros(nc), vtype(prec))
        lib.mg_restrict_residual(h, l, prec, xd, bd, rc)
        want = R @ (to_np(bd) - A @ to_np(xd))
        np.testing.assert_allclose(to_np(rc), want, rtol=0, atol=tol * 8 * (_scale(A, x) + np.abs(b).max()),
                                   err_msg=f"restriction, level {l}")
        ec = rng.standard_normal(nc)
        ecd, xd = to_dev(ec, vtype(prec)), to_dev(x, vtype(prec))
        xx = to_np(xd)
        lib.mg_prolong_add(h, l, prec, ecd, xd)
        np.testing.assert_allclose(to_np(xd), xx + P @ to_np(ecd), rtol=0,
                                   atol=(1e-15 if prec == 0 else 1e-6) * 4, err_msg=f"prolong, level {l}")


@pytest.mark.parametrize("name", list(SPHERES19))
def test_cut19_fp64_vcycle(lib, name):
    g = SPHERES19[name]
    h, hier, fm = make19(lib, g, 0, coarse_max=32)
    rng = np.random.default_rng(42)
    n = grid.shell(g).n
    x0 = rng.standard_normal(n)
    b, _ = omg.prepare_rhs(fm["J"], rng.standard_normal(n))
    xd, bd = to_dev(x0, vtype(0)), to_dev(b, vtype(0))
    lib.mg_vcycle(h, 0, xd, bd)
    ref = hier.vcycle(0, x0, b)
    np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("iters", [1, 3])
@pytest.mark.parametrize("name", list(SPHERES19))
def test_cut19_batched_iterates(lib, name, iters):
    """Plain FP64 V(2,2) cycles through the batched engine (the outer residual
    from the assembled rows across the pole): iterates and residual histories."""
    torch, _ = _torch()
    g = SPHERES19[name]
    n = grid.shell(g).n
    f = np.random.default_rng(43).standard_normal(n)
    h, hier, fm = make19(lib, g, 0, coarse_max=16, max_iters=iters)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
    xo, info = omg.solve(g, f, tol=1e-300, hier=hier, fm=fm, max_iters=iters, stencil=19)
    assert rep["iters"] == info["iters"] == iters
    np.testing.assert_allclose(to_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    np.testing.assert_allclose(rep["res_hist"][:iters + 1], info["hist"], rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cut19_solve_matches_oracle(lib, prec):
    """An oblate full sphere 16 x 16 x 32 to 1e-12 (FP16 coefficients: the
    refinement reaches the same FP64 solution)."""
    torch, _ = _torch()
    g = W.grid_desc(16, 16, 32, mapping=1, flattening=0.1, r_out=1 / 0.6, stretch=1.0, cut=True)
    f = W.rhs_modes(g, seed=4)
    h, hier, fm = make19(lib, g, prec, max_iters=400)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    xo, info = omg.solve(g, f.ravel(), tol=1e-12, hier=hier, fm=fm, max_iters=400, stencil=19)
    assert rep["rel_res"] <= 1e-12 and info["converged"]
    assert np.abs(to_np(xd) - xo).max() <= 1e-9 * np.abs(xo).max()
    if prec == 0:
        assert rep["iters"] == info["iters"]


def test_cut19_pressure_correction_steps(lib):
    """Right side of Eq. PC_6 and the correction of Eq. PC_7 with the cross
    terms' tangential differences across the pole."""
    torch, dev = _torch()
    from test_gpu_pc import to_gpu_layout, from_gpu_layout
    g = SPHERES19["oblate_cut_8"]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    h = lib.mg_setup(g, dict(precision=0))
    rng = np.random.default_rng(45)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    x = rng.standard_normal(sh.n)
    ud = torch.from_numpy(to_gpu_layout(sh, u)).to(dev)
    fd = torch.empty(sh.n, dtype=torch.float64, device=dev)
    lib.mg_pc_rhs(h, ud, fd)
    ref = pc.rhs(sh, fm, u).ravel()
    np.testing.assert_allclose(fd.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    lib.mg_pc_correct(h, torch.from_numpy(x).to(dev), ud)
    got = from_gpu_layout(sh, ud.cpu().numpy(), u)
    want = pc.project(sh, fm, x, u, 19)
    for d in range(3):
        np.testing.assert_allclose(got[d], want[d], rtol=0, atol=1e-12 * np.abs(want[d]).max())
