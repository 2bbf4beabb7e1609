"""Parity of every CUDA level operation and of whole solves with the FP64 oracle.

All inputs come from ``workloads`` or seeded numpy generators; the GPU side is
called only through the C ABI (``paper_2305_17875_gb300``).  Tolerances:
FP64 kernels agree to 1e-12 of the stencil scale (rounding order only); FP32
kernels to 1e-5 of the scale (single rounding of coefficients and operands,
a few ulps of accumulation); FP16-coefficient kernels to 2e-3 of the scale
(coefficient rounding 2^-11).  The scale of an apply is max_c sum_n |A_cn x_n|.
Solves: relative residual <= tol, and max pointwise error <= 1e-9 of max|x|
against the oracle solution when both run to 1e-12.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, mg as omg

pytestmark = pytest.mark.gpu

GRIDS = {
    "sphere_uniform": W.grid_desc(8, 8, 16),
    "sphere_stretched_ragged": W.grid_desc(12, 10, 24, stretch=2.0),
    "oblate": W.grid_desc(8, 8, 16, r_out=1 / 0.6, mapping=1, flattening=0.1),
    "triaxial_stretched": W.grid_desc(8, 12, 16, mapping=2, flattening=0.1, e2=0.05, stretch=1.5),
}


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def to_dev(a, dtype):
    torch, dev = torch_dev()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64).ravel()


def stencil_of(g):
    return 7 if g["mapping"] == 0 else 19


def make(lib, g, prec, **opts):
    h = lib.mg_setup(g, dict(precision=prec, **opts))
    hier, fm = omg.setup(g, stencil_of(g), policy=opts.get("coarsen", 0),
                         max_levels=opts.get("max_levels", 16), coarse_max=opts.get("coarse_max", 512))
    return h, hier, fm


def vtype(prec):
    import torch
    return torch.float64 if prec == 0 else torch.float32


TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3}


# ------------------------------------------------------------------ hierarchy / metric
@pytest.mark.parametrize("name", list(GRIDS))
def test_hierarchy_and_face_metric_match_oracle(lib, name):
    torch, dev = torch_dev()
    g = GRIDS[name]
    h, hier, fm = make(lib, g, 0, coarse_max=32)
    info = lib.mg_get_level_info(h, 0)
    assert info["levels"] == len(hier.levels)
    for l, lv in enumerate(hier.levels):
        li = lib.mg_get_level_info(h, l)
        assert (li["nr"], li["nth"], li["nph"]) == lv.shape
        if lv.factors:
            assert (li["cz"], li["ce"], li["cx"]) == lv.factors
        nr, nth, nph = lv.shape
        # oracle face rows -> "lower face of each cell" layout, walls zero
        G0 = lv.fm["G0"][:, :nth, :, :].copy()
        G0[:, 0] = 0
        G1 = lv.fm["G1"][:nr].copy()
        G1[0] = 0
        G2 = lv.fm["G2"]
        rows = [G0, G1, G2]
        buf = torch.empty(lv.n, dtype=torch.float64, device=dev)
        for d in range(3):
            for q in range(3):
                if stencil_of(g) == 7 and q != d:
                    continue
                lib.mg_get_metric(h, l, 3 * d + q, buf)
                ref = rows[d][..., q].ravel()
                scale = np.abs(rows[d][..., d]).max()
                np.testing.assert_allclose(to_np(buf), ref, rtol=0, atol=1e-12 * scale,
                                           err_msg=f"level {l} G[{d}][{q}]")
    lib.mg_get_metric(h, 0, 9, buf := torch.empty(grid.shell(g).n, dtype=torch.float64, device=dev))
    np.testing.assert_allclose(to_np(buf), fm["J"].ravel(), rtol=1e-12)


# ------------------------------------------------------------------ level operations
def _scale(A, x):
    return float((abs(A) @ np.abs(x)).max())


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(GRIDS))
def test_apply_matches_oracle(lib, name, prec):
    g = GRIDS[name]
    h, hier, fm = make(lib, g, prec, coarse_max=32)
    rng = np.random.default_rng(10)
    for l, lv in enumerate(hier.levels):
        x = rng.standard_normal(lv.n)
        xd = to_dev(x, vtype(prec))
        yd = to_dev(np.zeros(lv.n), vtype(prec))
        lib.mg_apply(h, l, prec, xd, yd)
        ref = lv.A @ to_np(xd)
        np.testing.assert_allclose(to_np(yd), ref, rtol=0, atol=TOL[prec] * _scale(lv.A, x),
                                   err_msg=f"level {l}")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", list(GRIDS))
def test_smoother_matches_oracle(lib, name, kind, prec):
    g = GRIDS[name]
    h, hier, fm = make(lib, g, prec, coarse_max=32)
    rng = np.random.default_rng(11)
    for l, lv in enumerate(hier.levels[:2]):
        x0 = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        xd, bd = to_dev(x0, vtype(prec)), to_dev(b, vtype(prec))
        lib.mg_smooth(h, l, prec, xd, bd, 2, kind)
        ref = omg.smooth(lv, to_np(to_dev(x0, vtype(prec))), to_np(bd), 2, kind)
        tol = 1e-12 if prec == 0 else 1e-5
        np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max(),
                                   err_msg=f"level {l}")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(GRIDS))
def test_restriction_and_prolongation_match_oracle(lib, name, prec):
    g = GRIDS[name]
    h, hier, fm = make(lib, g, prec, coarse_max=32)
    rng = np.random.default_rng(12)
    for l, lv in enumerate(hier.levels[:-1]):
        R, P = hier.transfers[l]
        nxt = hier.levels[l + 1]
        x = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        xd, bd = to_dev(x, vtype(prec)), to_dev(b, vtype(prec))
        rc = to_dev(np.zeros(nxt.n), vtype(prec))
        lib.mg_restrict_residual(h, l, prec, xd, bd, rc)
        xx, bb = to_np(xd), to_np(bd)
        ref = R @ (bb - lv.A @ xx)
        sc = float((R @ (np.abs(bb) + abs(lv.A) @ np.abs(xx))).max())
        np.testing.assert_allclose(to_np(rc), ref, rtol=0, atol=TOL[prec] * sc)
        ec = rng.standard_normal(nxt.n)
        ecd = to_dev(ec, vtype(prec))
        lib.mg_prolong_add(h, l, prec, ecd, xd)
        ref = xx + P @ to_np(ecd)
        np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=(1e-15 if prec == 0 else 1e-6) * 4)


@pytest.mark.parametrize("name", ["sphere_uniform", "triaxial_stretched"])
def test_coarse_solve_matches_oracle(lib, name):
    g = GRIDS[name]
    h, hier, fm = make(lib, g, 0, coarse_max=64)
    lv = hier.levels[-1]
    r = np.random.default_rng(13).standard_normal(lv.n)
    e = to_dev(np.zeros(lv.n), vtype(0))
    lib.mg_coarse_solve(h, 0, to_dev(r, vtype(0)), e)
    ref = omg.coarse_solve(lv, r)
    np.testing.assert_allclose(to_np(e), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("tail", [False, True])
@pytest.mark.parametrize("name", list(GRIDS))
def test_fp64_vcycle_matches_oracle(lib, name, tail, monkeypatch):
    if tail:
        monkeypatch.setenv("MG_TAIL", "1")
    g = GRIDS[name]
    h, hier, fm = make(lib, g, 0, coarse_max=32)
    rng = np.random.default_rng(14)
    n = grid.shell(g).n
    x0 = rng.standard_normal(n)
    b, _ = omg.prepare_rhs(fm["J"], rng.standard_normal(n))
    xd, bd = to_dev(x0, vtype(0)), to_dev(b, vtype(0))
    lib.mg_vcycle(h, 0, xd, bd)
    ref = hier.vcycle(0, x0, b)
    np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


# ------------------------------------------------------------------ batched iterates
ITER_GRIDS = {
    # nph % 4 == 0: four-cell groups on every level down to nph = 4
    "sphere_groups": W.grid_desc(8, 8, 16),
    # nph % 4 == 2: scalar forms
    "sphere_stretched_nph18": W.grid_desc(6, 10, 18, stretch=2.0),
    "triaxial_stretched": GRIDS["triaxial_stretched"],
    # the smallest longitude ring (nph = 4; the coarse levels reach nph = 2)
    "sphere_nph4": W.grid_desc(6, 4, 4),
    "triaxial_nph4": W.grid_desc(4, 4, 4, mapping=2, flattening=0.1, e2=0.05),
    # 19 points: odd colatitude count (rows of one parity one longer), and
    # a longitude count that is not a multiple of 4 (scalar forms)
    "triaxial_odd_nth": W.grid_desc(6, 9, 12, mapping=2, flattening=0.1, e2=0.05),
    "oblate_nph10": W.grid_desc(4, 6, 10, r_out=1 / 0.6, mapping=1, flattening=0.1),
}


@pytest.mark.parametrize("iters", [1, 3])
@pytest.mark.parametrize("name", list(ITER_GRIDS))
def test_fp64_batched_iterates_match_oracle(lib, name, iters):
    """Plain FP64 multigrid through the batched engine: the iterate after k
    V-cycles and the residual history (assembled FP64 rows) against the
    oracle's V-cycles on the same right side."""
    torch, dev = torch_dev()
    g = ITER_GRIDS[name]
    n = grid.shell(g).n
    f = np.random.default_rng(21).standard_normal(n)
    h, hier, fm = make(lib, g, 0, coarse_max=16, max_iters=iters)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-300, allow=(lib.MG_ENOCONV,))
    xo, info = omg.solve(g, f, tol=1e-300, hier=hier, fm=fm, max_iters=iters)
    assert rep["iters"] == info["iters"] == iters
    np.testing.assert_allclose(to_np(xd), xo, rtol=0, atol=1e-11 * np.abs(xo).max())
    # FP64 evaluation of b - A x rounds at about eps * cond(A) of ||b||:
    # an absolute floor in relative-residual units beside the relative check
    np.testing.assert_allclose(rep["res_hist"], info["hist"], rtol=1e-9, atol=1e-13)


# ------------------------------------------------------------------ solves
SOLVES = [
    ("single_sphere_32", 1, 0, dict(max_levels=4, coarsen=1)),
    ("single_sphere_32", 1, 1, {}),
    ("single_sphere_128", 4, 0, {}),
    ("single_sphere_128", 4, 1, {}),
    ("single_oblate_256", 8, 1, {}),
    ("single_oblate_256", 8, 2, {}),
    # the 256 x 256 x 512 oblate shell at a quarter of its size (64 x 64 x 128):
    # a deeper hierarchy and the four-cell group paths at 524,288 cells
    ("single_oblate_256", 4, 1, {}),
    ("single_oblate_256", 4, 2, {}),
]

_ORACLE = {}


def _oracle_problem(wl, scale, opts):
    """The oracle's hierarchy, right side and solution to 1e-12 for one
    workload (FP64: shared by every precision and schedule of the GPU side)."""
    key = (wl, scale, tuple(sorted(opts.items())))
    if key not in _ORACLE:
        w = W.single(wl, scale)
        g, f = w["grid"], w["f"]
        hier, fm = omg.setup(g, stencil_of(g), policy=opts.get("coarsen", 0),
                             max_levels=opts.get("max_levels", 16))
        b, mean = omg.prepare_rhs(fm["J"], f)
        xo, info = omg.solve(g, f.ravel(), tol=1e-12, hier=hier, fm=fm, max_iters=400)
        _ORACLE[key] = (hier, fm, b, mean, xo, info)
    return _ORACLE[key]


@pytest.mark.parametrize("path", ["default", "tail", "no_graph"])
@pytest.mark.parametrize("wl,scale,prec,opts", SOLVES)
def test_solve_matches_oracle(lib, wl, scale, prec, opts, path, monkeypatch):
    if path == "tail":
        monkeypatch.setenv("MG_TAIL", "1")
    elif path == "no_graph":
        monkeypatch.setenv("MG_NO_GRAPH", "1")
    torch, dev = torch_dev()
    w = W.single(wl, scale)
    g, f = w["grid"], w["f"]
    h = lib.mg_setup(g, dict(precision=prec, max_iters=200, **opts))
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-10)
    assert rep["rel_res"] <= 1e-10 and rep["status"] == "MG_OK"
    # independent residual check with the oracle's operator
    hier, fm, b, mean, xo, info = _oracle_problem(wl, scale, opts)
    x = to_np(xd)
    assert abs(rep["removed_mean"] - mean) <= 1e-12 * max(1.0, abs(mean))
    rel = np.linalg.norm(b - hier.levels[0].A @ x) / np.linalg.norm(b)
    assert rel <= 1.05e-10
    assert abs((fm["J"].ravel() * x).sum()) <= 1e-12 * np.abs(fm["J"].ravel() * x).sum()
    # error against the oracle solution, both to 1e-12
    xd.zero_()
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    assert info["converged"]
    err = np.abs(to_np(xd) - xo).max() / np.abs(xo).max()
    assert err <= 1e-9, err


@pytest.mark.parametrize("wl,scale,prec", [("single_sphere_128", 4, 1), ("single_sphere_128", 4, 0),
                                             ("single_oblate_256", 8, 1), ("single_sphere_32", 1, 2)])
def test_schedules_give_bitwise_identical_solves(lib, wl, scale, prec, monkeypatch):
    """The coarse tail, the one-pass sweeps (several tile shapes) and the
    per-level launches share the per-cell arithmetic, so every schedule gives
    the same bits."""
    torch, dev = torch_dev()
    w = W.single(wl, scale)
    fd = to_dev(w["f"], torch.float64)
    out = {}
    for name, env, tune in [("default", {}, 0), ("tuned", {}, 1), ("tuned_again", {}, 1), ("cached", {}, 2),
                            ("tail", {"MG_TAIL": "1", "MG_TAIL_CELLS": "8192"}, 1),
                            ("tail_big", {"MG_TAIL": "1", "MG_TAIL_CELLS": "65536", "MG_TAIL_CLUSTER": "4"}, 1),
                            ("tail_global", {"MG_TAIL": "1", "MG_TAIL_CELLS": "8192", "MG_TAIL_GLOBAL": "1"}, 1),
                            ("tail_big_global", {"MG_TAIL": "1", "MG_TAIL_CELLS": "65536", "MG_TAIL_CLUSTER": "4",
                                                 "MG_TAIL_GLOBAL": "1"}, 1),
                            ("fused", {"MG_FUSED_RB": "1"}, 1),
                            ("fused_narrow", {"MG_FUSED_RB": "1", "MG_TILE": "256,3,32"}, 1),
                            ("fused_tail", {"MG_FUSED_RB": "1", "MG_TILE": "1024,2,256", "MG_TAIL": "1"}, 1),
                            ("no_graph", {"MG_NO_GRAPH": "1"}, 0)]:
        for k in ("MG_TAIL", "MG_TAIL_CELLS", "MG_TAIL_CLUSTER", "MG_FUSED_RB", "MG_NO_GRAPH", "MG_TILE",
                  "MG_TAIL_GLOBAL"):
            monkeypatch.delenv(k, raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        h = lib.mg_setup(w["grid"], dict(precision=prec, autotune=tune))
        sc = lib.mg_get_schedule(h)
        if env.get("MG_TAIL") or env.get("MG_FUSED_RB"):
            assert sc["source"] == 3
        elif tune:
            assert sc["source"] in (1, 2) and sc["ms_per_iteration"] > 0
            assert sc["blocks_per_sm"] in (4, 8, 16, 32)
        else:
            assert sc["source"] == 0 and sc["blocks_per_sm"] == 16 and sc["tail_level"] == 0
        if name in ("tuned_again", "cached"):
            assert sc["source"] == 2           # same hierarchy shape: from the process cache
        if name.endswith("global"):
            assert sc["tail_smem_bytes"] == 0, name
        elif name == "tail":
            # a small tail lives in the cluster's shared memory (the big one
            # falls back to global memory where it does not fit)
            assert sc["tail_level"] > 0 and sc["tail_smem_bytes"] > 0, name
        xd = torch.zeros_like(fd)
        rep = lib.mg_solve(h, fd, xd, tol=1e-10)
        out[name] = (to_np(xd), rep["iters"])
        h.close()
    for name, (x, it) in out.items():
        assert it == out["default"][1], name
        assert np.array_equal(x, out["default"][0]), name


def test_cached_schedules_without_timing(lib):
    """autotune = 2 (the serve loop's set-up) times nothing: the default
    schedule for a shape not tuned yet, the tuned one once a set-up with
    autotune = 1 has cached it."""
    g = W.grid_desc(12, 10, 24, stretch=1.5)
    sc0 = lib.mg_get_schedule(lib.mg_setup(g, dict(precision=1, autotune=2)))
    assert sc0["source"] == 0 and sc0["candidates"] == 0
    tuned = lib.mg_get_schedule(lib.mg_setup(g, dict(precision=1, autotune=1)))
    assert tuned["source"] == 1 and tuned["candidates"] > 1
    again = lib.mg_get_schedule(lib.mg_setup(g, dict(precision=1, autotune=2)))
    assert again["source"] == 2
    for k in ("blocks_per_sm", "tail_level", "one_pass_tiles", "tile0"):
        assert again[k] == tuned[k], k


def test_solve_warm_start_and_host_buffers(lib):
    torch, dev = torch_dev()
    w = W.single("single_sphere_128", 4)
    g, f = w["grid"], w["f"]
    h = lib.mg_setup(g, dict(precision=1))
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    r1 = lib.mg_solve(h, fd, xd, tol=1e-10)
    r2 = lib.mg_solve(h, fd, xd, tol=1e-10)          # warm start: already converged
    assert r2["iters"] <= 1
    xh = np.zeros_like(f)
    r3 = lib.mg_solve_host(h, f, xh, tol=1e-10)
    assert r3["iters"] == r1["iters"]
    np.testing.assert_allclose(xh.ravel(), to_np(xd), atol=1e-9 * np.abs(xh).max())


@pytest.mark.parametrize("loop", ["device", "host", "events"])
@pytest.mark.parametrize("wl,scale,prec", [("single_sphere_128", 4, 1), ("single_oblate_256", 8, 2)])
def test_kernel_clocks_cover_every_launch_and_change_nothing(lib, wl, scale, prec, loop, monkeypatch):
    """Kernel timing on: the solve's iterates are bitwise those of an untimed
    solve; every launch but the clock bookkeeping lands in exactly one slot,
    with a positive span; the spans and the gaps between them add up to no
    more than the solve's wall time.  Bookkeeping kernels: with the loop on
    the host, a clock reset per outer iteration and one each for the
    prologue and the epilogue; with the loop on the device, a stop test and a
    clock accumulation per iteration, and three resets.  "events": CUDA
    events around eager launches instead of clocks (no bookkeeping kernels,
    no gap slot)."""
    import time
    torch, dev = torch_dev()
    if loop == "host":
        monkeypatch.setenv("MG_HOST_LOOP", "1")
    else:
        monkeypatch.delenv("MG_HOST_LOOP", raising=False)
    w = W.single(wl, scale)
    h = lib.mg_setup(w["grid"], dict(precision=prec))
    fd = to_dev(w["f"], torch.float64)
    x0 = torch.zeros_like(fd)
    r0 = lib.mg_solve(h, fd, x0, tol=1e-10)
    mode = 2 if loop == "events" else 1
    lib.mg_profile_enable(h, mode)
    for rep in range(2):             # the second solve replays the clocked graph
        x1 = torch.zeros_like(fd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r1 = lib.mg_solve(h, fd, x1, tol=1e-10)
        torch.cuda.synchronize()
        wall_ms = (time.perf_counter() - t0) * 1e3
        slots = [lib.mg_profile_read(h, s) for s in range(lib.PROF_SLOTS)]
        lib.mg_profile_enable(h, mode)           # resets the accumulators
        assert r1["iters"] == r0["iters"]
        assert torch.equal(x1, x0)
        n = sum(k for s, (_, k) in enumerate(slots) if s != lib.PROF_GAPS)
        it = r1["iters"]
        book = {"host": it + 2, "device": 2 * it + 3, "events": 0}[loop]
        assert n == r1["launches"] - book
        ms = sum(t for t, _ in slots)
        assert 0 < ms <= wall_ms
        assert all(t > 0 for s, (t, k) in enumerate(slots) if k and s != lib.PROF_GAPS)
        assert slots[lib.PROF_GAPS][0] >= 0
        if loop == "events":
            assert slots[lib.PROF_GAPS][1] == 0
    lib.mg_profile_enable(h, False)
    x2 = torch.zeros_like(fd)
    r2 = lib.mg_solve(h, fd, x2, tol=1e-10)
    assert r2["launches"] == r0["launches"] and torch.equal(x2, x0)
    # untimed, the device loop's stop test is a kernel of each iteration
    assert r0["launches"] == n + (0 if loop == "host" else it)


def test_nan_rhs_is_reported(lib):
    torch, dev = torch_dev()
    g = W.grid_desc(8)
    h = lib.mg_setup(g)
    f = np.zeros((8, 8, 16))
    f[3, 3, 3] = np.nan
    with pytest.raises(lib.MGError) as e:
        lib.mg_solve(h, to_dev(f, torch.float64), to_dev(np.zeros_like(f), torch.float64))
    assert e.value.status == lib.MG_ENAN


def test_max_iters_reports_noconv(lib):
    torch, dev = torch_dev()
    w = W.single("single_sphere_128", 4)
    h = lib.mg_setup(w["grid"], dict(max_iters=2))
    fd = to_dev(w["f"], torch.float64)
    rep = lib.mg_solve(h, fd, torch.zeros_like(fd), tol=1e-10, allow=(lib.MG_ENOCONV,))
    assert rep["status"] == "MG_ENOCONV" and rep["iters"] == 2


FUSED_GRIDS = {
    # with MG_FUSED_RB=1 every level a tile fits takes the one-pass sweep;
    # ragged last tiles in colatitude and radius
    "fused_ragged": W.grid_desc(6, 20, 96),
    "fused_stretched": W.grid_desc(12, 20, 72, stretch=2.0),
    "fused_exact_tiles": W.grid_desc(8, 16, 64),
    "fused_many_tiles": W.grid_desc(16, 24, 192, stretch=1.0),
}


@pytest.mark.parametrize("path", ["one_pass", "colour_passes"])
@pytest.mark.parametrize("sweeps", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(FUSED_GRIDS))
def test_fused_red_black_sweep_matches_oracle(lib, name, prec, sweeps, path, monkeypatch):
    if path == "one_pass":
        monkeypatch.setenv("MG_FUSED_RB", "1")
    g = FUSED_GRIDS[name]
    h = lib.mg_setup(g, dict(precision=prec))
    fm = grid.face_metrics(grid.shell(g))
    lv = omg.make_level(grid.shell(g).shape, fm, 7)
    rng = np.random.default_rng(15)
    x0 = rng.standard_normal(lv.n)
    b = rng.standard_normal(lv.n) * np.abs(lv.D)
    xd, bd = to_dev(x0, vtype(prec)), to_dev(b, vtype(prec))
    lib.mg_smooth(h, 0, prec, xd, bd, sweeps, 0)
    ref = omg.smooth(lv, to_np(to_dev(x0, vtype(prec))), to_np(bd), sweeps, omg.GS)
    tol = {0: 1e-12, 1: 1e-5, 2: 3e-3}[prec]
    np.testing.assert_allclose(to_np(xd), ref, rtol=0, atol=tol * np.abs(ref).max())


# ------------------------------------------------------------------ analytic metric option
@pytest.mark.parametrize("name", ["sphere_stretched_ragged", "triaxial_stretched"])
def test_analytic_metric_matches_oracle(lib, name):
    """metric = analytic: the face rows and cell volumes against the oracle's
    exact-derivative metric (FP64, 1e-12), and a solve against the oracle's
    solve on that metric."""
    torch, dev = torch_dev()
    g = GRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics_analytic(sh)
    h = lib.mg_setup(g, dict(precision=1, metric=1))
    nr, nth, nph = sh.shape
    G0 = fm["G0"][:, :nth, :, :].copy()
    G0[:, 0] = 0
    G1 = fm["G1"][:nr].copy()
    G1[0] = 0
    rows = [G0, G1, fm["G2"]]
    buf = torch.empty(sh.n, dtype=torch.float64, device=dev)
    for d in range(3):
        for q in range(3):
            if stencil_of(g) == 7 and q != d:
                continue
            lib.mg_get_metric(h, 0, 3 * d + q, buf)
            np.testing.assert_allclose(to_np(buf), rows[d][..., q].ravel(), rtol=0,
                                       atol=1e-12 * np.abs(rows[d][..., d]).max())
    lib.mg_get_metric(h, 0, 9, buf)
    np.testing.assert_allclose(to_np(buf), fm["J"].ravel(), rtol=1e-12)
    f = W.rhs_modes(g, seed=3)
    fd = to_dev(f, torch.float64)
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-12)
    xo, info = omg.solve(g, f.ravel(), tol=1e-12, fm=fm, max_iters=400)
    assert rep["rel_res"] <= 1e-12 and info["converged"]
    err = np.abs(to_np(xd) - xo).max() / np.abs(xo).max()
    assert err <= 1e-9, err
    # the steps around the solve need the discrete metric
    with pytest.raises(lib.MGError):
        lib.mg_pc_rhs(h, torch.zeros(9 * sh.n, dtype=torch.float64, device=dev), buf)


def test_setup_allocation_failures_release_everything(lib, monkeypatch):
    """A set-up whose n-th device allocation fails returns MG_ENOMEM and gives
    back every byte it took, for every n (fault injected on the host)."""
    import gc
    import torch
    g = GRIDS["triaxial_stretched"]
    gc.collect()
    torch.cuda.synchronize()
    base = lib.mg_device_bytes_in_use(0)
    n, failures = 0, 0
    while True:
        monkeypatch.setenv("MG_TEST_FAIL_ALLOC_AFTER", str(n))
        try:
            h = lib.mg_setup(g, dict(precision=1, autotune=0))
        except lib.MGError as e:
            assert e.status == lib.MG_ENOMEM
            torch.cuda.synchronize()          # the frees are stream ordered
            assert lib.mg_device_bytes_in_use(0) == base
            failures += 1
            n += 1
            continue
        h.close()
        break
    monkeypatch.delenv("MG_TEST_FAIL_ALLOC_AFTER")
    gc.collect()
    torch.cuda.synchronize()
    assert failures > 10 and lib.mg_device_bytes_in_use(0) == base


def test_axisymmetric_operator_matches_the_full_19_point_one(lib, monkeypatch):
    """The oblate shell's operator without the longitude cross terms (zero to
    rounding) and with all nine components (MG_FULL19) give the same solve to
    rounding, and the component arrays the former drops read back as zero."""
    import torch
    g = GRIDS["oblate"]
    n = grid.shell(g).n
    f = W.rhs_modes(g, seed=12)
    xs = {}
    for full in (False, True):
        if full:
            monkeypatch.setenv("MG_FULL19", "1")
        h = lib.mg_setup(g, dict(precision=0))
        fd = to_dev(f, torch.float64)
        xd = torch.zeros_like(fd)
        lib.mg_solve(h, fd, xd, tol=1e-13)
        xs[full] = to_np(xd)
        buf = torch.empty(n, dtype=torch.float64, device="cuda")
        lib.mg_get_metric(h, 0, 5, buf)          # eta-face row, xi column
        if not full:
            assert not buf.any()
        h.close()
    monkeypatch.delenv("MG_FULL19")
    np.testing.assert_allclose(xs[False], xs[True], rtol=0, atol=1e-11 * np.abs(xs[True]).max())
