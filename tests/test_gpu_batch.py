"""Batched solves: one launch per level operation over many shells.

A shell's result must not depend on its batch companions: the batch of one
(``mg_solve``) and the mixed batch give bitwise identical iterates, reports
and iteration counts; results match the FP64 oracle.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mg as omg

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _mixed_shells():
    """Uneven sizes, sphere (7-point) and oblate / triaxial (19-point), own RHS."""
    gs = [
        W.grid_desc(8, 8, 16),
        W.grid_desc(16, 16, 32, mapping=1, flattening=0.12, r_out=1 / 0.45),
        W.grid_desc(12, 12, 24, stretch=2.0),
        W.grid_desc(24, 24, 48, mapping=1, flattening=0.05, r_out=1 / 0.7),
        W.grid_desc(8, 16, 32, mapping=2, flattening=0.1, e2=0.05),
        W.grid_desc(32, 32, 64, mapping=1, flattening=0.15, r_out=2.5),
    ]
    fs = [W.rhs_modes(g, seed=1000 + s) for s, g in enumerate(gs)]
    tols = [1e-10, 1e-8, 1e-12, 1e-6, 1e-10, 1e-10]
    return gs, fs, tols


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_batch_result_equals_lone_solve_bitwise(lib, prec):
    import torch
    gs, fs, tols = _mixed_shells()
    hs = [lib.mg_setup(g, dict(precision=prec)) for g in gs]
    fd = [_dev(f) for f in fs]
    alone = []
    for h, f, t in zip(hs, fd, tols):
        x = torch.zeros_like(f)
        rep = lib.mg_solve(h, f, x, tol=t)
        alone.append((x.cpu().numpy(), rep))
    xs = [torch.zeros_like(f) for f in fd]
    reps = lib.mg_solve_batch(hs, fd, xs, tols)
    for s in range(len(gs)):
        xa, ra = alone[s]
        assert reps[s]["iters"] == ra["iters"], s
        assert reps[s]["rel_res"] == ra["rel_res"], s
        assert reps[s]["rel_res"] <= tols[s]
        assert np.array_equal(xs[s].cpu().numpy(), xa), s
    # the batch is reproducible run to run, and a different order gives the same shells
    order = list(reversed(range(len(gs))))
    xs2 = [torch.zeros_like(fd[s]) for s in order]
    reps2 = lib.mg_solve_batch([hs[s] for s in order], [fd[s] for s in order], xs2, [tols[s] for s in order])
    for q, s in enumerate(order):
        assert np.array_equal(xs2[q].cpu().numpy(), alone[s][0])
        assert reps2[q]["iters"] == alone[s][1]["iters"]


def test_batch_matches_oracle(lib):
    import torch
    gs, fs, _ = _mixed_shells()
    hs = [lib.mg_setup(g, dict(precision=1)) for g in gs]
    fd = [_dev(f) for f in fs]
    xs = [torch.zeros_like(f) for f in fd]
    reps = lib.mg_solve_batch(hs, fd, xs, [1e-12] * len(gs))
    for s, g in enumerate(gs):
        assert reps[s]["status"] == "MG_OK"
        xo, info = omg.solve(g, fs[s].ravel(), tol=1e-12, max_iters=400)
        x = xs[s].cpu().numpy().ravel()
        assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max(), s


def test_batch_of_uneven_shells_converges(lib):
    """The uneven-batch workload (nr in {32, 64, 96, 128}), 16 of its 64 shells."""
    import torch
    items = W.batch_shells(n=16)
    hs = [lib.mg_setup(it["grid"], dict(precision=1)) for it in items]
    fd = [_dev(W.batch_rhs(it)) for it in items]
    xs = [torch.zeros_like(f) for f in fd]
    reps = lib.mg_solve_batch(hs, fd, xs, [1e-10] * len(items))
    for r in reps:
        assert r["status"] == "MG_OK" and r["rel_res"] <= 1e-10
    # one of them checked against a lone solve
    x = torch.zeros_like(fd[3])
    lib.mg_solve(hs[3], fd[3], x, tol=1e-10)
    assert torch.equal(x, xs[3])


def test_batch_argument_errors(lib):
    import torch
    g = W.grid_desc(8)
    h = lib.mg_setup(g)
    f = _dev(W.rhs_modes(g))
    with pytest.raises(lib.MGError):
        lib.mg_solve_batch([h, h], [f, f], [torch.zeros_like(f), torch.zeros_like(f)], [1e-8, 1e-8])
    h64 = lib.mg_setup(g, dict(precision=0))
    with pytest.raises(lib.MGError):
        lib.mg_solve_batch([h, h64], [f, f], [torch.zeros_like(f), torch.zeros_like(f)], [1e-8, 1e-8])


@pytest.mark.parametrize("prec", [1, 2])
def test_device_loop_equals_host_loop(lib, prec, monkeypatch):
    """The outer loop on the device (a graph whose while node repeats the
    iteration and the stop tests) against the same loop driven by the host
    (MG_HOST_LOOP): bitwise the same iterates, counts, residual histories and
    statuses, for a mixed batch with its own tolerances and for a shell that
    stops at max_iters."""
    import torch
    gs, fs, tols = _mixed_shells()
    runs = {}
    for mode in ("device", "host"):
        if mode == "host":
            monkeypatch.setenv("MG_HOST_LOOP", "1")
        else:
            monkeypatch.delenv("MG_HOST_LOOP", raising=False)
        hs = [lib.mg_setup(g, dict(precision=prec)) for g in gs]
        fd = [_dev(f) for f in fs]
        xs = [torch.zeros_like(f) for f in fd]
        reps = lib.mg_solve_batch(hs, fd, xs, tols)
        h2 = lib.mg_setup(gs[3], dict(precision=prec, max_iters=3))
        x2 = torch.zeros_like(fd[3])
        r2 = lib.mg_solve(h2, fd[3], x2, tol=1e-14, allow=(lib.MG_ENOCONV,))
        runs[mode] = ([x.cpu().numpy() for x in xs], reps, x2.cpu().numpy(), r2)
    (xd, rd, x2d, r2d), (xh, rh, x2h, r2h) = runs["device"], runs["host"]
    for s in range(len(gs)):
        for k in ("iters", "status", "rel_res", "res_hist"):
            assert rd[s][k] == rh[s][k], (s, k)
        assert np.array_equal(xd[s], xh[s]), s
    assert r2d["status"] == r2h["status"] == "MG_ENOCONV" and r2d["iters"] == r2h["iters"] == 3
    assert r2d["res_hist"] == r2h["res_hist"] and np.array_equal(x2d, x2h)

