"""The serve loop: continuous batching of solve requests.

Requests admitted while others iterate join at the next step; each result is
bitwise the lone mg_solve result for the same grid, options and right side;
admission respects the slot count and the device-memory budget; idle
hierarchies are reused.
"""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _requests(n=10, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        nr = int(rng.choice([8, 12, 16, 24, 32]))
        fl = float(rng.uniform(0.0, 0.15))
        g = W.grid_desc(nr, r_out=2.0, mapping=1 if q % 3 else 0, flattening=fl if q % 3 else 0.0)
        tol = float(rng.choice([1e-6, 1e-8, 1e-10]))
        out.append((g, W.rhs_modes(g, seed=2000 + q), tol))
    return out


def _drain(lib, sv, tickets, shapes, timeout=120.0, order=None):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t, shp in zip(tickets, shapes):
            if t in res:
                continue
            x = np.empty(shp)
            r = lib.mg_serve_poll(sv, t, x)
            if r is not None:
                res[t] = (x, r[0], r[1])
                if order is not None:
                    order.append(t)
        assert time.time() - t0 < timeout, "serve loop did not finish"
        time.sleep(0.002)
    return res


def _lone(lib, g, f, tol, opts=None):
    import torch
    h = lib.mg_setup(g, opts or {})
    fd = torch.from_numpy(f).to("cuda:0")
    x = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, x, tol=tol, allow=(lib.MG_OK, lib.MG_ENOCONV))
    h.close()
    return x.cpu().numpy(), rep


def test_served_results_equal_lone_solves_bitwise(lib):
    reqs = _requests(12)
    sv = lib.mg_serve_create(max_slots=6, setup_threads=3)
    tickets = [lib.mg_serve_submit(sv, g, f, tol) for g, f, tol in reqs]
    res = _drain(lib, sv, tickets, [f.shape for _, f, _ in reqs])
    stats = lib.mg_serve_stats(sv)
    sv.close()
    assert stats["retired"] == len(reqs)
    for t, (g, f, tol) in zip(tickets, reqs):
        x, status, rep = res[t]
        assert status == "MG_OK" and rep["rel_res"] <= tol
        xl, rl = _lone(lib, g, f, tol)
        assert rep["iters"] == rl["iters"]
        assert np.array_equal(x, xl)


def test_admission_respects_slots_and_memory(lib):
    reqs = _requests(8, seed=1)
    g0 = reqs[0][0]
    one = lib.mg_footprint_bytes(g0) + 2 * 8 * g0["nr"] * g0["nth"] * g0["nph"]
    # a budget below two requests of the largest size admits them one or two at a time
    big = max(lib.mg_footprint_bytes(g) + 16 * g["nr"] * g["nth"] * g["nph"] for g, _, _ in reqs)
    sv = lib.mg_serve_create(max_slots=3, setup_threads=2, max_bytes=int(1.5 * big))
    tickets = [lib.mg_serve_submit(sv, g, f, tol) for g, f, tol in reqs]
    peak_active, peak_bytes = 0, 0
    t0 = time.time()
    while lib.mg_serve_stats(sv)["retired"] < len(reqs):
        s = lib.mg_serve_stats(sv)
        peak_active = max(peak_active, s["active"])
        peak_bytes = max(peak_bytes, s["bytes_reserved"])
        assert time.time() - t0 < 120
        time.sleep(0.001)
    res = _drain(lib, sv, tickets, [f.shape for _, f, _ in reqs])
    sv.close()
    assert peak_active <= 3
    assert peak_bytes <= max(int(1.5 * big), one)
    assert all(v[1] == "MG_OK" for v in res.values())


def test_arrivals_join_while_others_iterate(lib):
    """Requests submitted while a long solve iterates join it: they finish
    first, share its steps, and still give the lone-solve results bitwise."""
    g_big = W.grid_desc(48, stretch=2.0)
    f_big = W.rhs_modes(g_big, seed=5)
    sv = lib.mg_serve_create(max_slots=8)
    # tol 0 never converges: the request iterates until max_iters
    t_big = lib.mg_serve_submit(sv, g_big, f_big, 0.0, opts=dict(max_iters=3000))
    t0 = time.time()
    while lib.mg_serve_stats(sv)["steps"] < 3:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    small = _requests(5, seed=3)
    tickets = [lib.mg_serve_submit(sv, g, f, 1e-8) for g, f, _ in small]
    order = []
    res = _drain(lib, sv, tickets + [t_big], [f.shape for _, f, _ in small] + [f_big.shape], order=order)
    stats = lib.mg_serve_stats(sv)
    sv.close()
    assert res[t_big][1] == "MG_ENOCONV" and res[t_big][2]["iters"] == 3000
    assert order[-1] == t_big
    assert stats["steps"] < sum(r[2]["iters"] for r in res.values())   # steps were shared
    for t, (g, f, _) in zip(tickets, small):
        assert res[t][1] == "MG_OK"
        xl, rl = _lone(lib, g, f, 1e-8)
        assert res[t][2]["iters"] == rl["iters"]
        assert np.array_equal(res[t][0], xl)


def test_hierarchy_reuse(lib):
    g = W.grid_desc(16, mapping=1, flattening=0.07)
    f1, f2 = W.rhs_modes(g, seed=1), W.rhs_modes(g, seed=2)
    sv = lib.mg_serve_create(max_slots=2)
    t1 = lib.mg_serve_submit(sv, g, f1, 1e-10)
    r1 = _drain(lib, sv, [t1], [f1.shape])
    t2 = lib.mg_serve_submit(sv, g, f2, 1e-10)
    r2 = _drain(lib, sv, [t2], [f2.shape])
    stats = lib.mg_serve_stats(sv)
    sv.close()
    assert stats["cache_hits"] >= 1
    xl, _ = _lone(lib, g, f2, 1e-10)
    assert np.array_equal(r2[t2][0], xl)


def test_served_line_smoother_requests(lib):
    """Requests asking for the radial-line smoother are served like any other
    and give the lone-solve bits."""
    g = W.grid_desc(16, 16, 32, r_out=1.05, stretch=2.0)
    f = W.rhs_modes(g, seed=9)
    sv = lib.mg_serve_create(max_slots=2)
    t = lib.mg_serve_submit(sv, g, f, 1e-10, opts=dict(smoother=2))
    r = _drain(lib, sv, [t], [f.shape])
    sv.close()
    assert r[t][1] == "MG_OK"
    xl, rl = _lone(lib, g, f, 1e-10, dict(smoother=2))
    assert r[t][2]["iters"] == rl["iters"] and np.array_equal(r[t][0], xl)


def test_serve_errors(lib):
    sv = lib.mg_serve_create()
    g = W.grid_desc(8)
    f = W.rhs_modes(g)
    with pytest.raises(lib.MGError):
        lib.mg_serve_submit(sv, dict(g, nph=15), np.zeros(8 * 8 * 15), 1e-8)
    bad = f.copy()
    bad[0, 0, 0] = np.inf
    t = lib.mg_serve_submit(sv, g, bad, 1e-8)
    t0 = time.time()
    while True:
        try:
            r = lib.mg_serve_poll(sv, t, np.empty_like(f))
        except lib.MGError as e:
            assert e.status == lib.MG_ENAN
            break
        assert r is None and time.time() - t0 < 60
        time.sleep(0.002)
    with pytest.raises(lib.MGError):
        lib.mg_serve_poll(sv, 987654321, None)
    sv.close()
