"""Seeded input generators: determinism, shapes and the closed-form RHS."""
import numpy as np
import pytest

import workloads as W


def test_pstar_rhs_matches_symbolic_spherical_laplacian():
    sy = pytest.importorskip("sympy")
    g = W.grid_desc(8)
    f = W.rhs_pstar(g, noise=0)
    r, t, p = sy.symbols("r t p")
    P = sy.cos(sy.pi * (r - 1)) * sy.cos(3 * t) * sy.sin(2 * p)
    lap = (sy.diff(r ** 2 * sy.diff(P, r), r) / r ** 2
           + sy.diff(sy.sin(t) * sy.diff(P, t), t) / (r ** 2 * sy.sin(t))
           + sy.diff(P, p, 2) / (r ** 2 * sy.sin(t) ** 2))
    fl = sy.lambdify((r, t, p), lap)
    rh = 1 + (np.arange(8) + 0.5) / 8
    th = np.pi / 6 + (np.arange(8) + 0.5) * (2 * np.pi / 3) / 8
    ph = 2 * np.pi * (np.arange(16) + 0.5) / 16
    R, T, Ph = np.meshgrid(rh, th, ph, indexing="ij")
    np.testing.assert_allclose(f, fl(R, T, Ph), atol=1e-12)


def test_generators_are_seeded_and_contiguous():
    g = W.grid_desc(8, stretch=2.0)
    a, b = W.rhs_modes(g, 3), W.rhs_modes(g, 3)
    assert a.shape == (8, 8, 16) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    assert np.array_equal(a, b) and not np.array_equal(a, W.rhs_modes(g, 4))
    n1 = W.rhs_pstar(W.grid_desc(8), seed=0)
    assert np.array_equal(n1, W.rhs_pstar(W.grid_desc(8), seed=0))


def test_batch_and_stream_draws():
    shells = W.batch_shells()
    assert len(shells) == 64
    assert {s["grid"]["nr"] for s in shells} <= {32, 64, 96, 128}
    for s in shells:
        g = s["grid"]
        assert 1 / 0.8 <= g["r_out"] <= 1 / 0.35 and 0 <= g["flattening"] <= 0.15
    reqs = W.serve_stream(n=200, rate=100.0)
    t = np.array([q["t_arrive"] for q in reqs])
    assert np.all(np.diff(t) > 0)
    assert {q["grid"]["nr"] for q in reqs} <= set(W.FRIENDLY)
    assert {q["tol"] for q in reqs} <= {1e-6, 1e-8, 1e-10}
