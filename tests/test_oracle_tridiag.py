"""Pins of the oracle's line solves (Section 3.5) and of the radial-line
Gauss-Seidel smoother built on them.

The Thomas algorithm and its periodic variant are checked against dense
solves of the assembled matrices, against closed forms (the discrete
second difference of a quadratic; Fourier modes of a circulant system, with
unequal sub- and super-diagonals so that a transposed system fails), and
planted mistakes show that these checks catch a swapped pair of diagonals or
a dropped corner.  The smoother is checked against block Gauss-Seidel with
dense line blocks, and against the defining property of an exact block
update: after a colour is swept, the residual vanishes on its lines.
"""
import numpy as np
import pytest

from oracle import direct, grid, mg, tridiag


def _random_system(rng, n, lines, periodic):
    a = rng.uniform(-1.0, 0.0, (n,) + lines)
    c = rng.uniform(-1.0, 0.0, (n,) + lines)
    b = 2.2 + rng.uniform(0.0, 1.0, (n,) + lines)
    if not periodic:
        a[0] = 0.0
        c[-1] = 0.0
    g = rng.standard_normal((n,) + lines)
    return a, b, c, g


def _dense(a, b, c, periodic):
    n = len(b)
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    if periodic:
        M[0, n - 1] += a[0]
        M[n - 1, 0] += c[n - 1]
    return M


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("n", [3, 4, 17, 64])
def test_line_solves_match_dense_solves(periodic, n):
    rng = np.random.default_rng(n + 100 * periodic)
    a, b, c, g = _random_system(rng, n, (3, 5), periodic)
    solve = tridiag.thomas_periodic if periodic else tridiag.thomas
    psi = solve(a, b, c, g)
    for l1 in range(3):
        for l2 in range(5):
            M = _dense(a[:, l1, l2], b[:, l1, l2], c[:, l1, l2], periodic)
            want = np.linalg.solve(M, g[:, l1, l2])
            np.testing.assert_allclose(psi[:, l1, l2], want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_thomas_second_difference_of_a_quadratic():
    """-psi_{m-1} + 2 psi_m - psi_{m+1} = 2 with psi_{-1} = psi_n = 0 is solved by
    psi_m = (m + 1)(n - m)."""
    for n in (1, 2, 5, 100, 1000):
        m = np.arange(n)
        psi = tridiag.thomas(-np.ones(n), 2.0 * np.ones(n), -np.ones(n), 2.0 * np.ones(n))
        want = (m + 1.0) * (n - m)
        np.testing.assert_allclose(psi, want, rtol=1e-12 * n, atol=0)


def _circulant_mode(n, q, beta, lo, up):
    """a = lo, b = beta, c = up on a ring: the mode cos(2 pi q m / n) maps to
    Re(e^{i t m} (beta + lo e^{-i t} + up e^{i t})), t = 2 pi q / n."""
    t = 2 * np.pi * q / n
    m = np.arange(n)
    lam = beta + lo * np.exp(-1j * t) + up * np.exp(1j * t)
    g = np.cos(t * m)
    return g, np.real(np.exp(1j * t * m) / lam)


@pytest.mark.parametrize("n,q", [(3, 1), (8, 0), (8, 3), (64, 5), (512, 37)])
def test_periodic_thomas_fourier_modes(n, q):
    lo, up, beta = -1.2, -0.7, 2.5
    g, want = _circulant_mode(n, q, beta, lo, up)
    psi = tridiag.thomas_periodic(np.full(n, lo), np.full(n, beta), np.full(n, up), g)
    np.testing.assert_allclose(psi, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_planted_line_solve_mistakes_are_caught():
    n, q, lo, up, beta = 64, 5, -1.2, -0.7, 2.5
    g, want = _circulant_mode(n, q, beta, lo, up)
    A, B, C = np.full(n, lo), np.full(n, beta), np.full(n, up)
    # sub- and super-diagonal swapped
    assert np.abs(tridiag.thomas_periodic(C, B, A, g) - want).max() > 1e-3 * np.abs(want).max()
    # corners dropped (the periodic system solved as a plain one)
    Ap, Cp = A.copy(), C.copy()
    Ap[0] = Cp[-1] = 0.0
    assert np.abs(tridiag.thomas(Ap, B, Cp, g) - want).max() > 1e-3 * np.abs(want).max()
    # a plain solve with a swapped pair fails the dense check
    rng = np.random.default_rng(3)
    a, b, c, gg = _random_system(rng, 17, (), False)
    want2 = np.linalg.solve(_dense(a, b, c, False), gg)
    ash, csh = np.roll(c, 1), np.roll(a, -1)          # transposed matrix
    assert np.abs(tridiag.thomas(ash, b, csh, gg) - want2).max() > 1e-3 * np.abs(want2).max()


def test_periodic_line_needs_three_unknowns():
    with pytest.raises(ValueError):
        tridiag.thomas_periodic(np.ones(2), 3 * np.ones(2), np.ones(2), np.ones(2))


# ---------------------------------------------------------------- radial-line smoother
LINE_GRIDS = {
    "sphere_7": (dict(mapping=0, stretch=2.0), 7),
    "triaxial_19": (dict(mapping=2, flattening=0.1, e2=0.05, stretch=2.0), 19),
}


def _level(name, shape=(6, 8, 12)):
    kw, st = LINE_GRIDS[name]
    sh = grid.Shell(*shape, **kw)
    fm = grid.face_metrics(sh)
    return sh, fm, mg.make_level(sh.shape, fm, st)


@pytest.mark.parametrize("name", list(LINE_GRIDS))
def test_line_blocks_are_tridiagonal_and_colours_uncoupled(name):
    sh, fm, lv = _level(name)
    Ad = lv.A.toarray()
    col = mg.line_colour_of(lv.shape, lv.stencil)
    line = (np.arange(lv.n) % (sh.nth * sh.nph))        # (i, k) of every cell
    for cells, _, lower, diag, upper in mg.line_systems(lv):
        for l in range(cells.shape[1]):
            L = cells[:, l]
            B = Ad[np.ix_(L, L)]
            assert not np.triu(B, 2).any() and not np.tril(B, -2).any()
            np.testing.assert_array_equal(np.diag(B), diag[:, l])
            np.testing.assert_array_equal(np.diag(B, -1), lower[1:, l])
            np.testing.assert_array_equal(np.diag(B, 1), upper[:-1, l])
    # two cells on different lines of one colour are never coupled
    r, c = lv.A.nonzero()
    same = (col[r] == col[c]) & (line[r] != line[c])
    assert not same.any()


@pytest.mark.parametrize("name", list(LINE_GRIDS))
def test_line_sweep_is_block_gauss_seidel(name):
    sh, fm, lv = _level(name)
    rng = np.random.default_rng(6)
    b, _ = mg.prepare_rhs(fm["J"], rng.standard_normal(sh.n))
    x0 = rng.standard_normal(sh.n)
    Ad = lv.A.toarray()
    y = x0.copy()
    for cells, *_ in mg.line_systems(lv):
        for l in range(cells.shape[1]):
            L = cells[:, l]
            y[L] += np.linalg.solve(Ad[np.ix_(L, L)], b[L] - Ad[L] @ y)
        # exact block update: the residual vanishes on the lines just swept
        rr = b[cells.ravel()] - Ad[cells.ravel()] @ y
        assert np.abs(rr).max() <= 1e-12 * np.abs(b).max()
    x = mg.smooth(lv, x0, b, 1, mg.LINE)
    np.testing.assert_allclose(x, y, rtol=0, atol=1e-13 * np.abs(y).max())


def test_line_smoothed_multigrid_matches_direct_solve():
    kw, st = LINE_GRIDS["triaxial_19"]
    sh = grid.Shell(8, 8, 16, **kw)
    fm = grid.face_metrics(sh)
    f = np.random.default_rng(7).standard_normal(sh.n)
    x, info = mg.solve(sh, f, tol=1e-12, kind=mg.LINE, fm=fm)
    assert info["converged"]
    lv = mg.make_level(sh.shape, fm, st)
    b, _ = mg.prepare_rhs(fm["J"], f)
    xd, _ = direct.bordered_solve(lv.A, b, fm["J"].ravel())
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_line_smoother_handles_a_thin_shell():
    """Radius range 1 to 1.05 with stretching: the radial coupling dominates,
    point Gauss-Seidel stalls under full coarsening and radial lines do not."""
    sh = grid.Shell(16, 16, 32, r_in=1.0, r_out=1.05, stretch=2.0)
    f = np.random.default_rng(0).standard_normal(sh.n)
    rho = {}
    for kind in (mg.GS, mg.LINE):
        _, info = mg.solve(sh, f, tol=1e-10, policy=mg.FULL, kind=kind, max_iters=12)
        h = info["hist"]
        rho[kind] = (h[-1] / h[0]) ** (1.0 / info["iters"])
    assert rho[mg.GS] > 0.9 and rho[mg.LINE] < 0.15, rho
