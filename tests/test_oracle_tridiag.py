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


# ---------------------------------------------------------------- longitude-line smoother
@pytest.mark.parametrize("name", list(LINE_GRIDS))
def test_longitude_line_blocks_are_cyclic_tridiagonal_and_colours_uncoupled(name):
    sh, fm, lv = _level(name)
    Ad = lv.A.toarray()
    col = mg.xline_colour_of(lv.shape, lv.stencil)
    line = np.arange(lv.n) // sh.nph                  # (j, i) of every cell
    n = sh.nph
    for cells, _, a, b, c in mg.xline_systems(lv):
        for l in range(cells.shape[1]):
            L = cells[:, l]
            B = Ad[np.ix_(L, L)]
            band = np.eye(n, dtype=bool) | np.eye(n, k=1, dtype=bool) | np.eye(n, k=-1, dtype=bool)
            band[0, n - 1] = band[n - 1, 0] = True
            assert not B[~band].any()
            np.testing.assert_array_equal(np.diag(B), b[:, l])
            np.testing.assert_array_equal([B[k, (k - 1) % n] for k in range(n)], a[:, l])
            np.testing.assert_array_equal([B[k, (k + 1) % n] for k in range(n)], c[:, l])
    r, cc = lv.A.nonzero()
    assert not ((col[r] == col[cc]) & (line[r] != line[cc])).any()


@pytest.mark.parametrize("name", list(LINE_GRIDS))
def test_longitude_line_sweep_is_block_gauss_seidel(name):
    sh, fm, lv = _level(name)
    rng = np.random.default_rng(16)
    b, _ = mg.prepare_rhs(fm["J"], rng.standard_normal(sh.n))
    x0 = rng.standard_normal(sh.n)
    Ad = lv.A.toarray()
    y = x0.copy()
    for cells, *_ in mg.xline_systems(lv):
        for l in range(cells.shape[1]):
            L = cells[:, l]
            y[L] += np.linalg.solve(Ad[np.ix_(L, L)], b[L] - Ad[L] @ y)
        rr = b[cells.ravel()] - Ad[cells.ravel()] @ y
        assert np.abs(rr).max() <= 1e-12 * np.abs(b).max()
    x = mg.smooth(lv, x0, b, 1, mg.XLINE)
    np.testing.assert_allclose(x, y, rtol=0, atol=1e-13 * np.abs(y).max())
    # alternating: the radial sweep, then the longitude sweep
    z = mg.smooth(lv, mg.smooth(lv, x0, b, 1, mg.LINE), b, 1, mg.XLINE)
    np.testing.assert_allclose(mg.smooth(lv, x0, b, 1, mg.ALT), z, rtol=0, atol=0)


@pytest.mark.parametrize("kind", ["XLINE", "ALT"])
def test_longitude_line_smoothed_multigrid_matches_direct_solve(kind):
    kw, st = LINE_GRIDS["triaxial_19"]
    for sh in (grid.Shell(8, 8, 16, **kw), grid.full_sphere(8, 8, 16, **kw)):
        fm = grid.face_metrics(sh)
        f = np.random.default_rng(17).standard_normal(sh.n)
        x, info = mg.solve(sh, f, tol=1e-12, kind=getattr(mg, kind), fm=fm)
        assert info["converged"]
        lv = mg.make_level(sh.shape, fm, st, sh.cut)
        b, _ = mg.prepare_rhs(fm["J"], f)
        xd, _ = direct.bordered_solve(lv.A, b, fm["J"].ravel())
        np.testing.assert_allclose(x, xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_alternating_lines_handle_the_poles_and_a_thin_shell():
    """The full sphere (longitude coupling grows like 1/sin^2(theta) toward
    the poles) defeats point and radial-line smoothing; alternating radial and
    longitude lines keep their rate there and on the thin stretched shell."""
    f_iters = {}
    for name, sh in (("sphere", grid.full_sphere(16, 16, 32)),
                     ("thin", grid.Shell(16, 16, 32, r_out=1.05, stretch=2.0))):
        f = np.random.default_rng(3).standard_normal(sh.n)
        hier, fm = mg.setup(sh, 7)
        for kind in (mg.GS, mg.LINE, mg.ALT):
            _, info = mg.solve(sh, f, tol=1e-10, hier=hier, fm=fm, kind=kind, max_iters=60)
            f_iters[name, kind] = info["iters"]
    assert f_iters["sphere", mg.ALT] <= 10 and f_iters["thin", mg.ALT] <= 6, f_iters
    assert f_iters["sphere", mg.GS] >= 3 * f_iters["sphere", mg.ALT], f_iters
    assert f_iters["sphere", mg.LINE] >= 3 * f_iters["sphere", mg.ALT], f_iters


# ---------------------------------------------------------------- ADI-CN sweeps (Section 3.4)
from oracle import adi, operator  # noqa: E402

ADI_GRIDS = {
    "sphere_stretched": dict(mapping=0, stretch=2.0),
    "triaxial": dict(mapping=2, flattening=0.1, e2=0.05, stretch=1.0),
}


def _adi_grid(name, shape=(6, 8, 12)):
    sh = grid.Shell(*shape, **ADI_GRIDS[name])
    return sh, grid.face_metrics(sh)


@pytest.mark.parametrize("name", list(ADI_GRIDS))
def test_diagonal_terms_sum_to_the_seven_point_operator(name):
    """With zero-flux walls, L_zeta + L_eta + L_xi is the 7-point conservative
    operator (Eq. PC_term1 in each direction) assembled independently."""
    sh, fm = _adi_grid(name)
    u = np.random.default_rng(1).standard_normal(sh.n)
    bc = adi.walls((adi.FLUX0, 0, 0), (adi.FLUX0, 0, 0))
    L = sum(adi.apply_diag(sh, fm, u, d, bc) for d in range(3)).ravel()
    A = operator.assemble(sh, fm, 7)
    np.testing.assert_allclose(L, A @ u, rtol=0, atol=1e-13 * np.abs(A @ u).max())


@pytest.mark.parametrize("name", list(ADI_GRIDS))
def test_constants_are_steady(name):
    """A constant field with zero-flux walls, or with wall values equal to the
    constant, has L = 0 and is unchanged by a sub-step."""
    sh, fm = _adi_grid(name)
    u = np.full(sh.shape, 0.7)
    for bc in (adi.walls((adi.FLUX0, 0, 0), (adi.FLUX0, 0, 0)),
               adi.walls((adi.VALUE, 0.7, 0.7), (adi.VALUE, 0.7, 0.7))):
        for d in range(3):
            assert np.abs(adi.apply_diag(sh, fm, u, d, bc)).max() < 1e-13
        np.testing.assert_allclose(adi.substep(sh, fm, u, 0.3, bc), u, rtol=1e-13)


@pytest.mark.parametrize("name", list(ADI_GRIDS))
def test_each_sweep_solves_its_system(name):
    """(J - kappa L_d) u = rhs holds after the sweep, with L_d applied by the
    flux form (not the tridiagonal assembly), for each direction and wall kind."""
    sh, fm = _adi_grid(name)
    rng = np.random.default_rng(2)
    J = fm["J"]
    for bc in (adi.walls(), adi.walls((adi.VALUE, 1.0, 0.0), (adi.FLUX0, 0, 0))):
        for d in range(3):
            rhs = rng.standard_normal(sh.shape)
            u = adi.sweep(sh, fm, d, 0.8, rhs, bc)
            res = J * u - 0.8 * adi.apply_diag(sh, fm, u, d, bc) - rhs
            assert np.abs(res).max() < 1e-12 * np.abs(rhs).max(), (d, np.abs(res).max())


def test_substep_without_viscosity_adds_the_explicit_terms():
    sh, fm = _adi_grid("triaxial")
    rng = np.random.default_rng(3)
    un, s = rng.standard_normal(sh.shape), rng.standard_normal(sh.shape)
    np.testing.assert_allclose(adi.substep(sh, fm, un, 0.0, adi.walls(), src=s), un + s / fm["J"], rtol=1e-13)


def _exact(sh, fm, un, kappa, bc):
    """exp(2 kappa J^{-1} L) u^n for zero-flux walls (L = sum of the diagonal
    terms), by the matrix exponential of the assembled operator."""
    import scipy.linalg
    A = operator.assemble(sh, fm, 7).toarray()
    M = A / fm["J"].ravel()[:, None]
    return scipy.linalg.expm(2.0 * kappa * M) @ un.ravel()


@pytest.mark.parametrize("name", list(ADI_GRIDS))
def test_substep_is_second_order_in_time(name):
    """The sub-step factorises (I - kM_1)(I - kM_2)(I - kM_3)(u - u^n) = 2kM u^n
    (M_p = J^{-1} L_p): it matches exp(2 k M) u^n to O(k^3) (a first-order
    splitting or a misplaced factor 2 would leave O(k^2))."""
    sh, fm = _adi_grid(name, (4, 6, 8))
    bc = adi.walls((adi.FLUX0, 0, 0), (adi.FLUX0, 0, 0))
    un = np.random.default_rng(4).standard_normal(sh.shape)
    scale = np.abs(operator.assemble(sh, fm, 7).diagonal() / fm["J"].ravel()).max()
    errs = []
    for k in (0.02, 0.01, 0.005):
        kappa = k / scale
        errs.append(np.abs(adi.substep(sh, fm, un, kappa, bc).ravel() - _exact(sh, fm, un, kappa, bc)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 7.0 < r1 < 9.0 and 7.0 < r2 < 9.0, errs


def test_planted_adi_mistakes_are_caught(monkeypatch):
    """Explicit terms with weight kappa instead of 2 kappa, or a sweep that
    solves with +kappa, break second order or the sweep residual."""
    sh, fm = _adi_grid("sphere_stretched", (4, 6, 8))
    bc = adi.walls((adi.FLUX0, 0, 0), (adi.FLUX0, 0, 0))
    un = np.random.default_rng(4).standard_normal(sh.shape)
    scale = np.abs(operator.assemble(sh, fm, 7).diagonal() / fm["J"].ravel()).max()
    kap = [k / scale for k in (0.02, 0.01)]
    good = [np.abs(adi.substep(sh, fm, un, k, bc).ravel() - _exact(sh, fm, un, k, bc)).max() for k in kap]
    orig = adi.apply_diag

    def halved(shh, fmm, u, d, b):
        return 0.5 * orig(shh, fmm, u, d, b) if d != 0 else orig(shh, fmm, u, d, b)

    monkeypatch.setattr(adi, "apply_diag", halved)
    bad = [np.abs(adi.substep(sh, fm, un, k, bc).ravel() - _exact(sh, fm, un, k, bc)).max() for k in kap]
    monkeypatch.setattr(adi, "apply_diag", orig)
    assert good[0] / good[1] > 7.0 and bad[0] / bad[1] < 4.5
    origls = adi.line_system

    def flipped(shh, fmm, d, kappa, b):
        return origls(shh, fmm, d, -kappa, b)

    monkeypatch.setattr(adi, "line_system", flipped)
    rhs = np.random.default_rng(5).standard_normal(sh.shape)
    u = adi.sweep(sh, fm, 1, 0.8, rhs, bc)
    monkeypatch.setattr(adi, "line_system", origls)
    res = fm["J"] * u - 0.8 * adi.apply_diag(sh, fm, u, 1, bc) - rhs
    assert np.abs(res).max() > 1e-3 * np.abs(rhs).max()


@pytest.mark.parametrize("d", [0, 1])
def test_wall_values_sit_on_the_wall_face(d):
    """u linear in the index along d (u = m + 1/2 at cell m) with wall values 0
    and n (its values on the wall faces): every face, walls included, carries
    the flux G_dd x 1, so L_d u = G(upper face) - G(lower face) exactly."""
    sh, fm = _adi_grid("triaxial")
    ax = {0: 1, 1: 0}[d]
    n = sh.shape[ax]
    shape = [1, 1, 1]
    shape[ax] = n
    u = np.broadcast_to((np.arange(n) + 0.5).reshape(shape), sh.shape)
    bc = adi.walls((adi.VALUE, 0.0, float(n)), (adi.VALUE, 0.0, float(n)))
    G = np.moveaxis(adi.face_G(sh, fm, d), ax, 0)
    want = np.moveaxis(G[1:] - G[:-1], 0, ax)
    np.testing.assert_allclose(adi.apply_diag(sh, fm, u, d, bc), want, rtol=0, atol=1e-13 * np.abs(G).max())
