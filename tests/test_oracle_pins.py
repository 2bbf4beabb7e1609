"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: closed forms
(shell volume, textbook spherical metric, manufactured Laplacians, the
harmonic conductive profile), exact invariants of the conservative operator,
brute force on tiny grids (sparse direct solve) and exact properties of the
transfers.  The mutation tests at the end plant plausible mistakes in the
oracle and check that a pin catches each one.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import grid, operator, mg, direct, mms

MAPS = {
    "sphere": dict(mapping=0),
    "sphere_stretched": dict(mapping=0, stretch=2.0),
    "oblate": dict(mapping=1, flattening=0.1, r_out=1 / 0.6),
    "triaxial_stretched": dict(mapping=2, flattening=0.1, e2=0.05, stretch=2.0),
}


def sh_of(n, **kw):
    return grid.Shell(n, n, 2 * n, **kw)


# ---------------------------------------------------------------- Eq. stretching
@pytest.mark.parametrize("rx", [0.0, 1.0, 2.0, 3.5])
def test_stretching_endpoints_symmetry_and_slope(rx):
    n = 16
    j = np.arange(n + 1)
    s = grid.stretch_unit(j, n, rx)
    assert s[0] == pytest.approx(-0.5, abs=1e-15) and s[-1] == pytest.approx(0.5, abs=1e-15)
    assert s[n // 2] == pytest.approx(0.0, abs=1e-15)
    np.testing.assert_allclose(s + s[::-1], 0.0, atol=1e-15)      # odd about the middle
    assert np.all(np.diff(s) > 0)
    if rx > 0:
        # wall/centre spacing ratio of tanh clustering is sech^2(rx/2)
        ds = grid.d_stretch_unit(np.array([0.0, n / 2]), n, rx)
        assert ds[0] / ds[1] == pytest.approx(1 / np.cosh(rx / 2) ** 2, rel=1e-13)
        # the analytic derivative agrees with a fine central difference
        h = 1e-5
        fd = (grid.stretch_unit(3 + h, n, rx) - grid.stretch_unit(3 - h, n, rx)) / (2 * h)
        assert grid.d_stretch_unit(3.0, n, rx) == pytest.approx(fd, rel=1e-8)


# ---------------------------------------------------------------- Section 3.2
def test_analytic_sphere_metric_matches_textbook():
    """Analytic metric code vs spherical coordinates: in index units
    G_rr = r^2 sin(th) dth dph / dr, G_thth = sin(th) dr dph / dth,
    G_phph = dr dth / (sin(th) dph), det = r^2 sin(th) dr dth dph."""
    sh = sh_of(6)
    an = grid.analytic_face_metrics(sh)
    dr = (sh.r_out - sh.r_in) / sh.nr
    dth = (sh.th1 - sh.th0) / sh.nth
    dph = 2 * np.pi / sh.nph
    # eta (radial) faces at vertex radius j, centre colatitude i + 1/2
    j, i, k = np.meshgrid(np.arange(sh.nr + 1), np.arange(sh.nth), np.arange(sh.nph), indexing="ij")
    r = sh.r_in + j * dr
    th = sh.th0 + (i + 0.5) * dth
    np.testing.assert_allclose(an["G1"][..., 1], r ** 2 * np.sin(th) * dth * dph / dr, rtol=1e-13)
    np.testing.assert_allclose(an["det1"], r ** 2 * np.sin(th) * dr * dth * dph, rtol=1e-13)
    np.testing.assert_allclose(an["G1"][..., 0], 0, atol=1e-15)
    # zeta (colatitude) faces at vertex colatitude i, centre radius j + 1/2
    j, i, k = np.meshgrid(np.arange(sh.nr), np.arange(sh.nth + 1), np.arange(sh.nph), indexing="ij")
    r = sh.r_in + (j + 0.5) * dr
    th = sh.th0 + i * dth
    np.testing.assert_allclose(an["G0"][..., 0], np.sin(th) * dr * dph / dth, rtol=1e-13)
    # xi faces
    j, i, k = np.meshgrid(np.arange(sh.nr), np.arange(sh.nth), np.arange(sh.nph), indexing="ij")
    th = sh.th0 + (i + 0.5) * dth
    np.testing.assert_allclose(an["G2"][..., 2], dr * dth / (np.sin(th) * dph), rtol=1e-13)


@pytest.mark.parametrize("name", list(MAPS))
def test_face_metric_second_order(name):
    """The paper's discrete face metric converges to the exact metric at O(h^2)."""
    errs = []
    for n in (8, 16, 32):
        sh = sh_of(n, **MAPS[name])
        fm = grid.face_metrics(sh)
        an = grid.analytic_face_metrics(sh)
        e = 0.0
        for d in range(3):
            scale = np.abs(an[f"G{d}"][..., d]).max()
            e = max(e, np.abs(fm[f"G{d}"] - an[f"G{d}"]).max() / scale)
            e = max(e, np.abs(fm[f"det{d}"] / an[f"det{d}"] - 1).max())
        errs.append(e)
    assert errs[-1] < 5e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


@pytest.mark.parametrize("name", list(MAPS))
def test_cell_volumes_sum_to_shell_volume(name):
    """Sum of cell |J^{-1}| (step 3) -> exact sector volume, O(h^2)."""
    errs = []
    for n in (8, 16, 32):
        sh = sh_of(n, **MAPS[name])
        errs.append(abs(grid.face_metrics(sh)["J"].sum() / grid.shell_volume(sh) - 1))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_metric_inverse_matches_library_inverse():
    sh = sh_of(4, **MAPS["triaxial_stretched"])
    M = grid.face_jacobian(sh, 0, *np.meshgrid(np.arange(5), np.arange(4), np.arange(8), indexing="ij"))
    adet, G, C = grid.metric_from_jacobian(M)
    inv = np.linalg.inv(M)                       # inv[p, a] = dzeta_p / dx_a
    np.testing.assert_allclose(C, adet[..., None, None] * inv, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(adet, np.abs(np.linalg.det(M)), rtol=1e-13)


# ---------------------------------------------------------------- Section 3.3 operator
@pytest.mark.parametrize("name", list(MAPS))
@pytest.mark.parametrize("stencil", [7, 19])
def test_operator_invariants(name, stencil):
    sh = sh_of(6, **MAPS[name])
    fm = grid.face_metrics(sh)
    A = operator.assemble(sh, fm, stencil)
    one = np.ones(sh.n)
    scale = abs(A).max()
    assert np.abs(A @ one).max() < 1e-13 * scale          # constants in the kernel
    assert np.abs(A.T @ one).max() < 1e-13 * scale        # conservation (zero wall flux)
    if stencil == 7:
        assert abs(A - A.T).max() == 0.0                   # exact symmetry
    S = ((A + A.T) / 2).toarray()
    ev = np.linalg.eigvalsh(S)
    assert ev.max() < 1e-12 * scale                        # symmetric part is NSD
    assert np.sum(ev > -1e-10 * scale) == 1                # one-dimensional null space


def test_19pt_asymmetry_vanishes_at_first_order():
    """The cross-term discretisation of Eqs. PC_term2-3 is not exactly
    symmetric; its asymmetry decays at least linearly with h."""
    rel = []
    for n in (8, 16, 32):
        sh = sh_of(n, **MAPS["triaxial_stretched"])
        A = operator.assemble(sh, grid.face_metrics(sh), 19)
        rel.append(abs(A - A.T).max() / abs(A).max())
    assert rel[0] / rel[1] > 1.8 and rel[1] / rel[2] > 1.8


def test_19pt_stencil_footprint():
    sh = sh_of(6, **MAPS["triaxial_stretched"])
    A = operator.assemble(sh, grid.face_metrics(sh), 19)
    # an interior cell couples to itself, 6 faces and 12 edges: 19 points
    c = (3 * 6 + 3) * 12 + 5
    assert A[c].nnz == 19
    A7 = operator.assemble(sh, grid.face_metrics(sh), 7)
    assert A7[c].nnz == 7


@pytest.mark.parametrize("name,stencil", [("sphere", 7), ("sphere", 19), ("oblate", 19),
                                          ("triaxial_stretched", 19)])
def test_sampled_rows_match_assembly(name, stencil):
    sh = grid.Shell(5, 6, 8, **MAPS[name])
    fm = grid.face_metrics(sh)
    A = operator.assemble(sh, fm, stencil)
    x = np.random.default_rng(1).standard_normal(sh.n)
    cells = np.unravel_index(np.arange(sh.n), sh.shape)
    y = operator.apply_rows(sh, x, cells, stencil)
    np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-13 * abs(A).max() * np.abs(x).max())


def _interior_truncation(sh, kind, stencil):
    fm = grid.face_metrics(sh)
    A = operator.assemble(sh, fm, stencil)
    p, lap = mms.manufactured(sh, kind)
    res = (A @ p.ravel()) / fm["J"].ravel() - lap.ravel()
    res = res.reshape(sh.shape)[1:-1, 1:-1, :]
    return np.abs(res).max() / np.abs(lap).max()


@pytest.mark.parametrize("name,kind,stencil", [("sphere", "cosine", 7),
                                               ("sphere_stretched", "cosine", 7),
                                               ("oblate", "bump", 19),
                                               ("triaxial_stretched", "bump", 19)])
def test_truncation_error_second_order(name, kind, stencil):
    """(A p)/J approximates the closed-form Laplacian at O(h^2) in the interior."""
    e = [_interior_truncation(sh_of(n, **MAPS[name]), kind, stencil) for n in (8, 16, 32)]
    assert e[1] / e[2] > 3.5 and e[2] < 2e-2


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_conductive_profile_is_discretely_harmonic(stretch):
    """T_c = a/r + b (Eq. conductive profile) solves d/dr(r^2 dT/dr) = 0; the
    discrete operator annihilates it to O(h^2) away from the walls."""
    e = []
    for n in (8, 16, 32):
        sh = sh_of(n, stretch=stretch)
        fm = grid.face_metrics(sh)
        A = operator.assemble(sh, fm, 7)
        p, lap = mms.manufactured(sh, "conductive")
        assert np.abs(lap).max() < 1e-12
        ref = (A @ mms.manufactured(sh, "cosine")[0].ravel()) / fm["J"].ravel()
        y = ((A @ p.ravel()) / fm["J"].ravel()).reshape(sh.shape)[1:-1]
        e.append(np.abs(y).max() / np.abs(ref).max())
    assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.4


# ---------------------------------------------------------------- transfers / hierarchy
@pytest.mark.parametrize("c", [(2, 2, 2), (1, 2, 1), (2, 1, 2), (1, 1, 2)])
def test_transfers_exact_properties(c):
    shape = (8, 8, 16)
    R, P = mg.transfer_matrices(shape, c)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(R.shape[1])
    assert (R @ r).sum() == pytest.approx(r.sum(), rel=1e-13)      # children sum conserves
    np.testing.assert_allclose(P @ np.ones(P.shape[1]), 1.0, rtol=0, atol=1e-15)
    # trilinear: a function linear in the cell-centre coordinate is reproduced
    # exactly away from walls (fine centre of child s of C: C + (2s - 1)/4)
    nr, nth, nph = shape
    ncr, nct, ncp = nr // c[1], nth // c[0], nph // c[2]
    J, I, K = np.meshgrid(np.arange(ncr), np.arange(nct), np.arange(ncp), indexing="ij")
    lin = 0.3 * J + 0.7 * I
    fine = P @ lin.ravel()
    jf, if_, kf = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nph), indexing="ij")
    cj = (jf + 0.5) / c[1] - 0.5
    ci = (if_ + 0.5) / c[0] - 0.5
    exact = 0.3 * cj + 0.7 * ci
    inner = (cj >= 0) & (cj <= ncr - 1) & (ci >= 0) & (ci <= nct - 1)
    np.testing.assert_allclose(fine.reshape(shape)[inner], exact[inner], atol=1e-13)


def test_aggregated_coarse_metric_matches_coarse_grid_metric():
    """G aggregated from a fine grid approximates the paper's metric evaluated
    directly on the twice coarser grid (same mapping), at O(h^2)."""
    errs = []
    for n in (8, 16, 32):
        fine = sh_of(2 * n, **MAPS["triaxial_stretched"])
        coarse = sh_of(n, **MAPS["triaxial_stretched"])
        _, cfm = mg.coarsen_faces(fine.shape, grid.face_metrics(fine), (2, 2, 2))
        dfm = grid.face_metrics(coarse)
        e = max(np.abs(cfm[f"G{d}"] - dfm[f"G{d}"]).max() / np.abs(dfm[f"G{d}"][..., d]).max()
                for d in range(3))
        errs.append(e)
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.5


def test_colours_are_independent_sets():
    for stencil, name in ((7, "sphere"), (19, "triaxial_stretched")):
        sh = sh_of(4, **MAPS[name])
        lv = mg.make_level(sh.shape, grid.face_metrics(sh), stencil)
        for idx in lv.colours:
            sub = lv.A[idx][:, idx].tocoo()
            assert np.all(sub.row == sub.col)


def test_gauss_seidel_sweep_is_block_gauss_seidel_in_colour_order():
    """One multicolour Gauss-Seidel sweep is block Gauss-Seidel over the colour
    sets taken in order 0, 1 (7 points) or 0, 1, 2, 3 (19 points): with
    d_c = y_c - x_c the change of colour c, the final residual on colour c is
    exactly -sum over the later colours c' of A[c, c'] d_c' (the residual of
    colour c is zero right after its own update).  A swapped colour order, a
    skipped colour or a wrong diagonal breaks this identity."""
    rng = np.random.default_rng(11)
    for stencil, name in ((7, "sphere_stretched"), (19, "triaxial_stretched"), (19, "oblate")):
        sh = grid.Shell(4, 6, 8, **MAPS[name])
        lv = mg.make_level(sh.shape, grid.face_metrics(sh), stencil)
        x0 = rng.standard_normal(lv.n)
        b = rng.standard_normal(lv.n)
        _check_block_gauss_seidel(lv, x0, b, stencil, name)


def _colour_sets(shape, stencil):
    """The colour sets of the smoother's ordering, from the cell indices:
    (i + j + k) mod 2 for 7 points, ((i + j) mod 2) + 2 ((j + k) mod 2) for 19."""
    j, i, k = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    col = ((i + j + k) % 2 if stencil == 7 else (i + j) % 2 + 2 * ((j + k) % 2)).ravel()
    return [np.nonzero(col == c)[0] for c in range(2 if stencil == 7 else 4)]


def _check_block_gauss_seidel(lv, x0, b, stencil, name):
    y = mg.smooth(lv, x0, b, 1, mg.GS)
    r = b - lv.A @ y
    scale = np.abs(lv.A).max() * np.abs(y).max()
    sets = _colour_sets(lv.shape, stencil)
    for c, idx in enumerate(sets):
        want = np.zeros(len(idx))
        for later in sets[c + 1:]:
            want -= lv.A[idx][:, later] @ (y[later] - x0[later])
        np.testing.assert_allclose(r[idx], want, rtol=0, atol=1e-12 * scale, err_msg=f"{name} colour {c}")
        if c < len(sets) - 1:
            assert np.abs(r[idx]).max() > 1e-3 * scale       # not an already-converged colour
    assert np.abs(r[sets[-1]]).max() < 1e-12 * scale


@pytest.mark.parametrize("stencil,factor", [(7, -5.0 / 7.0), (19, -3.0 / 5.0)])
def test_weighted_jacobi_damps_the_checkerboard_by_one_minus_two_omega(stencil, factor):
    """On the constant-coefficient operator (G_pp = 1, no cross terms) the
    checkerboard (-1)^(i+j+k) is an eigenvector at cells away from the walls
    with D^-1 A e = 2 e, so one weighted-Jacobi step multiplies it by
    1 - 2 omega: -5/7 for omega = 6/7 (7 points), -3/5 for omega = 4/5
    (19 points)."""
    nr, nth, nph = 6, 6, 8
    fm = {"G0": np.zeros((nr, nth + 1, nph, 3)), "G1": np.zeros((nr + 1, nth, nph, 3)),
          "G2": np.zeros((nr, nth, nph, 3)), "J": np.ones((nr, nth, nph))}
    fm["G0"][..., 0] = 1.0
    fm["G1"][..., 1] = 1.0
    fm["G2"][..., 2] = 1.0
    lv = mg.make_level((nr, nth, nph), fm, stencil)
    j, i, k = np.meshgrid(np.arange(nr), np.arange(nth), np.arange(nph), indexing="ij")
    e = ((-1.0) ** (i + j + k)).ravel()
    y = mg.smooth(lv, e, np.zeros(lv.n), 1, mg.JACOBI).reshape(nr, nth, nph)
    inner = (slice(1, nr - 1), slice(1, nth - 1), slice(None))
    np.testing.assert_allclose(y[inner], factor * e.reshape(nr, nth, nph)[inner], rtol=0, atol=1e-14)


def test_plan_factors_policies():
    sh = sh_of(16, **MAPS["sphere"])
    fm = grid.face_metrics(sh)
    assert mg.plan_factors(sh.shape, fm, mg.FULL) == (2, 2, 2)
    # radial coupling dominates on this shell: semi-coarsening halves eta only
    assert mg.plan_factors(sh.shape, fm, mg.SEMI) == (1, 2, 1)
    assert mg.plan_factors((2, 2, 6), None, mg.FULL) is None


# ---------------------------------------------------------------- solves
@pytest.mark.parametrize("name", list(MAPS))
def test_multigrid_matches_direct_solve(name):
    sh = sh_of(8, **MAPS[name])
    stencil = 7 if MAPS[name]["mapping"] == 0 else 19
    f = np.random.default_rng(3).standard_normal(sh.n)
    x, info = mg.solve(sh, f, tol=1e-14, stencil=stencil, coarse_max=64)
    assert info["converged"] and info["levels"] >= 2
    fm = grid.face_metrics(sh)
    A = operator.assemble(sh, fm, stencil)
    b, _ = mg.prepare_rhs(fm["J"], f)
    xd, lam = direct.bordered_solve(A, b, fm["J"].ravel())
    assert abs(lam) < 1e-12 * np.abs(b).max()
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-11 * np.abs(xd).max())
    assert abs((fm["J"].ravel() * x).sum()) < 1e-12 * np.abs(x).max() * fm["J"].sum()


def test_gauss_seidel_and_jacobi_are_convergent_iterations():
    sh = grid.Shell(4, 4, 8, **MAPS["oblate"])
    fm = grid.face_metrics(sh)
    lv = mg.make_level(sh.shape, fm, 19)
    b, _ = mg.prepare_rhs(fm["J"], np.random.default_rng(4).standard_normal(sh.n))
    xd, _ = direct.bordered_solve(lv.A, b, fm["J"].ravel())
    for kind, sweeps in ((mg.GS, 2000), (mg.JACOBI, 6000)):
        x = mg.gauge(fm["J"], mg.smooth(lv, np.zeros(sh.n), b, sweeps, kind))
        assert np.abs(x - xd).max() < 1e-6 * np.abs(xd).max()


def test_coarse_solve_is_bordered_solution():
    sh = grid.Shell(2, 4, 8, **MAPS["oblate"])
    lv = mg.make_level(sh.shape, grid.face_metrics(sh), 19)
    r = np.random.default_rng(5).standard_normal(lv.n)
    e = mg.coarse_solve(lv, r)
    assert abs(e.sum()) < 1e-12
    np.testing.assert_allclose(lv.A @ e, r - r.mean(), atol=1e-12 * np.abs(r).max())


@pytest.mark.parametrize("name,kind,stencil", [("sphere", "cosine", 7),
                                               ("triaxial_stretched", "bump", 19)])
def test_discrete_solution_converges_second_order(name, kind, stencil):
    errs = []
    for n in (8, 16, 32):
        sh = sh_of(n, **MAPS[name])
        p, lap = mms.manufactured(sh, kind)
        hier, fm = mg.setup(sh, stencil)
        x, info = mg.solve(sh, lap.ravel(), tol=1e-11, hier=hier, fm=fm)
        assert info["converged"]
        pe = mg.gauge(fm["J"], p.ravel())
        errs.append(np.abs(x - pe).max() / np.abs(pe).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


def test_rhs_compatibility_and_gauge():
    sh = sh_of(4, **MAPS["oblate"])
    J = grid.face_metrics(sh)["J"]
    f = np.random.default_rng(6).standard_normal(sh.n) + 3.0
    b, mean = mg.prepare_rhs(J, f)
    assert abs(b.sum()) < 1e-13 * np.abs(b).sum()
    assert mean == pytest.approx((J.ravel() * f).sum() / J.sum(), rel=1e-14)
    x = mg.gauge(J, f)
    assert abs((J.ravel() * x).sum()) < 1e-13 * np.abs(J.ravel() * x).sum()


# ---------------------------------------------------------------- planted mistakes
def _metric_pin_error(sh):
    fm = grid.face_metrics(sh)
    an = grid.analytic_face_metrics(sh)
    return max(np.abs(fm[f"G{d}"] - an[f"G{d}"]).max() / np.abs(an[f"G{d}"][..., d]).max()
               for d in range(3))


def test_planted_metric_mistakes_are_caught(monkeypatch):
    sh = sh_of(16, **MAPS["triaxial_stretched"])
    good = _metric_pin_error(sh)
    orig = grid.face_jacobian

    def halved_normal(shh, d, i, j, k):      # 0.25 instead of 0.125 on the normal derivative
        M = orig(shh, d, i, j, k).copy()
        M[..., :, d] *= 2.0
        return M

    def transposed(shh, d, i, j, k):          # rows and columns of J^{-1} swapped
        return np.swapaxes(orig(shh, d, i, j, k), -1, -2)

    for bad in (halved_normal, transposed):
        monkeypatch.setattr(grid, "face_jacobian", bad)
        assert _metric_pin_error(sh) > 20 * good
        monkeypatch.setattr(grid, "face_jacobian", orig)


def test_planted_operator_mistakes_are_caught(monkeypatch):
    sh = sh_of(16, **MAPS["triaxial_stretched"])
    good = _interior_truncation(sh, "bump", 19)
    orig = operator._face_terms

    def flipped_cross(d, L, U, g, n, stencil, cut=False):   # wrong sign on the cross terms
        t = orig(d, L, U, g, n, stencil, cut)
        return t[:2] + [(c, -w) for c, w in t[2:]]

    def swapped_component(d, L, U, g, n, stencil, cut=False):  # G_pq from the wrong column
        return orig(d, L, U, g[..., ::-1], n, stencil, cut)

    for bad in (flipped_cross, swapped_component):
        monkeypatch.setattr(operator, "_face_terms", bad)
        assert _interior_truncation(sh, "bump", 19) > 4 * good
        monkeypatch.setattr(operator, "_face_terms", orig)


def test_two_cell_longitude_ring_is_rejected():
    """With nph = 2 the longitude-face normal derivative of Section 3.2
    differences one vertex plane against itself: the determinant is exactly
    zero, so such grids are refused rather than given an infinite metric."""
    with pytest.raises(ValueError):
        grid.Shell(8, 8, 2)
    with pytest.raises(ValueError):
        grid.Shell(8, 8, 6 + 1)
    assert grid.Shell(8, 8, 4).n == 256


# ------------------------------------------------------------------ Section 3.6 steps (Eqs. PC_6, PC_7)
from oracle import pc  # noqa: E402
import workloads as W  # noqa: E402

PC_GRIDS = {
    "sphere_stretched": (W.grid_desc(8, 8, 16, stretch=1.0), 7),
    "oblate": (W.grid_desc(6, 8, 12, r_out=1 / 0.6, mapping=1, flattening=0.1), 19),
    "triaxial": (W.grid_desc(8, 10, 16, mapping=2, flattening=0.1, e2=0.05, stretch=1.5), 19),
}


def _face_centres(sh, d):
    fj, fi, fk = np.meshgrid(*[np.arange(s) for s in pc.face_shapes(sh)[d]], indexing="ij")
    e = np.eye(3, dtype=int)
    t = [a for a in range(3) if a != d]
    acc = 0.0
    for a in (0, 1):
        for b in (0, 1):
            o = a * e[t[0]] + b * e[t[1]]
            acc = acc + grid.vertex(sh, fi + o[0], fj + o[1], fk + o[2])
    return acc / 4.0


@pytest.mark.parametrize("name", list(PC_GRIDS))
def test_uniform_flow_is_discretely_divergence_free(name):
    """Geometric conservation: the face C of Section 3.2 balance exactly, so a
    uniform Cartesian velocity has zero flux balance in every interior cell."""
    g, _ = PC_GRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    u = [np.broadcast_to(np.array([1.0, 0.5, -0.3]), s + (3,)).copy() for s in pc.face_shapes(sh)]
    D = pc.divergence(sh, fm, u)[1:-1, 1:-1, :]
    scale = max(np.abs(pc.contravariant_flux(sh, fm, u, d)).max() for d in range(3))
    assert np.abs(D).max() <= 1e-13 * scale


@pytest.mark.parametrize("name", ["sphere_stretched", "oblate"])
def test_rigid_rotation_is_discretely_divergence_free(name):
    """Rotation about the polar axis is tangential to every wall of an
    axisymmetric shell and solenoidal: its discrete divergence vanishes in all
    cells, walls included."""
    g, _ = PC_GRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    u = []
    for d in range(3):
        X = _face_centres(sh, d)
        u.append(np.stack([np.zeros(X.shape[:-1]), -X[..., 2], X[..., 1]], axis=-1))
    scale = max(np.abs(pc.contravariant_flux(sh, fm, u, d)).max() for d in range(3))
    assert np.abs(pc.divergence(sh, fm, u)).max() <= 1e-13 * scale


@pytest.mark.parametrize("name", list(PC_GRIDS))
def test_correction_removes_exactly_the_operator_flux(name):
    """D(U) - D(U corrected by x) equals A x for the assembled operator of
    Eqs. PC_8 / PC_term1-3 (7 or 19 points): the correction's face flux is the
    operator's face flux."""
    g, st = PC_GRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    rng = np.random.default_rng(3)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    x = rng.standard_normal(sh.n)
    Ax = operator.assemble(sh, fm, st) @ x
    lhs = (pc.divergence(sh, fm, u) - pc.divergence(sh, fm, pc.project(sh, fm, x, u, st))).ravel()
    np.testing.assert_allclose(lhs, Ax, rtol=0, atol=1e-13 * np.abs(Ax).max())


@pytest.mark.parametrize("name", list(PC_GRIDS))
def test_corrected_velocity_is_divergence_free(name):
    """The pressure-correction step: f = D(U***)/|J^{-1}|, solve for x = h dP,
    correct; the new field's divergence is the solver's residual."""
    g, st = PC_GRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    rng = np.random.default_rng(4)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    hier, fm2 = mg.setup(sh, st)
    x, info = mg.solve(sh, pc.rhs(sh, fm, u).ravel(), tol=1e-12, hier=hier, fm=fm2, max_iters=400)
    assert info["converged"]
    D0 = pc.divergence(sh, fm, u)
    D1 = pc.divergence(sh, fm, pc.project(sh, fm, x, u, st))
    assert np.linalg.norm(D1) <= 2e-12 * np.linalg.norm(D0)


def test_planted_smoother_mistakes_are_caught():
    """A reversed colour order and a wrong diagonal each break a smoother pin."""
    rng = np.random.default_rng(12)
    sh = grid.Shell(4, 6, 8, **MAPS["triaxial_stretched"])
    fm = grid.face_metrics(sh)
    x0, b = rng.standard_normal(sh.n), rng.standard_normal(sh.n)
    lv = mg.make_level(sh.shape, fm, 19)
    lv.colours, lv.colour_rows = lv.colours[::-1], lv.colour_rows[::-1]
    with pytest.raises(AssertionError):
        _check_block_gauss_seidel(lv, x0, b, 19, "reversed order")
    lv = mg.make_level(sh.shape, fm, 19)
    lv.D = lv.D * 1.1
    with pytest.raises(AssertionError):
        _check_block_gauss_seidel(lv, x0, b, 19, "wrong diagonal")


def test_planted_correction_mistakes_are_caught():
    """A transposed C, a dropped 1/|J^{-1}| or the cell instead of the face
    determinant breaks the flux identity; a C column for the flux breaks
    geometric conservation."""
    g, st = PC_GRIDS["triaxial"]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    rng = np.random.default_rng(5)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    x = rng.standard_normal(sh.n)
    Ax = operator.assemble(sh, fm, st) @ x

    def gap(fmx):
        lhs = (pc.divergence(sh, fm, u) - pc.divergence(sh, fm, pc.project(sh, fmx, x, u, st))).ravel()
        return np.abs(lhs - Ax).max() / np.abs(Ax).max()

    assert gap(fm) < 1e-13
    transposed = dict(fm, **{f"C{d}": np.swapaxes(fm[f"C{d}"], -1, -2) for d in range(3)})
    assert gap(transposed) > 1e-3
    no_det = dict(fm, **{f"det{d}": np.ones_like(fm[f"det{d}"]) for d in range(3)})
    assert gap(no_det) > 1e-3
    uu = [np.broadcast_to(np.array([1.0, 0.5, -0.3]), s + (3,)).copy() for s in pc.face_shapes(sh)]
    cols = dict(fm, **{f"C{d}": np.swapaxes(fm[f"C{d}"], -1, -2) for d in range(3)})
    D = pc.divergence(sh, cols, uu)[1:-1, 1:-1, :]
    assert np.abs(D).max() > 1e-6 * max(np.abs(pc.contravariant_flux(sh, fm, uu, d)).max() for d in range(3))


# ---------------------------------------------------------------- analytic metric option
@pytest.mark.parametrize("name", list(MAPS))
def test_analytic_metric_volumes_converge_second_order(name):
    """Cells from the exact face determinants (step 3 of Section 3.2) tile the
    closed-form shell volume to O(h^2), like the discrete metric."""
    errs = []
    for n in (8, 16, 32):
        sh = sh_of(n, **MAPS[name])
        fm = grid.face_metrics_analytic(sh)
        errs.append(abs(fm["J"].sum() - grid.shell_volume(sh)) / grid.shell_volume(sh))
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0, errs


def test_analytic_metric_keeps_the_operator_invariants():
    """A 1 = 0 and 1^T A = 0 hold for the operator on the analytic metric too
    (conservation does not depend on where the metric comes from)."""
    sh = sh_of(6, **MAPS["triaxial_stretched"])
    A = operator.assemble(sh, grid.face_metrics_analytic(sh), 19)
    one = np.ones(sh.n)
    scale = abs(A).sum(axis=1).max()
    assert np.abs(A @ one).max() < 1e-13 * scale
    assert np.abs(A.T @ one).max() < 1e-13 * scale


@pytest.mark.parametrize("name", ["oblate"])
def test_axisymmetric_mapping_has_no_longitude_cross_metric(name):
    """An axisymmetric map (the oblate shell) keeps the longitude direction
    orthogonal to the meridional plane face by face in the discrete metric of
    Section 3.2 too (the edge sums of step 1 are symmetric about the face's
    mid-longitude): G_r,phi and G_th,phi vanish to rounding, while G_r,th
    does not."""
    sh = sh_of(16, **MAPS[name])
    fm = grid.face_metrics(sh)
    scale = max(np.abs(fm[f"G{d}"][..., d]).max() for d in range(3))
    for arr, q in (("G0", 2), ("G1", 2), ("G2", 0), ("G2", 1)):
        assert np.abs(fm[arr][..., q]).max() < 1e-14 * scale, (arr, q)
    assert np.abs(fm["G0"][..., 1]).max() > 1e-3 * scale
