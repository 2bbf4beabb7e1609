"""Pins of the oracle's full sphere (shell cut) and semi-coarsening multigrid.

Full sphere (Sections 3.5 and 3.7, shell cut): the checks tie the cut to the
mapping's own geometry (the cell across a pole is where the mapping puts the
point beyond the pole), to exact invariants of the conservative operator, to
the reflection symmetry of the sphere through its equator, to the closed-form
volume and to manufactured solutions regular at the poles.

Semi-coarsening multigrid with plane relaxation (Section 3.6's solver class):
the plane relaxation is checked to be an exact block solve, the solver
against the bordered direct solve, and its robustness where point smoothing
degrades.  Planted mistakes at the end show that each pin fails on them.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import grid, operator, mg, smg, direct, mms

MAPS = {
    "sphere": dict(mapping=0),
    "oblate": dict(mapping=1, flattening=0.1, r_out=1 / 0.6),
    "triaxial_stretched": dict(mapping=2, flattening=0.1, e2=0.05, stretch=2.0),
}


def sphere_of(n, **kw):
    return grid.full_sphere(n, n, 2 * n, **kw)


def stencil_of(name):
    return 7 if name == "sphere" else 19


# ---------------------------------------------------------------- grid and metric
def test_cut_needs_the_full_colatitude_range():
    with pytest.raises(ValueError):
        grid.Shell(4, 4, 8, cut=True)
    assert grid.full_sphere(4, 4, 8).cut


@pytest.mark.parametrize("name", list(MAPS))
def test_full_sphere_volume_second_order(name):
    """Sum of the cell |J^{-1}| -> 4/3 pi (r_out^3 - r_in^3)(1 - fl)(1 + e2)."""
    errs = []
    for n in (8, 16, 32):
        sh = sphere_of(n, **MAPS[name])
        fm = grid.face_metrics(sh)
        assert all(np.isfinite(v).all() for v in fm.values())
        errs.append(abs(fm["J"].sum() / grid.shell_volume(sh) - 1))
    fl = MAPS[name].get("flattening", 0.0)
    e2 = MAPS[name].get("e2", 0.0) if MAPS[name]["mapping"] == 2 else 0.0
    r_out = MAPS[name].get("r_out", 2.0)
    assert grid.shell_volume(sphere_of(8, **MAPS[name])) == pytest.approx(
        4.0 / 3.0 * np.pi * (r_out ** 3 - 1.0) * (1 - fl) * (1 + e2), rel=1e-14)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.7


@pytest.mark.parametrize("name", list(MAPS))
def test_pole_faces_are_degenerate_and_carry_no_flux(name):
    """The zeta faces on the polar axis have (numerically) zero determinant
    straight from the vertex stencil; the metric zeroes exactly those."""
    sh = sphere_of(6, **MAPS[name])
    fm = grid.face_metrics(sh)
    jj, kk = np.meshgrid(np.arange(sh.nr), np.arange(sh.nph), indexing="ij")
    typical = np.median(fm["det0"][:, 1:-1])
    for i in (0, sh.nth):
        with np.errstate(divide="ignore", invalid="ignore"):
            adet, _, _ = grid.metric_from_jacobian(grid.face_jacobian(sh, 0, np.full_like(jj, i), jj, kk))
        assert adet.max() < 1e-12 * typical
        assert not fm["G0"][:, i].any() and not fm["det0"][:, i].any()
    assert (fm["det0"][:, 1:-1] > 0.01 * typical).all()


@pytest.mark.parametrize("name", list(MAPS))
def test_cell_across_the_pole_is_where_the_mapping_puts_it(name):
    """The operator's neighbour one row beyond a pole is the cell whose centre
    the mapping gives for the computational point half a cell beyond the pole."""
    sh = sphere_of(6, **MAPS[name])
    n = (sh.nth, sh.nr, sh.nph)
    jj, kk = np.meshgrid(np.arange(sh.nr), np.arange(sh.nph), indexing="ij")
    for i, s in ((0, -1), (sh.nth - 1, +1)):
        ii = np.full_like(jj, i)
        i2, j2, k2 = operator._shift((ii, jj, kk), 0, s, n, cut=True)
        want = grid.vertex(sh, i + s + 0.5, jj + 0.5, kk + 0.5)
        got = grid.vertex(sh, i2 + 0.5, j2 + 0.5, k2 + 0.5)
        np.testing.assert_allclose(got, want, atol=1e-13)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("name", list(MAPS))
@pytest.mark.parametrize("stencil", [7, 19])
def test_cut_operator_invariants(name, stencil):
    sh = sphere_of(6, **MAPS[name])
    A = operator.assemble(sh, grid.face_metrics(sh), stencil)
    one = np.ones(sh.n)
    scale = abs(A).max()
    assert np.abs(A @ one).max() < 1e-13 * scale
    assert np.abs(A.T @ one).max() < 1e-13 * scale
    if stencil == 7:
        assert abs(A - A.T).max() == 0.0
    ev = np.linalg.eigvalsh(((A + A.T) / 2).toarray())
    assert ev.max() < 1e-12 * scale
    assert np.sum(ev > -1e-10 * scale) == 1


def _equator_reflection(sh):
    """Cell permutation of the reflection x1 -> -x1 (theta -> pi - theta)."""
    j, i, k = np.meshgrid(np.arange(sh.nr), np.arange(sh.nth), np.arange(sh.nph), indexing="ij")
    return ((j * sh.nth + (sh.nth - 1 - i)) * sh.nph + k).ravel()


def _reflection_defect(sh, stencil):
    A = operator.assemble(sh, grid.face_metrics(sh), stencil).tocsr()
    s = _equator_reflection(sh)
    return abs(A[s][:, s] - A).max() / abs(A).max()


@pytest.mark.parametrize("name", list(MAPS))
def test_cut_operator_commutes_with_the_equator_reflection(name):
    """Every mapping here is symmetric under x1 -> -x1, so the operator must
    commute with the row reversal: the two poles' cuts agree."""
    sh = sphere_of(6, **MAPS[name])
    assert _reflection_defect(sh, stencil_of(name)) < 1e-13
    assert _reflection_defect(sh, 19) < 1e-13


@pytest.mark.parametrize("name", list(MAPS))
def test_cut_sampled_rows_match_assembly(name):
    sh = sphere_of(4, **MAPS[name])
    A = operator.assemble(sh, grid.face_metrics(sh), 19)
    x = np.random.default_rng(3).standard_normal(sh.n)
    cells = np.unravel_index(np.arange(sh.n), sh.shape)
    y = operator.apply_rows(sh, x, cells, 19)
    np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-13 * abs(A).max() * np.abs(x).max())


@pytest.mark.parametrize("name", ["sphere", "triaxial_stretched"])
def test_full_sphere_solution_converges_second_order(name):
    """Manufactured p regular through both poles (mms ``polar``): the discrete
    solution's error falls like h^2."""
    errs = []
    for n in (4, 8, 16):
        sh = sphere_of(n, **MAPS[name])
        fm = grid.face_metrics(sh)
        A = operator.assemble(sh, fm, stencil_of(name))
        p, lap = mms.manufactured(sh, "polar")
        J = fm["J"].ravel()
        b, _ = mg.prepare_rhs(J, lap.ravel())
        x, _ = direct.bordered_solve(A, b, J)
        pe = mg.gauge(J, p.ravel())
        errs.append(np.abs(x - pe).max() / np.abs(pe).max())
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.7


@pytest.mark.parametrize("name", ["sphere", "triaxial_stretched"])
def test_full_sphere_correction_is_divergence_free(name):
    """Eq. PC_7 on the full sphere: the face gradient across the pole is the
    operator's, so the corrected field's divergence is the (zero) residual."""
    from oracle import pc
    sh = sphere_of(6, **MAPS[name])
    fm = grid.face_metrics(sh, with_C=True)
    rng = np.random.default_rng(4)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    D0 = pc.divergence(sh, fm, u)
    A = operator.assemble(sh, fm, stencil_of(name))
    J = fm["J"].ravel()
    b, _ = mg.prepare_rhs(J, pc.rhs(sh, fm, u).ravel())
    x, _ = direct.bordered_solve(A, b, J)
    D1 = pc.divergence(sh, fm, pc.project(sh, fm, x, u, stencil_of(name)))
    assert np.linalg.norm(D1) <= 1e-11 * np.linalg.norm(D0)


def test_full_sphere_zeta_sweep_is_the_merged_cut_system():
    """Section 3.5 merges the zeta line at longitude k with the line at
    k + nph/2 (run backwards) into one system of twice the length.  With the
    zero-area pole faces the merged system's couplings across the poles are
    zero: solving it whole gives the implicit zeta sweep of the two lines,
    and any wall value at the poles has no effect."""
    from oracle import adi, tridiag
    sh = sphere_of(6, **MAPS["sphere"])
    fm = grid.face_metrics(sh)
    rng = np.random.default_rng(9)
    rhs = rng.standard_normal(sh.shape)
    kappa = 0.3 * fm["J"].min() / np.abs(fm["G1"][..., 1]).max()
    got = adi.sweep(sh, fm, 0, kappa, rhs, adi.walls(colatitude=(adi.VALUE, 5.0, -3.0)))
    got0 = adi.sweep(sh, fm, 0, kappa, rhs, adi.walls(colatitude=(adi.FLUX0, 0.0, 0.0)))
    np.testing.assert_array_equal(got, got0)
    a, b, c, w = adi.line_system(sh, fm, 0, kappa, adi.walls())
    n, h = sh.nth, sh.nph // 2
    for j in range(sh.nr):
        for k in range(h):
            # merged line: line k + h from the south pole up to the north pole,
            # across it, then line k down to the south pole
            idx = [(i, k + h) for i in range(n - 1, -1, -1)] + [(i, k) for i in range(n)]
            A = np.zeros(2 * n)
            B = np.zeros(2 * n)
            Cc = np.zeros(2 * n)
            g = np.zeros(2 * n)
            for m, (i, kk) in enumerate(idx):
                # reversed part: lower and upper neighbours swap
                lo, up = (c[i, j, kk], a[i, j, kk]) if m < n else (a[i, j, kk], c[i, j, kk])
                A[m], B[m], Cc[m], g[m] = lo, b[i, j, kk], up, rhs[j, i, kk]
            # the joint between the two halves is the pole face: zero coupling
            assert A[n] == 0.0 and Cc[n - 1] == 0.0
            x = tridiag.thomas(A, B, Cc, g)
            want = np.array([got[j, i, kk] for (i, kk) in idx])
            np.testing.assert_allclose(x, want, rtol=0, atol=1e-13 * np.abs(want).max())


# ---------------------------------------------------------------- multigrid on the cut
def _prolongation_defect(nr, nth, nph):
    """Largest error of P on a coarse field linear in the colatitude measured
    through each pole: theta cos(phi) near theta = 0 (exact on all fine rows but
    the last two), (pi - theta) cos(phi) near theta = pi (all but the first two)."""
    _, P = mg.transfer_matrices((nr, nth, nph), (2, 1, 1), cut=True)
    dth = np.pi / nth
    thc = (np.arange(nth // 2) + 0.5) * 2 * dth
    thf = (np.arange(nth) + 0.5) * dth
    phi = (np.arange(nph) + 0.5) * 2 * np.pi / nph
    worst = 0.0
    for g, keep in ((lambda t: t, slice(0, nth - 2)), (lambda t: np.pi - t, slice(2, nth))):
        ec = np.broadcast_to(g(thc)[None, :, None] * np.cos(phi)[None, None, :], (nr, nth // 2, nph))
        ef = (P @ ec.ravel()).reshape(nr, nth, nph)
        want = g(thf)[None, :, None] * np.cos(phi)[None, None, :]
        worst = max(worst, np.abs(ef - want)[:, keep].max())
    return worst


def test_prolongation_across_the_pole_is_linear_in_colatitude():
    assert _prolongation_defect(2, 8, 8) < 1e-14
    for c in ((2, 2, 2), (2, 1, 2), (1, 2, 2), (2, 2, 1)):
        _, P = mg.transfer_matrices((4, 8, 16), c, cut=True)
        np.testing.assert_allclose(P @ np.ones(P.shape[1]), 1.0, rtol=0, atol=1e-15)
        _, Pw = mg.transfer_matrices((4, 8, 16), c, cut=False)
        # away from the poles the cut changes nothing
        rows = (np.arange(P.shape[0]).reshape(4, 8, 16)[:, 1:-1, :]).ravel()
        assert abs(P[rows] - Pw[rows]).max() == 0.0


def _same_colour_coupling(sh):
    A = operator.assemble(sh, grid.face_metrics(sh), 19).tocoo()
    col = mg.colour_of(sh.shape, 19)
    same = (A.row != A.col) & (col[A.row] == col[A.col])
    return (np.abs(A.data[same]).max() if same.any() else 0.0) / np.abs(A.data).max()


def test_four_colours_across_the_cut():
    """The 4-colour sweep stays an independent-set colouring on the cut rows
    for an axisymmetric mapping with nph/2 odd, and only then."""
    assert _same_colour_coupling(grid.full_sphere(4, 6, 14, **MAPS["oblate"])) < 1e-14
    assert _same_colour_coupling(grid.full_sphere(4, 6, 12, **MAPS["oblate"])) > 1e-5
    assert _same_colour_coupling(grid.full_sphere(4, 6, 14, **MAPS["triaxial_stretched"])) > 1e-5
    assert _same_colour_coupling(grid.Shell(4, 6, 12, **MAPS["triaxial_stretched"])) < 1e-14


@pytest.mark.parametrize("name", list(MAPS))
def test_multigrid_on_the_cut_matches_direct_solve(name):
    sh = sphere_of(8, **MAPS[name])
    f = np.random.default_rng(5).standard_normal(sh.n)
    hier, fm = mg.setup(sh, stencil_of(name))
    x, info = mg.solve(sh, f, tol=1e-12, hier=hier, fm=fm)
    assert info["converged"]
    J = fm["J"].ravel()
    b, _ = mg.prepare_rhs(J, f)
    xd, _ = direct.bordered_solve(hier.levels[0].A, b, J)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-9 * np.abs(xd).max())


# ---------------------------------------------------------------- semi-coarsening multigrid
def test_plane_relaxation_is_an_exact_block_solve():
    """After a zebra sweep the residual vanishes on the planes relaxed last."""
    sh = sphere_of(8, **MAPS["triaxial_stretched"])
    hier, fm = smg.setup(sh, 19)
    lv = hier.levels[0]
    rng = np.random.default_rng(7)
    b = rng.standard_normal(sh.n)
    b -= b.mean()
    x = hier.relax(lv, rng.standard_normal(sh.n), b)
    r = (b - lv.A @ x).reshape(sh.shape)
    assert np.abs(r[:, 1::2, :]).max() < 1e-12 * np.abs(b).max()
    assert np.abs(r[:, 0::2, :]).max() > 1e-3 * np.abs(b).max()


def _plane_contraction(sh, stencil, i, cycles=6):
    hier, _ = smg.setup(sh, stencil)
    lv = hier.levels[0]
    B = lv.plane_block(i).tocsr()
    ph = smg.PlaneHierarchy(B, lv.shape[0], lv.shape[2])
    r = np.random.default_rng(0).standard_normal(B.shape[0])
    xe = spla.spsolve(B.tocsc(), r)
    e = np.zeros_like(r)
    errs = []
    for _ in range(cycles):
        e = ph.cycle(0, e, r)
        errs.append(np.abs(e - xe).max() / np.abs(xe).max())
    return (errs[-1] / errs[0]) ** (1.0 / (cycles - 1))


def test_plane_cycle_contracts_toward_the_plane_solve():
    """One cycle of the 2-D construction (eta semi-coarsening, zebra xi-lines
    by the periodic Thomas algorithm) cuts the plane error by > 3x, on a
    thin stretched shell and on the pole row of the cut sphere."""
    assert _plane_contraction(grid.Shell(32, 8, 32, r_out=1.05, stretch=2.0), 7, 4) < 0.3
    assert _plane_contraction(sphere_of(16, **MAPS["triaxial_stretched"]), 19, 0) < 0.3


@pytest.mark.parametrize("sh,stencil", [
    (grid.full_sphere(8, 8, 16), 7),
    (grid.full_sphere(8, 8, 16, **MAPS["oblate"]), 19),
    (grid.Shell(8, 8, 16, **MAPS["triaxial_stretched"]), 19),
    (grid.Shell(8, 6, 16, r_out=1.05, stretch=2.0), 7),
])
@pytest.mark.parametrize("planes", [smg.EXACT, 1])
def test_smg_matches_direct_solve(sh, stencil, planes):
    f = np.random.default_rng(11).standard_normal(sh.n)
    hier, fm = smg.setup(sh, stencil)
    x, info = smg.solve(sh, f, tol=1e-12, hier=hier, fm=fm, plane_cycles=planes)
    assert info["converged"] and info["iters"] <= 15
    J = fm["J"].ravel()
    b, _ = mg.prepare_rhs(J, f)
    xd, _ = direct.bordered_solve(hier.levels[0].A, b, J)
    np.testing.assert_allclose(x, xd, rtol=0, atol=1e-9 * np.abs(xd).max())


def test_smg_is_robust_where_point_smoothing_degrades():
    """Thin, stretched shell: point Gauss-Seidel multigrid slows down, plane
    relaxation with semi-coarsening keeps its rate."""
    sh = grid.Shell(16, 16, 32, r_out=1.05, stretch=2.0)
    f = np.random.default_rng(2).standard_normal(sh.n)
    _, i_smg = smg.solve(sh, f, tol=1e-10, stencil=7)
    _, i_mg = mg.solve(sh, f, tol=1e-10, stencil=7)
    assert i_smg["converged"] and i_smg["iters"] <= 14
    assert i_mg["iters"] >= 2 * i_smg["iters"]


# ---------------------------------------------------------------- planted mistakes
def test_planted_cut_mistakes_are_caught(monkeypatch):
    sh = sphere_of(6, **MAPS["oblate"])
    n = (sh.nth, sh.nr, sh.nph)
    jj, kk = np.meshgrid(np.arange(sh.nr), np.arange(sh.nph), indexing="ij")
    orig = operator._shift

    def quarter_turn(idx, q, s, n, cut=False):          # wrong longitude offset
        out = list(orig(idx, q, s, n, cut))
        if q == 0 and cut:
            across = (idx[0] + s < 0) | (idx[0] + s > n[0] - 1)
            out[2] = np.where(across, np.mod(idx[2] + n[2] // 4, n[2]), out[2])
        return tuple(out)

    def north_only(idx, q, s, n, cut=False):            # south pole mirrored instead
        return orig(idx, q, s, n, cut and bool(np.all(np.asarray(idx[0]) + s <= n[0] - 1)))

    def mirror(idx, q, s, n, cut=False):                # the walls' ghost at the poles
        return orig(idx, q, s, n, False)

    i, s = 0, -1
    want = grid.vertex(sh, i + s + 0.5, jj + 0.5, kk + 0.5)
    for bad in (quarter_turn, mirror):
        i2, j2, k2 = bad((np.full_like(jj, i), jj, kk), 0, s, n, cut=True)
        assert np.abs(grid.vertex(sh, i2 + 0.5, j2 + 0.5, k2 + 0.5) - want).max() > 0.1
    monkeypatch.setattr(operator, "_shift", north_only)
    assert _reflection_defect(sh, 19) > 1e-6
    monkeypatch.setattr(operator, "_shift", orig)

    origP = mg._prolong_sphere_plane

    def mirrored_plane(nct, ncp, cz, cx):
        import scipy.sparse as sp
        return sp.kron(mg._prolong_1d(nct, cz, False), mg._prolong_1d(ncp, cx, True)).tocsr()

    monkeypatch.setattr(mg, "_prolong_sphere_plane", mirrored_plane)
    assert _prolongation_defect(2, 8, 8) > 0.1
    monkeypatch.setattr(mg, "_prolong_sphere_plane", origP)


def test_planted_plane_cycle_mistake_is_caught(monkeypatch):
    """A coarse plane operator without the 1/2 of the coarsened direction
    (R B R^T) loses the plane cycle's rate."""
    import scipy.sparse as sp
    orig = smg._coarsen_rows_2d

    def doubled(B, nr, nph):
        R = sp.kron(smg._children(nr // 2), sp.identity(nph)).tocsr()
        P = sp.kron(smg._prolong_eta(nr // 2), sp.identity(nph)).tocsr()
        return (R @ B @ R.T).tocsr(), R, P

    monkeypatch.setattr(smg, "_coarsen_rows_2d", doubled)
    assert _plane_contraction(grid.Shell(32, 8, 32, r_out=1.05, stretch=2.0), 7, 4) > 0.5
    monkeypatch.setattr(smg, "_coarsen_rows_2d", orig)
