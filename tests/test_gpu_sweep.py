"""One-pass multicolour Gauss-Seidel sweeps (all colours in one launch, the
iterate staged plane by plane in shared memory) against the oracle's
sequential colour sweep, and bit for bit against the colour-pass kernels.

The operator is that of Eqs. PC_8 and PC_term1-3 (Section 3.3); the colour
orders are red/black by (i + j + k) mod 2 for 7 points and the four colours
((i + j) mod 2) + 2 ((j + k) mod 2) for 19 points.  Tile shapes are forced
through MG_TILE ("cells,planes,kmax"): whole longitude rows, tiles narrower
than the grid (both longitude seams), chunks of one to three planes, ragged
last tiles in every direction; grids with odd counts, stretched radii, the
axisymmetric 19-point operator and the full one.  The 7-point sweep of the
FP32 and FP16-coefficient cycles (whole rows, one thread per four
longitudes, x, b and the face coefficients staged by bulk copies) takes its
rows from the plane area (cells / nph, at least one) and the chunk depth
from MG_TILE.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, mg as omg

pytestmark = pytest.mark.gpu

GRIDS = {
    "sphere_ragged": W.grid_desc(6, 20, 96),
    "sphere_stretched": W.grid_desc(12, 21, 72, stretch=2.0),
    "sphere_wide": W.grid_desc(5, 9, 320, stretch=1.0),          # wider than one copy: longitude tiles
    "oblate": W.grid_desc(10, 12, 32, r_out=1 / 0.6, mapping=1, flattening=0.1, stretch=1.5),
    "oblate_odd": W.grid_desc(7, 9, 48, r_out=1 / 0.6, mapping=1, flattening=0.1),
    "triaxial": W.grid_desc(6, 11, 24, mapping=2, flattening=0.1, e2=0.05, stretch=1.0),
}
TILES = {
    "default": None,
    "small_shallow": "64,1,256",      # four rows, one plane per chunk
    "narrow": "128,3,16",             # 16-longitude tiles: seams on both sides
    "mid": "512,2,32",
}
TOL = {0: 1e-12, 1: 1e-5, 2: 3e-3}


def _torch():
    import torch
    return torch, torch.device("cuda:0")


def _dev(a, prec):
    torch, dev = _torch()
    dt = torch.float64 if prec == 0 else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dt)


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64).ravel()


def _stencil(g):
    return 7 if g["mapping"] == 0 else 19


def _sweep(lib, g, prec, x0, b, sweeps, tile, monkeypatch, one_pass=True, level=0):
    monkeypatch.delenv("MG_TILE", raising=False)
    monkeypatch.delenv("MG_FUSED_RB", raising=False)
    if one_pass:
        monkeypatch.setenv("MG_FUSED_RB", "1")
        if tile:
            monkeypatch.setenv("MG_TILE", tile)
    h = lib.mg_setup(g, dict(precision=prec, coarse_max=64))
    sc = lib.mg_get_schedule(h)
    xd, bd = _dev(x0, prec), _dev(b, prec)
    lib.mg_smooth(h, level, prec, xd, bd, sweeps, 0)
    h.close()
    return _np(xd), sc


@pytest.mark.parametrize("tile", list(TILES))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(GRIDS))
def test_one_pass_sweep_matches_oracle(lib, name, prec, tile, monkeypatch):
    g = GRIDS[name]
    st = _stencil(g)
    fm = grid.face_metrics(grid.shell(g))
    lv = omg.make_level(grid.shell(g).shape, fm, st)
    rng = np.random.default_rng(77)
    x0 = rng.standard_normal(lv.n)
    b = rng.standard_normal(lv.n) * np.abs(lv.D)
    for sweeps in (1, 2, 3):
        x, sc = _sweep(lib, g, prec, x0, b, sweeps, TILES[tile], monkeypatch)
        assert sc["one_pass_tiles"] == 1, sc
        # the 7-point FP32 / FP16 sweep takes whole rows of at most 256
        # longitudes; wider grids keep the colour passes
        assert sc["tile0"][0] > 0 or (st == 7 and prec != 0 and g["nph"] > 256), sc
        ref = omg.smooth(lv, _np(_dev(x0, prec)), _np(_dev(b, prec)), sweeps, omg.GS)
        np.testing.assert_allclose(x, ref, rtol=0, atol=TOL[prec] * np.abs(ref).max(),
                                   err_msg=f"{sweeps} sweeps, tile {sc['tile0']}")


@pytest.mark.parametrize("tile", list(TILES))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("name", list(GRIDS))
def test_one_pass_sweep_is_the_colour_passes_bit_for_bit(lib, name, prec, tile, monkeypatch):
    """Same per-cell arithmetic and neighbour values: the one-pass sweep and
    the C colour-pass launches give the same bits, on every level."""
    g = GRIDS[name]
    h = lib.mg_setup(g, dict(precision=prec, coarse_max=64))
    levels = lib.mg_get_level_info(h, 0)["levels"]
    shapes = [lib.mg_get_level_info(h, l) for l in range(levels)]
    h.close()
    rng = np.random.default_rng(5)
    for l in range(levels - 1):
        n = shapes[l]["nr"] * shapes[l]["nth"] * shapes[l]["nph"]
        x0, b = rng.standard_normal(n), rng.standard_normal(n)
        a, sc = _sweep(lib, g, prec, x0, b, 2, TILES[tile], monkeypatch, True, l)
        c, _ = _sweep(lib, g, prec, x0, b, 2, None, monkeypatch, False, l)
        assert np.array_equal(a, c), f"level {l} {shapes[l]}"


def test_one_pass_sweep_covers_the_bench_shapes(lib, monkeypatch):
    """The fine levels of the 128 x 128 x 256 sphere and the 256 x 256 x 512
    oblate shell take one-pass tiles (at half size here)."""
    for wl, st in (("single_sphere_128", 7), ("single_oblate_256", 19)):
        w = W.single(wl, 2)
        monkeypatch.setenv("MG_FUSED_RB", "1")
        h = lib.mg_setup(w["grid"], dict(precision=1))
        sc = lib.mg_get_schedule(h)
        assert sc["one_pass_tiles"] == 1 and min(sc["tile0"]) > 0, (wl, sc)
        h.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_red_black_sweep_at_full_size_is_the_colour_passes(lib, prec, monkeypatch):
    """The 128 x 128 x 256 sphere's two finest levels in the automatic tile
    shape (the one the solves use): one-pass sweeps bit for bit the colour
    passes, and the tile is whole rows."""
    g = W.single("single_sphere_128", 1)["grid"]
    rng = np.random.default_rng(11)
    for level in (0, 1):
        h = lib.mg_setup(g, dict(precision=1))
        info = lib.mg_get_level_info(h, level)
        h.close()
        n = info["nr"] * info["nth"] * info["nph"]
        x0, b = rng.standard_normal(n), rng.standard_normal(n)
        a, sc = _sweep(lib, g, prec, x0, b, 2, None, monkeypatch, True, level)
        c, _ = _sweep(lib, g, prec, x0, b, 2, None, monkeypatch, False, level)
        if level == 0:
            assert sc["tile0"][2] == g["nph"] and sc["tile0"][0] >= 1, sc
        assert np.array_equal(a, c), f"level {level}"
