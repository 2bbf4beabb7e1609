"""The ADI-CN implicit viscous sweeps (Section 3.4, Eqs. solve_2 to solve_4)
on the GPU against the oracle.

Small grids (ragged sizes, 7- and 19-point metrics, the smallest longitude
ring) for every wall kind, compared value by value (FP64 on both sides:
1e-12 of the largest |u|); the 128 x 128 x 256 bench grid checked by
properties that hold at any size: with zero-flux walls the volume integral
sum J u changes by exactly sum src, a constant field with matching wall
values is steady, and kappa = 0 gives u^n + src / J.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adi, grid

pytestmark = pytest.mark.gpu

AGRIDS = {
    "sphere_stretched_ragged": W.grid_desc(10, 12, 20, stretch=2.0),
    "triaxial": W.grid_desc(8, 7, 12, mapping=2, flattening=0.1, e2=0.05, stretch=1.0),
    "oblate_nph4": W.grid_desc(6, 6, 4, r_out=1 / 0.6, mapping=1, flattening=0.1),
    # odd line lengths in radius and colatitude, six longitudes
    "sphere_odd": W.grid_desc(9, 5, 6, stretch=1.0),
}
WALLS = {
    "no_slip": (None, adi.walls()),
    "temperature": (dict(radius=1, colatitude=0, v_r_in=1.0, v_r_out=0.0),
                    adi.walls((adi.VALUE, 1.0, 0.0), (adi.FLUX0, 0, 0))),
    "values": (dict(radius=1, colatitude=1, v_r_in=0.3, v_r_out=-0.2, v_th0=0.5, v_th1=0.1),
               adi.walls((adi.VALUE, 0.3, -0.2), (adi.VALUE, 0.5, 0.1))),
    "flux0": (dict(radius=0, colatitude=0), adi.walls((adi.FLUX0, 0, 0), (adi.FLUX0, 0, 0))),
}


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("walls", list(WALLS))
@pytest.mark.parametrize("name", list(AGRIDS))
def test_substep_matches_oracle(lib, name, walls):
    import torch
    g = AGRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh)
    h = lib.mg_setup(g, dict(precision=1))
    rng = np.random.default_rng(50)
    un = rng.standard_normal(sh.shape)
    src = 0.1 * rng.standard_normal(sh.shape) * fm["J"]
    wg, wo = WALLS[walls]
    scale = np.abs(fm["G1"][..., 1]).max() / fm["J"].min()
    for kappa in (0.0, 0.3 / scale, 3.0 / scale):
        u = torch.empty(sh.shape, dtype=torch.float64, device="cuda")
        lib.mg_adi_substep(h, kappa, _dev(un), u, src=_dev(src), walls=wg)
        want = adi.substep(sh, fm, un, kappa, wo, src=src)
        np.testing.assert_allclose(u.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max(),
                                   err_msg=f"kappa {kappa}")


@pytest.mark.parametrize("name", list(AGRIDS))
def test_three_fields_share_the_matrix(lib, name):
    """Three fields in one call (one launch per sweep, shared rows and
    divisions) with their own wall values: each equals the oracle's sub-step
    of that field, and the single-field call gives the same bits."""
    import torch
    g = AGRIDS[name]
    sh = grid.shell(g)
    fm = grid.face_metrics(sh)
    h = lib.mg_setup(g, dict(precision=1))
    rng = np.random.default_rng(51)
    uns = [rng.standard_normal(sh.shape) for _ in range(3)]
    srcs = [0.1 * rng.standard_normal(sh.shape) * fm["J"] for _ in range(3)]
    vals = [(0.0, 0.0, 0.0, 0.0), (0.2, -0.1, 0.05, 0.3), (1.0, 0.0, -0.5, 0.5)]
    wg = [dict(radius=1, colatitude=1, v_r_in=a, v_r_out=b, v_th0=c, v_th1=d) for a, b, c, d in vals]
    kappa = 1.0 / (np.abs(fm["G1"][..., 1]).max() / fm["J"].min())
    outs = [torch.empty(sh.shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    lib.mg_adi_substep(h, kappa, [_dev(x) for x in uns], outs, src=[_dev(x) for x in srcs], walls=wg)
    for f in range(3):
        a, b, c, d = vals[f]
        want = adi.substep(sh, fm, uns[f], kappa, adi.walls((adi.VALUE, a, b), (adi.VALUE, c, d)), src=srcs[f])
        np.testing.assert_allclose(outs[f].cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())
        one = torch.empty_like(outs[f])
        lib.mg_adi_substep(h, kappa, _dev(uns[f]), one, src=_dev(srcs[f]), walls=wg[f])
        assert torch.equal(one, outs[f])
    # five fields: two launches of sweeps (four, then one)
    five = [torch.empty(sh.shape, dtype=torch.float64, device="cuda") for _ in range(5)]
    lib.mg_adi_substep(h, kappa, [_dev(uns[f % 3]) for f in range(5)], five)
    ref = torch.empty_like(five[0])
    lib.mg_adi_substep(h, kappa, _dev(uns[1]), ref)
    assert torch.equal(five[4], ref)


def test_substep_rejects_bad_arguments(lib):
    import torch
    g = AGRIDS["triaxial"]
    h = lib.mg_setup(g, dict(precision=1))
    n = g["nr"] * g["nth"] * g["nph"]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for kw in (dict(kappa=-1.0), dict(kappa=float("nan")), dict(walls=dict(radius=3))):
        with pytest.raises(lib.MGError) as e:
            lib.mg_adi_substep(h, kw.get("kappa", 1.0), x, x.clone(), walls=kw.get("walls"))
        assert e.value.status == lib.MG_EINVAL
    with pytest.raises(lib.MGError):
        lib.mg_adi_substep(h, 1.0, x, x)       # u aliasing un
    with pytest.raises(lib.MGError):          # wall kinds differ between fields
        lib.mg_adi_substep(h, 1.0, [x, x.clone()], [x.clone(), x.clone()],
                           walls=[dict(radius=1, colatitude=1), dict(radius=0, colatitude=1)])


def test_bench_size_properties(lib):
    import torch
    w = W.single("single_sphere_128")
    g = w["grid"]
    shape = (g["nr"], g["nth"], g["nph"])
    N = int(np.prod(shape))
    h = lib.mg_setup(g, dict(precision=1))
    J = torch.empty(N, dtype=torch.float64, device="cuda")
    lib.mg_get_metric(h, 0, 9, J)
    J = J.reshape(shape)
    gen = torch.Generator(device="cuda").manual_seed(7)
    un = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64)
    src = 0.01 * torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64) * J
    u = torch.empty_like(un)
    # a sub-step of diffusion number kappa G / J up to 10
    G = torch.empty(N, dtype=torch.float64, device="cuda")
    gmax = 0.0
    for comp in (0, 4, 8):
        lib.mg_get_metric(h, 0, comp, G)
        gmax = max(gmax, G.abs().max().item())
    kappa = 10.0 * J.min().item() / gmax
    # conservation with zero-flux walls (flux form telescopes)
    lib.mg_adi_substep(h, kappa, un, u, src=src, walls=dict(radius=0, colatitude=0))
    before = (J * un).sum().item() + src.sum().item()
    after = (J * u).sum().item()
    assert abs(after - before) <= 1e-11 * (J * un.abs()).sum().item()
    assert not torch.equal(u, un)
    # constant field, walls at the same value
    c = torch.full(shape, 0.25, dtype=torch.float64, device="cuda")
    lib.mg_adi_substep(h, kappa, c, u, walls=dict(radius=1, colatitude=1, v_r_in=0.25, v_r_out=0.25,
                                                 v_th0=0.25, v_th1=0.25))
    assert (u - 0.25).abs().max().item() <= 1e-13
    # no viscosity: u^n + src / J
    lib.mg_adi_substep(h, 0.0, un, u, src=src)
    assert (u - (un + src / J)).abs().max().item() <= 1e-14 * un.abs().max().item()
