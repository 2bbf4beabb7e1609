"""The steps either side of the pressure solve (Section 3.6) on the GPU.

Right side of Eq. PC_6 and correction of Eq. PC_7 for a staggered velocity
against the oracle (FP64 kernels: 1e-12 of the scale), and the whole
pressure-correction step (right side, solve, correction) removing the
divergence down to the solver's residual, on small grids and on the
128 x 128 x 256 bench workload.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, pc

pytestmark = pytest.mark.gpu

PC_GRIDS = {
    "sphere_stretched": W.grid_desc(8, 8, 16, stretch=1.0),
    "sphere_ragged": W.grid_desc(6, 10, 18, stretch=2.0),
    "oblate": W.grid_desc(6, 8, 12, r_out=1 / 0.6, mapping=1, flattening=0.1),
    "triaxial": W.grid_desc(8, 10, 16, mapping=2, flattening=0.1, e2=0.05, stretch=1.5),
}


def to_gpu_layout(sh, u):
    """Oracle face arrays (both wall planes) -> 9 blocks of the cells' lower faces."""
    blocks = [u[0][:, :-1, :, :], u[1][:-1, :, :, :], u[2]]
    return np.stack([blocks[d][..., a] for d in range(3) for a in range(3)]).ravel()


def from_gpu_layout(sh, flat, like):
    out = [v.copy() for v in like]
    b = flat.reshape(9, *sh.shape)
    for a in range(3):
        out[0][:, :-1, :, a] = b[0 + a]
        out[1][:-1, :, :, a] = b[3 + a]
        out[2][..., a] = b[6 + a]
    return out


def _setup(lib, g, **opts):
    sh = grid.shell(g)
    fm = grid.face_metrics(sh, with_C=True)
    st = 7 if g["mapping"] == 0 else 19
    h = lib.mg_setup(g, dict(precision=0, **opts))
    return sh, fm, st, h


@pytest.mark.parametrize("name", list(PC_GRIDS))
def test_rhs_and_correction_match_oracle(lib, name):
    import torch
    g = PC_GRIDS[name]
    sh, fm, st, h = _setup(lib, g)
    rng = np.random.default_rng(8)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    x = rng.standard_normal(sh.n)
    ud = torch.from_numpy(to_gpu_layout(sh, u)).cuda()
    fd = torch.empty(sh.n, dtype=torch.float64, device="cuda")
    lib.mg_pc_rhs(h, ud, fd)
    ref = pc.rhs(sh, fm, u).ravel()
    np.testing.assert_allclose(fd.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    lib.mg_pc_correct(h, torch.from_numpy(x).cuda(), ud)
    got = from_gpu_layout(sh, ud.cpu().numpy(), u)
    want = pc.project(sh, fm, x, u, st)
    for d in range(3):
        np.testing.assert_allclose(got[d], want[d], rtol=0, atol=1e-12 * np.abs(want[d]).max())
    # wall faces are left as they were
    np.testing.assert_array_equal(got[0][:, 0], u[0][:, 0])
    np.testing.assert_array_equal(got[1][0], u[1][0])


def _step(lib, h, sh, u_flat, tol):
    import torch
    ud = torch.from_numpy(u_flat).cuda()
    f0 = torch.empty(sh.n, dtype=torch.float64, device="cuda")
    lib.mg_pc_rhs(h, ud, f0)
    x = torch.zeros_like(f0)
    lib.mg_solve(h, f0, x, tol=tol)
    lib.mg_pc_correct(h, x, ud)
    f1 = torch.empty_like(f0)
    lib.mg_pc_rhs(h, ud, f1)
    return f0, f1, ud


@pytest.mark.parametrize("name", list(PC_GRIDS))
@pytest.mark.parametrize("prec", [0, 1])
def test_correction_step_removes_divergence(lib, name, prec):
    """Right side, solve to 1e-12, correct: the flux balance of the corrected
    field is the solver's residual."""
    g = PC_GRIDS[name]
    sh, fm, st, h = _setup(lib, g)
    h = lib.mg_setup(g, dict(precision=prec))
    J = fm["J"].ravel()
    rng = np.random.default_rng(9)
    u = [rng.standard_normal(s + (3,)) for s in pc.face_shapes(sh)]
    f0, f1, _ = _step(lib, h, sh, to_gpu_layout(sh, u), 1e-12)
    d0 = np.linalg.norm(J * f0.cpu().numpy())
    d1 = np.linalg.norm(J * f1.cpu().numpy())
    assert d1 <= 5e-12 * d0, (d1, d0)


def test_correction_step_at_bench_size(lib):
    """The 128 x 128 x 256 stretched sphere (bench workload, FP32-IR to 1e-10):
    the divergence drops to the solve tolerance."""
    g = W.grid_desc(128, stretch=2.0)
    sh = grid.shell(g)
    h = lib.mg_setup(g, dict(precision=1))
    rng = np.random.default_rng(10)
    u_flat = rng.standard_normal(9 * sh.n)
    f0, f1, _ = _step(lib, h, sh, u_flat, 1e-10)
    import torch
    Jd = torch.empty(sh.n, dtype=torch.float64, device="cuda")
    lib.mg_get_metric(h, 0, 9, Jd)
    d0 = torch.linalg.norm(Jd * f0).item()
    d1 = torch.linalg.norm(Jd * f1).item()
    assert d1 <= 2e-10 * d0, (d1, d0)
