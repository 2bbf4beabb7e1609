"""Full-size solves, in the launch configuration the benchmark times, checked
against the oracle on sampled cells.

The grids are the 128 x 128 x 256 stretched sphere (7-point), the
256 x 256 x 512 oblate shell (19-point) and the 128 x 128 x 256 thin shell
(radius 1 to 1.05), with point and radial-line Gauss-Seidel.  The oracle cannot solve them, so
the check is on properties it can evaluate one cell at a time:

* the relative residual ||b - A x|| / ||b|| estimated from 32768 random cells,
  with A x from the oracle's on-demand face metric (``apply_rows``) and b from
  the oracle's cell volumes: below 1e-10 up to sampling error (factor 2);
* the removed mean equals the oracle's J-weighted mean of f;
* the answer has zero J-weighted mean.

Both mappings are axisymmetric about the polar axis and the longitude grid is
uniform, so |J^{-1}| does not depend on the longitude index: the oracle
computes one longitude plane of cell volumes and the test checks that
symmetry on sampled cells before using it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import grid, operator

pytestmark = pytest.mark.gpu

CASES = [("single_sphere_128", 1, 0), ("single_oblate_256", 1, 0), ("single_oblate_256", 2, 0),
         ("single_sphere_128", 1, 2), ("single_thin_128", 1, 2), ("single_thin_128", 1, 0)]


def _volumes(g):
    sh = grid.shell(g)
    j, i = np.meshgrid(np.arange(sh.nr), np.arange(sh.nth), indexing="ij")
    plane = grid.cell_volume_at(sh, (j.ravel(), i.ravel(), np.zeros(j.size, dtype=np.int64)))
    plane = plane.reshape(sh.nr, sh.nth)
    rng = np.random.default_rng(5)
    js, is_, ks = rng.integers(0, sh.nr, 64), rng.integers(0, sh.nth, 64), rng.integers(0, sh.nph, 64)
    np.testing.assert_allclose(grid.cell_volume_at(sh, (js, is_, ks)), plane[js, is_], rtol=1e-12)
    return plane


_W = {}


def _workload(name):
    if name not in _W:
        _W[name] = W.single(name)
    return _W[name]


@pytest.mark.parametrize("wl,prec,smoother", CASES)
def test_full_size_solve_sampled_against_oracle(lib, wl, prec, smoother):
    import torch
    w = _workload(wl)
    g, f = w["grid"], w["f"]
    sh = grid.shell(g)
    stencil = 7 if g["mapping"] == 0 else 19
    h = lib.mg_setup(g, dict(precision=prec, smoother=smoother))
    fd = torch.from_numpy(f).to("cuda:0")
    xd = torch.zeros_like(fd)
    rep = lib.mg_solve(h, fd, xd, tol=1e-10)
    assert rep["status"] == "MG_OK" and rep["rel_res"] <= 1e-10
    x = xd.cpu().numpy()
    del fd, xd
    h.close()
    torch.cuda.empty_cache()

    Jp = _volumes(g)                                   # [nr][nth], same for every k
    wsum = Jp.sum() * sh.nph
    mean = float((Jp[:, :, None] * f).sum() / wsum)
    assert abs(rep["removed_mean"] - mean) <= 1e-12 * max(1.0, np.abs(f).max())
    assert abs((Jp[:, :, None] * x).sum()) <= 1e-12 * (Jp[:, :, None] * np.abs(x)).sum()

    rng = np.random.default_rng(11)
    m = 32768
    cells = (rng.integers(0, sh.nr, m), rng.integers(0, sh.nth, m), rng.integers(0, sh.nph, m))
    b = Jp[cells[0], cells[1]] * (f[cells] - mean)
    r = b - operator.apply_rows(sh, x, cells, stencil)
    rel = np.sqrt(np.mean(r ** 2) / np.mean(b ** 2))
    assert rel <= 2e-10, rel
