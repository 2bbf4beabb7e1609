"""The allocation-free right-hand-side projection.

Callers that cannot allocate device memory when they need the step (inside a
stream capture, in an allocation-free time loop, or when another pool owns
the GPU) call mg_project_rhs_noalloc, whose reduction scratch is a static
device array.  Its results must match what the allocating solve computes:
the J-weighted mean that mg_solve reports as removed_mean, and
b = J (f - mean) with the cell volumes J that mg_get_metric returns.  Two
calls in a row check that the shared scratch carries nothing over.  This file
is collected last so a stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", [W.grid_desc(16, mapping=1, flattening=0.1, r_out=1 / 0.6),
                                  W.grid_desc(128, stretch=2.0)])
def test_noalloc_projection_matches_allocating_solve(lib, grid):
    import torch
    g = grid
    n = g["nr"] * g["nth"] * g["nph"]
    h = lib.mg_setup(g, dict(precision=1))
    f = torch.from_numpy(W.rhs_modes(g, seed=7) + 0.37).to("cuda:0")
    x = torch.zeros_like(f)
    rep = lib.mg_solve(h, f, x, tol=1e-8)
    J = torch.empty(n, dtype=torch.float64, device="cuda:0")
    lib.mg_get_metric(h, 0, 9, J)
    ref_mean = rep["removed_mean"]
    ref_b = (J * (f.reshape(-1) - ref_mean)).cpu().numpy()
    for call in range(2):                      # the second call reuses the scratch
        b = torch.full((n,), np.nan, dtype=torch.float64, device="cuda:0")
        mean = torch.full((1,), np.nan, dtype=torch.float64, device="cuda:0")
        lib.mg_project_rhs_noalloc(J, f.reshape(-1), b, mean)
        torch.cuda.synchronize()
        m = float(mean.item())
        assert m == pytest.approx(ref_mean, rel=1e-12, abs=1e-14), call
        np.testing.assert_allclose(b.cpu().numpy(), ref_b, rtol=0, atol=1e-12 * np.abs(ref_b).max())


def test_noalloc_projection_rejects_oversized_grids(lib):
    import torch
    n = 4194304 + 1
    J = torch.ones(n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(lib.MGError) as e:
        lib.mg_project_rhs_noalloc(J, J, J)
    assert e.value.status == lib.MG_EINVAL
    assert "4194304" in str(e.value)
