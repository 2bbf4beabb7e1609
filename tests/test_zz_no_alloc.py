"""The allocation-free right-hand-side projection.

Callers that cannot allocate device memory when they need the step (a time
loop that must not stall on the allocator, or a program whose GPU memory is
owned by another pool) call mg_project_rhs_noalloc, whose reduction scratch
is a static device array.  Its results must match the oracle's projection of
Eq. PC_6's right side (b = J (f - mean_J f), the J-weighted mean of
Section 3.7's volume average) on the same J and f, and what the allocating
solve computes: the mean that mg_solve reports as removed_mean and b with the
cell volumes that mg_get_metric returns.  Two calls in a row check that the
shared scratch carries nothing over; the mean output is optional and the
call runs on any stream.  This file is collected last so a
stop-at-first-failure run has run everything else.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mg as omg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", [W.grid_desc(16, mapping=1, flattening=0.1, r_out=1 / 0.6),
                                  W.grid_desc(128, stretch=2.0)])
def test_noalloc_projection_matches_oracle_and_allocating_solve(lib, grid):
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
    ob, omean = omg.prepare_rhs(J.cpu().numpy(), f.reshape(-1).cpu().numpy())
    ob = np.asarray(ob).ravel()
    for call in range(2):                      # the second call reuses the scratch
        b = torch.full((n,), np.nan, dtype=torch.float64, device="cuda:0")
        mean = torch.full((1,), np.nan, dtype=torch.float64, device="cuda:0")
        lib.mg_project_rhs_noalloc(J, f.reshape(-1), b, mean)
        torch.cuda.synchronize()
        m = float(mean.item())
        assert m == pytest.approx(ref_mean, rel=1e-12, abs=1e-14), call
        assert m == pytest.approx(omean, rel=1e-12, abs=1e-14), call
        np.testing.assert_allclose(b.cpu().numpy(), ref_b, rtol=0, atol=1e-12 * np.abs(ref_b).max())
        np.testing.assert_allclose(b.cpu().numpy(), ob, rtol=0, atol=1e-12 * np.abs(ob).max())
    h.close()


def test_noalloc_projection_without_mean_on_a_side_stream(lib):
    import torch
    g = W.grid_desc(24, 20, 40, mapping=2, flattening=0.1, e2=0.05)
    n = g["nr"] * g["nth"] * g["nph"]
    h = lib.mg_setup(g, dict(precision=1))
    J = torch.empty(n, dtype=torch.float64, device="cuda:0")
    lib.mg_get_metric(h, 0, 9, J)
    f = torch.from_numpy(W.rhs_modes(g, seed=9).ravel() - 1.5).to("cuda:0")
    ob, _ = omg.prepare_rhs(J.cpu().numpy(), f.cpu().numpy())
    ob = np.asarray(ob).ravel()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        b = torch.full((n,), np.nan, dtype=torch.float64, device="cuda:0")
        s.wait_stream(torch.cuda.current_stream())
        lib.mg_project_rhs_noalloc(J, f, b, None, stream=s)
        s.synchronize()
        np.testing.assert_allclose(b.cpu().numpy(), ob, rtol=0, atol=1e-12 * np.abs(ob).max())
    h.close()


def test_noalloc_projection_rejects_oversized_grids(lib):
    import torch
    n = 4194304 + 1
    J = torch.ones(n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(lib.MGError) as e:
        lib.mg_project_rhs_noalloc(J, J, J)
    assert e.value.status == lib.MG_EINVAL
    assert "4194304" in str(e.value)


def test_noalloc_projection_refuses_memory_of_no_device(lib):
    """Arrays that are not device memory of the current device are refused on
    the host, before any kernel is queued (here: pageable and pinned host
    memory handed to the C call directly)."""
    import ctypes
    import torch
    n = 4096
    J = torch.ones(n, dtype=torch.float64, device="cuda:0")
    pageable = np.ones(n)
    pinned = torch.ones(n, dtype=torch.float64).pin_memory()
    for host in (pageable.ctypes.data, pinned.data_ptr()):
        st = lib._lib.mg_project_rhs_noalloc(ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(J.data_ptr()),
                                             ctypes.c_void_p(host), ctypes.c_longlong(n), None, None)
        assert st == lib.MG_EINVAL
        assert "current device" in lib.mg_last_error() or "not a CUDA pointer" in lib.mg_last_error()
