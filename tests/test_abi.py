"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/mg.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w]+\s*\**\s+(mg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def so():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("mg_setup", "mg_solve", "mg_solve_batch", "mg_destroy", "mg_apply", "mg_smooth",
                 "mg_restrict_residual", "mg_prolong_add", "mg_coarse_solve", "mg_footprint_bytes"):
        assert name in d


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in sorted(_declared()) if not hasattr(so, n)]
    assert not missing, missing


def test_binding_resolves_every_declared_symbol(so):
    import paper_2305_17875_gb300 as mgs
    assert set(mgs.exported_symbols()) == _declared()


def test_host_side_validation_without_gpu(so):
    import paper_2305_17875_gb300 as mgs
    g = dict(nr=8, nth=8, nph=16, r_in=1.0, r_out=2.0, th0=0.5, th1=2.6)
    assert mgs.mg_footprint_bytes(g) > 8 * 8 * 8 * 16
    assert mgs.mg_footprint_bytes(dict(g, nph=15)) == 0           # odd longitude count
    assert mgs.mg_footprint_bytes(dict(g, nph=2)) == 0            # degenerate longitude faces
    assert mgs.mg_footprint_bytes(dict(g, r_out=0.5)) == 0        # r_out < r_in
    assert mgs.mg_footprint_bytes(dict(g, th1=3.5)) == 0          # beyond the pole
    import math
    sphere = dict(g, th0=0.0, th1=math.pi, cut=1)                      # full sphere, shell cut
    assert mgs.mg_footprint_bytes(sphere) > 0
    assert mgs.mg_footprint_bytes(dict(sphere, cut=2)) == 0
    assert mgs.mg_footprint_bytes(dict(g, cut=1)) == 0               # cut needs [0, pi]
    assert mgs.mg_footprint_bytes(dict(sphere, th0=0.0, cut=0)) == 0  # walls need th0 > 0
    assert mgs.mg_footprint_bytes(dict(sphere, mapping=1, flattening=0.1)) > 0    # 19 points, axisymmetric
    assert mgs.mg_footprint_bytes(dict(sphere, mapping=2, flattening=0.1, e2=0.05)) == 0   # 19 points, triaxial
    assert mgs.mg_footprint_bytes(sphere, dict(stencil=19)) > 0
    assert mgs.mg_footprint_bytes(sphere, dict(stencil=19, smoother=2)) == 0   # 19 points, radial lines
    with pytest.raises(mgs.MGError) as e:
        mgs.mg_setup(dict(g, nph=15), stream=0)
    assert e.value.status == mgs.MG_EINVAL
    with pytest.raises(mgs.MGError) as e:
        mgs.mg_setup(g, dict(precision=7), stream=0)
    assert e.value.status == mgs.MG_EINVAL
    with pytest.raises(mgs.MGError) as e:
        mgs.mg_setup(g, dict(metric=2), stream=0)
    assert e.value.status == mgs.MG_EINVAL
    o = mgs.default_opts()
    assert (o.precision, o.nu1, o.nu2, o.smoother) == (1, 2, 2, 0)


def test_line_solve_and_adi_validation_without_gpu(so):
    """Geometry and argument checks of mg_thomas / mg_adi_substep happen on
    the host, before any device work."""
    import paper_2305_17875_gb300 as mgs
    L = dict(n=5, n1=3, n2=4, sm=12, s1=4, s2=1)
    assert mgs.mg_thomas_work_bytes(L) == 8 * 4 * 12
    assert mgs.mg_thomas_work_bytes(L, periodic=True) == 8 * 2 * 4 * 12
    assert mgs.mg_thomas_work_bytes(dict(L, n=2), periodic=True) == 0
    assert mgs.mg_thomas_work_bytes(dict(L, n=0)) == 0
    assert mgs.mg_thomas_work_bytes(dict(L, n1=-1)) == 0
    assert mgs.lines_along((2, 3, 4), 0) == dict(n=2, n1=3, n2=4, sm=12, s1=4, s2=1)
    assert mgs.lines_along((2, 3, 4), 2) == dict(n=4, n1=2, n2=3, sm=1, s1=12, s2=4)
    dummy = 4096   # never dereferenced: the checks fail first
    for geom, per in ((dict(L, n=2), True), (dict(L, n=0), False)):
        with pytest.raises(mgs.MGError) as e:
            mgs.mg_thomas(geom, dummy, dummy + 8, dummy + 16, dummy + 24, dummy + 32, periodic=per, work=dummy + 40,
                          stream=0)
        assert e.value.status == mgs.MG_EINVAL
    with pytest.raises(mgs.MGError) as e:       # x aliasing a coefficient
        mgs.mg_thomas(L, dummy, dummy + 8, dummy + 16, dummy + 24, dummy, work=dummy + 40, stream=0)
    assert e.value.status == mgs.MG_EINVAL
    st = mgs._lib.mg_adi_substep(None, 1.0, 1, None, None, None, None)
    assert st == mgs.MG_EINVAL


def test_buffers_are_checked_for_their_memory_kind(so):
    """Device arguments refuse host memory (numpy arrays, CPU tensors) before
    any call: the kernels would read it as device memory.  Host arguments
    refuse CUDA tensors and other dtypes."""
    import torch
    import paper_2305_17875_gb300 as mgs
    host_t = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        mgs._ptr(host_t, "float64")
    with pytest.raises(ValueError):
        mgs._ptr(np.zeros(4), "float64")
    with pytest.raises(TypeError):
        mgs._ptr(torch.zeros(4, dtype=torch.float32), "float64")
    assert mgs._ptr(1234, "float64") == 1234              # raw device address
    assert mgs._hptr(host_t) == host_t.data_ptr()
    a = np.zeros(4)
    assert mgs._hptr(a) == a.ctypes.data
    with pytest.raises(TypeError):
        mgs._hptr(np.zeros(4, dtype=np.float32))
    with pytest.raises(ValueError):
        mgs._hptr(np.zeros((4, 4))[:, 0])
