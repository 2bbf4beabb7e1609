"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/mg.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

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
    with pytest.raises(mgs.MGError) as e:
        mgs.mg_setup(dict(g, nph=15), stream=0)
    assert e.value.status == mgs.MG_EINVAL
    with pytest.raises(mgs.MGError) as e:
        mgs.mg_setup(g, dict(precision=7), stream=0)
    assert e.value.status == mgs.MG_EINVAL
    o = mgs.default_opts()
    assert (o.precision, o.nu1, o.nu2, o.smoother) == (1, 2, 2, 0)
