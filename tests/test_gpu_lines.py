"""Batched tridiagonal line solves (Section 3.5) on the GPU against the
oracle's Thomas algorithm and its periodic variant.

Lines along each axis of a C-contiguous [d0][d1][d2] array (strided radial
and colatitude lines, contiguous longitude lines), ragged sizes, the smallest
line lengths, solves in place, and the 128 x 128 x 256 and 256 x 256 x 512
fields of the bench workloads (sampled lines, and a Fourier mode of a
circulant system checked at every line).  FP64 on both sides: 1e-12 of the
largest |psi|.
"""
import numpy as np
import pytest

from oracle import tridiag

pytestmark = pytest.mark.gpu


def _system(rng, shape, axis, periodic):
    a = rng.uniform(-1.0, 0.0, shape)
    c = rng.uniform(-1.0, 0.0, shape)
    b = 2.2 + rng.uniform(0.0, 1.0, shape)
    g = rng.standard_normal(shape)
    return a, b, c, g


def _oracle(a, b, c, g, axis, periodic):
    f = tridiag.thomas_periodic if periodic else tridiag.thomas
    mv = [np.moveaxis(v, axis, 0) for v in (a, b, c, g)]
    return np.moveaxis(f(*mv), 0, axis)


SHAPES = [(9, 10, 12), (1, 5, 8), (2, 3, 4), (3, 7, 6), (130, 3, 33)]


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("shape", SHAPES)
def test_line_solves_match_oracle(lib, shape, axis, periodic):
    import torch
    if periodic and shape[axis] < 3:
        pytest.skip("periodic lines need 3 unknowns")
    rng = np.random.default_rng(hash((shape, axis, periodic)) % 2**32)
    a, b, c, g = _system(rng, shape, axis, periodic)
    want = _oracle(a, b, c, g, axis, periodic)
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, g)]
    x = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
    L = lib.lines_along(shape, axis)
    lib.mg_thomas(L, *t, x, periodic=periodic)
    got = x.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    # in place: x is g
    lib.mg_thomas(L, t[0], t[1], t[2], t[3], t[3], periodic=periodic)
    np.testing.assert_array_equal(t[3].cpu().numpy(), got)


def test_empty_batch_is_a_no_op(lib):
    import torch
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib.mg_thomas(dict(n=5, n1=0, n2=7, sm=1, s1=5, s2=5), z, z, z, z, z.clone(), work=z.clone())


def test_invalid_geometry_is_rejected(lib):
    import torch
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    for L, per in ((dict(n=2, n1=1, n2=1, sm=1, s1=2, s2=2), True),
                   (dict(n=0, n1=1, n2=1, sm=1, s1=1, s2=1), False)):
        with pytest.raises(lib.MGError) as e:
            lib.mg_thomas(L, z, z, z, z, z.clone(), periodic=per, work=z.clone())
        assert e.value.status == lib.MG_EINVAL
    with pytest.raises(lib.MGError):        # x aliasing a coefficient
        lib.mg_thomas(dict(n=4, n1=1, n2=2, sm=2, s1=8, s2=1), z, z.clone(), z.clone(), z.clone(), z)


@pytest.mark.parametrize("shape", [(128, 128, 256), (256, 256, 512)])
def test_bench_size_fields(lib, shape):
    """Every axis at full size: sampled lines against the oracle; the periodic
    longitude solve of a circulant Fourier mode checked everywhere."""
    import torch
    rng = np.random.default_rng(21)
    N = int(np.prod(shape))
    gen = torch.Generator(device="cuda").manual_seed(3)
    a = -torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
    c = -torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
    b = 2.2 + torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
    g = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64)
    x = torch.empty_like(g)
    for axis in (0, 1, 2):
        for periodic in (False, True):
            L = lib.lines_along(shape, axis)
            lib.mg_thomas(L, a, b, c, g, x, periodic=periodic)
            other = [d for d in range(3) if d != axis]
            for _ in range(6):
                idx = [slice(None)] * 3
                for d in other:
                    idx[d] = int(rng.integers(0, shape[d]))
                idx = tuple(idx)
                want = (tridiag.thomas_periodic if periodic else tridiag.thomas)(
                    *(v[idx].cpu().numpy() for v in (a, b, c, g)))
                got = x[idx].cpu().numpy()
                np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    del a, b, c, g
    # circulant Fourier mode along longitude: lo psi_{m-1} + beta psi_m + up psi_{m+1}
    n = shape[2]
    lo, up, beta, q = -1.2, -0.7, 2.5, 7
    t = 2 * np.pi * q / n
    lam = beta + lo * np.exp(-1j * t) + up * np.exp(1j * t)
    m = np.arange(n)
    want = np.real(np.exp(1j * t * m) / lam)
    gg = torch.from_numpy(np.cos(t * m)).cuda().expand(shape).contiguous()
    A = torch.full(shape, lo, dtype=torch.float64, device="cuda")
    B = torch.full(shape, beta, dtype=torch.float64, device="cuda")
    Cc = torch.full(shape, up, dtype=torch.float64, device="cuda")
    lib.mg_thomas(lib.lines_along(shape, 2), A, B, Cc, gg, gg, periodic=True)
    err = (gg - torch.from_numpy(want).cuda()).abs().max().item()
    assert err <= 1e-12 * np.abs(want).max(), err
    assert N == gg.numel()


def test_one_unknown_lines_give_the_reciprocal(lib):
    """n = 1: psi = g / b.  With g = 1 this is the kernel's reciprocal: the
    correctly rounded 1/b (IEEE division) across the exponent range."""
    import torch
    rng = np.random.default_rng(4)
    mag = np.concatenate([rng.uniform(-300, 300, 4000), rng.uniform(-30, 30, 4000)])
    b = np.where(rng.random(mag.size) < 0.5, -1.0, 1.0) * 10.0 ** mag
    n = b.size
    L = dict(n=1, n1=1, n2=n, sm=n, s1=n, s2=1)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    lib.mg_thomas(L, t(np.zeros(n)), t(b), t(np.zeros(n)), t(np.ones(n)), x)
    got = x.cpu().numpy()
    want = 1.0 / b
    np.testing.assert_array_equal(got, want)
