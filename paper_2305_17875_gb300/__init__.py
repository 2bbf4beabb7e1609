"""Python binding of the GB300 shell pressure-correction Poisson solver.

Argument marshalling only: every function forwards to the C ABI of
``include/mg.h`` (same names) in ``_lib/libmgshell.so``; all computation runs
in the library's CUDA kernels.  Device buffers are torch CUDA tensors
(float64 or float32, C-contiguous); streams default to torch's current stream.
Importing fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmgshell.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'` "
                      "or `python -m paper_2305_17875_gb300.build`")
_lib = C.CDLL(LIB_PATH)

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ENOCONV, MG_ENAN, MG_EDIVERGED, MG_ETIMEOUT, MG_EAGAIN, MG_ECUDA = range(9)
STATUS = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ENOCONV", 4: "MG_ENAN",
          5: "MG_EDIVERGED", 6: "MG_ETIMEOUT", 7: "MG_EAGAIN", 8: "MG_ECUDA"}
PREC_FP64, PREC_FP32_IR, PREC_FP16C_IR = 0, 1, 2
MG_HIST = 64
MG_SMOOTH_GS, MG_SMOOTH_JACOBI, MG_SMOOTH_LINE, MG_SMOOTH_XLINE, MG_SMOOTH_ALT, MG_SMOOTH_PLANE = range(6)
MG_METRIC_DISCRETE, MG_METRIC_ANALYTIC = range(2)


class mg_grid_desc(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("nph", C.c_int),
                ("r_in", C.c_double), ("r_out", C.c_double),
                ("th0", C.c_double), ("th1", C.c_double),
                ("mapping", C.c_int), ("flattening", C.c_double), ("e2", C.c_double),
                ("stretch", C.c_double), ("cut", C.c_int)]


class mg_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("smoother", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("max_levels", C.c_int), ("coarsen", C.c_int), ("coarse_max", C.c_int),
                ("max_iters", C.c_int), ("stencil", C.c_int), ("autotune", C.c_int), ("metric", C.c_int),
                ("plane_cycles", C.c_int)]


class mg_lines(C.Structure):
    _fields_ = [("n", C.c_int), ("n1", C.c_int), ("n2", C.c_int),
                ("sm", C.c_longlong), ("s1", C.c_longlong), ("s2", C.c_longlong)]


class mg_walls(C.Structure):
    _fields_ = [("radius", C.c_int), ("colatitude", C.c_int), ("v_r_in", C.c_double), ("v_r_out", C.c_double),
                ("v_th0", C.c_double), ("v_th1", C.c_double)]


class mg_schedule(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int), ("tail_level", C.c_int), ("tail_cluster", C.c_int),
                ("one_pass_tiles", C.c_int), ("source", C.c_int), ("candidates", C.c_int),
                ("ms_per_iteration", C.c_double), ("tile_cells", C.c_int), ("tile_planes", C.c_int),
                ("tile_kmax", C.c_int), ("tile_min_cells", C.c_longlong), ("tile0", C.c_int * 3),
                ("tail_smem_bytes", C.c_int)]


class mg_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("levels", C.c_int), ("stencil", C.c_int), ("status", C.c_int),
                ("rel_res", C.c_double), ("res_hist", C.c_double * MG_HIST),
                ("seconds", C.c_double), ("removed_mean", C.c_double), ("model_bytes", C.c_double),
                ("launches", C.c_longlong)]

    def as_dict(self):
        n = min(self.iters + 1, MG_HIST)
        return dict(iters=self.iters, levels=self.levels, stencil=self.stencil,
                    status=STATUS.get(self.status, self.status), rel_res=self.rel_res,
                    res_hist=list(self.res_hist[:n]), seconds=self.seconds,
                    removed_mean=self.removed_mean, model_bytes=self.model_bytes,
                    launches=self.launches)


class mg_serve_opts(C.Structure):
    _fields_ = [("max_bytes", C.c_size_t), ("max_slots", C.c_int), ("setup_threads", C.c_int),
                ("cache_bytes", C.c_size_t), ("device", C.c_int)]


class mg_serve_stats_t(C.Structure):
    _fields_ = [("queued", C.c_longlong), ("active", C.c_longlong), ("steps", C.c_longlong),
                ("retired", C.c_longlong), ("cache_hits", C.c_longlong),
                ("cached_hierarchies", C.c_longlong), ("bytes_reserved", C.c_size_t),
                ("t_start", C.c_double), ("t_plan", C.c_double), ("t_step", C.c_double),
                ("t_retire", C.c_double), ("plan_rebuilds", C.c_longlong)]


class mg_level_info(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("nph", C.c_int), ("cz", C.c_int),
                ("ce", C.c_int), ("cx", C.c_int), ("stencil", C.c_int), ("levels", C.c_int)]


_vp, _dp, _i, _d = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double
_SIGS = {
    "mg_version": ([], C.c_char_p),
    "mg_last_error": ([], C.c_char_p),
    "mg_default_opts": ([C.POINTER(mg_opts)], _i),
    "mg_footprint_bytes": ([C.POINTER(mg_grid_desc), C.POINTER(mg_opts)], C.c_size_t),
    "mg_setup": ([C.POINTER(mg_grid_desc), C.POINTER(mg_opts), _vp, C.POINTER(_vp)], _i),
    "mg_destroy": ([_vp], None),
    "mg_set_stream": ([_vp, _vp], _i),
    "mg_solve": ([_vp, _vp, _vp, _d, C.POINTER(mg_report)], _i),
    "mg_solve_host": ([_vp, _vp, _vp, _d, C.POINTER(mg_report)], _i),
    "mg_solve_batch": ([_vp, _i, _vp, _vp, _vp, _vp], _i),
    "mg_get_level_info": ([_vp, _i, C.POINTER(mg_level_info)], _i),
    "mg_get_metric": ([_vp, _i, _i, _vp], _i),
    "mg_apply": ([_vp, _i, _i, _vp, _vp], _i),
    "mg_smooth": ([_vp, _i, _i, _vp, _vp, _i, _i], _i),
    "mg_restrict_residual": ([_vp, _i, _i, _vp, _vp, _vp], _i),
    "mg_prolong_add": ([_vp, _i, _i, _vp, _vp], _i),
    "mg_coarse_solve": ([_vp, _i, _vp, _vp], _i),
    "mg_vcycle": ([_vp, _i, _vp, _vp], _i),
    "mg_profile_enable": ([_vp, _i], _i),
    "mg_profile_read": ([_vp, _i, C.POINTER(C.c_double), C.POINTER(C.c_longlong)], _i),
    "mg_project_rhs_noalloc": ([_vp, _vp, _vp, C.c_longlong, _vp, _vp], _i),
    "mg_get_schedule": ([_vp, C.POINTER(mg_schedule)], _i),
    "mg_pc_rhs": ([_vp, _vp, _vp], _i),
    "mg_pc_correct": ([_vp, _vp, _vp], _i),
    "mg_adi_substep": ([_vp, _d, _i, C.POINTER(mg_walls), _vp, _vp, _vp], _i),
    "mg_device_bytes_in_use": ([_i], C.c_size_t),
    "mg_thomas_work_bytes": ([C.POINTER(mg_lines), _i], C.c_size_t),
    "mg_thomas": ([C.POINTER(mg_lines), _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp], _i),
    "mg_serve_default_opts": ([C.POINTER(mg_serve_opts)], _i),
    "mg_serve_create": ([C.POINTER(mg_serve_opts), C.POINTER(_vp)], _i),
    "mg_serve_submit": ([_vp, C.POINTER(mg_grid_desc), C.POINTER(mg_opts), _vp, _d,
                         C.POINTER(C.c_uint64)], _i),
    "mg_serve_poll": ([_vp, C.c_uint64, _vp, C.POINTER(mg_report)], _i),
    "mg_serve_stats": ([_vp, C.POINTER(mg_serve_stats_t)], _i),
    "mg_serve_destroy": ([_vp], None),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


class MGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.mg_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}")


def _check(st, where, ok=(MG_OK,)):
    if st not in ok:
        raise MGError(st, where)
    return st


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ptr(t, dtype=None):
    """Device buffer: a C-contiguous CUDA tensor of ``dtype`` (or a raw device
    address as an int).  Host memory is refused here: the kernels would read
    it as device memory."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be C-contiguous")
        if dtype is not None and str(t.dtype) != f"torch.{dtype}":
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor (device buffer), got a host tensor")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        raise ValueError("expected a CUDA tensor (device buffer), got a numpy array")
    return int(t)


def _hptr(t):
    """Host buffer of float64: a C-contiguous numpy array or CPU tensor (or a
    raw host address as an int)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be C-contiguous")
        if str(t.dtype) != "torch.float64":
            raise TypeError(f"expected float64, got {t.dtype}")
        if t.is_cuda:
            raise ValueError("expected a host buffer, got a CUDA tensor")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if t.dtype != np.float64:
            raise TypeError(f"expected float64, got {t.dtype}")
        return t.ctypes.data
    return int(t)


def grid_desc(d) -> mg_grid_desc:
    """mg_grid_desc from a dict with the C field names."""
    g = mg_grid_desc()
    for k, _ in mg_grid_desc._fields_:
        if k in d:
            setattr(g, k, d[k])
    return g


def default_opts(**kw) -> mg_opts:
    o = mg_opts()
    _check(_lib.mg_default_opts(C.byref(o)), "mg_default_opts")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, int(v))
    return o


def mg_version() -> str:
    return _lib.mg_version().decode()


def mg_last_error() -> str:
    return _lib.mg_last_error().decode()


def mg_footprint_bytes(grid, opts=None) -> int:
    g = grid if isinstance(grid, mg_grid_desc) else grid_desc(grid)
    o = opts if isinstance(opts, mg_opts) or opts is None else default_opts(**opts)
    return int(_lib.mg_footprint_bytes(C.byref(g), C.byref(o) if o is not None else None))


class Handle:
    """Owner of an mg_handle*; ``close()`` (or garbage collection) destroys it."""

    def __init__(self, ptr, grid, opts):
        self.ptr = ptr
        self.grid = grid
        self.opts = opts

    @property
    def shape(self):
        return (self.grid.nr, self.grid.nth, self.grid.nph)

    def close(self):
        if self.ptr:
            _lib.mg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_setup(grid, opts=None, stream=None) -> Handle:
    g = grid if isinstance(grid, mg_grid_desc) else grid_desc(grid)
    o = opts if isinstance(opts, mg_opts) else default_opts(**(opts or {}))
    h = C.c_void_p()
    _check(_lib.mg_setup(C.byref(g), C.byref(o), _stream(stream), C.byref(h)), "mg_setup")
    return Handle(h, g, o)


def mg_destroy(h: Handle):
    h.close()


def mg_set_stream(h: Handle, stream=None):
    _check(_lib.mg_set_stream(h.ptr, _stream(stream)), "mg_set_stream")


def mg_solve(h: Handle, f, x, tol=1e-10, allow=(MG_OK,)):
    """Solve in place on device tensors; returns the report as a dict."""
    rep = mg_report()
    st = _lib.mg_solve(h.ptr, _ptr(f, "float64"), _ptr(x, "float64"), float(tol), C.byref(rep))
    _check(st, "mg_solve", allow)
    return rep.as_dict()


def mg_solve_host(h: Handle, f, x, tol=1e-10, allow=(MG_OK,)):
    """Solve from host arrays (numpy or pinned torch CPU tensors); x in place."""
    rep = mg_report()
    st = _lib.mg_solve_host(h.ptr, _hptr(f), _hptr(x), float(tol), C.byref(rep))
    _check(st, "mg_solve_host", allow)
    return rep.as_dict()


def mg_solve_batch(hs, fs, xs, tols, allow=(MG_OK,)):
    n = len(hs)
    H = (C.c_void_p * n)(*[h.ptr for h in hs])
    F = (C.c_void_p * n)(*[_ptr(f, "float64") for f in fs])
    X = (C.c_void_p * n)(*[_ptr(x, "float64") for x in xs])
    T = (C.c_double * n)(*[float(t) for t in tols])
    reps = (mg_report * n)()
    st = _lib.mg_solve_batch(H, n, F, X, T, reps)
    _check(st, "mg_solve_batch", allow)
    return [r.as_dict() for r in reps]


def mg_get_level_info(h: Handle, level: int) -> dict:
    info = mg_level_info()
    _check(_lib.mg_get_level_info(h.ptr, level, C.byref(info)), "mg_get_level_info")
    return {k: getattr(info, k) for k, _ in mg_level_info._fields_}


def mg_get_metric(h: Handle, level: int, component: int, dst):
    _check(_lib.mg_get_metric(h.ptr, level, component, _ptr(dst, "float64")), "mg_get_metric")


def _vdtype(prec):
    return "float64" if prec == PREC_FP64 else "float32"


def mg_apply(h: Handle, level: int, prec: int, x, y):
    _check(_lib.mg_apply(h.ptr, level, prec, _ptr(x, _vdtype(prec)), _ptr(y, _vdtype(prec))), "mg_apply")


def mg_smooth(h: Handle, level: int, prec: int, x, b, sweeps: int, kind: int = 0):
    _check(_lib.mg_smooth(h.ptr, level, prec, _ptr(x, _vdtype(prec)), _ptr(b, _vdtype(prec)),
                          sweeps, kind), "mg_smooth")


def mg_restrict_residual(h: Handle, level: int, prec: int, x, b, rc):
    _check(_lib.mg_restrict_residual(h.ptr, level, prec, _ptr(x, _vdtype(prec)), _ptr(b, _vdtype(prec)),
                                     _ptr(rc, _vdtype(prec))), "mg_restrict_residual")


def mg_prolong_add(h: Handle, level: int, prec: int, ec, x):
    _check(_lib.mg_prolong_add(h.ptr, level, prec, _ptr(ec, _vdtype(prec)), _ptr(x, _vdtype(prec))),
           "mg_prolong_add")


def mg_coarse_solve(h: Handle, prec: int, r, e):
    _check(_lib.mg_coarse_solve(h.ptr, prec, _ptr(r, _vdtype(prec)), _ptr(e, _vdtype(prec))),
           "mg_coarse_solve")


def mg_vcycle(h: Handle, prec: int, x, b):
    _check(_lib.mg_vcycle(h.ptr, prec, _ptr(x, _vdtype(prec)), _ptr(b, _vdtype(prec))), "mg_vcycle")


def mg_pc_rhs(h: Handle, u_face, f):
    """Right side of Eq. PC_6 from the staggered velocity u_face (9 * N doubles)."""
    _check(_lib.mg_pc_rhs(h.ptr, _ptr(u_face, "float64"), _ptr(f, "float64")), "mg_pc_rhs")


def mg_pc_correct(h: Handle, x, u_face):
    """Correction of Eq. PC_7 of u_face (in place) by x = h dP."""
    _check(_lib.mg_pc_correct(h.ptr, _ptr(x, "float64"), _ptr(u_face, "float64")), "mg_pc_correct")


def lines_along(shape, axis) -> dict:
    """mg_lines fields for the lines along ``axis`` of a C-contiguous 3-d array."""
    d0, d1, d2 = shape
    return [dict(n=d0, n1=d1, n2=d2, sm=d1 * d2, s1=d2, s2=1),
            dict(n=d1, n1=d0, n2=d2, sm=d2, s1=d1 * d2, s2=1),
            dict(n=d2, n1=d0, n2=d1, sm=1, s1=d1 * d2, s2=d2)][axis]


def _lines(d) -> mg_lines:
    L = mg_lines()
    for k, _ in mg_lines._fields_:
        setattr(L, k, int(d[k]))
    return L


def mg_thomas_work_bytes(lines: dict, periodic=False) -> int:
    return int(_lib.mg_thomas_work_bytes(C.byref(_lines(lines)), int(bool(periodic))))


def mg_thomas(lines: dict, a, b, c, g, x, periodic=False, work=None, stream=None):
    """Tridiagonal solves of Section 3.5 along every line of ``lines``
    (mg_lines fields); device float64 tensors; ``work`` is allocated when None."""
    L = _lines(lines)
    if work is None:
        import torch
        nbytes = _lib.mg_thomas_work_bytes(C.byref(L), int(bool(periodic)))
        work = torch.empty(max(nbytes // 8, 1), dtype=torch.float64, device=x.device)
    _check(_lib.mg_thomas(C.byref(L), _ptr(a, "float64"), _ptr(b, "float64"), _ptr(c, "float64"),
                          _ptr(g, "float64"), _ptr(x, "float64"), _ptr(work, "float64"),
                          int(bool(periodic)), _stream(stream)), "mg_thomas")


MG_WALL_FLUX0, MG_WALL_VALUE = 0, 1


def mg_device_bytes_in_use(device: int = 0) -> int:
    return int(_lib.mg_device_bytes_in_use(int(device)))


def mg_adi_substep(h: Handle, kappa, un, u, src=None, walls=None):
    """ADI-CN sub-step of Section 3.4 (Eqs. solve_2 to solve_4): u = u*** from
    un.  un, u (and src) are one device tensor or equal-length lists of them
    (fields sharing kappa and wall kinds); walls: None for no-slip, a dict of
    mg_walls fields, or one dict per field."""
    many = isinstance(un, (list, tuple))
    uns, us = (list(un), list(u)) if many else ([un], [u])
    n = len(uns)
    srcs = (list(src) if many else [src]) if src is not None else None
    wp = None
    if walls is not None:
        wl = walls if isinstance(walls, (list, tuple)) else [walls] * n
        W = (mg_walls * n)()
        for f, d in enumerate(wl):
            for k, v in d.items():
                setattr(W[f], k, v)
        wp = W
    UN = (C.c_void_p * n)(*[_ptr(t, "float64") for t in uns])
    U = (C.c_void_p * n)(*[_ptr(t, "float64") for t in us])
    S = (C.c_void_p * n)(*[_ptr(t, "float64") for t in srcs]) if srcs is not None else None
    _check(_lib.mg_adi_substep(h.ptr, float(kappa), n, wp, UN, S, U), "mg_adi_substep")


def mg_get_schedule(h: Handle) -> dict:
    sc = mg_schedule()
    _check(_lib.mg_get_schedule(h.ptr, C.byref(sc)), "mg_get_schedule")
    out = {k: getattr(sc, k) for k, _ in mg_schedule._fields_}
    out["tile0"] = list(sc.tile0)
    return out


PROF_SMOOTH0, PROF_RESIDUAL, PROF_RESTRICT0, PROF_PROLONG0, PROF_UPDATE, PROF_TAIL, PROF_OTHER, PROF_GAPS = range(8)
PROF_LEVEL_BASE, PROF_SLOTS = 8, 24   # slot PROF_LEVEL_BASE + l: level l's operations (1 <= l < 16)


def mg_profile_enable(h: Handle, on=True):
    """on: True / 1 = launch clocks, 2 = CUDA events around eager launches, False / 0 = off."""
    mode = int(on) if not isinstance(on, bool) else int(on)
    _check(_lib.mg_profile_enable(h.ptr, mode), "mg_profile_enable")


def mg_profile_read(h: Handle, slot: int):
    ms, n = C.c_double(), C.c_longlong()
    _check(_lib.mg_profile_read(h.ptr, slot, C.byref(ms), C.byref(n)), "mg_profile_read")
    return ms.value, n.value


class Server:
    """Owner of an mg_server*."""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            _lib.mg_serve_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_serve_create(**kw) -> Server:
    o = mg_serve_opts()
    _check(_lib.mg_serve_default_opts(C.byref(o)), "mg_serve_default_opts")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, int(v))
    p = C.c_void_p()
    _check(_lib.mg_serve_create(C.byref(o), C.byref(p)), "mg_serve_create")
    return Server(p)


def mg_serve_submit(sv: Server, grid, f, tol=1e-10, opts=None) -> int:
    g = grid if isinstance(grid, mg_grid_desc) else grid_desc(grid)
    o = opts if isinstance(opts, mg_opts) else default_opts(**(opts or {}))
    f = np.ascontiguousarray(f, dtype=np.float64)
    if f.size != g.nr * g.nth * g.nph:
        raise ValueError("f has the wrong size")
    t = C.c_uint64()
    _check(_lib.mg_serve_submit(sv.ptr, C.byref(g), C.byref(o), f.ctypes.data, float(tol), C.byref(t)),
           "mg_serve_submit")
    return t.value


def mg_serve_poll(sv: Server, ticket: int, x=None):
    """None while the request runs; else (status name, report dict)."""
    rep = mg_report()
    st = _lib.mg_serve_poll(sv.ptr, C.c_uint64(ticket), _hptr(x), C.byref(rep))
    if st == MG_EAGAIN:
        return None
    if st not in (MG_OK, MG_ENOCONV):
        raise MGError(st, "mg_serve_poll")
    return STATUS[st], rep.as_dict()


def mg_serve_stats(sv: Server) -> dict:
    s = mg_serve_stats_t()
    _check(_lib.mg_serve_stats(sv.ptr, C.byref(s)), "mg_serve_stats")
    return {k: getattr(s, k) for k, _ in mg_serve_stats_t._fields_}


def mg_serve_destroy(sv: Server):
    sv.close()


def mg_project_rhs_noalloc(J, f, b, mean=None, stream=None):
    """b = J (f - mean_J f) with no device allocation (the library's static
    scratch holds the partial sums), for callers that cannot allocate when
    they need the step (a time loop that must not stall on the allocator, or
    a program whose GPU memory belongs to another pool).  J, f, b: float64
    tensors of one size on one CUDA device; mean: optional float64 tensor of
    one element there.  The call runs with the tensors' device current;
    stream=None means torch.cuda.current_stream() of that device (not the
    legacy default stream the C call takes for NULL)."""
    import torch
    n = J.numel()
    if f.numel() != n or b.numel() != n:
        raise ValueError("J, f and b must have the same size")
    with torch.cuda.device(J.device):
        _check(_lib.mg_project_rhs_noalloc(_ptr(J, "float64"), _ptr(f, "float64"), _ptr(b, "float64"), n,
                                           _stream(stream), _ptr(mean, "float64")), "mg_project_rhs_noalloc")


def exported_symbols():
    """Names declared in include/mg.h that this binding resolves."""
    return sorted(_SIGS)
