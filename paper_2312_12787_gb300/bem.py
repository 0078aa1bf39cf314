"""Thin ctypes binding of libbem (include/bem.h).  Argument marshalling only: every step runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (complex128 for bem_c64 blocks); streams
are torch CUDA streams.

The functions keep the C names.  Each raises BemError on a non-OK status (BEM_ENOCONV is returned as
the status code in the result instead, because the best iterate is still written).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbem.so")

BEM_OK, BEM_EINVAL, BEM_ENOMEM, BEM_ENOCONV, BEM_ETIMEOUT, BEM_ECUDA, BEM_ESTATE = range(7)
BEM_FORM_MOD, BEM_FORM_ORIG, BEM_FORM_BETA1, BEM_FORM_CONV = range(4)
BEM_PREC_FP64, BEM_PREC_MIXED, BEM_PREC_MIXED_TC = range(3)
FORMS = {"mod": BEM_FORM_MOD, "orig": BEM_FORM_ORIG, "beta1": BEM_FORM_BETA1, "conv": BEM_FORM_CONV}
PRECS = {"fp64": BEM_PREC_FP64, "mixed": BEM_PREC_MIXED, "mixed_tc": BEM_PREC_MIXED_TC}

EXPORTS = [
    "bem_default_opts", "bem_problem_create", "bem_problem_destroy", "bem_set_opts", "bem_set_domains",
    "bem_add_segment", "bem_num_elements", "bem_num_unknowns", "bem_footprint_bytes", "bem_assemble",
    "bem_get_matrix", "bem_rhs_planewave", "bem_matvec", "bem_residual", "bem_residual_noalloc", "bem_solve", "bem_solve_planewave", "bem_far_field",
    "bem_solve_planewave_host", "bem_near_field", "bem_profile_enable", "bem_profile_read", "bem_last_error", "bem_version",
    "bem_batch_create", "bem_batch_destroy", "bem_batch_admit", "bem_batch_step", "bem_batch_query",
    "bem_batch_take", "bem_batch_free_units", "bem_batch_solve_planewave", "bem_test_set_wait_limit",
    "bem_test_set_fused_iteration",
]
PHASES = ["geometry", "assemble", "rhs", "matvec", "arnoldi", "givens", "update", "residual", "farfield", "other",
          "reduce", "relaxed"]


class BemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libbem status {status}: {msg}")
        self.status = status


class bem_opts(ctypes.Structure):
    _fields_ = [("quad_order", ctypes.c_int), ("form", ctypes.c_int), ("prec", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("max_refine", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("orth_passes", ctypes.c_int), ("matrix_free", ctypes.c_int),
                ("store_bytes", ctypes.c_longlong)]


_lib = None


def load(path: str | None = None):
    """Load libbem.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing; build it with paper_2312_12787_gb300.build.build()")
    L = ctypes.CDLL(p)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    L.bem_default_opts.argtypes = [P(bem_opts)]
    L.bem_default_opts.restype = None
    L.bem_problem_create.argtypes = [P(vp), P(bem_opts)]
    L.bem_problem_destroy.argtypes = [vp]
    L.bem_problem_destroy.restype = None
    L.bem_set_opts.argtypes = [vp, P(bem_opts)]
    L.bem_set_domains.argtypes = [vp, i, vp, vp]
    L.bem_add_segment.argtypes = [vp, i, vp, i, i, i]
    L.bem_num_elements.argtypes = [vp]
    L.bem_num_unknowns.argtypes = [vp]
    L.bem_footprint_bytes.argtypes = [vp, i]
    L.bem_footprint_bytes.restype = sz
    L.bem_assemble.argtypes = [vp, vp]
    L.bem_get_matrix.argtypes = [vp, i, vp, vp]
    L.bem_rhs_planewave.argtypes = [vp, i, vp, vp, vp]
    L.bem_matvec.argtypes = [vp, i, vp, vp, vp]
    L.bem_residual.argtypes = [vp, i, vp, vp, vp, vp]
    L.bem_residual_noalloc.argtypes = [vp, i, vp, vp, vp, vp]
    L.bem_solve.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.bem_solve_planewave.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.bem_far_field.argtypes = [vp, i, vp, i, vp, vp, vp]
    L.bem_solve_planewave_host.argtypes = [vp, i, vp, vp, i, vp, vp, vp, vp, vp]
    L.bem_near_field.argtypes = [vp, i, vp, vp, i, vp, vp, vp, vp]
    L.bem_near_field.restype = i
    L.bem_profile_enable.argtypes = [vp, i]
    L.bem_profile_read.argtypes = [vp, vp, vp]
    ll = ctypes.c_longlong
    L.bem_batch_create.argtypes = [P(vp), P(bem_opts), i, ll]
    L.bem_batch_destroy.argtypes = [vp]
    L.bem_batch_destroy.restype = None
    L.bem_batch_admit.argtypes = [vp, i, vp, vp, vp, vp]
    L.bem_batch_step.argtypes = [vp, vp, vp]
    L.bem_batch_query.argtypes = [vp, i, vp, vp, vp]
    L.bem_batch_take.argtypes = [vp, i, vp, vp]
    L.bem_batch_free_units.argtypes = [vp]
    L.bem_batch_free_units.restype = ll
    L.bem_batch_solve_planewave.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    for name in ("bem_batch_create", "bem_batch_admit", "bem_batch_step", "bem_batch_query", "bem_batch_take",
                 "bem_batch_solve_planewave"):
        getattr(L, name).restype = i
    L.bem_test_set_wait_limit.argtypes = [d]
    L.bem_test_set_wait_limit.restype = i
    L.bem_test_set_fused_iteration.argtypes = [i]
    L.bem_test_set_fused_iteration.restype = i
    L.bem_last_error.argtypes = []
    L.bem_last_error.restype = ctypes.c_char_p
    L.bem_version.argtypes = []
    L.bem_version.restype = ctypes.c_char_p
    for name in ("bem_problem_create", "bem_set_opts", "bem_set_domains", "bem_add_segment", "bem_assemble",
                 "bem_get_matrix", "bem_rhs_planewave", "bem_matvec", "bem_residual", "bem_residual_noalloc", "bem_solve", "bem_solve_planewave",
                 "bem_far_field", "bem_solve_planewave_host", "bem_profile_enable", "bem_profile_read"):
        getattr(L, name).restype = i
    _lib = L
    return L


def _check(st, allow_noconv=False):
    if st == BEM_OK or (allow_noconv and st == BEM_ENOCONV):
        return st
    raise BemError(st, load().bem_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _hbuf(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def bem_default_opts() -> bem_opts:
    o = bem_opts()
    load().bem_default_opts(ctypes.byref(o))
    return o


def make_opts(quad_order=4, form="mod", prec="fp64", max_iter=500, max_refine=6, tol=1e-10, inner_tol=1e-5,
              orth_passes=0, matrix_free=0, store_bytes=0):
    o = bem_default_opts()
    o.quad_order = quad_order
    o.form = FORMS[form] if isinstance(form, str) else form
    o.prec = PRECS[prec] if isinstance(prec, str) else prec
    o.max_iter = max_iter
    o.max_refine = max_refine
    o.tol = tol
    o.inner_tol = inner_tol
    o.orth_passes = orth_passes
    o.matrix_free = int(matrix_free)
    o.store_bytes = int(store_bytes)
    return o


class Problem:
    """Owns a bem_problem handle; methods map one to one onto the C entry points."""

    def __init__(self, opts: bem_opts | None = None, **kw):
        L = load()
        self._h = ctypes.c_void_p()
        o = opts if opts is not None else make_opts(**kw)
        _check(L.bem_problem_create(ctypes.byref(self._h), ctypes.byref(o)))
        self.opts = o

    def close(self):
        if self._h:
            load().bem_problem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup ---------------------------------------------------------------------------------
    def bem_set_opts(self, opts):
        _check(load().bem_set_opts(self._h, ctypes.byref(opts)))
        self.opts = opts

    def bem_set_domains(self, k, eps):
        ka, kp = _hbuf(k, np.float64)
        ea, ep = _hbuf(eps, np.float64)
        _check(load().bem_set_domains(self._h, len(ka), kp, ep))

    def bem_add_segment(self, xy, P, M, closed):
        a, ptr = _hbuf(xy, np.float64)
        _check(load().bem_add_segment(self._h, a.shape[0], ptr, int(P), int(M), int(bool(closed))))

    @classmethod
    def from_workload(cls, wp, **kw):
        """Build from a workloads.Problem (geometry + domain table)."""
        p = cls(**kw)
        p.bem_set_domains(wp.k, wp.eps)
        for s in wp.segments:
            p.bem_add_segment(s.xy, s.P, s.M, s.closed)
        return p

    def bem_num_elements(self):
        return load().bem_num_elements(self._h)

    def bem_num_unknowns(self):
        return load().bem_num_unknowns(self._h)

    def bem_footprint_bytes(self, n_rhs=1):
        return load().bem_footprint_bytes(self._h, n_rhs)

    # -- compute -------------------------------------------------------------------------------
    def bem_assemble(self, stream=None):
        _check(load().bem_assemble(self._h, _stream_ptr(stream)))

    def bem_get_matrix(self, out, which=0, stream=None):
        _check(load().bem_get_matrix(self._h, which, _dptr(out), _stream_ptr(stream)))
        return out

    def bem_rhs_planewave(self, angles, b_out, stream=None):
        a, ptr = _hbuf(angles, np.float64)
        _check(load().bem_rhs_planewave(self._h, len(a), ptr, _dptr(b_out), _stream_ptr(stream)))
        return b_out

    def bem_matvec(self, x, y, n_rhs=1, stream=None):
        _check(load().bem_matvec(self._h, n_rhs, _dptr(x), _dptr(y), _stream_ptr(stream)))
        return y

    def bem_residual(self, x, b, r, n_rhs=1, stream=None):
        _check(load().bem_residual(self._h, n_rhs, _dptr(x), _dptr(b), _dptr(r), _stream_ptr(stream)))
        return r

    def bem_residual_noalloc(self, x, b, r, n_rhs=1, stream=None):
        """bem_residual without device allocation (static scratch; see include/bem.h)."""
        _check(load().bem_residual_noalloc(self._h, n_rhs, _dptr(x), _dptr(b), _dptr(r), _stream_ptr(stream)))
        return r

    def bem_solve(self, b, x, n_rhs=1, stream=None):
        it = np.zeros(n_rhs, np.int32)
        rs = np.zeros(n_rhs, np.float64)
        st = _check(load().bem_solve(self._h, n_rhs, _dptr(b), _dptr(x), it.ctypes.data_as(ctypes.c_void_p),
                                     rs.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)), allow_noconv=True)
        return st, it, rs

    def bem_solve_planewave(self, angles, x, stream=None):
        a, ptr = _hbuf(angles, np.float64)
        it = np.zeros(len(a), np.int32)
        rs = np.zeros(len(a), np.float64)
        st = _check(load().bem_solve_planewave(self._h, len(a), ptr, _dptr(x), it.ctypes.data_as(ctypes.c_void_p),
                                               rs.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
                    allow_noconv=True)
        return st, it, rs

    def bem_far_field(self, x, angles, out, n_rhs=1, stream=None):
        a, ptr = _hbuf(angles, np.float64)
        _check(load().bem_far_field(self._h, n_rhs, _dptr(x), len(a), ptr, _dptr(out), _stream_ptr(stream)))
        return out

    def bem_near_field(self, x, pts, dom, out, angles=None, n_rhs=1, stream=None):
        pa, pp = _hbuf(pts, np.float64)
        da, dp = _hbuf(dom, np.int32)
        if angles is not None:
            aa, ap = _hbuf(angles, np.float64)
        else:
            ap = None
        _check(load().bem_near_field(self._h, n_rhs, _dptr(x), ap, len(da), pp, dp, _dptr(out), _stream_ptr(stream)))
        return out

    def bem_profile_enable(self, on=True):
        _check(load().bem_profile_enable(self._h, int(bool(on))))

    def bem_profile_read(self):
        """{phase: (device ms, kernel launches)} since the last bem_profile_enable."""
        ms = np.zeros(len(PHASES), np.float64)
        nl = np.zeros(len(PHASES), np.int64)
        _check(load().bem_profile_read(self._h, ms.ctypes.data_as(ctypes.c_void_p), nl.ctypes.data_as(ctypes.c_void_p)))
        return {ph: (float(ms[k]), int(nl[k])) for k, ph in enumerate(PHASES)}

    def bem_solve_planewave_host(self, angles, ff_angles=None, want_traces=True, stream=None):
        """Host buffers in and out: returns (status, traces (n_rhs, 2N) or None, far field or None, iters, resid)."""
        a, ptr = _hbuf(angles, np.float64)
        nr = len(a)
        n2 = self.bem_num_unknowns()
        x = np.zeros((nr, n2), np.complex128) if want_traces else None
        ff = None
        fa, fptr, na = None, None, 0
        if ff_angles is not None:
            fa, fptr = _hbuf(ff_angles, np.float64)
            na = len(fa)
            ff = np.zeros((nr, na), np.complex128)
        it = np.zeros(nr, np.int32)
        rs = np.zeros(nr, np.float64)
        st = _check(load().bem_solve_planewave_host(
            self._h, nr, ptr, x.ctypes.data_as(ctypes.c_void_p) if x is not None else None, na, fptr,
            ff.ctypes.data_as(ctypes.c_void_p) if ff is not None else None, it.ctypes.data_as(ctypes.c_void_p),
            rs.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)), allow_noconv=True)
        return st, x, ff, it, rs


class Batch:
    """Owns a bem_batch engine (batched mixed-precision solves of many problems; see include/bem.h)."""

    def __init__(self, max_slots, pool_unknowns, opts: bem_opts | None = None, **kw):
        L = load()
        self._h = ctypes.c_void_p()
        o = opts if opts is not None else make_opts(**({"prec": "mixed"} | kw))
        _check(L.bem_batch_create(ctypes.byref(self._h), ctypes.byref(o), int(max_slots), int(pool_unknowns)))
        self.opts = o

    def close(self):
        if self._h:
            load().bem_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bem_batch_admit(self, problems, angles, stream=None):
        """Returns (status, slots); slots[i] = -1 for problems that did not fit."""
        n = len(problems)
        hs = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
        a, ptr = _hbuf(angles, np.float64)
        slots = np.full(n, -1, np.int32)
        st = load().bem_batch_admit(self._h, n, ctypes.cast(hs, ctypes.c_void_p), ptr,
                                    slots.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream))
        if st not in (BEM_OK, BEM_ENOMEM):
            _check(st)
        return st, slots

    def bem_batch_step(self, stream=None):
        r = ctypes.c_int(0)
        _check(load().bem_batch_step(self._h, ctypes.byref(r), _stream_ptr(stream)))
        return r.value

    def bem_batch_query(self, slot):
        st, it, rs = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        _check(load().bem_batch_query(self._h, int(slot), ctypes.byref(st), ctypes.byref(it), ctypes.byref(rs)))
        return st.value, it.value, rs.value

    def bem_batch_take(self, slot, x=None, stream=None):
        _check(load().bem_batch_take(self._h, int(slot), _dptr(x) if x is not None else None, _stream_ptr(stream)))
        return x

    def bem_batch_free_units(self):
        return load().bem_batch_free_units(self._h)

    def bem_batch_solve_planewave(self, problems, angles, xs, stream=None):
        n = len(problems)
        hs = (ctypes.c_void_p * n)(*[p._h.value for p in problems])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        a, ptr = _hbuf(angles, np.float64)
        it = np.zeros(n, np.int32)
        rs = np.zeros(n, np.float64)
        st = _check(load().bem_batch_solve_planewave(self._h, n, ctypes.cast(hs, ctypes.c_void_p), ptr,
                                                     ctypes.cast(xp, ctypes.c_void_p),
                                                     it.ctypes.data_as(ctypes.c_void_p),
                                                     rs.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
                    allow_noconv=True)
        return st, it, rs


def bem_test_set_wait_limit(seconds: float) -> None:
    """Wait limit of the tensor-core main loops and of the fused iteration kernel's barriers, for kernels
    launched from now on (0 = defaults); for failure tests."""
    _check(load().bem_test_set_wait_limit(float(seconds)))


def bem_test_set_fused_iteration(on: bool) -> None:
    """False: later solves run each iteration's tail as separate kernels (the non-cooperative path); for tests."""
    _check(load().bem_test_set_fused_iteration(1 if on else 0))


def bem_version() -> str:
    return load().bem_version().decode()


def bem_last_error() -> str:
    return load().bem_last_error().decode()
