"""The C-ABI library builds, loads without a GPU and exports every symbol include/bem.h declares;
host-side argument validation (no device work)."""
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_12787_gb300 import build as B
    B.build()
    import paper_2312_12787_gb300 as P
    return P


def _declared():
    txt = open(os.path.join(ROOT, "include", "bem.h")).read()
    return sorted(set(re.findall(r"BEM_API\s+[\w\s\*]+?\b(bem_\w+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared()
    assert "bem_solve" in names and "bem_assemble" in names and len(names) >= 19


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.bem.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(bem_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    L = lib.load()
    for n in _declared():
        assert hasattr(L, n)
    assert set(lib.EXPORTS) == set(_declared())


def test_version_and_defaults(lib):
    assert "sm_103a" in lib.bem_version()
    o = lib.bem.bem_default_opts()
    assert o.quad_order == 4 and o.form == lib.BEM_FORM_MOD and o.prec == lib.BEM_PREC_FP64
    assert o.tol == 1e-10 and o.max_iter == 500 and o.orth_passes == 0


def test_host_validation(lib):
    P = lib.Problem
    with pytest.raises(lib.BemError):
        P(quad_order=0)
    with pytest.raises(lib.BemError):
        P(max_iter=5000)
    p = P()
    with pytest.raises(lib.BemError) as e:
        p.bem_set_domains([1.0, 2.0], [2.0, 1.0])          # host eps must be 1
    assert e.value.status == lib.BEM_EINVAL
    with pytest.raises(lib.BemError):
        p.bem_set_domains([1.0, -2.0], [1.0, 1.0])         # k <= 0
    with pytest.raises(lib.BemError):
        p.bem_set_domains([1.0, 2.0], [1.0, -1.0])         # eps = -1: cluster at the origin (Sec. 5)
    with pytest.raises(lib.BemError):
        p.bem_set_domains([1.0, np.nan], [1.0, 1.0])
    p.bem_set_domains([5.0, 7.5], [1.0, 2.25])
    with pytest.raises(lib.BemError):
        p.bem_add_segment(np.array([[0, 0], [1, 0.0]]), 0, 1, True)      # closed needs 3 vertices
    with pytest.raises(lib.BemError):
        p.bem_add_segment(np.array([[0, 0], [1, 0.0], [1, 0.0]]), 0, 1, False)   # zero-length element
    with pytest.raises(lib.BemError):
        p.bem_add_segment(np.array([[0, 0], [1, 0.0], [0, 1.0]]), 1, 1, True)    # P == M
    with pytest.raises(lib.BemError):
        p.bem_add_segment(np.array([[0, 0], [1, np.inf], [0, 1.0]]), 0, 1, True)
    p.bem_add_segment(np.array([[0, 0], [1, 0.0], [0, 1.0]]), 0, 1, True)
    assert p.bem_num_elements() == 3 and p.bem_num_unknowns() == 6
    assert p.bem_footprint_bytes(1) > 6 * 6 * 16
    p.close()
    # matrix-free: FP64 and MIXED (with stored rows) are valid, MIXED_TC is not; stored bytes must be >= 0
    with pytest.raises(lib.BemError):
        P(prec="mixed_tc", matrix_free=1)
    with pytest.raises(lib.BemError):
        P(prec="mixed", matrix_free=1, store_bytes=-1)
    for kw in (dict(prec="fp64", matrix_free=1), dict(prec="mixed", matrix_free=1, store_bytes=1 << 20)):
        q = P(**kw)
        q.bem_set_domains([5.0, 7.5], [1.0, 2.25])
        q.bem_add_segment(W.circle(40), 0, 1, True)
        if kw["prec"] == "mixed":
            # stored element rows: 1 MiB / (2 rows x 80 complex FP32) = 819 >= 40, so the whole matrix is kept
            full = P(prec="mixed")
            full.bem_set_domains([5.0, 7.5], [1.0, 2.25])
            full.bem_add_segment(W.circle(40), 0, 1, True)
            assert q.bem_footprint_bytes(1) < full.bem_footprint_bytes(1)
            full.close()
        q.close()


def test_workload_generators_shapes():
    import workloads as W
    assert W.cfg_circle_c1().n_elem == 256
    assert W.cfg_star_c2().n_elem == 4096
    p3 = W.cfg_junction_c3()
    assert p3.n_elem == 8192 and len(p3.segments) == 3
    c4 = W.cfg_random_stars_c4()
    assert len(c4) == 256 and all(128 <= q.n_elem <= 2048 for q in c4)
    c5 = W.cfg_serving_c5(count=50)
    assert all(t2 > t1 for (t1, _), (t2, _) in zip(c5, c5[1:]))
    # the sweeps of Sec. 7.1 / 7.2: k_d = omega sqrt(eps_d) in every domain (Sec. 2)
    sw = W.cfg_omega_eps_sweep()
    assert len(sw) == 128 and {lab for lab, _, _ in sw} == {"omega", "eps"}
    for lab, v, q in sw:
        assert q.n_elem == 600 and q.eps[0] == 1.0
        om = q.k[0]
        assert np.allclose(q.k, [om * np.sqrt(e) for e in q.eps], rtol=1e-14)
        assert (om == v) if lab == "omega" else (q.eps[1] == v and om == 5.0)
    cs = W.cfg_concentric_sweep()
    assert len(cs) == 64
    for lab, v, q in cs:
        assert q.n_elem == 1800 and len(q.k) == 3
        assert np.allclose(q.k, [q.k[0] * np.sqrt(e) for e in q.eps], rtol=1e-14)
        if lab == "eps":
            assert q.eps[2] == v and abs(q.eps[1] * q.eps[2] - 1.0) < 1e-14


def test_empty_and_null_arguments_rejected_before_device_work(lib):
    """Empty inputs (n_rhs = 0, n_ang = 0, n_pts = 0) and NULL buffers are argument errors, reported before any
    device call: on a machine without a GPU a call that reached the device would answer BEM_ECUDA instead."""
    import ctypes
    L = lib.load()
    p = lib.Problem(prec="mixed")
    p.bem_set_domains([5.0, 7.5], [1.0, 2.25])
    p.bem_add_segment(np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0], [0.0, -1.0]]), 0, 1, True)
    h = p._h
    ang = np.zeros(2)
    ap = ang.ctypes.data_as(ctypes.c_void_p)
    buf = ctypes.c_void_p(1 << 20)          # never dereferenced: every call below fails validation first
    it = np.zeros(2, np.int32)
    rs = np.zeros(2)
    itp, rsp = it.ctypes.data_as(ctypes.c_void_p), rs.ctypes.data_as(ctypes.c_void_p)
    calls = {
        "rhs n_rhs=0": lambda: L.bem_rhs_planewave(h, 0, ap, buf, None),
        "rhs NULL angles": lambda: L.bem_rhs_planewave(h, 1, None, buf, None),
        "matvec n_rhs=0": lambda: L.bem_matvec(h, 0, buf, buf, None),
        "matvec NULL y": lambda: L.bem_matvec(h, 1, buf, None, None),
        "residual n_rhs=0": lambda: L.bem_residual(h, 0, buf, buf, buf, None),
        "residual NULL r": lambda: L.bem_residual(h, 1, buf, buf, None, None),
        "noalloc n_rhs=0": lambda: L.bem_residual_noalloc(h, 0, buf, buf, buf, None),
        "noalloc r aliases x": lambda: L.bem_residual_noalloc(h, 1, buf, ctypes.c_void_p(1 << 21), buf, None),
        "solve n_rhs=0": lambda: L.bem_solve(h, 0, buf, buf, itp, rsp, None),
        "solve NULL b": lambda: L.bem_solve(h, 1, None, buf, itp, rsp, None),
        "solve_planewave n_rhs=0": lambda: L.bem_solve_planewave(h, 0, ap, buf, itp, rsp, None),
        "solve_planewave NULL x": lambda: L.bem_solve_planewave(h, 1, ap, None, itp, rsp, None),
        "far_field n_ang=0": lambda: L.bem_far_field(h, 1, buf, 0, ap, buf, None),
        "far_field n_rhs=0": lambda: L.bem_far_field(h, 0, buf, 2, ap, buf, None),
        "near_field n_pts=0": lambda: L.bem_near_field(h, 1, buf, None, 0, ap, ap, buf, None),
        "host solve n_rhs=0": lambda: L.bem_solve_planewave_host(h, 0, ap, None, 0, None, None, itp, rsp, None),
        "NULL problem": lambda: L.bem_matvec(None, 1, buf, buf, None),
    }
    for what, call in calls.items():
        assert call() == lib.BEM_EINVAL, what
        assert L.bem_last_error().decode(), what
    # the no-allocation residual never assembles: an unassembled problem is a state error, again host-side
    assert L.bem_residual_noalloc(h, 1, buf, ctypes.c_void_p(1 << 21), ctypes.c_void_p(1 << 22), None) == lib.BEM_ESTATE
    assert L.bem_num_unknowns(None) == 0 and L.bem_footprint_bytes(h, 0) == 0
    p.close()


def test_binding_signatures_match_the_header(lib):
    """Every entry point of include/bem.h has ctypes argument types in the binding, one per declared parameter
    and of the declared kind (pointers as pointers, so that no 64-bit address is passed as a C int)."""
    import ctypes
    L = lib.load()
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bem.h")).read(), flags=re.S)
    decls = re.findall(r"BEM_API\s+([\w\s\*]+?)\b(bem_\w+)\s*\(([^)]*)\)", txt)
    assert len(decls) == len(_declared())
    ptr_types = (ctypes.c_void_p, ctypes.c_char_p)
    for ret, name, params in decls:
        params = [q.strip() for q in params.split(",") if q.strip() and q.strip() != "void"]
        f = getattr(L, name)
        assert f.argtypes is not None and len(f.argtypes) == len(params), name
        for q, t in zip(params, f.argtypes):
            if "*" in q:
                assert t in ptr_types or issubclass(t, ctypes._Pointer), (name, q, t)
            elif "long long" in q:
                assert t is ctypes.c_longlong, (name, q, t)
            elif "size_t" in q:
                assert t is ctypes.c_size_t, (name, q, t)
            elif "double" in q:
                assert t is ctypes.c_double, (name, q, t)
            else:
                assert t is ctypes.c_int, (name, q, t)
        ret = ret.strip()
        if "*" in ret:
            assert f.restype in ptr_types, (name, ret)
        elif ret == "void":
            assert f.restype is None, name
        elif ret == "long long":
            assert f.restype is ctypes.c_longlong, name
        elif ret == "size_t":
            assert f.restype is ctypes.c_size_t, name
        else:
            assert f.restype is ctypes.c_int, (name, ret, f.restype)


def test_missing_library_fails_loudly(tmp_path):
    """There is no CPU fallback: without libbem.so the binding raises instead of computing anything."""
    import subprocess
    import sys
    code = ("import paper_2312_12787_gb300.bem as b\n"
            "b.LIB_PATH = %r\n"
            "try:\n"
            "    b.Problem()\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n" % str(tmp_path / "libbem.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and "raised:" in out.stdout and "missing" in out.stdout, out.stdout + out.stderr
