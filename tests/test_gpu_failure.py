"""Failure paths through the C interface: iteration limits (BEM_ENOCONV with the best iterate written) and
bounded device waits that run out (BEM_ETIMEOUT, with the context still usable afterwards).

No test here faults, traps or hangs the GPU: the timeouts are provoked by a short main-loop wait limit of
the tensor-core product, whose drain waits keep their full limit, and by a short barrier wait limit of the
fused GMRES iteration kernel, whose waits then give up and let the kernel run on with every access in bounds.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_12787_gb300 import build as bld
    bld.build()
    import paper_2312_12787_gb300 as P
    P.load()
    return P


def test_fp64_iteration_limit_returns_enoconv_with_the_gmres_iterate(B):
    """max_iter = 5 on the circle of 256 elements: BEM_ENOCONV, five iterations, and the written x is the
    fifth GMRES iterate (the minimiser of the residual over the Krylov space K_5, Sec. 3.2), which the
    oracle's GMRES stopped after five iterations gives independently."""
    import torch
    wp = W.cfg_circle_c1(256)
    p = B.Problem.from_workload(wp, prec="fp64", tol=1e-10, max_iter=5)
    x = torch.full((1, 512), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave(np.array([0.0]), x)
    assert st == B.BEM_ENOCONV and "iteration limit" in B.bem_last_error()
    assert it[0] == 5 and rs[0] > 1e-10
    xg = x[0].cpu().numpy()
    assert np.all(np.isfinite(xg))
    A = O.assemble(wp, Q=4)
    b = O.rhs_planewave(wp, 0.0)
    x5, m, hist = O.gmres(A, b, tol=0.0, maxit=5)
    assert m == 5
    assert np.linalg.norm(xg - x5) / np.linalg.norm(x5) < 1e-9
    true_res = np.linalg.norm(b - A @ xg) / np.linalg.norm(b)
    assert abs(rs[0] - true_res) <= 1e-6 * true_res
    assert abs(rs[0] - hist[-1]) <= 1e-6 * hist[-1]
    p.close()


@pytest.mark.parametrize("prec", ["mixed", "mixed_tc"])
def test_mixed_refinement_limit_returns_enoconv_with_its_residual(B, prec):
    """Mixed paths with two refinement steps of five inner iterations: BEM_ENOCONV, a finite x, and the
    reported residual is the FP64 residual of that x (checked with the oracle's matrix)."""
    import torch
    wp = W.cfg_circle_c1(256)
    ang = np.array([0.0, 1.1])
    p = B.Problem.from_workload(wp, prec=prec, tol=1e-10, max_iter=5, max_refine=2)
    x = torch.full((2, 512), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave(ang, x)
    assert st == B.BEM_ENOCONV
    assert np.all(it == 10) and np.all(rs > 1e-10)
    xs = x.cpu().numpy()
    assert np.all(np.isfinite(xs))
    A = O.assemble(wp, Q=4)
    for r, t in enumerate(ang):
        b = O.rhs_planewave(wp, t)
        true_res = np.linalg.norm(b - A @ xs[r]) / np.linalg.norm(b)
        assert abs(rs[r] - true_res) <= 1e-6 * true_res
    p.close()


def test_batch_iteration_limit_returns_enoconv(B):
    import torch
    probs = [B.Problem.from_workload(W.circle_problem(n, 5.0, 7.5), prec="mixed", max_iter=5, max_refine=1)
             for n in (200, 330)]
    xs = [torch.full((p.bem_num_unknowns(),), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
          for p in probs]
    bt = B.Batch(4, 2000, max_iter=5, max_refine=1)
    st, it, rs = bt.bem_batch_solve_planewave(probs, np.zeros(2), xs)
    assert st == B.BEM_ENOCONV
    assert np.all(it == 5) and np.all(rs > 1e-10) and np.all(np.isfinite(rs))
    for x in xs:
        assert torch.isfinite(x).all()
    bt.close()
    for p in probs:
        p.close()


def test_tensor_core_wait_expiry_returns_etimeout_and_the_next_call_succeeds(B):
    """A main-loop wait limit of 1 ns makes waits of the tensor-core product run out: the kernel records the
    expiry, drains its own copies and MMAs with the full limit and returns; bem_matvec reads the error word
    and returns BEM_ETIMEOUT.  With the default limit restored, the same product on the same problem succeeds
    and matches the FP64 product of the stored matrix."""
    import torch
    wp = W.cfg_star_c2(2048)
    p = B.Problem.from_workload(wp, prec="mixed_tc")
    p.bem_assemble()
    n2 = p.bem_num_unknowns()
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn((4, n2), dtype=torch.complex128, generator=g).cuda()
    y = torch.zeros_like(x)
    try:
        B.bem_test_set_wait_limit(1e-9)
        with pytest.raises(B.BemError) as e:
            p.bem_matvec(x, y, n_rhs=4)
        assert e.value.status == B.BEM_ETIMEOUT
        assert "wait expired" in B.bem_last_error()
    finally:
        B.bem_test_set_wait_limit(0.0)
    torch.cuda.synchronize()
    p.bem_matvec(x, y, n_rhs=4)
    A = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
    p.bem_get_matrix(A, which=0)
    ref = (A @ x.T).T
    err = ((y - ref).abs().max(dim=1).values / ref.abs().max(dim=1).values).max().item()
    assert err < 5e-6
    with pytest.raises(B.BemError):
        B.bem_test_set_wait_limit(-1.0)
    p.close()


def test_gram_schmidt_barrier_expiry_returns_etimeout_and_the_next_solve_succeeds(B):
    """A barrier wait limit of 1 ns makes the per-system barrier waits of the fused iteration kernel run out:
    the kernel records the expiry and goes on without waiting (every later wait of the run is skipped), the
    solve runs to its iteration limit and returns BEM_ETIMEOUT.  A problem created after the default is
    restored solves to the tolerance (mixed path: no tensor-core waits are involved)."""
    import torch
    wp = W.cfg_circle_c1(256)
    ang = np.array([0.0, 0.7, 1.9])
    x = torch.zeros((3, 512), dtype=torch.complex128, device="cuda")
    try:
        B.bem_test_set_wait_limit(1e-9)
        p = B.Problem.from_workload(wp, prec="mixed", tol=1e-10, max_iter=30, max_refine=1)
        with pytest.raises(B.BemError) as e:
            p.bem_solve_planewave(ang, x)
        assert e.value.status == B.BEM_ETIMEOUT
        assert "barrier" in B.bem_last_error()
        p.close()
    finally:
        B.bem_test_set_wait_limit(0.0)
    torch.cuda.synchronize()
    p = B.Problem.from_workload(wp, prec="mixed", tol=1e-10)
    st, it, rs = p.bem_solve_planewave(ang, x)
    assert st == B.BEM_OK and np.all(rs <= 1e-10)
    A = O.assemble(wp, Q=4)
    xs = x.cpu().numpy()
    for r, t in enumerate(ang):
        b = O.rhs_planewave(wp, t)
        assert np.linalg.norm(b - A @ xs[r]) / np.linalg.norm(b) < 1e-9
    p.close()
