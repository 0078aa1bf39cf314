"""Serving loop (continuous batching) on a short Poisson stream mixing circles, ellipses and two-material
junction disks: every result equals the one the same problem gets alone, and matches the FP64 path."""
import numpy as np
import pytest

import workloads as W
from tests.util import SOLUTION_TOL_MIXED, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2312_12787_gb300 import build as bld
    bld.build()
    import paper_2312_12787_gb300 as M
    M.load()
    return M


def test_serving_stream_results_equal_alone(P):
    import torch
    from paper_2312_12787_gb300 import serve
    stream = W.cfg_serving_c5(count=14, seed=9, rate=400.0, n_min=64, n_max=700)
    requests = [(t, wp, 0.0) for t, wp in stream]
    srv = serve.Server(max_slots=6, pool_unknowns=6000, tol=1e-10, max_iter=300)
    out = {}
    st = srv.run(requests, out=out, time_limit_s=120)
    srv.close()
    s = st.summary()
    assert s["solves"] == len(requests) and s["p99_ms"] >= s["p50_ms"] > 0
    assert st.max_resident >= 2                        # requests really overlapped on the device
    for rid, (t, wp, ang) in enumerate(requests):
        bt = P.Batch(1, wp.n_unknowns, tol=1e-10, max_iter=300)
        p = P.Problem.from_workload(wp, prec="mixed", tol=1e-10, max_iter=300)
        x = torch.empty(wp.n_unknowns, dtype=torch.complex128, device="cuda")
        status, it, rs = bt.bem_batch_solve_planewave([p], [ang], [x])
        bt.close()
        p.close()
        assert rel(out[rid].cpu().numpy(), x.cpu().numpy()) <= 1e-12
        if rid % 4 == 0:
            q = P.Problem.from_workload(wp, prec="fp64", tol=1e-12, max_iter=600)
            x64 = torch.empty((1, wp.n_unknowns), dtype=torch.complex128, device="cuda")
            q.bem_solve_planewave([ang], x64)
            q.close()
            assert rel(out[rid].cpu().numpy(), x64[0].cpu().numpy()) <= SOLUTION_TOL_MIXED


def test_serving_defers_when_budget_is_full(P):
    from paper_2312_12787_gb300 import serve
    stream = W.cfg_serving_c5(count=6, seed=4, rate=1e6, n_min=200, n_max=260)
    requests = [(0.0, wp, 0.0) for _, wp in stream]
    one = max(serve.matrix_bytes(wp) for _, wp, _ in requests)
    srv = serve.Server(max_slots=6, pool_unknowns=100000, hbm_budget_bytes=2 * one, tol=1e-8)
    st = srv.run(requests, time_limit_s=120)
    srv.close()
    assert st.n_done == 6 and st.max_resident <= 2 and st.deferred > 0


def test_serving_routes_oversized_requests_matrix_free(P):
    """Requests whose complex-FP32 matrix exceeds the limit are solved matrix-free (rows within the limit stored,
    the rest recomputed) on a worker stream while the batch engine serves the rest; every result matches the
    stored-matrix FP64 solve."""
    import torch
    from paper_2312_12787_gb300 import serve
    stream = W.cfg_serving_c5(count=8, seed=21, rate=400.0, n_min=64, n_max=500)
    requests = [(t, wp, 0.3) for t, wp in stream]
    sizes = sorted(serve.c32_matrix_bytes(wp) for _, wp, _ in requests)
    limit = sizes[len(sizes) // 2]                         # the larger half goes matrix-free
    n_mf = sum(serve.c32_matrix_bytes(wp) > limit for _, wp, _ in requests)
    assert 1 <= n_mf < len(requests)
    srv = serve.Server(max_slots=6, pool_unknowns=6000, tol=1e-10, max_iter=300, matrix_free_bytes=limit)
    out = {}
    st = srv.run(requests, out=out, time_limit_s=300)
    srv.close()
    assert st.n_done == len(requests) and st.matrix_free == n_mf
    for rid, (t, wp, ang) in enumerate(requests):
        q = P.Problem.from_workload(wp, prec="fp64", tol=1e-12, max_iter=600)
        x64 = torch.empty((1, wp.n_unknowns), dtype=torch.complex128, device="cuda")
        q.bem_solve_planewave([ang], x64)
        q.close()
        assert rel(out[rid].cpu().numpy(), x64[0].cpu().numpy()) <= SOLUTION_TOL_MIXED, rid
