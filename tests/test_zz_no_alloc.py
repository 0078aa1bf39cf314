"""bem_residual_noalloc: the refinement residual for callers that cannot let the library allocate device
memory (for example because their device memory belongs to their own arena or caching allocator, or
because a cudaMalloc in a latency-bound loop would stall).  It must agree with bem_residual, which may
allocate the problem's solver workspace to get the same scratch.

Kept in a file that pytest collects last; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_12787_gb300 import build as bld
    bld.build()
    import paper_2312_12787_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("prec,nrhs", [("mixed", 3), ("mixed", 5), ("mixed_tc", 5)])
def test_residual_noalloc_matches_residual(B, prec, nrhs):
    """n_rhs = 3 takes the per-row residual kernel, n_rhs = 5 the tiled one; on a tensor-core problem
    bem_residual forms the small terms on the tensor cores and the no-allocation call on the FP32 pipes.
    Free device memory is unchanged across every no-allocation call, the first one after assembly included
    (assembly does the one-time set-up)."""
    import torch
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                   segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)])
    p = B.Problem.from_workload(wp, prec=prec)
    p.bem_assemble()                         # all allocation happens here, before the no-alloc calls
    n2 = p.bem_num_unknowns()
    g = torch.Generator(device="cpu").manual_seed(42 + nrhs)
    for call in range(2):                    # two calls in a row, different inputs each time
        x = torch.randn((nrhs, n2), dtype=torch.complex128, generator=g).cuda()
        b = torch.randn((nrhs, n2), dtype=torch.complex128, generator=g).cuda()
        r_na = torch.full_like(b, complex(np.nan, np.nan))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        p.bem_residual_noalloc(x, b, r_na, n_rhs=nrhs)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, call     # nothing allocated by the call
        r_ref = torch.empty_like(b)
        p.bem_residual(x, b, r_ref, n_rhs=nrhs)                     # existing entry point
        A = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
        p.bem_get_matrix(A, which=1)
        scale = (A.abs().max() * x.abs().max()).item() * np.sqrt(n2)
        # same tolerance as the residual parity test
        assert torch.isfinite(r_na).all()
        assert (r_na - r_ref).abs().max().item() <= 1e-12 * scale
    p.close()


def test_residual_noalloc_rejects_what_it_cannot_do(B):
    import torch
    wp = W.Problem(k=[5.0, 7.5], eps=[1.0, 2.25], segments=[W.Segment(W.circle(600), P=0, M=1, closed=True)])
    x = torch.zeros((1, 1200), dtype=torch.complex128, device="cuda")
    r = torch.zeros_like(x)
    p = B.Problem.from_workload(wp, prec="mixed")
    with pytest.raises(B.BemError) as e:                 # not assembled: it never assembles itself
        p.bem_residual_noalloc(x, x, r)
    assert e.value.status == B.BEM_ESTATE
    p.bem_assemble()
    big = torch.zeros((437, 1200), dtype=torch.complex128, device="cuda")   # 437 * 1200 > 524288
    with pytest.raises(B.BemError) as e:
        p.bem_residual_noalloc(big, big.clone(), torch.zeros_like(big), n_rhs=437)
    assert e.value.status == B.BEM_EINVAL and "524288" in B.bem_last_error()
    p.close()
    q = B.Problem.from_workload(wp, prec="fp64")
    q.bem_assemble()
    with pytest.raises(B.BemError) as e:                 # FP64 problems have no split matrix
        q.bem_residual_noalloc(x, x, r)
    assert e.value.status == B.BEM_ESTATE
    q.close()
