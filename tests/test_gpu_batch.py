"""GPU tests of the batched engine: many problems of different sizes solved together (random-star sweep)
and continuous batching (problems admitted while others iterate), through the C-ABI."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.util import SOLUTION_TOL_MIXED, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_12787_gb300 import build as bld
    bld.build()
    import paper_2312_12787_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _solve_alone(B, torch, wp, angle, **kw):
    p = B.Problem.from_workload(wp, prec="mixed", **kw)
    x = torch.empty((1, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave([angle], x)
    p.close()
    return x[0].cpu().numpy(), int(it[0]), float(rs[0])


def test_batch_matches_single_problem_solves_and_oracle(B, torch):
    stars = W.cfg_random_stars_c4(count=7, seed=11, n_min=40, n_max=260)
    probs = [B.Problem.from_workload(wp, prec="mixed", tol=1e-10) for wp in stars]
    angles = np.linspace(0.0, 2.0, len(stars))
    xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
    bt = B.Batch(8, sum(p.bem_num_unknowns() for p in probs), tol=1e-10, max_iter=300)
    st, it, rs = bt.bem_batch_solve_planewave(probs, angles, xs)
    assert st == B.BEM_OK and np.all(rs <= 1e-10), (st, rs)
    for k, (wp, a) in enumerate(zip(stars, angles)):
        xa, ita, rsa = _solve_alone(B, torch, wp, a, tol=1e-10)
        assert rel(xs[k].cpu().numpy(), xa) <= 1e-8
    for k in (0, 3):
        wp = stars[k]
        xl = O.solve_lu(O.assemble(wp, Q=4), O.rhs_planewave(wp, angles[k]))
        assert rel(xs[k].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED
    bt.close()
    for p in probs:
        p.close()


def test_continuous_batching_same_result_alone_and_in_mix(B, torch):
    """A problem admitted while others are mid-solve gets exactly the result it gets alone."""
    stars = W.cfg_random_stars_c4(count=4, seed=5, n_min=100, n_max=300)
    angles = [0.3, 1.1, 2.0, 4.0]
    pool = sum(wp.n_unknowns for wp in stars)

    def run(order_groups, steps_between):
        bt = B.Batch(4, pool, tol=1e-10, max_iter=300)
        probs = {k: B.Problem.from_workload(stars[k], prec="mixed", tol=1e-10) for k in range(4)}
        slot_of = {}
        out = {}
        for gi, group in enumerate(order_groups):
            st, slots = bt.bem_batch_admit([probs[k] for k in group], [angles[k] for k in group])
            assert st == B.BEM_OK
            slot_of.update({k: int(s) for k, s in zip(group, slots)})
            for _ in range(steps_between):
                bt.bem_batch_step()
        running = 1
        while running:
            running = bt.bem_batch_step()
        for k, s in slot_of.items():
            state, it, rs = bt.bem_batch_query(s)
            assert state == 2 and rs <= 1e-10
            x = torch.empty(stars[k].n_unknowns, dtype=torch.complex128, device="cuda")
            bt.bem_batch_take(s, x)
            out[k] = (x.cpu().numpy(), it)
        bt.close()
        for p in probs.values():
            p.close()
        return out

    mixed = run([[0], [1, 2], [3]], steps_between=3)
    for k in range(4):
        alone = run([[k]], steps_between=0)[k]
        assert rel(mixed[k][0], alone[0]) <= 1e-12
        assert mixed[k][1] == alone[1]


def test_batch_admission_by_pool_footprint(B, torch):
    stars = W.cfg_random_stars_c4(count=3, seed=2, n_min=100, n_max=120)
    probs = [B.Problem.from_workload(wp, prec="mixed", tol=1e-8) for wp in stars]
    n2 = [p.bem_num_unknowns() for p in probs]
    bt = B.Batch(3, n2[0] + n2[1], tol=1e-8)          # room for two of them
    st, slots = bt.bem_batch_admit(probs, [0.0, 0.0, 0.0])
    assert st == B.BEM_ENOMEM and slots[2] == -1 and slots[0] >= 0 and slots[1] >= 0
    while bt.bem_batch_step():
        pass
    bt.bem_batch_take(int(slots[0]))
    bt.bem_batch_take(int(slots[1]))
    assert bt.bem_batch_free_units() >= n2[2]
    st, s2 = bt.bem_batch_admit([probs[2]], [0.0])
    assert st == B.BEM_OK and s2[0] >= 0
    while bt.bem_batch_step():
        pass
    assert bt.bem_batch_query(int(s2[0]))[0] == 2
    bt.close()
    for p in probs:
        p.close()


@pytest.mark.slow
def test_random_star_sweep_full_c4(B, torch):
    """256 random stars, N_e uniform in [128, 2048], k_e uniform in [1, 40], contrast 1.2-2.0: one batch.
    Every problem reaches the tolerance; sampled problems match their FP64 single-problem solves and the
    smallest sampled one matches the oracle's LU solution."""
    stars = W.cfg_random_stars_c4()
    probs = [B.Problem.from_workload(wp, prec="mixed", tol=1e-8, max_iter=400) for wp in stars]
    xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
    bt = B.Batch(256, sum(p.bem_num_unknowns() for p in probs), tol=1e-8, max_iter=400)
    st, it, rs = bt.bem_batch_solve_planewave(probs, np.zeros(256), xs)
    assert st == B.BEM_OK and np.all(rs <= 1e-8)
    rng = np.random.default_rng(0)
    for k in rng.choice(256, 4, replace=False):
        p64 = B.Problem.from_workload(stars[k], prec="fp64", tol=1e-12, max_iter=600)
        x64 = torch.empty((1, p64.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
        p64.bem_solve_planewave([0.0], x64)
        p64.close()
        assert rel(xs[k].cpu().numpy(), x64[0].cpu().numpy()) <= SOLUTION_TOL_MIXED
    k = int(np.argmin([wp.n_elem for wp in stars]))
    xl = O.solve_lu(O.assemble(stars[k], Q=4), O.rhs_planewave(stars[k], 0.0))
    assert rel(xs[k].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED
    bt.close()
    for p in probs:
        p.close()


def test_high_contrast_concentric_converges_on_every_mixed_path(B, torch):
    """The concentric case of Sec. 7.2 at the high-contrast end of its sweep (eps_2 = 1/eps_3 = 10, omega = 5,
    600 + 1200 elements), where the FP32 inner solves lose orthogonality under the selective second
    Gram-Schmidt pass: the stagnation test must switch the system to two passes, so that the single-problem
    path, the tensor-core path and the batched engine all reach the tolerance and agree with the FP64 solve."""
    wp = W.concentric(600, 1200, 5.0, eps=(1.0, 10.0, 0.1))
    n2 = 2 * wp.n_elem
    p = B.Problem.from_workload(wp, prec="fp64", tol=1e-10, max_iter=1000)
    x64 = torch.empty((1, n2), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave([0.0], x64)
    p.close()
    assert st == B.BEM_OK
    ref = x64[0].cpu().numpy()
    for prec, nr in (("mixed", 1), ("mixed_tc", 2)):
        p = B.Problem.from_workload(wp, prec=prec, tol=1e-8, max_iter=1000)
        x = torch.empty((nr, n2), dtype=torch.complex128, device="cuda")
        st, it, rs = p.bem_solve_planewave([0.0] * nr, x)
        p.close()
        assert st == B.BEM_OK and np.all(rs <= 1e-8), (prec, st, it, rs)
        assert rel(x[0].cpu().numpy(), ref) <= SOLUTION_TOL_MIXED, prec
    q = B.Problem.from_workload(wp, prec="mixed")
    xb = [torch.empty(n2, dtype=torch.complex128, device="cuda")]
    bt = B.Batch(2, n2, tol=1e-8, max_iter=1000)
    st, it, rs = bt.bem_batch_solve_planewave([q], np.zeros(1), xb)
    bt.close()
    q.close()
    assert st == B.BEM_OK and rs[0] <= 1e-8, (st, it, rs)
    assert rel(xb[0].cpu().numpy(), ref) <= SOLUTION_TOL_MIXED


@pytest.mark.parametrize("form", ["orig", "conv", "beta1"])
def test_batch_engine_forms_match_oracle_lu(B, torch, form):
    """The comparison arrangements of Sec. 5-7 through the batched engine (which the omega / eps sweeps and
    the junction study use): a few concentric and junction problems in one batch, each against the oracle's
    LU solution of the same arrangement, element by element."""
    cases = [W.concentric(30, 60, 1.0, eps=(1.0, 2.0, 3.0)),
             W.concentric(40, 80, 2.0, eps=(1.0, 0.5, 2.0)),
             W.junction_disk(120, k=(4.0, 6.0, 7.2)),
             W.junction_disk(160, k=(3.0, 4.5, 6.0))]
    angles = np.array([0.0, 0.7, 1.9, 3.3])
    probs = [B.Problem.from_workload(wp, prec="mixed", form=form, tol=1e-10, max_iter=1000) for wp in cases]
    xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
    bt = B.Batch(len(cases), sum(p.bem_num_unknowns() for p in probs), form=form, tol=1e-10, max_iter=1000)
    st, it, rs = bt.bem_batch_solve_planewave(probs, angles, xs)
    assert st == B.BEM_OK and np.all(rs <= 1e-10), (form, st, it, rs)
    for k, wp in enumerate(cases):
        xl = O.solve_lu(O.assemble(wp, Q=4, form=form), O.rhs_planewave(wp, angles[k], form=form))
        assert rel(xs[k].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED, (form, k)
    bt.close()
    for p in probs:
        p.close()


def test_device_loop_matches_host_stepped_solve(B, torch):
    """bem_batch_solve_planewave runs the whole batched solve as one graph launch (a conditional loop whose
    refinement decisions are taken on the device); admitting the same problems and stepping them from the host
    (bem_batch_step) gives the same solutions and iteration counts."""
    stars = W.cfg_random_stars_c4(count=6, seed=17, n_min=60, n_max=400)
    angles = np.linspace(0.2, 3.0, len(stars))
    pool = sum(wp.n_unknowns for wp in stars)
    probs = [B.Problem.from_workload(wp, prec="mixed", tol=1e-10) for wp in stars]
    xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
    bt = B.Batch(8, pool, tol=1e-10, max_iter=300)
    st, it_loop, rs_loop = bt.bem_batch_solve_planewave(probs, angles, xs)
    assert st == B.BEM_OK and np.all(rs_loop <= 1e-10), (st, rs_loop)
    st, slots = bt.bem_batch_admit(probs, angles)
    assert st == B.BEM_OK
    while bt.bem_batch_step():
        pass
    for k, s in enumerate(slots):
        state, it, rs = bt.bem_batch_query(int(s))
        assert state == 2 and it == it_loop[k] and abs(rs - rs_loop[k]) <= 1e-12 * max(rs, 1e-30) + 1e-30
        x = torch.empty_like(xs[k])
        bt.bem_batch_take(int(s), x)
        assert rel(x.cpu().numpy(), xs[k].cpu().numpy()) <= 1e-12
    bt.close()
    for p in probs:
        p.close()


def test_junction_study_ordering_and_parity_on_gpu(B, torch):
    """Sec. 7.2's junction study through the batched engine: on the junction disk (eps_i = i, omega = 5) the
    modified Calderon arrangement needs the fewest GMRES iterations, then the original one, then the
    conventional one, at N = 200 and 400; the solutions match the oracle's LU solutions of each arrangement."""
    cases = [W.junction_material(200, 5.0, 2.0, 3.0), W.junction_material(400, 5.0, 2.0, 3.0)]
    its = {}
    for form in ("mod", "orig", "conv"):
        probs = [B.Problem.from_workload(wp, prec="mixed", form=form, tol=1e-8, max_iter=1000) for wp in cases]
        xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
        bt = B.Batch(2, sum(p.bem_num_unknowns() for p in probs), form=form, tol=1e-8, max_iter=1000)
        st, it, rs = bt.bem_batch_solve_planewave(probs, np.zeros(2), xs)
        assert st == B.BEM_OK and np.all(rs <= 1e-8), (form, st, it, rs)
        its[form] = it
        wp = cases[0]
        xl = O.solve_lu(O.assemble(wp, Q=4, form=form), O.rhs_planewave(wp, 0.0, form=form))
        assert rel(xs[0].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED, form
        bt.close()
        for p in probs:
            p.close()
    for k in range(2):
        assert its["mod"][k] < its["orig"][k] < its["conv"][k], (k, its)
