"""The serving loop's scheduling on the CPU, with a stand-in for the batch engine (no GPU, no library calls):
requests are admitted in arrival order, the HBM budget is never exceeded, requests that do not fit wait
(deferred admissions), every request completes exactly once, and requests whose complex-FP32 matrix exceeds the
matrix-free limit go to the matrix-free worker instead of a batch slot.  The stand-in engine finishes a problem
a fixed number of steps after its admission; the real engine is covered by the GPU serving tests."""
import time

import numpy as np
import pytest

import workloads as W


class FakeProblem:
    def __init__(self, wp, **opts):
        self.n2 = wp.n_unknowns
        self.opts = opts
        self.closed = False

    @classmethod
    def from_workload(cls, wp, **opts):
        return cls(wp, **opts)

    def bem_num_unknowns(self):
        return self.n2

    def close(self):
        self.closed = True


class FakeBatch:
    """Slots and a pool of unknowns; a problem finishes `steps` engine steps after its admission."""
    steps = 3
    log = None

    def __init__(self, max_slots, pool_unknowns, **opts):
        self.cap, self.pool = max_slots, pool_unknowns
        self.slots = {}
        FakeBatch.log = {"admitted": [], "max_used_bytes": 0, "server": None}

    def bem_batch_free_units(self):
        return self.pool - sum(n for n, _ in self.slots.values())

    def bem_batch_admit(self, probs, angles, stream=None):
        srv = FakeBatch.log["server"]
        FakeBatch.log["max_used_bytes"] = max(FakeBatch.log["max_used_bytes"], srv.used_bytes)
        out = []
        for p in probs:
            free = [s for s in range(self.cap) if s not in self.slots]
            if not free or self.bem_batch_free_units() < p.n2:
                out.append(-1)
                continue
            self.slots[free[0]] = (p.n2, self.steps)
            FakeBatch.log["admitted"].append(p)
            out.append(free[0])
        return 0, out

    def bem_batch_step(self, stream=None):
        for s, (n, left) in list(self.slots.items()):
            self.slots[s] = (n, max(0, left - 1))

    def bem_batch_query(self, slot):
        n, left = self.slots[slot]
        return (2 if left == 0 else 1), self.steps, 1e-9

    def bem_batch_take(self, slot, x=None, stream=None):
        del self.slots[slot]

    def close(self):
        pass


class FakeStream:
    def synchronize(self):
        pass


@pytest.fixture
def serve(monkeypatch):
    import torch
    from paper_2312_12787_gb300 import serve as S
    monkeypatch.setattr(S._bem, "Batch", FakeBatch)
    monkeypatch.setattr(S._bem, "Problem", FakeProblem)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: real_empty(*a, **k))
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)

    def mf_worker(self, device):          # the matrix-free worker without the device: echo a result
        while True:
            item = self._mf_in.get()
            if item is None:
                return
            rid, wp, ang = item
            self._mf_out.put((rid, real_empty(wp.n_unknowns, dtype=torch.complex128), 7, time.perf_counter(), None))

    monkeypatch.setattr(S.Server, "_mf_worker", mf_worker)
    return S


def _requests(sizes, rng):
    """all requests arrive at the start (ties keep their index order), so the admission limits bind"""
    return [(0.0, W.circle_problem(int(n), float(rng.uniform(1, 10)), 7.5), 0.0) for n in sizes]


def test_admission_order_budget_and_completion(serve):
    rng = np.random.default_rng(1)
    reqs = _requests(rng.integers(16, 64, 40), rng)
    budget = 3 * 16 * (2 * 64) ** 2           # room for about three of the largest matrices at a time
    srv = serve.Server(max_slots=8, pool_unknowns=1 << 12, hbm_budget_bytes=budget)
    FakeBatch.log["server"] = srv
    out = {}
    st = srv.run(reqs, out=out, stream=FakeStream(), time_limit_s=60)
    assert st.n_done == len(reqs) and sorted(out) == list(range(len(reqs)))
    assert FakeBatch.log["max_used_bytes"] <= budget
    assert st.deferred > 0 and st.max_resident <= 8
    # admitted in arrival order: the admitted problems' sizes follow the request order
    assert [p.n2 for p in FakeBatch.log["admitted"]] == [wp.n_unknowns for _, wp, _ in reqs]
    assert all(p.closed for p in FakeBatch.log["admitted"])
    assert srv.used_bytes == 0 and not srv.resident
    assert len(st.latencies_s) == len(reqs) and min(st.latencies_s) >= 0
    srv.close()


def test_slot_limit_and_pool_limit_defer(serve):
    rng = np.random.default_rng(2)
    reqs = _requests([40] * 12, rng)
    srv = serve.Server(max_slots=2, pool_unknowns=200, hbm_budget_bytes=1 << 40)
    FakeBatch.log["server"] = srv
    st = srv.run(reqs, stream=FakeStream(), time_limit_s=60)
    assert st.n_done == 12 and st.max_resident <= 2 and st.deferred > 0
    srv.close()


def test_oversized_requests_go_matrix_free(serve):
    rng = np.random.default_rng(3)
    sizes = [20, 200, 24, 180, 30]
    reqs = _requests(sizes, rng)
    limit = 8 * (2 * 100) ** 2                 # complex-FP32 matrices above N_e = 100 go matrix-free
    srv = serve.Server(max_slots=4, pool_unknowns=1 << 12, hbm_budget_bytes=1 << 40, matrix_free_bytes=limit)
    FakeBatch.log["server"] = srv
    out = {}
    st = srv.run(reqs, out=out, stream=FakeStream(), time_limit_s=60)
    assert st.n_done == 5 and st.matrix_free == 2 and sorted(out) == list(range(5))
    assert [p.n2 for p in FakeBatch.log["admitted"]] == [2 * n for n in sizes if n <= 100]
    assert out[1].shape == (400,) and out[3].shape == (360,)
    assert srv.used_bytes == 0
    srv.close()
