"""Request loop for solve requests arriving over time (continuous batching on the batch engine).

Requests (a workloads.Problem and an incident angle each) arrive at given times.  The loop admits arrived
requests in arrival order as long as they fit: a free slot, a contiguous run of free unknowns in the engine's
pools (Krylov bases, solutions, residuals, right-hand sides) and room in the HBM budget for their matrices
(complex FP32 plus remainder, 16 bytes per entry).  Admitted requests are assembled together in one launch and
then iterate together with the ones already on the device; finished solves are taken out at once, which frees
their slot, pool space and matrix.  Latency is measured from arrival to the moment the solution is back in a
device buffer.  All compute runs in libbem; this module only schedules.

Requests whose complex-FP32 matrix would exceed `matrix_free_bytes` (8e9 by default: N_e above ~15.8k) are
recomputed above that limit: a worker thread solves them one at a time with the matrix-free mixed path, which keeps
the leading rows that fit in `matrix_free_bytes` as complex FP32 and recomputes the others in every inner product
(the refinement residual recomputes every entry with FP64 sums), on a CUDA stream of its own, while the batch
engine keeps iterating the others.  Their HBM footprint (stored rows and Krylov basis) is charged to the budget
while they run.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import bem as _bem


@dataclass
class ServeStats:
    n_done: int = 0
    wall_s: float = 0.0
    latencies_s: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    max_resident: int = 0
    admissions: int = 0
    deferred: int = 0          # admission attempts that had to wait for space
    matrix_free: int = 0       # requests solved by the matrix-free path
    overlapped: int = 0        # matrix-free solves that finished while batch slots were resident

    def summary(self):
        lat = np.array(self.latencies_s) if self.latencies_s else np.zeros(1)
        return {"solves": self.n_done, "wall_s": self.wall_s,
                "solves_per_s": self.n_done / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_iters": float(np.mean(self.iters)) if self.iters else 0.0,
                "max_resident": self.max_resident, "deferred_admissions": self.deferred,
                "matrix_free": self.matrix_free, "matrix_free_overlapped": self.overlapped}


def matrix_bytes(wp) -> int:
    n2 = wp.n_unknowns
    return 16 * n2 * n2


def c32_matrix_bytes(wp) -> int:
    n2 = wp.n_unknowns
    return 8 * n2 * n2


def mf_footprint_bytes(wp, max_iter, store_bytes=0) -> int:
    """Device bytes of a matrix-free mixed solve: the stored rows (whole elements, two rows of 2N complex FP32
    each, within store_bytes), the FP32 Krylov basis and the Hessenberg data."""
    n2 = wp.n_unknowns
    per_elem = 2 * n2 * 8
    stored = min(wp.n_elem, int(store_bytes) // per_elem) * per_elem
    return stored + 8 * (max_iter + 1) * n2 + 16 * max_iter * (max_iter + 1) + 64 * n2


class Server:
    """Continuous-batching solver: slots of a bem_batch engine plus an HBM budget for matrices."""

    def __init__(self, max_slots=128, pool_unknowns=1 << 21, hbm_budget_bytes=64 << 30, tol=1e-8, max_iter=300,
                 prec="mixed", quad_order=4, matrix_free_bytes=8e9, mf_max_iter=600, inner_tol=1e-5, orth_passes=0):
        self.opts = dict(prec=prec, tol=tol, max_iter=max_iter, quad_order=quad_order, inner_tol=inner_tol,
                         orth_passes=orth_passes)
        self.batch = _bem.Batch(max_slots, pool_unknowns, **self.opts)
        self.batch_max_slots = max_slots
        self.budget = hbm_budget_bytes
        self.resident = {}          # slot -> (request id, problem, matrix bytes)
        self.used_bytes = 0
        self.mf_limit = matrix_free_bytes
        self.mf_opts = dict(prec="mixed", matrix_free=1, store_bytes=int(matrix_free_bytes), tol=tol,
                            max_iter=mf_max_iter, quad_order=quad_order, inner_tol=inner_tol, orth_passes=orth_passes)
        self._mf_in = queue.Queue()
        self._mf_out = queue.Queue()
        self._mf_thread = None

    def close(self):
        for (_, p, _) in self.resident.values():
            p.close()
        self.resident.clear()
        if self._mf_thread is not None:
            self._mf_in.put(None)
            self._mf_thread.join()
            self._mf_thread = None
        self.batch.close()

    def _mf_worker(self, device):
        """Matrix-free solves, one at a time, on a stream of their own (ctypes releases the GIL in the calls)."""
        import torch
        torch.cuda.set_device(device)
        stream = torch.cuda.Stream()
        while True:
            item = self._mf_in.get()
            if item is None:
                return
            rid, wp, ang = item
            try:
                p = _bem.Problem.from_workload(wp, **self.mf_opts)
                with torch.cuda.stream(stream):
                    x = torch.empty((1, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
                st, it, rs = p.bem_solve_planewave([ang], x, stream=stream)
                stream.synchronize()
                p.close()
                self._mf_out.put((rid, x[0], int(it[0]), time.perf_counter(), None))
            except Exception as e:   # reported to the loop, which re-raises
                self._mf_out.put((rid, None, 0, time.perf_counter(), e))

    def run(self, requests, out=None, stream=None, time_limit_s=600.0):
        """requests: list of (arrival_s, workloads.Problem, angle).  Arrival times are relative to the start
        of the run (wall clock).  Returns ServeStats; if `out` is a dict, solutions (torch tensors) are stored
        there by request index."""
        import torch
        st = ServeStats()
        order = sorted(range(len(requests)), key=lambda i: requests[i][0])
        waiting = []                # arrived, not admitted
        nxt = 0
        t0 = time.perf_counter()
        pending = len(requests)
        mf_running = {}             # request id -> footprint bytes (queued at or running in the worker)
        while pending:
            now = time.perf_counter() - t0
            if now > time_limit_s:
                raise TimeoutError("serving run exceeded its time limit")
            while nxt < len(order) and requests[order[nxt]][0] <= now:
                waiting.append(order[nxt])
                nxt += 1
            # finished matrix-free solves
            while True:
                try:
                    rid, x, it, t_done, err = self._mf_out.get_nowait()
                except queue.Empty:
                    break
                if err is not None:
                    raise err
                self.used_bytes -= mf_running.pop(rid)
                st.latencies_s.append(t_done - t0 - requests[rid][0])
                st.iters.append(it)
                st.n_done += 1
                st.matrix_free += 1
                if self.resident:
                    st.overlapped += 1
                pending -= 1
                if out is not None:
                    out[rid] = x
            # admit in arrival order while the head of the queue fits
            batch_ids, batch_probs, batch_angles = [], [], []
            while waiting:
                rid = waiting[0]
                wp = requests[rid][1]
                if c32_matrix_bytes(wp) > self.mf_limit:
                    need = mf_footprint_bytes(wp, self.mf_opts["max_iter"], self.mf_opts["store_bytes"])
                    if self.used_bytes + need > self.budget:
                        st.deferred += 1
                        break
                    waiting.pop(0)
                    if self._mf_thread is None:
                        self._mf_thread = threading.Thread(target=self._mf_worker, args=(torch.cuda.current_device(),),
                                                           daemon=True)
                        self._mf_thread.start()
                    mf_running[rid] = need
                    self.used_bytes += need
                    self._mf_in.put((rid, wp, requests[rid][2]))
                    continue
                need = matrix_bytes(wp)
                units = sum(p.bem_num_unknowns() for p in batch_probs) + wp.n_unknowns
                if (self.used_bytes + need > self.budget or self.batch.bem_batch_free_units() < units or
                        len(self.resident) + len(batch_probs) >= self.batch_max_slots):
                    st.deferred += 1
                    break
                waiting.pop(0)
                p = _bem.Problem.from_workload(wp, **self.opts)
                batch_ids.append(rid)
                batch_probs.append(p)
                batch_angles.append(requests[rid][2])
                self.used_bytes += need
            if batch_probs:
                status, slots = self.batch.bem_batch_admit(batch_probs, batch_angles, stream)
                for rid, p, s in zip(batch_ids, batch_probs, slots):
                    if s < 0:           # did not fit after all (fragmented pool): back to the queue head
                        self.used_bytes -= matrix_bytes(requests[rid][1])
                        p.close()
                        waiting.insert(0, rid)
                    else:
                        self.resident[int(s)] = (rid, p, matrix_bytes(requests[rid][1]))
                        st.admissions += 1
                st.max_resident = max(st.max_resident, len(self.resident))
            if not self.resident:
                # idle until the next arrival or the next matrix-free result
                if nxt < len(order):
                    time.sleep(max(0.0, min(0.002, requests[order[nxt]][0] - (time.perf_counter() - t0))))
                elif mf_running:
                    time.sleep(0.002)
                continue
            self.batch.bem_batch_step(stream)
            for s in list(self.resident):
                state, it, rs = self.batch.bem_batch_query(s)
                if state != 2:
                    continue
                rid, p, nbytes = self.resident.pop(s)
                x = torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda")
                self.batch.bem_batch_take(s, x, stream)
                (stream or torch.cuda.current_stream()).synchronize()
                st.latencies_s.append(time.perf_counter() - t0 - requests[rid][0])
                st.iters.append(it)
                st.n_done += 1
                pending -= 1
                if out is not None:
                    out[rid] = x
                p.close()
                self.used_bytes -= nbytes
        st.wall_s = time.perf_counter() - t0
        return st


def serve_fp64_sequential(requests, tol=1e-8, max_iter=600, quad_order=4, out=None, time_limit_s=600.0):
    """Baseline: the same requests through the plain FP64 single-problem path, one at a time in arrival
    order (no batching).  Returns ServeStats."""
    import torch
    st = ServeStats()
    order = sorted(range(len(requests)), key=lambda i: requests[i][0])
    t0 = time.perf_counter()
    for rid in order:
        arr, wp, ang = requests[rid]
        now = time.perf_counter() - t0
        if now > time_limit_s:
            raise TimeoutError("FP64 serving run exceeded its time limit")
        if now < arr:
            time.sleep(arr - now)
        p = _bem.Problem.from_workload(wp, prec="fp64", tol=tol, max_iter=max_iter, quad_order=quad_order)
        x = torch.empty((1, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
        status, it, rs = p.bem_solve_planewave([ang], x)
        torch.cuda.synchronize()
        st.latencies_s.append(time.perf_counter() - t0 - arr)
        st.iters.append(int(it[0]))
        st.n_done += 1
        if out is not None:
            out[rid] = x[0]
        p.close()
    st.wall_s = time.perf_counter() - t0
    return st
