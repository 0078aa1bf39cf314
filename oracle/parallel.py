"""Row-parallel driver of the oracle's assembly (test infrastructure, like the rest of this package).

The arithmetic is the oracle's own: every row block is `assemble_rows` of bem_oracle.py (Sec. 6 recipe,
Sec. 7 quadrature), run unchanged in a pool of spawned worker processes that write their rows into one
shared-memory matrix.  Only the work split differs from `assemble`, so the result is identical to it.
Workers are spawned (never forked), which keeps a parent that already holds a CUDA context safe.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from .bem_oracle import assemble_rows, elements

__all__ = ["assemble_parallel", "default_workers"]


def default_workers() -> int:
    """Host cores this process may use."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _rows_into_shared(args):
    name, shape, problem, rows, Q, form = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        A = np.ndarray(shape, dtype=np.complex128, buffer=shm.buf)
        A[rows] = assemble_rows(problem, rows, Q=Q, form=form)
    finally:
        shm.close()
    return len(rows)


def assemble_parallel(problem, Q: int = 4, form: str = "mod", workers: int | None = None, block: int = 64):
    """The full 2N x 2N collocation matrix, equal to `assemble(problem, Q, form)`, with its rows computed in
    blocks of `block` rows by `workers` spawned processes."""
    n2 = 2 * elements(problem).n
    workers = workers or default_workers()
    if workers <= 1:
        return assemble_rows(problem, np.arange(n2), Q=Q, form=form)
    shape = (n2, n2)
    shm = shared_memory.SharedMemory(create=True, size=n2 * n2 * 16)
    try:
        # interleave the blocks so that upper (interior-domain) and lower (host) rows mix in every worker
        blocks = [np.arange(s, min(s + block, n2)) for s in range(0, n2, block)]
        jobs = [(shm.name, shape, problem, rows, Q, form) for rows in blocks]
        with mp.get_context("spawn").Pool(workers) as pool:
            done = sum(pool.imap_unordered(_rows_into_shared, jobs, chunksize=1))
        assert done == n2
        A = np.array(np.ndarray(shape, dtype=np.complex128, buffer=shm.buf))
    finally:
        shm.close()
        shm.unlink()
    return A
