"""Shared helpers for the GPU parity tests (tolerance metrics and device plumbing)."""
import numpy as np

# Entry parity for the FP64 path (per 2x2 block of the matrix):
#   max |dA| / max |A| <= 1e-12 over each of the four N x N blocks, and
#   |dA_ij| / |A_ij| <= 1e-10 for entries with |A_ij| >= 1e-6 * max |A| of their block.
ENTRY_BLOCK_TOL = 1e-12
ENTRY_REL_TOL = 1e-10
SOLUTION_TOL_FP64 = 1e-10     # ||x_gpu - x_lu|| / ||x_lu||, FP64 path
SOLUTION_TOL_MIXED = 1e-6     # same after mixed-precision refinement


def block_errors(A_gpu, A_ref):
    n = A_ref.shape[0] // 2
    worst_blk, worst_rel = 0.0, 0.0
    for bi in range(2):
        for bj in range(2):
            g = A_gpu[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n]
            r = A_ref[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n]
            mx = np.max(np.abs(r))
            if mx == 0:
                assert np.max(np.abs(g)) == 0
                continue
            d = np.abs(g - r)
            worst_blk = max(worst_blk, np.max(d) / mx)
            big = np.abs(r) >= 1e-6 * mx
            worst_rel = max(worst_rel, np.max(d[big] / np.abs(r[big])))
    return worst_blk, worst_rel


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
