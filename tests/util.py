"""Shared helpers for the GPU parity tests (tolerance metrics and device plumbing)."""
import numpy as np

# Entry parity for the FP64 path (per 2x2 block of the matrix):
#   max |dA| / max |A| <= 1e-12 over each of the four N x N blocks, and
#   |dA_ij| / |A_ij| <= 1e-10 for entries with |A_ij| >= 1e-4 * max |A| of their block.
# Below 1e-4 of the block maximum the relative check says nothing about either side: FP64 evaluations of the
# quadrature rule differ by ~5e-15 of the block maximum (the absolute bar covers that), and the double-layer
# entries of neighbouring, nearly collinear elements are that small because their kernel's cosine cancels (at
# 2e-6 of the block maximum on the star of 4096 elements, a 40-digit evaluation of the same rule puts the
# oracle 2.5e-9 to 5e-9 and the library 1.1e-9 to 3.4e-9 away, relative to the entry).
ENTRY_BLOCK_TOL = 1e-12
ENTRY_REL_TOL = 1e-10
ENTRY_REL_FLOOR = 1e-4
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
            big = np.abs(r) >= ENTRY_REL_FLOOR * mx
            worst_rel = max(worst_rel, np.max(d[big] / np.abs(r[big])))
    return worst_blk, worst_rel


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
