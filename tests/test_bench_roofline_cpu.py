"""bench.py's roofline entry on the CPU: the dominant phase it picks and the arithmetic of its figures.

The algorithmic bytes of one tensor-core product are fixed by the layout of its operands: A with n x n complex
entries for n unknowns, each stored as the FP16 hi and lo parts of its real and imaginary parts (8 bytes), the
basis block X and the product Y (64 complex FP32 columns of n entries each).  A relaxed product reads A's hi
parts only (4 bytes per entry).
"""
import pytest

import bench

HBM = 6794.1


def _prof(**kw):
    base = {"assemble": (4.4, 1), "rhs": (0.03, 1), "matvec": (0.0, 0), "arnoldi": (6.4, 120),
            "residual": (0.0, 0), "relaxed": (0.0, 0)}
    base.update(kw)
    return base


def test_gemm_bytes_at_the_benchmarked_size():
    # 4096 elements: 8192 complex unknowns, 8192^2 entries of A x 8 bytes, plus X and Y (64 x 8192 x 8 bytes each)
    roof = bench.roofline(_prof(matvec=(9.6, 100)), 4096, HBM, "measured")
    full = 8192 * 8192 * 8 + 2 * 64 * 8192 * 8
    assert full == 545_259_520
    assert roof["kernel"].startswith("k_gemm_tc") and roof["bound"] == "hbm"
    assert roof["full_launches"] == 100 and roof["relaxed_launches"] == 0
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(full, rel=1e-15)
    assert roof["avg_launch_ms"] == pytest.approx(0.096)
    assert roof["achieved"] == pytest.approx(full / 96e-6 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / HBM)
    assert roof["traffic"] == pytest.approx(bench.GEMM_DRAM_BYTES_N4096)


def test_relaxed_launches_average_bytes_and_traffic():
    roof = bench.roofline(_prof(matvec=(11.7, 117), relaxed=(0.0, 21)), 4096, HBM, "measured")
    full = 8192 * 8192 * 8 + 2 * 64 * 8192 * 8
    rel = 8192 * 8192 * 4 + 2 * 64 * 8192 * 8
    assert rel == 276_824_064
    assert roof["full_launches"] == 96 and roof["relaxed_launches"] == 21
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx((96 * full + 21 * rel) / 117)
    want_t = (96 * bench.GEMM_DRAM_BYTES_N4096 + 21 * bench.GEMM_DRAM_BYTES_RELAXED_N4096) / 117
    assert roof["traffic"] == pytest.approx(want_t)
    # the measured traffic of either kind of launch stays within 5 % of its algorithmic bytes
    assert bench.GEMM_DRAM_BYTES_N4096 / full == pytest.approx(1.0, abs=0.05)
    assert bench.GEMM_DRAM_BYTES_RELAXED_N4096 / rel == pytest.approx(1.0, abs=0.05)


def test_relaxed_count_is_capped_and_sizes_scale():
    # more relaxed launches recorded than products timed (gated launches): every timed product counts as relaxed
    roof = bench.roofline(_prof(matvec=(7.0, 100), relaxed=(0.0, 130)), 2048, HBM, "fallback")
    rel = 4096 * 4096 * 4 + 2 * 64 * 4096 * 8
    assert roof["relaxed_launches"] == 100 and roof["full_launches"] == 0
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(rel)
    assert roof["traffic"] == pytest.approx(bench.GEMM_DRAM_BYTES_RELAXED_N4096 / 4)
    assert roof["peak_source"] == "fallback"


def test_dominant_phase_selection():
    # assembly dominant: the issue-rate model scaled by the number of element pairs
    roof = bench.roofline(_prof(assemble=(20.0, 1), matvec=(9.6, 100)), 8192, HBM, "measured")
    assert roof["kernel"].startswith("k_assemble") and roof["bound"] == "alu"
    want = bench.ASM_WARP_INST_N4096 * 4.0 / 20e-3 / 1e9
    assert roof["achieved"] == pytest.approx(want)
    assert roof["frac"] == pytest.approx(want / bench.ISSUE_PEAK_G)
    assert roof["traffic"] == pytest.approx(bench.ASM_DRAM_BYTES_N4096 * 4.0)
    # residual dominant: one double-float product per group of launches of the residual
    roof = bench.roofline(_prof(residual=(30.0, 2 * bench.RESID_LAUNCHES_TC)), 4096, HBM, "measured")
    assert roof["kernel"].startswith("k_resid_df_gemm") and roof["launches"] == 2
    ops = bench.RESID_FP32_OPS_PER_CMAC * 8192 * 8192 * 64
    assert roof["achieved"] == pytest.approx(ops / 15e-3 / 1e12)
    # phases without a model (Arnoldi here) are never picked, however long
    roof = bench.roofline(_prof(arnoldi=(99.0, 120), matvec=(9.6, 100)), 4096, HBM, "measured")
    assert roof["kernel"].startswith("k_gemm_tc")
