"""The library's Bessel routines (bessel.cuh, host-and-device code) built for the host and checked against
mpmath on every branch: the ascending series (x < 1/4 on the double-float path, x < 2 on the FP64 path), the
Taylor steps from the tabulated coefficients (1/4 <= x < 128: spacing 1/128 below 1, 1/32 above), Hankel's
expansion (x >= 128), and the branch boundaries.  Errors are measured relative to
|H0| for J0, Y0 and to |H1| for J1, Y1 (the Hankel functions the kernels are made of, Sec. 3.3).

Three paths are checked: bessel01_f2, the double-float path of the assembly and matrix-free kernels;
bessel01, the FP64 path of the self terms and the near field; and the FP64 routines (Miller's recurrence below
18, the 22-term expansion beyond) from which the host builds the Taylor table.  The host build runs the same
source as the device build except for the table loads, the warp-uniform choices and the FP32
reciprocal-square-root seed (refined by Newton steps on both)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_12787_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def values(tmp_path_factory):
    mpmath = pytest.importorskip("mpmath")
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("bessel") / "bessel_host_check")
    # -ffp-contract=off: the double-float error-free transformations must not be fused on any host
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off", "-I" + CSRC,
                    "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "bessel_host_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    rng = np.random.default_rng(7)
    xs = np.concatenate([
        np.geomspace(1e-3, 1.999, 40),
        [2.0 - 2.0 ** -40, 2.0, 2.0 + 2.0 ** -40],
        2.0 + np.arange(1, 4032, 7) / 32.0 + rng.uniform(-1 / 64, 1 / 64, 576),   # around the grid points
        2.0 + (np.arange(0, 4032, 11) + 0.5) / 32.0,                             # half-way between them
        [18.0, 25.0, 35.0, 128.0 - 2.0 ** -40, 128.0, 128.0 + 2.0 ** -40],
        2.0 + (np.arange(2, 4032, 13) + 0.5) / 32.0 + 2.0 ** -33,                 # just past half-grid points
        [8.328125 + 5.16e-11, 2.0 + 0.046875, 2.0 - 1e-9],
        np.geomspace(128.0, 2000.0, 120),
        # the table's first segment, 1 <= x < 2 (the derivatives of Y0, Y1 grow toward the origin)
        [1.0 - 2.0 ** -40, 1.0, 1.0 + 2.0 ** -40, 1.0 + 2.0 ** -30, 1.0 + 1 / 64, 1.0 + 1 / 64 + 2.0 ** -33],
        1.0 + np.arange(0, 32) / 32.0 + rng.uniform(-1 / 64, 1 / 64, 32),
        1.0 + (np.arange(0, 32) + 0.5) / 32.0,
        np.geomspace(0.5, 0.999, 12),
        # the fine segment, 1/4 <= x < 1 (spacing 1/128), and the series below it
        [0.25 - 2.0 ** -40, 0.25, 0.25 + 2.0 ** -40, 1.0 - 1 / 256, 1.0 - 1 / 256 - 2.0 ** -33],
        0.25 + np.arange(0, 96) / 128.0 + rng.uniform(-1 / 256, 1 / 256, 96),
        0.25 + (np.arange(0, 96) + 0.5) / 128.0,
        np.geomspace(1e-3, 0.249, 24),
    ])
    out = subprocess.run([exe], input="\n".join(repr(float(v)) for v in xs), capture_output=True, text=True,
                         check=True).stdout
    got = np.array([[float.fromhex(t) for t in line.split()] for line in out.strip().splitlines()])
    assert got.shape == (len(xs), 21) and np.array_equal(got[:, 0], xs)
    mpmath.mp.dps = 30
    ref = np.array([[float(mpmath.besselj(0, x)), float(mpmath.bessely(0, x)), float(mpmath.besselj(1, x)),
                     float(mpmath.bessely(1, x))] for x in xs])
    return xs, got, ref


def _rel_err(got4, ref):
    h0 = np.hypot(ref[:, 0], ref[:, 1])
    h1 = np.hypot(ref[:, 2], ref[:, 3])
    scale = np.stack([h0, h0, h1, h1], 1)
    return np.max(np.abs(got4 - ref) / scale, axis=1)


@pytest.mark.parametrize("lo,hi,bound", [(0.0, 0.25, 3e-15), (0.25, 1.0, 1e-14), (1.0, 2.0, 1e-14),
                                         (2.0, 128.0, 1e-14), (128.0, np.inf, 2.5e-14)])
def test_double_float_path_matches_mpmath(values, lo, hi, bound):
    xs, got, ref = values
    sel = (xs >= lo) & (xs < hi)
    err = _rel_err(got[sel, 1:5], ref[sel])
    assert sel.sum() > 30 and err.max() <= bound, (err.max(), xs[sel][np.argmax(err)])


@pytest.mark.parametrize("lo,hi,bound", [(0.0, 2.0, 1e-15), (2.0, 35.0, 1e-13), (35.0, np.inf, 2.5e-14)])
def test_fp64_path_matches_mpmath(values, lo, hi, bound):
    xs, got, ref = values
    sel = (xs >= lo) & (xs < hi)
    err = _rel_err(got[sel, 5:9], ref[sel])
    assert sel.sum() > 30 and err.max() <= bound, (err.max(), xs[sel][np.argmax(err)])


@pytest.mark.parametrize("lo,hi,bound", [(0.0, 2.0, 1e-15), (2.0, 18.0, 3e-15), (18.0, np.inf, 2e-15)])
def test_table_builders_match_mpmath(values, lo, hi, bound):
    xs, got, ref = values
    sel = (xs >= lo) & (xs < hi)
    err = _rel_err(got[sel, 9:13], ref[sel])
    assert sel.sum() > 30 and err.max() <= bound, (err.max(), xs[sel][np.argmax(err)])


@pytest.mark.parametrize("lo,hi,bound", [(0.0, 0.25, 3e-15), (0.25, 1.0, 1e-14), (1.0, 2.0, 1e-14),
                                         (2.0, 128.0, 1e-14), (128.0, np.inf, 2.5e-14)])
def test_split_argument_path_matches_mpmath(values, lo, hi, bound):
    """The assembly passes x as an FP64 base (per element pair) plus a double-float offset (per node); with the
    base and the node on different table grid points, near half-grid points and across the branch boundaries."""
    xs, got, ref = values
    sel = (xs >= lo) & (xs < hi)
    for c0 in (13, 17):
        err = _rel_err(got[sel, c0:c0 + 4], ref[sel])
        assert sel.sum() > 30 and err.max() <= bound, (c0, err.max(), xs[sel][np.argmax(err)])

