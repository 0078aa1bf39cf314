"""The library's entry formulas (pair.cuh, the code of the assembly kernels) built for the host and compared with
the oracle's matrix entry by entry, on the CPU: operators S, D, D*, N of Sec. 3.3 with exact self terms,
placed by the Sec. 6 recipe or a comparison form, for one-, two- and three-material geometries, Q = 4 and 10.
The bar is the GPU parity test's: max |dA| / max |A| <= 1e-12 per N x N block and 1e-10 relative on the
entries above 1e-6 of their block's largest.  The host build runs the same source as the device build except
for the table loads, the warp-uniform choices and the FP32 reciprocal-square-root seeds."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.util import ENTRY_BLOCK_TOL, ENTRY_REL_TOL, block_errors

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2312_12787_gb300", "csrc")
FORMS = {"mod": 0, "orig": 1, "beta1": 2, "conv": 3}


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = next((c for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("pair") / "pair_host_check")
    # -ffp-contract=off: the double-float error-free transformations must not be fused on any host
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    "--expt-relaxed-constexpr", "-Xcompiler", "-ffp-contract=off", "-I" + CSRC,
                    "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "pair_host_check.cu"),
                    "-o", exe], check=True, capture_output=True)
    return exe


def host_matrix(exe, wp, Q, form):
    """Elements from the segments as the C interface forms them (closed: the last vertex joins the first)."""
    t, w = np.polynomial.legendre.leggauss(Q)
    rows = []
    for s in wp.segments:
        xy = np.asarray(s.xy, float)
        ne = len(xy) if s.closed else len(xy) - 1
        for e in range(ne):
            a, b = xy[e], xy[(e + 1) % len(xy)]
            rows.append(" ".join(repr(float(v)) for v in (a[0], a[1], b[0], b[1])) + f" {int(s.P)} {int(s.M)}")
    n = len(rows)
    head = [f"{n} {Q} {FORMS[form]} {len(wp.k)}", " ".join(repr(float(v)) for v in wp.k),
            " ".join(repr(float(v)) for v in wp.eps), " ".join(repr(float(v)) for v in t),
            " ".join(repr(float(v)) for v in w)]
    out = subprocess.run([exe], input="\n".join(head + rows) + "\n", capture_output=True, text=True, check=True).stdout
    v = np.array([float.fromhex(x) for x in out.split()])
    assert v.size == 2 * (2 * n) ** 2
    return (v[0::2] + 1j * v[1::2]).reshape(2 * n, 2 * n)


CASES = [
    ("triangle", lambda: W.Problem(k=[2.0, 3.0], eps=[1.0, 2.25],
                                   segments=[W.Segment(W.circle(3), P=0, M=1, closed=True)]), 4, "mod"),
    ("circle33_q10", lambda: W.circle_problem(33, 5.0, 7.5), 10, "mod"),
    ("star90", lambda: W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                                 segments=[W.Segment(W.star(90, 0.3, 5), P=0, M=1, closed=True)]), 4, "mod"),
    ("concentric_orig", lambda: W.concentric(21, 41, 2.0), 4, "orig"),
    ("concentric_conv", lambda: W.concentric(21, 41, 2.0), 10, "conv"),
    ("junction_mod", lambda: W.junction_disk(60, k=(5.0, 7.5, 10.0)), 4, "mod"),
    ("junction_beta1", lambda: W.junction_disk(60, k=(5.0, 7.5, 10.0)), 4, "beta1"),
    ("equal_density", lambda: W.circle_problem(29, 5.0, 7.5, eps_i=1.0), 4, "mod"),
]


@pytest.mark.parametrize("name,mk,Q,form", CASES, ids=[c[0] for c in CASES])
def test_host_entries_match_oracle(harness, name, mk, Q, form):
    wp = mk()
    got = host_matrix(harness, wp, Q, form)
    ref = O.assemble(wp, Q=Q, form=form)
    blk, rl = block_errors(got, ref)
    assert blk <= ENTRY_BLOCK_TOL and rl <= ENTRY_REL_TOL, (name, blk, rl)
