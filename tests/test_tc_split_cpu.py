"""The FP16 x 3 operand format of the tensor-core block product, emulated on the CPU.

The GPU product reads the complex FP32 matrix as a real n x 2n matrix (Re, Im interleaved along K), scales
row r by a power of two 2^-e_r that maps its largest magnitude into [1/2, 1), and stores each scaled value v
as hi = fp16(v) and lo = fp16(2^11 (v - hi)).  The right-hand sides become the K-major rows (Re x, -Im x) and
(Im x, Re x), split the same way with one power-of-two scale per column.  The tensor cores form
D1 = A_hi B_hi and D2 = A_lo B_hi + A_hi B_lo with FP32 accumulation, and y = (D1 + 2^-11 D2) / scales.
This file checks the claims that format rests on, with numpy's correctly rounded FP16 conversions:
  * hi + 2^-11 lo holds v to 2^-22 |v| plus an absolute 2^-36 of the row's largest entry (the floor set by
    lo's subnormal spacing, for the entries far below the row maximum);
  * the product error on BEM matrices stays within the 5e-6 (relative, per column) that the GPU parity test
    allows, and the lo terms are what make it so: hi alone is two orders of magnitude worse.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

f16, f32 = np.float16, np.float32
LO = 2048.0


def pow2_scale(m):
    """2^-e with m = f 2^e, f in [1/2, 1): maps m into [1/2, 1) (1 for m = 0)"""
    _, e = np.frexp(np.asarray(m, np.float64))
    return np.where(m == 0, 1.0, np.ldexp(1.0, -e))


def split16(v32):
    """hi = fp16(v), lo = fp16(2^11 (v - hi)); v - hi is exact in FP32 (both lie in one binade or hi = 0)"""
    hi = v32.astype(f16)
    lo = ((v32 - hi.astype(f32)) * f32(LO)).astype(f16)
    return hi, lo


def real_rows(A32):
    """n x n complex -> n x 2n real, (Re, Im) interleaved along K"""
    R = np.empty((A32.shape[0], 2 * A32.shape[1]), f32)
    R[:, 0::2], R[:, 1::2] = A32.real, A32.imag
    return R


def bt_rows(X32):
    """columns x_s -> the K-major rows (Re x, -Im x) (real part of y) and (Im x, Re x) (imaginary part)"""
    s, n = X32.shape
    Bre = np.empty((s, 2 * n), f32)
    Bim = np.empty((s, 2 * n), f32)
    Bre[:, 0::2], Bre[:, 1::2] = X32.real, -X32.imag
    Bim[:, 0::2], Bim[:, 1::2] = X32.imag, X32.real
    return np.concatenate([Bre, Bim])


def tc_product(A32, X32, seg=256, lo_terms=True):
    """Y = A X by the split format with FP32 accumulation in segments of `seg` K values (each segment's sum is
    folded into an FP32 total, as the accumulator readers do)."""
    Ar = real_rows(A32)
    rs = pow2_scale(np.abs(Ar).max(1)).astype(f32)
    ahi, alo = split16(Ar * rs[:, None])
    Bt = bt_rows(X32)
    ns = X32.shape[0]
    ts = pow2_scale(np.maximum(np.abs(X32.real), np.abs(X32.imag)).max(1)).astype(f32)
    ts2 = np.concatenate([ts, ts])
    bhi, blo = split16(Bt * ts2[:, None])
    a_h, a_l = ahi.astype(f32), alo.astype(f32)
    b_h, b_l = bhi.astype(f32), blo.astype(f32)
    D1 = np.zeros((Ar.shape[0], 2 * ns), f32)
    D2 = np.zeros_like(D1)
    for k0 in range(0, Ar.shape[1], seg):
        k = slice(k0, k0 + seg)
        D1 += a_h[:, k] @ b_h[:, k].T
        if lo_terms:
            D2 += a_l[:, k] @ b_h[:, k].T + a_h[:, k] @ b_l[:, k].T
    D = (D1.astype(np.float64) + D2.astype(np.float64) / LO) / (rs[:, None].astype(np.float64) * ts2[None, :])
    return (D[:, :ns] + 1j * D[:, ns:]).T          # ns x n


@pytest.fixture(scope="module")
def bem():
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(240, 0.3, 5), P=0, M=1, closed=True)])
    A = O.assemble(wp, Q=4)
    b = np.stack([O.rhs_planewave(wp, t) for t in np.linspace(0.0, 3.0, 4)])
    x = np.linalg.solve(A, b.T).T
    return A.astype(np.complex64), x


def test_split_round_trip_bound(bem):
    A32, _ = bem
    Ar = real_rows(A32)
    rs = pow2_scale(np.abs(Ar).max(1)).astype(f32)
    v = Ar * rs[:, None]
    assert np.all(np.abs(v).max(1) >= 0.5) and np.all(np.abs(v) < 1.0)
    hi, lo = split16(v)
    rec = hi.astype(np.float64) + lo.astype(np.float64) / LO
    err = np.abs(rec - v.astype(np.float64))
    assert np.all(err <= 2.0 ** -22 * np.abs(v) + 2.0 ** -36)
    # the relative part of the bound is reached (it is not slack by orders of magnitude)
    big = np.abs(v) > 2.0 ** -10
    assert np.max(err[big] / np.abs(v[big])) > 2.0 ** -24
    # tiny entries keep their absolute accuracy through lo's subnormals
    tiny = np.array([2.0 ** -30, 3.3e-9, -7.1e-10, 2.0 ** -36], f32)
    th, tl = split16(tiny)
    assert np.all(np.abs(th.astype(np.float64) + tl.astype(np.float64) / LO - tiny) <= 2.0 ** -36)


@pytest.mark.parametrize("kind", ["solution", "random", "unit"])
def test_product_error_within_parity_bound(bem, kind):
    A32, x = bem
    rng = np.random.default_rng(4)
    n = A32.shape[0]
    if kind == "random":
        x = rng.normal(size=(4, n)) + 1j * rng.normal(size=(4, n))
    elif kind == "unit":                    # unit-norm Krylov vectors, the operand the solver feeds it
        x = rng.normal(size=(4, n)) + 1j * rng.normal(size=(4, n))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
    X32 = x.astype(np.complex64)
    ref = (A32.astype(np.complex128) @ X32.astype(np.complex128).T).T
    got = tc_product(A32, X32)
    err = np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err <= 5e-6, err
    hi_only = tc_product(A32, X32, lo_terms=False)
    err_hi = np.max(np.linalg.norm(hi_only - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err_hi > 100 * err, (err_hi, err)
