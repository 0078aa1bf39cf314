"""The refinement residual's offset accumulation, emulated on the CPU with correctly rounded FP32 arithmetic.

The GPU residual kernel sums the leading products hi * x_hi of b - (hi + lo)(x_hi + x_lo) in runs of 8
columns.  For each run it takes a power of two sigma > 64 M, where M bounds the run's |product| from the
row and column maxima.  The accumulator starts at sigma and each product a b enters as
    t = fma(a, b, acc),   d = t - acc,   c += fma(a, b, -d),   acc = t.
At the end of the run, acc - sigma joins a double-float total by one two-sum step and c joins its low part.
The scheme rests on two facts, which this file checks on BEM rows and on adversarial data:
  1. every difference d = t - acc and acc - sigma is exact (Sterbenz: acc never leaves [sigma/2, 2 sigma]),
     so the only roundings are those of the small corrections c;
  2. the sum is then accurate to far better than FP32: within 2^-34 of sum |a b| (plain FP32: ~2^-24).
A negative case shows the exactness check is not vacuous: with sigma ~ 4 M, a run of negative products
drives acc through zero, and d is no longer exact.

FP32 operations are numpy float32 operations (IEEE, correctly rounded); fma is emulated exactly: the
product of two FP32 values is exact in FP64, its sum with the addend is carried as an FP64 two-sum, and the
result is rounded once to FP32.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

f32 = np.float32


def fma32(a, b, c):
    a, b, c = (np.asarray(v, np.float64) for v in (a, b, c))
    p = a * b                                   # exact: 24 + 24 significant bits
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)               # s + e = p + c exactly
    r = s.astype(f32)
    # s exactly between two FP32 neighbours: the sign of e decides
    rn = np.nextafter(r, np.where(e > 0, np.inf, -np.inf).astype(f32))
    tie = (e != 0) & (np.abs(r.astype(np.float64) - s) == np.abs(rn.astype(np.float64) - s))
    return np.where(tie, rn, r)


def two_sum32(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def offset_of(m, margin):
    """power of two sigma with M < 2^e -> sigma = 2^(e + margin)"""
    _, ex = np.frexp(np.asarray(m, np.float64))
    return np.where(m == 0, 2.0 ** -120, np.ldexp(1.0, ex + margin)).astype(f32)


def offset_sum(ar, ai, xr, xi, run=8, margin=6):
    """Re sum_k a[r, k] x[s, k] for complex FP32 rows a = ar + i ai and columns x = xr + i xi, by the offset
    scheme; returns (rows x columns result in FP64, number of inexact differences seen)."""
    R, S_, n = ar.shape[0], xr.shape[0], ar.shape[1]
    S = np.zeros((R, S_), f32)
    L = np.zeros((R, S_), f32)
    inexact = 0
    for k0 in range(0, n, run):
        k1 = min(n, k0 + run)
        amax = np.maximum(np.abs(ar[:, k0:k1]), np.abs(ai[:, k0:k1])).max(1)
        xmax = np.maximum(np.abs(xr[:, k0:k1]), np.abs(xi[:, k0:k1])).max(1)
        sig = offset_of((amax[:, None] * xmax[None, :]).astype(f32), margin)
        acc = sig.copy()
        c = np.zeros_like(acc)
        for k in range(k0, k1):
            for a, b in ((ar[:, k, None], xr[None, :, k]), (-ai[:, k, None], xi[None, :, k])):
                a, b = np.broadcast_to(a, acc.shape), np.broadcast_to(b, acc.shape)
                t = fma32(a, b, acc)
                d = t - acc
                inexact += int(np.count_nonzero(d.astype(np.float64) != t.astype(np.float64) - acc.astype(np.float64)))
                c = c + fma32(a, b, -d)
                acc = t
        run_sum = acc - sig
        inexact += int(np.count_nonzero(run_sum.astype(np.float64) != acc.astype(np.float64) - sig.astype(np.float64)))
        S, e = two_sum32(S, run_sum)
        L = L + (e + c)
    return S.astype(np.float64) + L.astype(np.float64), inexact


def exact_sum(ar, ai, xr, xi):
    out = np.empty((ar.shape[0], xr.shape[0]))
    for r in range(ar.shape[0]):
        for s in range(xr.shape[0]):
            out[r, s] = math.fsum(np.concatenate([ar[r].astype(np.float64) * xr[s],
                                                  -(ai[r].astype(np.float64) * xi[s])]))
    return out


def _split(z):
    z = np.asarray(z).astype(np.complex64)
    return z.real.astype(f32), z.imag.astype(f32)


@pytest.fixture(scope="module")
def bem_rows():
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(160, 0.3, 5), P=0, M=1, closed=True)])
    A = O.assemble(wp, Q=4)
    b = np.stack([O.rhs_planewave(wp, t) for t in (0.0, 1.0)])
    x = np.linalg.solve(A, b.T).T
    return A[::5], x


@pytest.mark.parametrize("kind", ["solution", "random", "spread"])
def test_offset_sum_exact_differences_and_accuracy_on_bem_rows(bem_rows, kind):
    """BEM rows of a star (k = 20 / 30) against the LU solution (the sum cancels to the residual), random
    columns and columns spread over 30 decades."""
    A, x = bem_rows
    rng = np.random.default_rng(11)
    n2 = A.shape[1]
    if kind == "random":
        x = rng.normal(size=(2, n2)) + 1j * rng.normal(size=(2, n2))
    elif kind == "spread":
        x = (rng.normal(size=(2, n2)) + 1j * rng.normal(size=(2, n2))) * 10.0 ** rng.uniform(-20, 10, (2, n2))
    ar, ai = _split(A)
    xr, xi = _split(x)
    got, inexact = offset_sum(ar, ai, xr, xi)
    assert inexact == 0
    ref = exact_sum(ar, ai, xr, xi)
    scale = np.abs(ar).astype(np.float64) @ np.abs(xr).T.astype(np.float64) \
        + np.abs(ai).astype(np.float64) @ np.abs(xi).T.astype(np.float64)
    rel = np.max(np.abs(got - ref) / scale)
    assert rel <= 2.0 ** -34, rel
    naive = (ar @ xr.T - ai @ xi.T).astype(np.float64)       # the same sums accumulated in FP32
    assert np.max(np.abs(naive - ref) / scale) > 2.0 ** 8 * rel


def test_offset_sum_worst_drift_stays_exact():
    """Every product of a run at the run's bound M, all of one sign, with M just below a power of two (so
    sigma is as close to 64 M as it gets): the accumulator drifts by the full 16 M, every difference stays
    exact, and the result keeps the accuracy bound."""
    n = 64
    m = np.nextafter(f32(1.0), f32(0.0))
    for sign in (1.0, -1.0):
        ar = np.full((1, n), f32(sign * m), f32)
        zero = np.zeros_like(ar)
        xr = np.full((1, n), m, f32)
        got, inexact = offset_sum(ar, zero, xr, zero.copy())
        assert inexact == 0
        ref = exact_sum(ar, zero, xr, zero.copy())[0, 0]
        assert abs(got[0, 0] - ref) <= 2.0 ** -34 * abs(ref)


def test_offset_too_small_is_caught():
    """sigma ~ 4 M (margin 2): a run of negative products takes the accumulator through zero, where
    t - acc is no longer exact; the exactness check must see it."""
    rng = np.random.default_rng(3)
    n = 64
    ar = (-rng.uniform(0.5, 1.0, (4, n))).astype(f32)
    xr = rng.uniform(0.5, 1.0, (3, n)).astype(f32)
    zero_a, zero_x = np.zeros_like(ar), np.zeros_like(xr)
    _, inexact_ok = offset_sum(ar, zero_a, xr, zero_x, margin=6)
    _, inexact_small = offset_sum(ar, zero_a, xr, zero_x, margin=2)
    assert inexact_ok == 0 and inexact_small > 0
