"""Series (Mie) solution for a penetrable circular cylinder (Sec. 7.1, eq. 2dom_anal).

TEST INFRASTRUCTURE ONLY.  The exterior field is u_in + sum_n a_n H_n(k_1 r) e^{in theta}, the interior
field sum_n b_n J_n(k_2 r) e^{in theta}.  For each n the pair (a_n, b_n) solves the two transmission
conditions at r = R: continuity of u (eq. jump_in_u) and of the flux (1/eps) du/dr (eq. jump_in_w).
The series is truncated at |n| <= nmax (the paper uses 50).
"""
from __future__ import annotations

import numpy as np
from scipy import special

__all__ = ["mie_coefficients", "mie_traces", "mie_far_field", "mie_field"]


def _nmax_default(k1, k2, R):
    return max(50, int(np.ceil(max(k1, k2) * R)) + 40)


def mie_coefficients(k1, k2, eps2, R=1.0, theta_inc=0.0, nmax=None):
    """(n, a_n, b_n, c_n) with c_n = i^n e^{-i n theta_inc} the plane-wave (Jacobi-Anger) coefficients."""
    if nmax is None:
        nmax = _nmax_default(k1, k2, R)
    n = np.arange(-nmax, nmax + 1)
    x1, x2 = k1 * R, k2 * R
    c = (1j ** n) * np.exp(-1j * n * theta_inc)
    a = np.zeros(len(n), dtype=np.complex128)
    b = np.zeros(len(n), dtype=np.complex128)
    for m, nn in enumerate(n):
        # [ H_n(x1)        -J_n(x2)            ] [a]   [ -c J_n(x1)       ]
        # [ k1 H_n'(x1)    -(k2/eps2) J_n'(x2) ] [b] = [ -c k1 J_n'(x1)   ]
        Mat = np.array([[special.hankel1(nn, x1), -special.jv(nn, x2)],
                        [k1 * special.h1vp(nn, x1), -(k2 / eps2) * special.jvp(nn, x2)]])
        rhs = -c[m] * np.array([special.jv(nn, x1), k1 * special.jvp(nn, x1)])
        a[m], b[m] = np.linalg.solve(Mat, rhs)
    return n, a, b, c


def mie_traces(k1, k2, eps2, theta, R=1.0, theta_inc=0.0, nmax=None):
    """Boundary traces (u, w) at polar angles theta on r = R.

    The normal points into the scatterer (n = -r_hat, Sec. 2), so w = (1/eps_1) du/dn = -du/dr from the
    host side."""
    n, a, b, c = mie_coefficients(k1, k2, eps2, R, theta_inc, nmax)
    x1, x2 = k1 * R, k2 * R
    E = np.exp(1j * np.outer(theta, n))
    u = E @ (b * special.jv(n, x2))
    w = -k1 * (E @ (c * special.jvp(n, x1) + a * special.h1vp(n, x1)))
    return u, w


def mie_far_field(k1, k2, eps2, angles, R=1.0, theta_inc=0.0, nmax=None):
    """u_inf(theta) = sqrt(2/(pi k1)) e^{-i pi/4} sum_n a_n (-i)^n e^{i n theta}
    (large-argument form of H_n; same normalisation as the oracle's far_field)."""
    n, a, b, c = mie_coefficients(k1, k2, eps2, R, theta_inc, nmax)
    E = np.exp(1j * np.outer(angles, n))
    return np.sqrt(2.0 / (np.pi * k1)) * np.exp(-0.25j * np.pi) * (E @ (a * (-1j) ** n))


def mie_field(k1, k2, eps2, pts, R=1.0, theta_inc=0.0, nmax=None):
    """Total field u at points pts (M,2): exterior series outside r = R, interior series inside."""
    n, a, b, c = mie_coefficients(k1, k2, eps2, R, theta_inc, nmax)
    r = np.hypot(pts[:, 0], pts[:, 1])
    th = np.arctan2(pts[:, 1], pts[:, 0])
    out = np.zeros(len(pts), dtype=np.complex128)
    for m in range(len(pts)):
        e = np.exp(1j * n * th[m])
        if r[m] >= R:
            out[m] = np.sum((c * special.jv(n, k1 * r[m]) + a * special.hankel1(n, k1 * r[m])) * e)
        else:
            out[m] = np.sum(b * special.jv(n, k2 * r[m]) * e)
    return out
