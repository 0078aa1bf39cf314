"""Series (Mie) solution for a penetrable circular cylinder (Sec. 7.1, eq. 2dom_anal).

TEST INFRASTRUCTURE ONLY.  The exterior field is u_in + sum_n a_n H_n(k_1 r) e^{in theta}, the interior
field sum_n b_n J_n(k_2 r) e^{in theta}.  For each n the pair (a_n, b_n) solves the two transmission
conditions at r = R: continuity of u (eq. jump_in_u) and of the flux (1/eps) du/dr (eq. jump_in_w).
The series is truncated at |n| <= nmax (the paper uses 50).
"""
from __future__ import annotations

import numpy as np
from scipy import special

__all__ = ["mie_coefficients", "mie_traces", "mie_far_field", "mie_field", "mie2_coefficients", "mie2_far_field"]


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


def mie2_coefficients(k, eps, R_out=2.0, R_in=1.0, theta_inc=0.0, nmax=None):
    """Two-layer cylinder of Sec. 7.2 (concentric circles): host k[0]; ring R_in < r < R_out with k[1], eps[1];
    core r < R_in with k[2], eps[2].  Host: c_n J_n + a_n H_n; ring: b_n J_n + d_n H_n; core: e_n J_n.
    Continuity of u and of (1/eps) du/dr at both radii gives a 4 x 4 system per n (eqs. jump_in_u, jump_in_w).
    Returns (n, a, b, d, e, c)."""
    k1, k2, k3 = k
    e1, e2, e3 = eps
    if nmax is None:
        nmax = max(50, int(np.ceil(max(k) * R_out)) + 40)
    n = np.arange(-nmax, nmax + 1)
    c = (1j ** n) * np.exp(-1j * n * theta_inc)
    out = np.zeros((4, len(n)), dtype=np.complex128)
    J, H, Jp, Hp = special.jv, special.hankel1, special.jvp, special.h1vp
    for m, nn in enumerate(n):
        x1, x2o, x2i, x3 = k1 * R_out, k2 * R_out, k2 * R_in, k3 * R_in
        Mat = np.array([
            [H(nn, x1), -J(nn, x2o), -H(nn, x2o), 0.0],
            [(k1 / e1) * Hp(nn, x1), -(k2 / e2) * Jp(nn, x2o), -(k2 / e2) * Hp(nn, x2o), 0.0],
            [0.0, J(nn, x2i), H(nn, x2i), -J(nn, x3)],
            [0.0, (k2 / e2) * Jp(nn, x2i), (k2 / e2) * Hp(nn, x2i), -(k3 / e3) * Jp(nn, x3)],
        ], dtype=np.complex128)
        rhs = np.array([-c[m] * J(nn, x1), -c[m] * (k1 / e1) * Jp(nn, x1), 0.0, 0.0], dtype=np.complex128)
        out[:, m] = np.linalg.solve(Mat, rhs)
    a, b, d, e = out
    return n, a, b, d, e, c


def mie2_far_field(k, eps, angles, R_out=2.0, R_in=1.0, theta_inc=0.0, nmax=None):
    """Far-field pattern of the two-layer cylinder, same normalisation as mie_far_field."""
    n, a, b, d, e, c = mie2_coefficients(k, eps, R_out, R_in, theta_inc, nmax)
    E = np.exp(1j * np.outer(angles, n))
    return np.sqrt(2.0 / (np.pi * k[0])) * np.exp(-0.25j * np.pi) * (E @ (a * (-1j) ** n))
