"""FP64 CPU oracle: collocation BEM with constant elements for the Helmholtz transmission problem.

TEST INFRASTRUCTURE ONLY (imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs).

What it follows, step by step (paper: "Automatically well-conditioned collocation BEM for transmission
problems based on the Burton-Miller formulation", arXiv 2312.12787):

* Sec. 2 (eqs. helmholtz .. radiation): domains Omega_d with wavenumber k_d and flux coefficient eps_d,
  flux w = (1/eps_d) du/dn, eps_1 = 1, time factor exp(-i omega t).
* Sec. 3.3 (eqs. stmp, dtmp, dstmp, ddtmp, fundamental_sol): the four boundary integral operators with
  G = (i/4) H0^(1)(k r).
* Sec. 3.3 (eq. bm_orig1): Burton-Miller coupling with alpha = -i/k_1.
* Sec. 5 (eq. calderon_bieb with beta = -alpha) and Sec. 6 (eq. 3dom_calderon_bie with gamma = alpha/eps_3
  and the general recipe at the end of Sec. 6): row placement of the standard and Burton-Miller equations.
* Sec. 7 (opening paragraph): constant elements, collocation at element centres, Gauss-Legendre
  quadrature, exact treatment of the singular self-element integrals, GMRES without restart from x0 = 0.

Readings taken where the paper is silent (each is also listed in the design notes):

* Self-element integrals use their exact closed forms (flat element, collocation at the centre):
  S_ii = (i/(2k)) [int_0^{ka} J0 + i int_0^{ka} Y0],  D_ii = D*_ii = 0,
  N_ii = k^2 S_ii - (ik/2) H1(ka),  a = h/2.
  These are the limits that the paper's "subtraction and addition" and hypersingular regularisation
  converge to.
* The general recipe is applied per interface segment: the upper row of an element is the standard
  equation of the domain its normal points into (M), scaled by -alpha; the lower row is the
  Burton-Miller equation of the domain its normal points out of (P), with coefficient alpha/eps_P.

Parity pins (tests/test_oracle_pins.py): kernels against finite differences of an independent Hankel
evaluation; self terms against independent quadrature; the printed Calderon-product errors on the unit
square (Sec. 4); the printed largest eigenvalue of A^2 for concentric circles (Sec. 7.2); the predicted
eigenvalue clusters (Sec. 5); Green's representation identities; the Mie series (Sec. 7.1, eq. 2dom_anal)
and the equal-material junction disk.  No function here is "parity unpinned".
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import special

__all__ = [
    "Elements", "elements", "gauss_legendre", "kernel_values", "self_terms", "operator_block",
    "sigma", "row_plan", "assemble", "assemble_rows", "rhs_planewave", "solve_lu", "gmres",
    "far_field", "near_field", "alpha_of", "FORMS",
]

FORMS = ("mod", "orig", "beta1", "conv")


@dataclass
class Elements:
    a: np.ndarray      # (N,2) start vertex
    b: np.ndarray      # (N,2) end vertex
    mid: np.ndarray    # (N,2) collocation point (element centre)
    h: np.ndarray      # (N,)  length
    tau: np.ndarray    # (N,2) unit tangent (a -> b)
    nrm: np.ndarray    # (N,2) unit normal, tangent turned by +90 degrees; points from P into M
    P: np.ndarray      # (N,)  domain the normal points out of
    M: np.ndarray      # (N,)  domain the normal points into

    @property
    def n(self) -> int:
        return len(self.h)


def elements(problem) -> Elements:
    """Constant elements of every segment in order (Sec. 7 opening paragraph; Sec. 2 for the normal)."""
    A, B, P, M = [], [], [], []
    for s in problem.segments:
        xy = np.asarray(s.xy, dtype=np.float64)
        nv = len(xy)
        ne = nv if s.closed else nv - 1
        for e in range(ne):
            A.append(xy[e])
            B.append(xy[(e + 1) % nv])
            P.append(s.P)
            M.append(s.M)
    a = np.array(A)
    b = np.array(B)
    d = b - a
    h = np.hypot(d[:, 0], d[:, 1])
    tau = d / h[:, None]
    nrm = np.stack([-tau[:, 1], tau[:, 0]], 1)
    return Elements(a=a, b=b, mid=0.5 * (a + b), h=h, tau=tau, nrm=nrm,
                    P=np.array(P, dtype=np.int64), M=np.array(M, dtype=np.int64))


def gauss_legendre(Q: int):
    """Q-point Gauss-Legendre nodes and weights on [-1, 1] (Sec. 7 opening paragraph)."""
    t, w = np.polynomial.legendre.leggauss(Q)
    return t, w


def alpha_of(k1: float) -> complex:
    """Burton-Miller coupling constant alpha = -i/k_1 (Sec. 3.3, after eq. fundamental_sol)."""
    return -1j / k1


def kernel_values(k, x, nx, y, ny):
    """Kernels of S, D, D*, N at (x, y) for G(x-y) = (i/4) H0^(1)(k|x-y|) (eqs. stmp-ddtmp, fundamental_sol).

    x, nx, y, ny broadcast to (..., 2).  With z = x - y, r = |z|, zh = z/r:
      S  : (i/4) H0(kr)
      D  : dG/dn(y)       =  (ik/4) H1(kr) (zh . n_y)
      D* : dG/dn(x)       = -(ik/4) H1(kr) (zh . n_x)
      N  : d2G/dn(x)dn(y) =  (ik/4) [ H1(kr)/r (n_x.n_y - 2 (n_x.zh)(n_y.zh)) + k H0(kr) (n_x.zh)(n_y.zh) ]
    """
    z = x - y
    r = np.hypot(z[..., 0], z[..., 1])
    zh = z / r[..., None]
    H0 = special.hankel1(0, k * r)
    H1 = special.hankel1(1, k * r)
    zx = np.sum(zh * nx, -1)
    zy = np.sum(zh * ny, -1)
    nn = np.sum(nx * ny, -1)
    S = 0.25j * H0
    D = 0.25j * k * H1 * zy
    Ds = -0.25j * k * H1 * zx
    N = 0.25j * k * (H1 / r * (nn - 2.0 * zx * zy) + k * H0 * zx * zy)
    return S, D, Ds, N


def self_terms(k, h):
    """Exact self-element integrals on a flat element of length h, collocated at its centre.

    S_ii = int_{-a}^{a} (i/4) H0(k|s|) ds = (i/(2k)) [int_0^{ka} J0 + i int_0^{ka} Y0]   (a = h/2)
    N_ii = finite part of int (ik/4) H1(k|s|)/|s| ds = k^2 S_ii - (ik/2) H1(ka)
    D_ii = D*_ii = 0 because the normal is orthogonal to the element.
    (Sec. 7 opening paragraph: the weakly singular and hypersingular self integrals.)
    """
    a = 0.5 * np.asarray(h, dtype=np.float64)
    ij0, iy0 = special.itj0y0(k * a)
    S = 0.5j / k * (ij0 + 1j * iy0)
    N = k * k * S - 0.5j * k * special.hankel1(1, k * a)
    return S, N


def operator_block(el: Elements, k: float, Q: int, rows=None):
    """Collocation matrices S, D, D*, N of wavenumber k for rows `rows` against every element.

    Entry (i, j) integrates the kernel over element j with Q-point Gauss-Legendre
    (y_q = mid_j + (h_j/2) t_q tau_j, weight (h_j/2) w_q); the diagonal uses self_terms.
    The normals are the fixed element normals; the domain signs are applied by the caller.
    """
    if rows is None:
        rows = np.arange(el.n)
    rows = np.asarray(rows)
    t, w = gauss_legendre(Q)
    yq = el.mid[:, None, :] + (0.5 * el.h)[:, None, None] * t[None, :, None] * el.tau[:, None, :]   # (N,Q,2)
    Wq = (0.5 * el.h)[:, None] * w[None, :]                                                      # (N,Q)
    out = [np.zeros((len(rows), el.n), dtype=np.complex128) for _ in range(4)]
    chunk = max(1, 2 ** 19 // max(1, el.n * Q))
    for c0 in range(0, len(rows), chunk):
        ri = rows[c0:c0 + chunk]
        x = el.mid[ri][:, None, None, :]
        nx = el.nrm[ri][:, None, None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            vals = kernel_values(k, x, nx, yq[None], el.nrm[None, :, None, :])
        for m in range(4):
            out[m][c0:c0 + chunk] = np.sum(vals[m] * Wq[None], axis=-1)
        # replace the (singular) self entries by the exact integrals
        Sii, Nii = self_terms(k, el.h[ri])
        loc = np.arange(len(ri))
        out[0][c0 + loc, ri] = Sii
        out[1][c0 + loc, ri] = 0.0
        out[2][c0 + loc, ri] = 0.0
        out[3][c0 + loc, ri] = Nii
    return out


def sigma(el: Elements, d: int) -> np.ndarray:
    """sigma_{d,j} = +1 if the normal of element j points out of domain d, -1 if into d, else 0.

    Domain d's boundary integrals run over the elements it touches, with its own outward normal
    sigma_{d,j} n_j (Sec. 2; Sec. 6, eq. 3dom_bies)."""
    return np.where(el.P == d, 1.0, 0.0) - np.where(el.M == d, 1.0, 0.0)


def row_plan(el: Elements, k, form: str = "mod"):
    """Which equation each row carries: (domain, kind, scale) for the upper and the lower half.

    kind is 'std' (traces of the representation, standard equation) or 'bm' (Burton-Miller: standard plus
    gamma_d times the normal-derivative equation, gamma_d = alpha/eps_d).

    * 'mod'   (Sec. 6 recipe; eq. calderon_bieb with beta = -alpha; eq. 3dom_calderon_bie with
               gamma = alpha/eps_3): upper = std of M(i) scaled by -alpha, lower = bm of P(i).
    * 'orig'  (eq. 3dom_calderon_bie0): as 'mod' but the lower row is bm only where P(i) is the host;
               elsewhere it is std of P(i) scaled by -alpha.
    * 'beta1' (eq. calderon_bie1): as 'mod' with the standard rows unscaled (beta = 1).
    * 'conv'  (eq. naive_bie, eq. 3dom_conv_bie up to row order): upper = equation of P(i) (bm on the
               host, std elsewhere), lower = std of M(i); nothing scaled.
    """
    alpha = alpha_of(k[0])
    n = el.n
    up_dom, lo_dom = el.M.copy(), el.P.copy()
    up_kind = np.array(["std"] * n, dtype=object)
    lo_kind = np.array(["bm"] * n, dtype=object)
    up_scale = np.full(n, -alpha, dtype=np.complex128)
    lo_scale = np.ones(n, dtype=np.complex128)
    if form == "mod":
        pass
    elif form == "orig":
        interior = el.P != 0
        lo_kind[interior] = "std"
        lo_scale[interior] = -alpha
    elif form == "beta1":
        up_scale[:] = 1.0
    elif form == "conv":
        up_dom, lo_dom = el.P.copy(), el.M.copy()
        up_kind = np.where(el.P == 0, "bm", "std").astype(object)
        lo_kind[:] = "std"
        up_scale[:] = 1.0
    else:
        raise ValueError(f"unknown form {form!r}")
    return (up_dom, up_kind, up_scale), (lo_dom, lo_kind, lo_scale)


def _equation_rows(el, k, eps, Q, rows, dom, kind, scale, alpha):
    """Coefficient rows [u-part | w-part] of one equation per row (Sec. 6, eq. 3dom_bies and recipe).

    Standard equation of domain d at x_i (traces of Green's representation in Omega_d):
        1/2 u_i + sum_j sig_dj D_d(i,j) u_j - sum_j sig_dj eps_d S_d(i,j) w_j = [u_in(x_i) if d is the host]
    Normal-derivative equation of domain d at x_i:
        sum_j sig_dj N_d(i,j) u_j + eps_d/2 w_i - sum_j sig_dj eps_d D*_d(i,j) w_j = [q_in(x_i) if host]
    Burton-Miller equation = standard + gamma_d * normal-derivative, gamma_d = alpha/eps_d (eq. bm_orig1
    for the host; Sec. 6 recipe for interior domains).
    """
    n = el.n
    out = np.zeros((len(rows), 2 * n), dtype=np.complex128)
    for d in np.unique(dom[rows]):
        sel = np.nonzero(dom[rows] == d)[0]
        ri = np.asarray(rows)[sel]
        S, D, Ds, N = operator_block(el, k[d], Q, ri)
        sg = sigma(el, d)[None, :]
        e = eps[d]
        g = alpha / e
        loc = np.arange(len(ri))
        for kd in ("std", "bm"):
            m = np.nonzero(kind[ri] == kd)[0]
            if len(m) == 0:
                continue
            Au = sg * D[m]
            Aw = -sg * e * S[m]
            Au[loc[:len(m)], ri[m]] += 0.5
            if kd == "bm":
                Au = Au + g * sg * N[m]
                Aw = Aw - g * sg * e * Ds[m]
                Aw[loc[:len(m)], ri[m]] += 0.5 * g * e
            out[sel[m], :n] = Au * scale[ri[m]][:, None]
            out[sel[m], n:] = Aw * scale[ri[m]][:, None]
    return out


def assemble_rows(problem, rows, Q: int = 4, form: str = "mod", el: Elements | None = None):
    """Rows `rows` (indices in [0, 2N)) of the collocation matrix A (Sec. 6 recipe, Sec. 7)."""
    if el is None:
        el = elements(problem)
    k = np.asarray(problem.k, dtype=np.float64)
    eps = np.asarray(problem.eps, dtype=np.float64)
    alpha = alpha_of(k[0])
    rows = np.asarray(rows)
    n = el.n
    (ud, uk, us), (ld, lk, ls) = row_plan(el, k, form)
    out = np.zeros((len(rows), 2 * n), dtype=np.complex128)
    up = rows < n
    if np.any(up):
        out[up] = _equation_rows(el, k, eps, Q, rows[up], ud, uk, us, alpha)
    if np.any(~up):
        out[~up] = _equation_rows(el, k, eps, Q, rows[~up] - n, ld, lk, ls, alpha)
    return out


def assemble(problem, Q: int = 4, form: str = "mod"):
    """The full 2N x 2N collocation matrix A; unknowns ordered [u_1..u_N, w_1..w_N] (Sec. 6)."""
    el = elements(problem)
    return assemble_rows(problem, np.arange(2 * el.n), Q, form, el)


def rhs_planewave(problem, theta: float, form: str = "mod", el: Elements | None = None):
    """Right-hand side for the plane wave u_in = exp(i k_1 d.x), d = (cos theta, sin theta) (Sec. 7.1).

    A host-domain standard row gets u_in(x_i); a host-domain Burton-Miller row gets
    u_in(x_i) + alpha q_in(x_i) with q_in = grad u_in . n_i = i k_1 (d.n_i) u_in (eq. naive_bie);
    each row carries the same scale as its matrix row.  Rows of interior domains are zero.
    """
    if el is None:
        el = elements(problem)
    k = np.asarray(problem.k, dtype=np.float64)
    k1 = k[0]
    alpha = alpha_of(k1)
    dvec = np.array([np.cos(theta), np.sin(theta)])
    uin = np.exp(1j * k1 * (el.mid @ dvec))
    qin = 1j * k1 * (el.nrm @ dvec) * uin
    b = np.zeros(2 * el.n, dtype=np.complex128)
    for half, (dom, kind, scale) in enumerate(row_plan(el, k, form)):
        host = dom == 0
        val = np.where(kind == "bm", uin + alpha * qin, uin)
        b[half * el.n:(half + 1) * el.n] = np.where(host, val * scale, 0.0)
    return b


def solve_lu(A, b):
    """Direct solve by LU with partial pivoting (LAPACK) - the exact discrete solution."""
    return np.linalg.solve(A, b)


def gmres(A, b, tol: float = 1e-8, maxit: int | None = None, matvec=None):
    """GMRES without restart from x0 = 0 (Sec. 3.2; Sec. 7 opening paragraph).

    Arnoldi with modified Gram-Schmidt, Givens rotations for the least-squares problem; stops when the
    estimated relative residual ||b - A x_j|| / ||b|| <= tol.  Returns (x, iterations, residual history).
    """
    if matvec is None:
        matvec = lambda v: A @ v  # noqa: E731
    n = len(b)
    if maxit is None:
        maxit = n
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros_like(b), 0, [0.0]
    V = np.zeros((maxit + 1, n), dtype=np.complex128)
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit, dtype=np.complex128)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    j = 0
    for j in range(maxit):
        w = matvec(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0.0:
            V[j + 1] = w / H[j + 1, j]
        # rotation i acts on rows (i, i+1) as [[conj(c), conj(s)], [-s, c]]
        for i in range(j):
            t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(abs(H[j, j]), abs(H[j + 1, j]))
        cs[j] = H[j, j] / den
        sn[j] = H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = np.conj(cs[j]) * g[j]
        hist.append(abs(g[j + 1]) / beta)
        if hist[-1] <= tol:
            break
    m = j + 1
    y = np.zeros(m, dtype=np.complex128)
    for i in range(m - 1, -1, -1):
        y[i] = (g[i] - H[i, i + 1:m] @ y[i + 1:m]) / H[i, i]
    x = V[:m].T @ y
    return x, m, hist


def far_field(problem, y, angles, Q: int = 4, el: Elements | None = None):
    """Far-field pattern of the scattered field in the host medium.

    Convention: u_s(x) = exp(i k_1 |x|)/sqrt(|x|) (u_inf(xh) + O(1/|x|)).  From the host's Green
    representation (traces u, w on elements bordering the host, outward normal sigma_{1,j} n_j, eps_1 = 1)
    and the large-argument form of H0:
      u_inf(xh) = exp(i pi/4)/sqrt(8 pi k_1) sum_j sigma_{1,j} sum_q W_q exp(-i k_1 xh.y_q)
                  [w_j + i k_1 (xh.n_j) u_j].
    """
    if el is None:
        el = elements(problem)
    k1 = float(problem.k[0])
    n = el.n
    u, w = y[:n], y[n:]
    t, wq = gauss_legendre(Q)
    yq = el.mid[:, None, :] + (0.5 * el.h)[:, None, None] * t[None, :, None] * el.tau[:, None, :]
    Wq = (0.5 * el.h)[:, None] * wq[None, :]
    sg = sigma(el, 0)
    out = np.zeros(len(angles), dtype=np.complex128)
    for a, th in enumerate(angles):
        xh = np.array([np.cos(th), np.sin(th)])
        ph = np.exp(-1j * k1 * (yq @ xh))                       # (N, Q)
        elem = np.sum(Wq * ph, axis=1) * (w + 1j * k1 * (el.nrm @ xh) * u)
        out[a] = np.sum(sg * elem)
    return out * np.exp(0.25j * np.pi) / np.sqrt(8.0 * np.pi * k1)


def near_field(problem, y, pts, dom, theta=None, Q: int = 4, el: Elements | None = None):
    """Total field u at points `pts` (M,2) lying in domains `dom` (M,) from the traces y = [u; w].

    Green's representation in the domain d that contains the point (Sec. 3.3; the same representation whose
    boundary traces give the standard equations of Sec. 6):
        u(x) = [u_in(x) if d is the host] + sum_j sigma_{d,j} int_j [ eps_d G_d(x-y) w_j - dG_d/dn(y) u_j ] dy
    with element integrals by the same Q-point Gauss-Legendre rule as the matrix.  theta = incident angle of
    the plane wave (None: scattered field only in the host).
    """
    if el is None:
        el = elements(problem)
    k = np.asarray(problem.k, dtype=np.float64)
    eps = np.asarray(problem.eps, dtype=np.float64)
    n = el.n
    u, w = y[:n], y[n:]
    t, wq = gauss_legendre(Q)
    yq = el.mid[:, None, :] + (0.5 * el.h)[:, None, None] * t[None, :, None] * el.tau[:, None, :]   # (N,Q,2)
    Wq = (0.5 * el.h)[:, None] * wq[None, :]
    out = np.zeros(len(pts), dtype=np.complex128)
    for m, (x, d) in enumerate(zip(np.asarray(pts, dtype=np.float64), np.asarray(dom))):
        sg = sigma(el, int(d))
        z = x[None, None, :] - yq
        r = np.hypot(z[..., 0], z[..., 1])
        kd = k[int(d)]
        G = 0.25j * special.hankel1(0, kd * r)
        dGdny = 0.25j * kd * special.hankel1(1, kd * r) * np.sum(z / r[..., None] * el.nrm[:, None, :], -1)
        S = np.sum(Wq * G, 1)
        D = np.sum(Wq * dGdny, 1)
        out[m] = np.sum(sg * (eps[int(d)] * S * w - D * u))
        if int(d) == 0 and theta is not None:
            out[m] += np.exp(1j * k[0] * (np.cos(theta) * x[0] + np.sin(theta) * x[1]))
    return out
