"""GPU parity: the CUDA path through the C-ABI against the CPU oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests.util import ENTRY_BLOCK_TOL, ENTRY_REL_TOL, SOLUTION_TOL_FP64, SOLUTION_TOL_MIXED, block_errors, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2312_12787_gb300 import build as bld
    bld.build()
    import paper_2312_12787_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    return T


def gpu_matrix(B, torch, wp, **kw):
    p = B.Problem.from_workload(wp, **kw)
    n2 = p.bem_num_unknowns()
    A = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
    p.bem_get_matrix(A, which=0)
    out = {"main": A.cpu().numpy()}
    if kw.get("prec", "fp64") != "fp64":
        p.bem_get_matrix(A, which=1)
        out["full"] = A.cpu().numpy()
    p.close()
    return out


CASES = [
    ("triangle", lambda: W.Problem(k=[2.0, 3.0], eps=[1.0, 2.25],
                                   segments=[W.Segment(W.circle(3), P=0, M=1, closed=True)])),
    ("circle17", lambda: W.circle_problem(17, 5.0, 7.5)),
    ("circle_c1", lambda: W.cfg_circle_c1()),
    ("star300", lambda: W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                                  segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)])),
    ("concentric", lambda: W.concentric(41, 83, 2.0)),
    ("junction", lambda: W.junction_disk(150, k=(5.0, 7.5, 10.0))),
    ("equal_density", lambda: W.circle_problem(65, 5.0, 7.5, eps_i=1.0)),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("Q", [4, 10])
def test_assembly_fp64_matches_oracle(B, torch, name, mk, Q):
    wp = mk()
    ref = O.assemble(wp, Q=Q)
    got = gpu_matrix(B, torch, wp, quad_order=Q)["main"]
    blk, rl = block_errors(got, ref)
    assert blk <= ENTRY_BLOCK_TOL, (blk, rl)
    assert rl <= ENTRY_REL_TOL, (blk, rl)


@pytest.mark.parametrize("form", ["orig", "beta1", "conv"])
def test_assembly_forms_match_oracle(B, torch, form):
    for wp in (W.concentric(30, 61, 1.0), W.junction_disk(96, k=(3.0, 4.5, 6.0))):
        ref = O.assemble(wp, Q=4, form=form)
        got = gpu_matrix(B, torch, wp, form=form)["main"]
        blk, rl = block_errors(got, ref)
        assert blk <= ENTRY_BLOCK_TOL and rl <= ENTRY_REL_TOL, (form, blk, rl)


@pytest.mark.parametrize("name,mk", [
    # k times the bounding-box diagonal below 127: the kernel without the reduction by pi/2
    ("star300", lambda: W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                                  segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)])),
    # far above it (arguments up to ~280 reach Hankel's expansion): the kernel with the reduction
    ("ellipse250_k40", lambda: W.Problem(k=[40.0, 70.0], eps=[1.0, (70.0 / 40.0) ** 2],
                                         segments=[W.Segment(W.ellipse(250, 4.0), P=0, M=1, closed=True)])),
], ids=["star300", "ellipse250_k40"])
def test_assembly_mixed_split_matches_oracle(B, torch, name, mk):
    wp = mk()
    ref = O.assemble(wp, Q=4)
    m = gpu_matrix(B, torch, wp, prec="mixed")
    blk, rl = block_errors(m["full"], ref)
    assert blk <= ENTRY_BLOCK_TOL and rl <= ENTRY_REL_TOL, (blk, rl)
    # hi alone is the FP32 rounding of each FP64 entry
    err = np.abs(m["main"] - ref)
    assert np.all(err <= 2.0 ** -24 * (np.abs(ref.real) + np.abs(ref.imag)) + 1e-12 * np.max(np.abs(ref)))


def test_rhs_matches_oracle(B, torch):
    for wp in (W.cfg_circle_c1(), W.junction_disk(96, k=(3.0, 4.5, 6.0)), W.concentric(30, 61, 1.0)):
        for form in ("mod", "orig", "conv"):
            p = B.Problem.from_workload(wp, form=form)
            ang = np.array([0.0, 0.7, 2.0])
            b = torch.empty((3, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
            p.bem_rhs_planewave(ang, b)
            got = b.cpu().numpy()
            for r, t in enumerate(ang):
                ref = O.rhs_planewave(wp, t, form=form)
                assert np.max(np.abs(got[r] - ref)) <= 1e-14 * np.max(np.abs(ref)), (form, r)
            p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [1, 3, 70])
def test_matvec_matches_reference(B, torch, prec, nrhs):
    wp = W.circle_problem(700, 5.0, 7.5)
    p = B.Problem.from_workload(wp, prec=prec)
    n2 = p.bem_num_unknowns()
    A = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
    p.bem_get_matrix(A, which=0)
    g = torch.Generator(device="cpu").manual_seed(7)
    x = torch.randn((nrhs, n2), dtype=torch.complex128, generator=g).cuda()
    y = torch.empty_like(x)
    p.bem_matvec(x, y, n_rhs=nrhs)
    ref = (A @ x.T).T.cpu().numpy()      # reference product of the same stored matrix
    tol = 1e-13 if prec == "fp64" else 2e-6
    for r in range(nrhs):
        assert rel(y[r].cpu().numpy(), ref[r]) <= tol
    p.close()


def test_solve_fp64_matches_oracle_lu(B, torch):
    wp = W.cfg_circle_c1()
    A = O.assemble(wp, Q=4)
    ang = np.array([0.0, 1.1])
    p = B.Problem.from_workload(wp, tol=1e-13)
    x = torch.empty((2, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave(ang, x)
    assert st == B.BEM_OK and np.all(rs <= 1e-13)
    for r, t in enumerate(ang):
        xl = O.solve_lu(A, O.rhs_planewave(wp, t))
        assert rel(x[r].cpu().numpy(), xl) <= SOLUTION_TOL_FP64
    # iteration count of the paper's stopping rule against the oracle's GMRES (MGS vs CGS2: +-2)
    p2 = B.Problem.from_workload(wp, tol=1e-10)
    st, it2, rs2 = p2.bem_solve_planewave(ang[:1], x[:1].contiguous())
    _, it_ref, _ = O.gmres(A, O.rhs_planewave(wp, 0.0), tol=1e-10)
    assert abs(int(it2[0]) - it_ref) <= 2
    p.close()
    p2.close()


@pytest.mark.parametrize("name,mk", [("star700", lambda: W.Problem(
    k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(700, 0.3, 5), P=0, M=1, closed=True)])),
    ("junction", lambda: W.junction_disk(400, k=(5.0, 7.5, 10.0)))])
def test_solve_mixed_matches_oracle_lu(B, torch, name, mk):
    wp = mk()
    A = O.assemble(wp, Q=4)
    ang = np.array([0.0, 0.9, 2.5])
    for prec in ("mixed",):
        p = B.Problem.from_workload(wp, prec=prec, tol=1e-10)
        x = torch.empty((3, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
        st, it, rs = p.bem_solve_planewave(ang, x)
        assert st == B.BEM_OK and np.all(rs <= 1e-10), (st, rs)
        for r, t in enumerate(ang):
            xl = O.solve_lu(A, O.rhs_planewave(wp, t))
            assert rel(x[r].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED
        p.close()


def test_far_field_matches_oracle_and_mie(B, torch):
    wp = W.cfg_circle_c1()
    p = B.Problem.from_workload(wp, tol=1e-12)
    ang = np.array([0.0])
    x = torch.empty((1, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
    p.bem_solve_planewave(ang, x)
    fa = np.linspace(0, 2 * np.pi, 37)
    ff = torch.empty((1, len(fa)), dtype=torch.complex128, device="cuda")
    p.bem_far_field(x, fa, ff)
    got = ff.cpu().numpy()[0]
    ref = O.far_field(wp, x.cpu().numpy()[0], fa, Q=4)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    mie = O.mie_far_field(5.0, 7.5, 2.25, fa)
    assert rel(got, mie) < 3e-3      # discretisation error at N = 256, Q = 4
    p.close()


def test_host_entry_point_round_trip(B, torch):
    wp = W.cfg_circle_c1()
    p = B.Problem.from_workload(wp, tol=1e-12)
    st, xh, ffh, it, rs = p.bem_solve_planewave_host([0.0, 1.0], ff_angles=np.linspace(0, 1, 5))
    xl = O.solve_lu(O.assemble(wp, Q=4), O.rhs_planewave(wp, 1.0))
    assert st == B.BEM_OK and rel(xh[1], xl) < 1e-10
    assert ffh.shape == (2, 5)
    p.close()


@pytest.fixture(scope="module")
def star_c2_oracle():
    """The oracle on the benchmarked star (r = 1 + 0.3 cos 5t, 4096 elements, k = 20/30, Q = 4): the whole
    matrix (rows split over host processes, the oracle's arithmetic unchanged) and its LU solutions for the
    64 plane waves of the benchmark."""
    wp = W.cfg_star_c2()
    ang = W.plane_wave_angles(64)
    A = O.assemble_parallel(wp, Q=4)
    el = O.elements(wp)
    Bm = np.stack([O.rhs_planewave(wp, t, el=el) for t in ang], 1)
    X = O.solve_lu(A, Bm).T.copy()
    return wp, ang, A, X


@pytest.mark.slow
def test_full_size_star_matrix_matches_oracle(B, torch, star_c2_oracle):
    """Every entry of the benchmarked 8192 x 8192 matrix, FP64 path and mixed split (hi + lo), against the
    oracle's at the entry-parity bar of the small cases."""
    wp, ang, A, X = star_c2_oracle
    for prec, which in (("fp64", 0), ("mixed_tc", 1)):
        p = B.Problem.from_workload(wp, prec=prec)
        n2 = p.bem_num_unknowns()
        G = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
        p.bem_get_matrix(G, which=which)
        got = G.cpu().numpy()
        del G
        p.close()
        blk, rl = block_errors(got, A)
        assert blk <= ENTRY_BLOCK_TOL and rl <= ENTRY_REL_TOL, (prec, blk, rl)
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_full_size_star_solutions_match_oracle_lu(B, torch, star_c2_oracle):
    """The measured configuration itself (mixed path, tensor-core product, CUDA-graph iterations, 64 plane
    waves, tol 1e-8) and the FP64 path at tol 1e-12, every column element by element against the oracle's LU
    solution: <= 1e-6 after mixed-precision refinement, <= 1e-10 for the FP64 path.  The GPU far field equals
    the oracle's far-field formula applied to the GPU traces."""
    wp, ang, A, X = star_c2_oracle
    el = O.elements(wp)
    for prec, tol, bar in (("mixed_tc", 1e-8, SOLUTION_TOL_MIXED), ("fp64", 1e-12, SOLUTION_TOL_FP64)):
        p = B.Problem.from_workload(wp, prec=prec, tol=tol, max_iter=400)
        n2 = p.bem_num_unknowns()
        x = torch.empty((64, n2), dtype=torch.complex128, device="cuda")
        st, it, rs = p.bem_solve_planewave(ang, x)
        assert st == B.BEM_OK and np.all(rs <= tol) and np.all(it > 0), (prec, st)
        xs = x.cpu().numpy()
        errs = np.linalg.norm(xs - X, axis=1) / np.linalg.norm(X, axis=1)
        assert np.max(errs) <= bar, (prec, np.max(errs))
        if prec == "mixed_tc":
            # the reported residual (updated with the tensor-core product after the first refinement step) is
            # the true residual of the returned x under the oracle's matrix
            Bm = np.stack([O.rhs_planewave(wp, t, el=el) for t in ang])
            true_res = np.linalg.norm(Bm - (A @ xs.T).T, axis=1) / np.linalg.norm(Bm, axis=1)
            assert np.all(np.abs(rs - true_res) <= 0.02 * true_res + 1e-12), np.max(np.abs(rs - true_res) / true_res)
        if prec == "mixed_tc":
            ffa = np.linspace(0.0, 2 * np.pi, 32, endpoint=False)
            ff = torch.empty((64, 32), dtype=torch.complex128, device="cuda")
            p.bem_far_field(x, ffa, ff, n_rhs=64)
            ffs = ff.cpu().numpy()
            for c in (0, 17, 40, 63):
                ref_ff = O.far_field(wp, xs[c], ffa, Q=4, el=el)
                assert np.max(np.abs(ffs[c] - ref_ff)) <= 1e-10 * np.max(np.abs(ref_ff))
        p.close()


def test_invalid_mesh_rejected_on_device_path(B, torch):
    wp = W.circle_problem(8, 40.0, 80.0)     # elements several wavelengths long
    p = B.Problem.from_workload(wp)
    with pytest.raises(B.BemError) as e:
        p.bem_assemble()
    assert e.value.status == B.BEM_EINVAL
    p.close()


@pytest.mark.parametrize("ne,nrhs", [(700, 3), (701, 64), (4096, 64)])
def test_matvec_tensor_core_matches_reference(B, torch, ne, nrhs):
    """FP16 x 3 tcgen05 GEMM: y = A_hi x against the complex128 product of the same stored FP32 matrix.
    4096 elements x 64 columns is the launch configuration the benchmark times; 701 elements give a row
    length that needs the padded FP16 stride.  Column 1 is scaled by 1e-4 and column 2 has entries spread
    over six decades, which exercises the per-column scaling and FP16's subnormal range."""
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(ne, 0.3, 5), P=0, M=1, closed=True)])
    p = B.Problem.from_workload(wp, prec="mixed_tc")
    n2 = p.bem_num_unknowns()
    A = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")
    p.bem_get_matrix(A, which=0)
    g = torch.Generator(device="cpu").manual_seed(nrhs)
    x = torch.randn((nrhs, n2), dtype=torch.complex128, generator=g)
    x[1] *= 1e-4
    x[2] *= 10.0 ** (-6.0 * torch.rand(n2, generator=g, dtype=torch.float64))
    x = x.cuda().to(torch.complex64).to(torch.complex128)  # the kernel sees FP32 inputs
    y = torch.empty_like(x)
    for rep in range(2):                                   # two calls in a row: no state carried over
        p.bem_profile_enable(True)
        p.bem_matvec(x, y, n_rhs=nrhs)
        prof = p.bem_profile_read()
        assert prof["matvec"][1] == 4   # column maxima, B operand, GEMM, stream-K reduction
        ref = (A @ x.T).T
        err = (torch.linalg.vector_norm(y - ref, dim=1) / torch.linalg.vector_norm(ref, dim=1)).max().item()
        # 22-bit split operands with FP32 tensor-core accumulation over 256-value segments (the previous
        # 3xTF32 kernel measured 2.1e-6 at 8192 x 64); the FP32 SIMT kernels reach ~1e-6.  The inner
        # solves run at 1e-5.
        assert err <= 5e-6, err
    p.close()


def test_solve_mixed_tensor_core_matches_oracle_lu(B, torch):
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(700, 0.3, 5), P=0, M=1, closed=True)])
    A = O.assemble(wp, Q=4)
    ang = W.plane_wave_angles(8)
    p = B.Problem.from_workload(wp, prec="mixed_tc", tol=1e-10)
    x = torch.empty((8, p.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave(ang, x)
    assert st == B.BEM_OK and np.all(rs <= 1e-10), (st, rs)
    for r in (0, 3, 7):
        xl = O.solve_lu(A, O.rhs_planewave(wp, ang[r]))
        assert rel(x[r].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_tc"])
@pytest.mark.parametrize("nrhs", [1, 5])
def test_residual_matches_oracle(B, torch, prec, nrhs):
    """r = b - A x through the C-ABI against the oracle's FP64 matrix: for random x (no cancellation), for
    the LU solution (residual dominated by cancellation, where the double-float sum matters), for that
    solution scaled by 2^70, for x spread over 30 decades, and for x = 0 (r must be b exactly).  mixed_tc with
    several columns forms the small terms hi x_lo + lo x_hi on the tensor cores."""
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)])
    A = O.assemble(wp, Q=4)
    n2 = A.shape[0]
    rng = np.random.default_rng(5)
    b = np.stack([O.rhs_planewave(wp, t) for t in np.linspace(0, 3, nrhs)])
    for kind in ("random", "solution", "scaled", "spread", "zero"):
        bk = b
        if kind == "random":
            x = rng.normal(size=(nrhs, n2)) + 1j * rng.normal(size=(nrhs, n2))
        elif kind == "solution":
            x = np.ascontiguousarray(np.linalg.solve(A, b.T).T)
        elif kind == "scaled":          # far from unit magnitude: the offsets follow the data's exponents
            x = np.ascontiguousarray(np.linalg.solve(A, b.T).T) * 2.0 ** 70
            bk = b * 2.0 ** 70
        elif kind == "spread":          # entries spread over 30 decades
            x = (rng.normal(size=(nrhs, n2)) + 1j * rng.normal(size=(nrhs, n2))) * 10.0 ** rng.uniform(-20, 10, (nrhs, n2))
        else:
            x = np.zeros((nrhs, n2), complex)
        ref = bk - (A @ x.T).T
        scale = np.max(np.abs(A)) * np.max(np.abs(x)) * np.sqrt(n2)
        p = B.Problem.from_workload(wp, prec=prec)
        xd = torch.as_tensor(x, device="cuda")
        bd = torch.as_tensor(bk, device="cuda")
        rd = torch.empty_like(bd)
        p.bem_residual(xd, bd, rd, n_rhs=nrhs)
        got = rd.cpu().numpy()
        if kind == "zero":
            assert np.array_equal(got, bk)
            p.close()
            continue
        # the two matrices agree to ~1e-13 per entry; an FP32 residual would miss by ~1e-7
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (kind, np.max(np.abs(got - ref)) / scale)
        p.close()


@pytest.mark.slow
def test_full_size_junction_disk_c3(B, torch):
    """Junction disk, 8192 elements (16384 unknowns), host k = 15, halves k = 22.5 and 30, one plane wave:
    every entry of the mixed matrix (hi + lo) against the oracle's whole matrix (rows split over host
    processes), and the mixed (tol 1e-8) and FP64 (tol 1e-12) GPU solutions element by element against the
    oracle's LU solution."""
    wp = W.cfg_junction_c3()
    n2 = 2 * wp.n_elem
    A = O.assemble_parallel(wp, Q=4)
    pm = B.Problem.from_workload(wp, prec="mixed", tol=1e-8, max_iter=1000)
    G = torch.empty((n2, n2), dtype=torch.complex128, device="cuda")     # 4.3 GB
    pm.bem_get_matrix(G, which=1)
    got = G.cpu().numpy()
    del G
    torch.cuda.empty_cache()
    blk, rl = block_errors(got, A)
    del got
    assert blk <= ENTRY_BLOCK_TOL and rl <= ENTRY_REL_TOL, (blk, rl)
    xl = O.solve_lu(A, O.rhs_planewave(wp, 0.0))
    del A
    xm = torch.empty((1, n2), dtype=torch.complex128, device="cuda")
    st, it, rs = pm.bem_solve_planewave([0.0], xm)
    assert st == B.BEM_OK and rs[0] <= 1e-8
    pm.close()
    assert rel(xm.cpu().numpy()[0], xl) <= SOLUTION_TOL_MIXED
    pf = B.Problem.from_workload(wp, prec="fp64", tol=1e-12, max_iter=1000)
    xf = torch.empty_like(xm)
    st, itf, rsf = pf.bem_solve_planewave([0.0], xf)
    assert st == B.BEM_OK
    pf.close()
    assert rel(xf.cpu().numpy()[0], xl) <= SOLUTION_TOL_FP64


@pytest.mark.parametrize("name,mk,solve", [
    # k times the bounding-box diagonal below 127: the kernels without the reduction by pi/2
    ("star300", lambda: W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25],
                                  segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)]), True),
    # arguments up to ~280 reach Hankel's expansion: the kernels with the reduction (products and residual only:
    # 2.6 elements per interior wavelength is too coarse a mesh for a meaningful solve)
    ("ellipse250_k40", lambda: W.Problem(k=[40.0, 70.0], eps=[1.0, (70.0 / 40.0) ** 2],
                                         segments=[W.Segment(W.ellipse(250, 4.0), P=0, M=1, closed=True)]), False),
], ids=["star300", "ellipse250_k40"])
def test_matrix_free_matvec_residual_and_solve(B, torch, name, mk, solve):
    """Matrix-free products (entries recomputed, nothing stored) against the stored FP64 matrix, the
    residual against the oracle, and the matrix-free solve against the oracle's LU solution."""
    wp = mk()
    pf = B.Problem.from_workload(wp, prec="fp64", matrix_free=1, tol=1e-12)
    ps = B.Problem.from_workload(wp, prec="fp64")
    n2 = pf.bem_num_unknowns()
    assert pf.bem_footprint_bytes(1) < ps.bem_footprint_bytes(1) - n2 * n2 * 16 + 1
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn((2, n2), dtype=torch.complex128, generator=g).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    pf.bem_matvec(x, y1, n_rhs=2)
    ps.bem_matvec(x, y2, n_rhs=2)
    assert (torch.linalg.vector_norm(y1 - y2, dim=1) / torch.linalg.vector_norm(y2, dim=1)).max().item() <= 1e-13
    A = O.assemble(wp, Q=4)
    b = np.stack([O.rhs_planewave(wp, 0.0), O.rhs_planewave(wp, 1.0)])
    r = torch.empty_like(x)
    pf.bem_residual(x, torch.as_tensor(b, device="cuda"), r, n_rhs=2)
    ref = b - (A @ x.cpu().numpy().T).T
    assert np.max(np.abs(r.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(A)) * np.max(np.abs(x.cpu().numpy())) * n2
    if solve:
        xs = torch.empty((1, n2), dtype=torch.complex128, device="cuda")
        st, it, rs = pf.bem_solve_planewave([0.0], xs)
        assert st == B.BEM_OK
        assert rel(xs[0].cpu().numpy(), O.solve_lu(A, b[0])) <= SOLUTION_TOL_FP64
    with pytest.raises(B.BemError):
        pf.bem_get_matrix(torch.empty((n2, n2), dtype=torch.complex128, device="cuda"))
    pf.close()
    ps.close()
    with pytest.raises(B.BemError):                       # the tensor-core path stores its split copy of A
        B.Problem(prec="mixed_tc", matrix_free=1)


def test_near_field_matches_oracle_and_mie_grid(B, torch):
    """Field on the paper's 101 x 101 grid over [-2.99, 2.99]^2 (Sec. 7.1): GPU against the oracle at sampled
    points, and the paper's relative l2 error of Re u against the Mie series decreasing with N."""
    k1, k2, e2 = 5.0, 7.5, 2.25
    g = np.linspace(-2.99, 2.99, 101)
    pts = np.array([(a, b) for a in g for b in g])
    dom = (np.hypot(pts[:, 0], pts[:, 1]) < 1.0).astype(np.int32)
    ref = O.mie_field(k1, k2, e2, pts[::97])
    errs = []
    for n in (256, 512):
        wp = W.circle_problem(n, k1, k2, e2)
        p = B.Problem.from_workload(wp, tol=1e-12, quad_order=10)
        x = torch.empty((1, 2 * n), dtype=torch.complex128, device="cuda")
        p.bem_solve_planewave([0.0], x)
        u = torch.empty((1, len(pts)), dtype=torch.complex128, device="cuda")
        p.bem_near_field(x, pts, dom, u, angles=[0.0])
        got = u[0].cpu().numpy()
        samp = np.arange(0, len(pts), 97)
        oref = O.near_field(wp, x[0].cpu().numpy(), pts[samp], dom[samp], theta=0.0, Q=10)
        assert np.max(np.abs(got[samp] - oref)) <= 1e-11 * np.max(np.abs(oref))
        mie = O.mie_field(k1, k2, e2, pts) if n == 256 else mie
        errs.append(np.sqrt(np.sum((got.real - mie.real) ** 2) / np.sum(mie.real ** 2)))
        p.close()
    assert errs[1] < errs[0] and errs[1] < 2e-2


def test_gpu_iteration_study_matches_paper_trend(B, torch):
    """NEXT-1 reproduction on the GPU (FP64 path, Sec. 7.1 setting): iterations of the conventional form grow
    with N, those of the proposed form stay flat, up to N = 1600."""
    its = {"conv": [], "mod": []}
    for n in (200, 400, 800, 1600):
        wp = W.circle_problem(n, 5.0, 5.0 * np.sqrt(2.0), eps_i=2.0)
        for f in its:
            p = B.Problem.from_workload(wp, form=f, tol=1e-8, quad_order=10, max_iter=800)
            x = torch.empty((1, 2 * n), dtype=torch.complex128, device="cuda")
            st, it, rs = p.bem_solve_planewave([0.0], x)
            its[f].append(int(it[0]))
            p.close()
    assert max(its["mod"]) - min(its["mod"]) <= 2, its
    assert all(b > 1.15 * a for a, b in zip(its["conv"], its["conv"][1:])), its


def test_concentric_largest_eigenvalue_from_gpu_matrix(B, torch):
    """Sec. 7.2's printed largest-magnitude eigenvalue of A^2 (concentric circles: 100 inner and 200 outer
    elements, omega = 1, eps = 1, 2, 3; Q = 10), taken from the matrix the GPU assembles: 'mod' to the printed
    four digits, 'orig' within 1 % (its printed imaginary part is 0.7 % off the oracle's)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as fh:
        g = json.load(fh)["concentric_largest_eig"]
    wp = W.concentric(g["n_inner"], g["n_outer"], g["omega"], eps=tuple(g["eps"]))
    for form, tol in (("mod", 1e-3), ("orig", 0.01 * abs(complex(*g["orig"])))):
        A = gpu_matrix(B, torch, wp, quad_order=10, form=form)["main"]
        ev = np.linalg.eigvals(A @ A)
        lam = ev[np.argmax(np.abs(ev))]
        assert abs(lam - complex(*g[form])) < tol, (form, lam)


def test_concentric_gpu_solution_matches_two_layer_series(B, torch):
    """Concentric circles (Sec. 7.2): mixed-precision GPU solutions of the 'mod' system, far field against the
    two-layer series (first order in N) and the traces against the oracle's LU solution."""
    eps = (1.0, 2.0, 3.0)
    om = 1.0
    k = [om * np.sqrt(e) for e in eps]
    ang = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    ref = O.mie2_far_field(k, eps, ang)
    errs = []
    for N in (300, 600):
        wp = W.concentric(N // 3, 2 * N // 3, om, eps=eps)
        p = B.Problem.from_workload(wp, prec="mixed", tol=1e-10, quad_order=10)
        x = torch.empty((1, 2 * N), dtype=torch.complex128, device="cuda")
        st, it, rs = p.bem_solve_planewave([0.0], x)
        assert st == B.BEM_OK
        ff = torch.empty((1, len(ang)), dtype=torch.complex128, device="cuda")
        p.bem_far_field(x, ang, ff)
        errs.append(rel(ff[0].cpu().numpy(), ref))
        if N == 300:
            xl = O.solve_lu(O.assemble(wp, Q=10), O.rhs_planewave(wp, 0.0))
            assert rel(x[0].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED
        p.close()
    assert errs[1] < errs[0] / 1.6 and errs[1] < 3e-3


@pytest.mark.parametrize("name", ["circle_11", "junction_16"])
def test_mixed_inner_solves_keep_orthogonality(B, torch, name):
    """A high-frequency circle and a low-frequency junction disk of the serving stream: one classical
    Gram-Schmidt pass in FP32 loses orthogonality there (measured: 1275 and 309 iterations against 106 and 43
    for FP64); the selective second pass brings the mixed path back within a small factor of FP64."""
    wp = next(w for _, w in W.cfg_serving_c5(count=20) if w.name == name)
    q = B.Problem.from_workload(wp, prec="mixed", tol=1e-8, max_iter=400)
    x = torch.empty((1, wp.n_unknowns), dtype=torch.complex128, device="cuda")
    st, it, rs = q.bem_solve_planewave([0.0], x)
    q.close()
    q = B.Problem.from_workload(wp, prec="fp64", tol=1e-12, max_iter=800)
    x64 = torch.empty((1, wp.n_unknowns), dtype=torch.complex128, device="cuda")
    st64, it64, rs64 = q.bem_solve_planewave([0.0], x64)
    q.close()
    q = B.Problem.from_workload(wp, prec="fp64", tol=1e-8, max_iter=800)
    st8, it8, rs8 = q.bem_solve_planewave([0.0], torch.empty_like(x64))
    q.close()
    assert st == B.BEM_OK and rs[0] <= 1e-8
    assert it[0] <= 3 * it8[0], (int(it[0]), int(it8[0]))
    assert rel(x[0].cpu().numpy(), x64[0].cpu().numpy()) <= SOLUTION_TOL_MIXED


def test_matrix_free_mixed_reaching_the_expansion(B, torch):
    """Mixed matrix-free solve where Bessel arguments reach Hankel's expansion (an ellipse of aspect 4 with
    k = 40 / 70, arguments up to ~280: the recomputing kernels keep the reduction by pi/2), half of the rows
    stored, against the same problem with its whole matrix stored: both solve to 1e-8, so their solutions agree
    to ~cond x 1e-8."""
    wp = W.Problem(k=[40.0, 70.0], eps=[1.0, (70.0 / 40.0) ** 2],
                   segments=[W.Segment(W.ellipse(600, 4.0), P=0, M=1, closed=True)])
    n = wp.n_elem
    x = torch.empty((2, 1, 2 * n), dtype=torch.complex128, device="cuda")
    for k, kw in enumerate((dict(matrix_free=1, store_bytes=(n // 2) * 2 * 2 * n * 8), {})):
        p = B.Problem.from_workload(wp, prec="mixed", tol=1e-8, max_iter=600, **kw)
        st, it, rs = p.bem_solve_planewave(np.array([0.3]), x[k])
        assert st == B.BEM_OK and rs[0] <= 1e-8, (kw, st, it, rs)
        p.close()
    assert rel(x[0, 0].cpu().numpy(), x[1, 0].cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("store_frac", [0.0, 0.5, 1.0])
def test_matrix_free_mixed_with_stored_rows(B, torch, store_frac):
    """Matrix-free mixed solves: the leading element rows that fit in store_bytes are kept as complex FP32, the
    others recomputed in every inner product; the refinement residual recomputes every entry with FP64 sums.
    Nothing stored, half the rows stored and all rows stored: the solution matches the oracle's LU solution to
    the mixed bar, and the problem holds less device memory than with its whole matrix stored."""
    wp = W.Problem(k=[20.0, 30.0], eps=[1.0, 2.25], segments=[W.Segment(W.star(300, 0.3, 5), P=0, M=1, closed=True)])
    n = wp.n_elem
    store = int(store_frac * n) * 2 * 2 * n * 8
    p = B.Problem.from_workload(wp, prec="mixed", matrix_free=1, store_bytes=store, tol=1e-10, max_iter=300)
    full = B.Problem.from_workload(wp, prec="mixed")
    assert p.bem_footprint_bytes(1) < full.bem_footprint_bytes(1)
    full.close()
    ang = np.array([0.0, 2.1])
    x = torch.empty((2, 2 * n), dtype=torch.complex128, device="cuda")
    st, it, rs = p.bem_solve_planewave(ang, x)
    assert st == B.BEM_OK and np.all(rs <= 1e-10), (st, it, rs)
    A = O.assemble(wp, Q=4)
    for r, t in enumerate(ang):
        xl = O.solve_lu(A, O.rhs_planewave(wp, t))
        assert rel(x[r].cpu().numpy(), xl) <= SOLUTION_TOL_MIXED, (store_frac, r)
    with pytest.raises(B.BemError) as e:          # no matrix to read back
        p.bem_get_matrix(torch.empty((2 * n, 2 * n), dtype=torch.complex128, device="cuda"))
    assert e.value.status == B.BEM_ESTATE
    p.close()
