"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances (derived in the design notes from the arithmetic):
  * sparsity: bit-exact;
  * FP64 values, operator, gradients: 1e-12 relative to the row (or vector)
    magnitude; the kernels sum at most a few hundred FP64 products per
    output, so the expected error is ~1e-15;
  * FP32 LOR values / FP32 smoother: 1e-5 relative (FP32 unit roundoff
    6e-8 times the short sums involved), stated per result.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import make_problem

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def setup(dims, p, seed=1, jitter=0.1, kappa="lognormal"):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("t", *dims, p, seed=seed, jitter=jitter, kappa=kappa, rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    op = LOR(p, *dims, torch.tensor(prob.vertices, device=DEV).contiguous())
    op.set_coefficient(torch.tensor(prob.kappa, device=DEV).reshape(-1), check=True)
    return prob, mesh, op


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def rowwise_rel_err(rp, v_gpu, v_ref):
    err = 0.0
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        scale = np.abs(v_ref[a:b]).max()
        err = max(err, np.abs(v_gpu[a:b] - v_ref[a:b]).max() / scale)
    return err


# every mesh at least two elements thick on each axis, so the jitter moves an
# interior vertex and the metric has off-diagonal entries
CASES = [((3, 2, 4), 1), ((2, 3, 2), 2), ((3, 3, 2), 3), ((4, 3, 3), 4), ((2, 2, 3), 5), ((2, 2, 2), 6),
         ((2, 2, 2), 7), ((2, 2, 2), 8), ((2, 2, 2), 9), ((2, 2, 2), 10)]


@pytest.mark.parametrize("dims,p", CASES)
def test_pattern_bit_exact(dims, p):
    prob, mesh, op = setup(dims, p)
    rp, ci = op.build_pattern()
    orp, oci, _ = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert op.nnz == len(oci)
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), oci)


@pytest.mark.parametrize("dims,p", CASES)
def test_lor_values_fp64(dims, p):
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12


@pytest.mark.parametrize("dims", [(3, 3, 3), (5, 2, 3)])
def test_lor_values_fp64_partial_last_cta(dims):
    """At p = 2 the FP64 assembly takes four elements per CTA; 27 and 30
    elements leave the last CTA three and two slots short, whose threads
    compute on a stand-in sub-hex and store nothing."""
    p = 2
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12


@pytest.mark.parametrize("dims,p", [((3, 2, 4), 2), ((4, 3, 3), 4), ((2, 1, 2), 6)])
def test_lor_values_fp32(dims, p):
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    v = op.assemble(torch.float32).cpu().numpy().astype(np.float64)
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert rowwise_rel_err(orp, v, ov) <= 1e-5


@pytest.mark.parametrize("dims,p", CASES)
def test_apply_fp64(dims, p):
    prob, mesh, op = setup(dims, p)
    x = np.random.default_rng(p).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dims,p", [((3, 2, 4), 1), ((3, 3, 2), 3), ((4, 3, 3), 4), ((1, 2, 1), 7)])
def test_apply_backward_fp64(dims, p):
    prob, mesh, op = setup(dims, p)
    rng = np.random.default_rng(10 + p)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    gx, gk = op.apply_backward(t(x), t(gy))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, p + 2, prob.kappa, x, gy)
    assert np.abs(gx.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    gk = gk.cpu().numpy().reshape(rgk.shape)
    assert np.abs(gk - rgk).max() <= 1e-12 * np.abs(rgk).max()
    _, gk_only = op.apply_backward(t(x), t(gy), want_gx=False)
    np.testing.assert_array_equal(gk_only.cpu().numpy().reshape(rgk.shape), gk)


@pytest.mark.parametrize("dims,p", [((3, 2, 2), 2), ((2, 3, 2), 5)])
def test_load_vector(dims, p):
    prob, mesh, op = setup(dims, p)
    b1 = op.load_vector().cpu().numpy()
    assert np.abs(b1 - oracle.load_vector(mesh, p, p + 2)).max() <= 1e-13 * np.abs(b1).max()
    f = np.random.default_rng(0).standard_normal((mesh.nel, (p + 2) ** 3))
    bf = op.load_vector(t(f).reshape(-1)).cpu().numpy()
    ref = oracle.load_vector(mesh, p, p + 2, f)
    assert np.abs(bf - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_spmv(dtype, tol):
    dims, p = (3, 4, 2), 3
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    x = np.random.default_rng(3).standard_normal(op.ndof)
    y = op.spmv(t(x), dtype).cpu().numpy()
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    ref = oracle.csr_spmv(*csr, x)
    assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_preconditioners(dtype, tol):
    dims, p = (3, 2, 3), 4
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    lam = op.precond_setup("cheb", dtype, degree=3, power_iters=20, v0=t(v0))
    lam_ref = oracle.power_lambda_max(*csr, v0, 20)
    assert abs(lam - lam_ref) <= (1e-10 if dtype == torch.float64 else 1e-5) * lam_ref
    r = np.random.default_rng(8).standard_normal(op.ndof)
    for k in (1, 2, 3, 5):
        op.precond_setup("cheb", dtype, degree=k, lambda_max=lam_ref)
        z = op.precond_apply(t(r)).cpu().numpy()
        ref = oracle.chebyshev(*csr, r, k, lam_ref / 30, 1.1 * lam_ref)
        assert np.abs(z - ref).max() <= tol * np.abs(ref).max(), k
    op.precond_setup("jacobi", dtype)
    z = op.precond_apply(t(r)).cpu().numpy()
    ref = r / oracle.csr_diagonal(*csr)
    assert np.abs(z - ref).max() <= tol * np.abs(ref).max()


def test_pcg_unit_source_jacobi_fp64():
    """4^3 undistorted, p = 3, kappa = 1, f = 1, Jacobi-on-LOR PCG to 1e-10."""
    prob, mesh, op = setup((4, 4, 4), 3, jitter=0.0, kappa="one")
    b = op.load_vector()
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    op.precond_setup("jacobi", torch.float64)
    x, it, rel = op.pcg_solve(b, 1e-10, 1000)
    csr = oracle.lor_assemble(mesh, 3, 5, prob.kappa, True)
    bo = oracle.load_vector(mesh, 3, 5)
    xo, ito, relo, _ = oracle.pcg(mesh, 3, 5, prob.kappa, csr, bo, 1e-10, 1000, oracle.PRECOND_JACOBI)
    assert rel <= 1e-10 and abs(it - ito) <= 1
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-9 * np.abs(xo).max()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_pcg_chebyshev_matches_oracle(dtype):
    dims, p = (3, 3, 4), 3
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    lam = oracle.power_lambda_max(*csr, v0, 20)
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    x, it, rel = op.pcg_solve(t(prob.rhs), 1e-10, 2000)
    xo, ito, relo, _ = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 2000, oracle.PRECOND_CHEB, 3,
                                  lam / 30, 1.1 * lam)
    assert rel <= 1e-10
    if dtype == torch.float64:
        assert abs(it - ito) <= 1
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max()


def test_pcg_no_convergence_reported():
    prob, mesh, op = setup((2, 2, 2), 3)
    op.precond_setup("none")
    x, it, rel = op.pcg_solve(t(prob.rhs), 1e-14, 3, raise_on_noconv=False)
    assert it == 3 and rel > 1e-14
    from paper_2210_12253_gb300 import LORError
    with pytest.raises(LORError) as ei:
        op.pcg_solve(t(prob.rhs), 1e-14, 3)
    assert ei.value.code == 5


def test_autograd_apply_matches_oracle():
    from paper_2210_12253_gb300 import LORApply
    dims, p = (2, 3, 2), 3
    prob, mesh, op = setup(dims, p)
    rng = np.random.default_rng(4)
    x = t(rng.standard_normal(op.ndof)).requires_grad_(True)
    kap = t(prob.kappa.reshape(-1)).requires_grad_(True)
    w = t(rng.standard_normal(op.ndof))
    L = (LORApply.apply(op, kap, x) * w).sum()
    L.backward()
    rgx, rgk = oracle.ho_apply_backward(mesh, p, p + 2, prob.kappa, x.detach().cpu().numpy(), w.cpu().numpy())
    assert np.abs(x.grad.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    assert np.abs(kap.grad.cpu().numpy() - rgk.ravel()).max() <= 1e-12 * np.abs(rgk).max()


def test_adjoint_gradient_against_finite_differences():
    """dJ/dtheta from the adjoint PCG + backward kernel vs central differences
    of the GPU's own J, and vs the oracle's gradient (dense solves)."""
    import scipy.linalg
    from meshutil import element_corners, element_dofs, eliminate, essential_mask
    from paper_2210_12253_gb300 import solve_with_adjoint
    from paper_2210_12253_gb300.inputs import make_problem as mp
    dims, p = (2, 2, 2), 3
    prob = mp("t", *dims, p, seed=3, kappa="theta", rhs="normal")
    from paper_2210_12253_gb300 import LOR
    op = LOR(p, *dims, t(prob.vertices))
    mesh = oracle.Mesh(*dims, prob.vertices)
    q = p + 2
    C, Dm = element_corners(mesh.V, *dims), element_dofs(*dims, p)
    ess = essential_mask(*dims, p)

    def dense_solve(theta, rhs):
        A = eliminate(oracle.dense_general(C, Dm, np.exp(theta), p, q, prob.ndof), ess)
        return scipy.linalg.solve(A, rhs, assume_a="pos")

    ustar = dense_solve(prob.theta_star, prob.rhs)
    opts = dict(rtol=1e-13, maxit=5000, precond="cheb", dtype=torch.float64)
    th = t(prob.theta.reshape(-1))
    J, g = solve_with_adjoint(op, th, t(prob.rhs), t(ustar), **opts)
    u = dense_solve(prob.theta, prob.rhs)
    lam = dense_solve(prob.theta, u - ustar)
    _, gk = oracle.ho_apply_backward(mesh, p, q, np.exp(prob.theta), u, lam, want_gx=False)
    gref = -np.exp(prob.theta) * gk
    g = g.cpu().numpy().reshape(gref.shape)
    assert np.abs(g - gref).max() <= 1e-8 * np.abs(gref).max()
    rng = np.random.default_rng(5)
    from paper_2210_12253_gb300 import solve
    for _ in range(4):
        v = rng.standard_normal(prob.theta.shape)
        eps = 1e-6 * np.linalg.norm(prob.theta) / np.linalg.norm(v)
        Jp = 0.5 * float(((solve(op, torch.exp(th + eps * t(v.ravel())), t(prob.rhs), **opts) - t(ustar)) ** 2).sum())
        Jm = 0.5 * float(((solve(op, torch.exp(th - eps * t(v.ravel())), t(prob.rhs), **opts) - t(ustar)) ** 2).sum())
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - (g * v).sum()) <= 1e-6 * abs(fd)


# ------------------------------------------------------------------ edge cases and errors
def test_single_element_p1_is_identity():
    """1 element, p = 1: every DOF is essential, so A_p and A_h are identities."""
    prob, mesh, op = setup((1, 1, 1), 1)
    rp, ci = op.build_pattern()
    v = op.assemble(torch.float64).cpu().numpy()
    A = np.zeros((8, 8))
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    for r in range(8):
        A[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    np.testing.assert_array_equal(A, np.eye(8))
    x = np.random.default_rng(0).standard_normal(8)
    np.testing.assert_array_equal(op.apply(t(x)).cpu().numpy(), x)


def test_inverted_element_rejected():
    from paper_2210_12253_gb300 import LOR, LORError
    from paper_2210_12253_gb300.inputs import unit_cube_vertices
    V = unit_cube_vertices(2, 2, 2)
    V[1 + 3 * (1 + 3 * 1)] = [0.5, 0.5, 1.2]
    with pytest.raises(LORError) as ei:
        LOR(2, 2, 2, 2, t(V))
    assert ei.value.code == 2


def test_injected_allocation_failure_leaves_the_context_usable(monkeypatch):
    """LOR_DEVICE_ALLOC_LIMIT makes the context's next allocation fail on the
    host: the call returns LOR_ENOMEM, and once the limit is lifted the same
    context assembles and applies as usual."""
    from paper_2210_12253_gb300 import LOR, LORError
    from paper_2210_12253_gb300.inputs import make_problem
    prob = make_problem("t", 2, 2, 2, 3, seed=4, jitter=0.1, kappa="lognormal", rhs="normal")
    op = LOR(3, 2, 2, 2, t(prob.vertices).contiguous())
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    monkeypatch.setenv("LOR_DEVICE_ALLOC_LIMIT", "1")
    with pytest.raises(LORError) as ei:
        op.build_pattern_internal()
    assert ei.value.code == 3 and "LOR_DEVICE_ALLOC_LIMIT" in str(ei.value)
    monkeypatch.delenv("LOR_DEVICE_ALLOC_LIMIT")
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    op.precond_setup("jacobi", torch.float64)
    mesh = oracle.Mesh(2, 2, 2, prob.vertices)
    x = np.random.default_rng(3).standard_normal(op.ndof)
    ref = oracle.ho_apply(mesh, 3, 5, prob.kappa, x)
    assert np.abs(op.apply(t(x)).cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()


def test_bad_coefficient_and_call_order():
    from paper_2210_12253_gb300 import LOR, LORError
    from paper_2210_12253_gb300.inputs import unit_cube_vertices
    op = LOR(2, 2, 2, 2, t(unit_cube_vertices(2, 2, 2)))
    x = torch.zeros(op.ndof, dtype=torch.float64, device=DEV)
    with pytest.raises(LORError) as ei:
        op.apply(x)
    assert ei.value.code == 7
    k = torch.ones(op.nqpt, dtype=torch.float64, device=DEV)
    k[17] = -1.0
    with pytest.raises(LORError) as ei:
        op.set_coefficient(k, check=True)
    assert ei.value.code == 1
    k[17] = float("nan")
    with pytest.raises(LORError):
        op.set_coefficient(k, check=True)
    op.set_coefficient(torch.ones_like(k), check=True)
    with pytest.raises(LORError) as ei:
        op.precond_setup("jacobi", torch.float64)
    assert ei.value.code == 7


@pytest.mark.parametrize("scale", [1e-9, 1e-3, 1e4, 1e9])
def test_fp64_path_at_extreme_mesh_scales(scale):
    """The FP64 setup and assembly form the metric from M = J^T J, whose
    determinant is det(J)^2, and take 1/sqrt(det M) by a range-reduced
    seed: meshes of any size give the oracle's LOR matrix and apply (both
    scale with the element size; det M spans 1e-60 .. 1e+54 here)."""
    from paper_2210_12253_gb300 import LOR
    dims, p = (3, 2, 2), 3
    prob = make_problem("t", *dims, p, seed=1, jitter=0.1, kappa="lognormal", rhs="normal")
    V = prob.vertices * scale
    mesh = oracle.Mesh(*dims, V)
    op = LOR(p, *dims, t(V))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    rp, ci = op.build_pattern()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, oci, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12
    x = np.random.default_rng(2).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("p", [2, 5, 8])
def test_fixed_point_operator_scale_invariance_and_zero(p):
    """The FP64 operator and its backward carry one power-of-two scale per
    element and stage: inputs scaled by 2^k (k = -600, 600) give each
    element's contributions scaled by exactly 2^k, so gkappa (one value per
    Gauss point) scales bit for bit and y, gx (sums of the elements'
    contributions by FP64 atomics, whose order varies from run to run) to
    within a few units of the last place; a zero input gives an exactly zero
    output."""
    dims = (2, 2, 2)
    prob, mesh, op = setup(dims, p)
    rng = np.random.default_rng(30 + p)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    gx, gk = (a.cpu().numpy() for a in op.apply_backward(t(x), t(gy)))
    def near(a, b):  # a few units of the last place of the largest entry
        assert np.abs(a - b).max() <= 4e-16 * np.abs(b).max()

    for k in (-600, 600):
        s = 2.0 ** k
        near(op.apply(t(x * s)).cpu().numpy() / s, y)
        gxs, gks = (a.cpu().numpy() for a in op.apply_backward(t(x * s), t(gy)))
        near(gxs, gx)
        np.testing.assert_array_equal(gks, gk * s)
        gxs, gks = (a.cpu().numpy() for a in op.apply_backward(t(x), t(gy * s)))
        near(gxs / s, gx)
        np.testing.assert_array_equal(gks, gk * s)
    z = np.zeros(op.ndof)
    assert not op.apply(t(z)).cpu().numpy().any()
    gxz, gkz = (a.cpu().numpy() for a in op.apply_backward(t(z), t(z)))
    assert not gxz.any() and not gkz.any()
    op.close()


@pytest.mark.parametrize("p", [3, 6])
def test_fixed_point_operator_mixed_magnitudes(p):
    """Nodal values spanning ten orders of magnitude inside each element (the
    element's largest value sets its fixed-point scale) and a coefficient
    spanning six: the apply and the backward stay within 1e-12 of the
    oracle relative to the output maximum."""
    from paper_2210_12253_gb300 import LOR
    dims = (3, 2, 2)
    prob = make_problem("t", *dims, p, seed=4, jitter=0.1, kappa="lognormal", rhs="normal")
    kappa = prob.kappa * np.exp(np.random.default_rng(5).uniform(-7, 7, prob.kappa.shape))
    mesh = oracle.Mesh(*dims, prob.vertices)
    op = LOR(p, *dims, t(prob.vertices))
    op.set_coefficient(t(kappa).reshape(-1), check=True)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(op.ndof) * 10.0 ** rng.uniform(-10, 0, op.ndof)
    gy = rng.standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, kappa, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    gx, gk = op.apply_backward(t(x), t(gy))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, p + 2, kappa, x, gy)
    assert np.abs(gx.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    gk = gk.cpu().numpy().reshape(rgk.shape)
    assert np.abs(gk - rgk).max() <= 1e-12 * np.abs(rgk).max()
    op.close()


@pytest.mark.parametrize("stretch,jitter,p", [((1000.0, 1.0, 1.0), 0.1, 3), ((1.0, 1e-3, 1e2), 0.1, 4),
                                              ((1.0, 1.0, 1.0), 0.3, 4), ((1.0, 1.0, 1.0), 0.3, 2),
                                              ((1.0, 1e-3, 1e2), 0.1, 1), ((1e2, 1.0, 1e-3), 0.2, 6)])
def test_fixed_point_metric_anisotropic_and_distorted(stretch, jitter, p):
    """The setup and the LOR assembly form adj(J^T J) from J's adjugate rows
    and det J from the first of them (fixed point from p = 2 in the assembly,
    everywhere in the setup): elements stretched 1000:1 (and 1e5 between two
    axes) and strongly distorted ones (vertices moved by up to 30% of the
    spacing) give the oracle's LOR values (1e-12 of the row maximum) and
    apply (1e-12 of the maximum).  Forming the cofactors of M = J^T J instead
    loses O(eps cond(J)^2) and fails the 1e5 case."""
    from paper_2210_12253_gb300 import LOR
    dims = (3, 2, 2)
    prob = make_problem("t", *dims, p, seed=9, jitter=jitter, kappa="lognormal", rhs="normal")
    V = prob.vertices.reshape(-1, 3) * np.asarray(stretch)
    V = V.reshape(prob.vertices.shape)
    mesh = oracle.Mesh(*dims, V)
    op = LOR(p, *dims, t(V))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12
    x = np.random.default_rng(3).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    op.close()
