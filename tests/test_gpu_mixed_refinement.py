"""GPU parity of the FP32-arithmetic high-order apply and of the
mixed-precision iterative refinement (lor_apply_f32, lor_pcg_solve_ir)
against the FP64 CPU oracle.

Tolerances:
  * FP32 apply: 2e-5 of max |A_p x| (FP32 unit roundoff 6e-8 times the
    growth of the six contraction stages and the D product, with margin);
    essential rows return x bit-exactly (they are written in FP64);
  * refinement: the reported residual is the FP64 one and must meet rtol;
    the solution matches the oracle's PCG solution as the FP64 solver's does.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import make_problem

pytestmark = pytest.mark.gpu

DEV = "cuda"
F32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def setup(dims, p, seed=1):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("t", *dims, p, seed=seed, jitter=0.1, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    op = LOR(p, *dims, t(prob.vertices).contiguous())
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    return prob, mesh, op


def essential(dims, p):
    n = [d * p + 1 for d in dims]
    I, J, K = np.meshgrid(*(np.arange(m) for m in n), indexing="ij")
    e = (I == 0) | (I == n[0] - 1) | (J == 0) | (J == n[1] - 1) | (K == 0) | (K == n[2] - 1)
    return e.transpose(2, 1, 0).reshape(-1)  # x fastest


# every mesh at least two elements thick on each axis, so the jitter moves an
# interior vertex and the metric has off-diagonal entries
CASES = [((3, 2, 4), 1), ((2, 3, 2), 2), ((3, 3, 2), 3), ((4, 3, 3), 4), ((2, 2, 3), 5), ((2, 2, 2), 6),
         ((2, 2, 2), 7), ((2, 2, 2), 8), ((2, 2, 2), 9), ((2, 2, 2), 10)]


@pytest.mark.parametrize("dims,p", CASES)
def test_apply_f32_matches_oracle(dims, p):
    prob, mesh, op = setup(dims, p)
    x = np.random.default_rng(p).standard_normal(op.ndof)
    y = op.apply_f32(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err <= F32_TOL, err
    assert err > 0.0  # FP32 arithmetic really ran (FP64 would agree to ~1e-15)
    ess = essential(dims, p)
    np.testing.assert_array_equal(y[ess], x[ess])


@pytest.mark.parametrize("dims,p", [((2, 3, 2), 2), ((3, 2, 2), 5)])
def test_apply_f32_with_reaction(dims, p):
    prob, mesh, op = setup(dims, p)
    rng = np.random.default_rng(11)
    beta = np.exp(rng.standard_normal(prob.kappa.shape))
    op.set_reaction(t(beta).reshape(-1), check=True)
    x = rng.standard_normal(op.ndof)
    y = op.apply_f32(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x, beta=beta)
    assert np.abs(y - ref).max() <= F32_TOL * np.abs(ref).max()
    # a later coefficient change refreshes the FP32 factors
    op.set_reaction(None)
    kappa2 = 2.0 * prob.kappa
    op.set_coefficient(t(kappa2).reshape(-1), check=True)
    y2 = op.apply_f32(t(x)).cpu().numpy()
    ref2 = oracle.ho_apply(mesh, p, p + 2, kappa2, x)
    assert np.abs(y2 - ref2).max() <= F32_TOL * np.abs(ref2).max()


@pytest.mark.parametrize("dims,p", [((2, 2, 2), 3), ((2, 2, 2), 8)])
def test_apply_f32_general_mesh(dims, p):
    from test_gpu_general import make
    prob, mesh, op, perm, *_ = make(dims, p)
    x = np.random.default_rng(5).standard_normal(op.ndof)
    xn = np.empty_like(x)
    xn[perm] = x
    y = op.apply_f32(t(xn)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    assert np.abs(y[perm] - ref).max() <= F32_TOL * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("scheme", ["restart", "replace"])
@pytest.mark.parametrize("inner_rtol", [1e-2, 1e-4])
def test_refinement_matches_oracle(inner_rtol, scheme):
    dims, p = (3, 3, 4), 3
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(torch.float32)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    lam = oracle.power_lambda_max(*csr, v0, 20)
    op.precond_setup("cheb", torch.float32, degree=3, lambda_max=lam)
    b = t(prob.rhs)
    x, outer, inner, rel = op.pcg_solve_ir(b, 1e-10, inner_rtol, 4000, scheme=scheme)
    # the reported residual is the FP64 one
    r = b - op.apply(x)
    true_rel = (torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)).item()
    assert rel <= 1e-10 and abs(true_rel - rel) <= 1e-3 * rel
    # each outer step gains about inner_rtol: 1e-10 needs at least log(1e-10)/log(inner_rtol) of them
    assert outer >= int(np.ceil(np.log(1e-10) / np.log(inner_rtol))) - 1 and inner >= outer
    xo, ito, relo, _ = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 2000, oracle.PRECOND_CHEB, 3,
                                  lam / 30, 1.1 * lam)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max()


def test_refinement_general_mesh_with_reaction():
    from test_gpu_general import make
    dims, p = (3, 2, 3), 3
    prob, mesh, op, perm, eperm, rot, to_new, *_ = make(dims, p)
    beta = np.exp(np.random.default_rng(21).standard_normal(prob.kappa.shape))
    op.set_reaction(t(to_new(beta)).reshape(-1), check=True)
    op.build_pattern_internal()
    op.assemble_internal(torch.float32)
    op.precond_setup("cheb", torch.float32, degree=3, power_iters=20)
    bn = np.empty(op.ndof)
    bn[perm] = prob.rhs
    for scheme in ("restart", "replace"):
        x, outer, inner, rel = op.pcg_solve_ir(t(bn), 1e-10, 1e-4, 4000, scheme=scheme)
        assert rel <= 1e-10
        # against the oracle's FP64 operator: residual of the permuted solution
        xs = x.cpu().numpy()[perm]
        r = prob.rhs - oracle.ho_apply(mesh, p, p + 2, prob.kappa, xs, beta=beta)
        assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(prob.rhs)
    op.close()


def test_refinement_limits_and_errors():
    from paper_2210_12253_gb300 import LORError
    prob, mesh, op = setup((2, 2, 2), 3)
    op.precond_setup("none")
    b = t(prob.rhs)
    for scheme in ("restart", "replace"):
        x, outer, inner, rel = op.pcg_solve_ir(b, 1e-14, 1e-4, 3, raise_on_noconv=False, scheme=scheme)
        assert inner == 3 and rel > 1e-14
        with pytest.raises(LORError) as ei:
            op.pcg_solve_ir(b, 1e-14, 1e-4, 3, scheme=scheme)
        assert ei.value.code == 5
    import ctypes
    no, ni, rel = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    rc = op._lib.lor_pcg_solve_ir(op._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-8, 1e-4,
                                  100, 7, ctypes.byref(no), ctypes.byref(ni), ctypes.byref(rel),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1
    with pytest.raises(LORError) as ei:
        op.pcg_solve_ir(b, 1e-8, 1.5, 100)
    assert ei.value.code == 1
    z = torch.zeros_like(b)
    x, outer, inner, rel = op.pcg_solve_ir(z, 1e-8, 1e-4, 100)
    assert outer == 0 and inner == 0 and rel == 0.0 and torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("dims,p,kind,degree", [((4, 3, 3), 1, "jacobi", 1), ((2, 2, 3), 2, "cheb", 1),
                                                ((2, 2, 2), 4, "cheb", 2), ((1, 2, 1), 8, "cheb", 5)])
def test_refinement_across_preconditioners_and_degrees(dims, p, kind, degree):
    """Every preconditioner mode of the fused PCG update (Jacobi, Chebyshev of
    degree 1 and >= 2) under both schemes, against the oracle's FP64 solve."""
    prob, mesh, op = setup(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(torch.float32)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    lam = oracle.power_lambda_max(*csr, v0, 20)
    if kind == "jacobi":
        op.precond_setup("jacobi", torch.float32)
        ref = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 4000, oracle.PRECOND_JACOBI)
    else:
        op.precond_setup("cheb", torch.float32, degree=degree, lambda_max=lam)
        ref = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 4000, oracle.PRECOND_CHEB, degree,
                         lam / 30, 1.1 * lam)
    xo = ref[0]
    b = t(prob.rhs)
    for scheme in ("replace", "restart"):
        x, outer, inner, rel = op.pcg_solve_ir(b, 1e-10, 1e-3, 4000, scheme=scheme)
        r = prob.rhs - oracle.ho_apply(mesh, p, p + 2, prob.kappa, x.cpu().numpy())
        assert rel <= 1e-10 and np.linalg.norm(r) <= 2e-10 * np.linalg.norm(prob.rhs), scheme
        assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max(), scheme
    op.close()
