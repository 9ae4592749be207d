"""GPU parity of the definite Helmholtz (diffusion-reaction) path, the
operator Section 4.1 solves: lor_set_reaction's beta enters the high-order
apply (mass term B_m^T (beta w detJ) B_m), its backward (gx), the LOR matrix
(sub-hex trilinear mass blocks, FP64 and FP32) and PCG, each checked against
the FP64 oracle on the same seeded inputs.  Tolerances as in
test_gpu_parity.py: 1e-12 relative for FP64 results, 1e-5 for FP32 values."""
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


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def setup(dims, p, seed=1, beta_scale=1.0):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("h", *dims, p, seed=seed, jitter=0.1, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    beta = beta_scale * np.exp(np.random.default_rng(100 + seed).standard_normal(prob.kappa.shape))
    op = LOR(p, *dims, t(prob.vertices))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    op.set_reaction(t(beta).reshape(-1), check=True)
    return prob, mesh, op, beta


def rowwise_rel_err(rp, v_gpu, v_ref):
    err = 0.0
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        err = max(err, np.abs(v_gpu[a:b] - v_ref[a:b]).max() / np.abs(v_ref[a:b]).max())
    return err


# every mesh at least two elements thick on each axis, so the jitter moves an
# interior vertex and the metric has off-diagonal entries
CASES = [((3, 2, 4), 1), ((2, 3, 2), 2), ((3, 3, 2), 3), ((4, 3, 3), 4), ((2, 2, 3), 5), ((2, 2, 2), 6),
         ((2, 2, 2), 7), ((2, 2, 2), 8), ((2, 2, 2), 9), ((2, 2, 2), 10)]


@pytest.mark.parametrize("dims,p", CASES)
def test_apply_with_reaction(dims, p):
    prob, mesh, op, beta = setup(dims, p)
    x = np.random.default_rng(p).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x, beta=beta)
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    # switching the term off gives the diffusion operator back
    op.set_reaction(None)
    y0 = op.apply(t(x)).cpu().numpy()
    ref0 = oracle.ho_apply(mesh, p, p + 2, prob.kappa, x)
    assert np.abs(y0 - ref0).max() <= 1e-12 * np.abs(ref0).max()
    assert np.abs(ref - ref0).max() > 1e-6 * np.abs(ref).max()
    op.close()


@pytest.mark.parametrize("dims,p", CASES)
def test_lor_values_with_reaction_fp64(dims, p):
    prob, mesh, op, beta = setup(dims, p)
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True, beta=beta)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12
    op.close()


def test_lor_values_with_reaction_partial_last_cta():
    """p = 2, 27 elements: the last four-element CTA of the FP64 assembly
    holds three empty slots."""
    prob, mesh, op, beta = setup((3, 3, 3), 2)
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    orp, _, ov = oracle.lor_assemble(mesh, 2, 4, prob.kappa, True, beta=beta)
    assert rowwise_rel_err(orp, v, ov) <= 1e-12
    op.close()


@pytest.mark.parametrize("dims,p", [((3, 2, 4), 2), ((4, 3, 3), 4), ((2, 2, 2), 6), ((2, 2, 2), 10)])
def test_lor_values_with_reaction_fp32(dims, p):
    prob, mesh, op, beta = setup(dims, p)
    op.build_pattern_internal()
    v = op.assemble(torch.float32).cpu().numpy().astype(np.float64)
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True, beta=beta)
    assert rowwise_rel_err(orp, v, ov) <= 1e-5
    op.close()


@pytest.mark.parametrize("dims,p", [((3, 2, 4), 1), ((3, 3, 2), 3), ((4, 3, 3), 4), ((2, 2, 2), 6),
                                    ((2, 2, 2), 7)])
def test_backward_with_reaction(dims, p):
    prob, mesh, op, beta = setup(dims, p)
    rng = np.random.default_rng(10 + p)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    gx, gk = op.apply_backward(t(x), t(gy))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, p + 2, prob.kappa, x, gy, beta=beta)
    assert np.abs(gx.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    gk = gk.cpu().numpy().reshape(rgk.shape)
    assert np.abs(gk - rgk).max() <= 1e-12 * np.abs(rgk).max()
    op.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_helmholtz_pcg_matches_oracle(dtype):
    dims, p = (3, 3, 4), 3
    prob, mesh, op, beta = setup(dims, p, beta_scale=30.0)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True, beta=beta)
    lam = oracle.power_lambda_max(*csr, v0, 20)
    lam_gpu = op.precond_setup("cheb", dtype, degree=3, power_iters=20, v0=t(v0))
    assert abs(lam_gpu - lam) <= (1e-10 if dtype == torch.float64 else 1e-5) * lam
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    x, it, rel = op.pcg_solve(t(prob.rhs), 1e-10, 2000)
    xo, ito, relo, _ = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 2000, oracle.PRECOND_CHEB, 3,
                                  lam / 30, 1.1 * lam, beta=beta)
    assert rel <= 1e-10
    if dtype == torch.float64:
        assert abs(it - ito) <= 1
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max()
    r = prob.rhs - oracle.ho_apply(mesh, p, p + 2, prob.kappa, x.cpu().numpy(), beta=beta)
    assert np.linalg.norm(r) <= 1.000001e-10 * np.linalg.norm(prob.rhs)
    op.close()


def test_bad_reaction_coefficient_reported():
    from paper_2210_12253_gb300 import LOR, LORError
    from paper_2210_12253_gb300.lor import LOR_EINVAL
    prob = make_problem("h", 2, 2, 2, 3, seed=1, kappa="lognormal", rhs="normal")
    op = LOR(3, 2, 2, 2, t(prob.vertices))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    beta = np.ones(prob.kappa.size)
    beta[17] = -1.0
    op.set_reaction(t(beta))
    with pytest.raises(LORError) as ei:
        op.check()
    assert ei.value.code == LOR_EINVAL
    beta[17] = np.nan
    op.set_reaction(t(beta))
    with pytest.raises(LORError):
        op.check()
    op.set_reaction(t(np.ones(prob.kappa.size)), check=True)
    op.close()
