"""Parity at the measured sizes, in the launch configuration bench.py times.

* 16^3 elements, p = 4 (274,625 DOFs; the benchmark step): the whole LOR
  CSR (pattern bit-exact, all 7,189,057 values in FP64 and FP32) against the
  oracle's assembled CSR, sampled rows against the oracle's rows computed
  alone, the full high-order apply and backward, SpMV and the
  Chebyshev-Jacobi smoother.
* 32^3 elements, p = 6 (7,189,057 DOFs; the PCG workload): sampled LOR rows,
  the full apply (FP64 and FP32 arithmetic), and PCG to 1e-8 in FP64, mixed
  precision and the mixed-precision refinement (both schemes), whose true
  residual is re-checked with the oracle's operator.
* the step workload with the reaction term (whole CSR, apply, backward), and
  handed over as a renumbered, rotated general mesh (whole CSR, apply,
  smoother).
* 24^3 elements, p = 5 (1,771,561 DOFs; the gradient workload): dJ/dtheta by
  the adjoint against fourth-order central differences on 16 random
  directions, and the
  gradient kernel against the oracle's on the same fields.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import power_start_vector, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def setup(name):
    from paper_2210_12253_gb300 import LOR
    prob = workload(name)
    mesh = oracle.Mesh(prob.nex, prob.ney, prob.nez, prob.vertices)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, t(prob.vertices))
    op.set_coefficient(t(prob.kappa.reshape(-1)), check=True)
    return prob, mesh, op


def sample_rows(prob, n, seed):
    """Random rows plus every corner/edge/face class of row."""
    nx, ny, nz = (prob.nex * prob.p + 1, prob.ney * prob.p + 1, prob.nez * prob.p + 1)
    rng = np.random.default_rng(seed)
    rows = set(rng.integers(0, nx * ny * nz, n).tolist())
    for I in (0, 1, prob.p, nx // 2, nx - 2, nx - 1):
        for J in (0, 1, prob.p, ny - 1):
            for K in (0, prob.p + 1, nz - 2, nz - 1):
                rows.add(I + nx * (J + ny * K))
    return np.array(sorted(rows), dtype=np.int64)


def check_rows(prob, mesh, op, rows, tol, dtype):
    rp, ci = op.build_pattern()
    rp, ci = rp.cpu().numpy(), ci.cpu().numpy()
    v = op.assemble(dtype).cpu().numpy().astype(np.float64)
    cnt, cols, vals = oracle.lor_rows(mesh, prob.p, prob.q, prob.kappa, rows, True)
    for k, r in enumerate(rows):
        a, b = rp[r], rp[r + 1]
        assert b - a == cnt[k]
        np.testing.assert_array_equal(ci[a:b].astype(np.int64), cols[k, :cnt[k]])
        ref = vals[k, :cnt[k]]
        assert np.abs(v[a:b] - ref).max() <= tol * np.abs(ref).max()


def rowwise_max_rel_err(rp, v, ref):
    """max over rows of max|v - ref| / max|ref| on the row (every row non-empty)."""
    err = np.maximum.reduceat(np.abs(v - ref), rp[:-1])
    scale = np.maximum.reduceat(np.abs(ref), rp[:-1])
    return (err / scale).max()


def test_step_workload_16x16x16_p4():
    prob, mesh, op = setup("c2_16x16x16_p4")
    p, q = prob.p, prob.q
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True)
    rp, ci = op.build_pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), csr[0])
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), csr[1])
    assert csr[2].size == 7189057
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = op.assemble(dtype).cpu().numpy().astype(np.float64)
        assert rowwise_max_rel_err(csr[0], v, csr[2]) <= tol, dtype
    rows = sample_rows(prob, 300, 1)
    check_rows(prob, mesh, op, rows, 1e-12, torch.float64)
    rng = np.random.default_rng(2)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ry = oracle.ho_apply(mesh, p, q, prob.kappa, x)
    assert np.abs(y - ry).max() <= 1e-12 * np.abs(ry).max()
    gx, gk = op.apply_backward(t(x), t(gy))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, q, prob.kappa, x, gy)
    assert np.abs(gx.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    assert np.abs(gk.cpu().numpy() - rgk.ravel()).max() <= 1e-12 * np.abs(rgk).max()
    # smoother and SpMV against the oracle's own CSR
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    v0 = power_start_vector(op.ndof)
    lam_ref = oracle.power_lambda_max(*csr, v0, 20)
    lam = op.precond_setup("cheb", torch.float64, degree=3, power_iters=20, v0=t(v0))
    assert abs(lam - lam_ref) <= 1e-10 * lam_ref
    op.precond_setup("cheb", torch.float64, degree=3, lambda_max=lam_ref)
    z = op.precond_apply(t(prob.rhs)).cpu().numpy()
    zr = oracle.chebyshev(*csr, prob.rhs, 3, lam_ref / 30, 1.1 * lam_ref)
    assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max()
    s = op.spmv(t(x), torch.float64).cpu().numpy()
    sr = oracle.csr_spmv(*csr, x)
    assert np.abs(s - sr).max() <= 1e-13 * np.abs(sr).max()
    op.close()


def test_pcg_workload_32x32x32_p6():
    prob, mesh, op = setup("c3_32x32x32_p6")
    p, q = prob.p, prob.q
    rows = sample_rows(prob, 2000, 3)
    check_rows(prob, mesh, op, rows, 1e-12, torch.float64)
    check_rows(prob, mesh, op, rows, 1e-5, torch.float32)
    x = np.random.default_rng(4).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ry = oracle.ho_apply(mesh, p, q, prob.kappa, x)
    assert np.abs(y - ry).max() <= 1e-12 * np.abs(ry).max()
    y32 = op.apply_f32(t(x)).cpu().numpy()
    assert np.abs(y32 - ry).max() <= 2e-5 * np.abs(ry).max()
    b = t(prob.rhs)
    v0 = t(power_start_vector(op.ndof))
    op.build_pattern_internal()
    its = {}
    for dt in (torch.float64, torch.float32):
        op.assemble_internal(dt)
        op.precond_setup("cheb", dt, degree=3, power_iters=20, v0=v0)
        u, it, rel = op.pcg_solve(b, 1e-8, 20000)
        its[dt] = it
        r = prob.rhs - oracle.ho_apply(mesh, p, q, prob.kappa, u.cpu().numpy())
        assert np.linalg.norm(r) <= 1.000001e-8 * np.linalg.norm(prob.rhs), dt
    # mixed precision reaches the same tolerance with a similar iteration count
    assert its[torch.float32] <= 1.25 * its[torch.float64]
    # the refinement (FP32 operator in the iterations), FP32 smoother as above
    for scheme in ("replace", "restart"):
        u, outer, inner, rel = op.pcg_solve_ir(b, 1e-8, 1e-4, 20000, scheme=scheme)
        r = prob.rhs - oracle.ho_apply(mesh, p, q, prob.kappa, u.cpu().numpy())
        assert np.linalg.norm(r) <= 1.000001e-8 * np.linalg.norm(prob.rhs), scheme
        assert inner <= 1.5 * its[torch.float32], scheme
    op.close()


def test_gradient_workload_24x24x24_p5():
    from paper_2210_12253_gb300 import LOR, solve, solve_with_adjoint
    prob = workload("c4_24x24x24_p5")
    mesh = oracle.Mesh(prob.nex, prob.ney, prob.nez, prob.vertices)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, t(prob.vertices))
    opts = dict(rtol=1e-12, maxit=50000, precond="cheb", dtype=torch.float64)
    b = t(prob.rhs)
    ustar = solve(op, torch.exp(t(prob.theta_star.ravel())), b, **opts).detach()
    th = t(prob.theta.ravel())
    J, g = solve_with_adjoint(op, th, b, ustar, **opts)
    g = g.cpu().numpy()
    # the gradient kernel against the oracle's on the same u and adjoint
    u = solve(op, torch.exp(th), b, **opts)
    lam, _, _ = op.pcg_solve((u - ustar).contiguous(), 1e-12, 50000)
    _, gk_ref = oracle.ho_apply_backward(mesh, prob.p, prob.q, np.exp(prob.theta), u.detach().cpu().numpy(),
                                         lam.cpu().numpy(), want_gx=False)
    gref = -np.exp(prob.theta).ravel() * gk_ref.ravel()
    assert np.abs(g - gref).max() <= 1e-8 * np.abs(gref).max()
    # fourth-order central differences (steps h and 2h, Richardson-combined)
    # on 16 random directions.  h = 1e-3 |theta| keeps the difference quotient
    # far above the solver's forward error (relative residual 1e-12 times the
    # condition number) while the O(h^4) truncation error stays below 1e-7.
    # The error is measured against |g|, the typical size of g.v for
    # v ~ N(0, I): a direction whose g.v happens to be near 0 makes a
    # relative-to-fd test ill-conditioned.
    rng = np.random.default_rng(6)
    gnorm = np.linalg.norm(g)

    def J_at(d):
        return 0.5 * float(((solve(op, torch.exp(th + t(d)), b, **opts) - ustar) ** 2).sum())

    for _ in range(16):
        v = rng.standard_normal(th.numel())
        h = 1e-3 * np.linalg.norm(prob.theta) / np.linalg.norm(v)
        d1 = J_at(h * v) - J_at(-h * v)
        d2 = J_at(2 * h * v) - J_at(-2 * h * v)
        fd = (8 * d1 - d2) / (12 * h)
        assert abs(fd - float(g @ v)) <= 1e-6 * gnorm
    op.close()


def test_step_workload_with_reaction_16x16x16_p4():
    """The definite Helmholtz variant of the step workload (beta = exp(N(0,1))
    per Gauss point, seed 777): the whole LOR CSR (pattern bit-exact, values
    FP64 1e-12 and FP32 1e-5 of the row maximum), the apply and the backward
    in full against the oracle with the reaction term."""
    prob, mesh, op = setup("c2_16x16x16_p4")
    p, q = prob.p, prob.q
    beta = np.exp(np.random.default_rng(777).standard_normal(prob.kappa.shape))
    op.set_reaction(t(beta.reshape(-1)), check=True)
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True, beta=beta)
    rp, ci = op.build_pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), csr[0])
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), csr[1])
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = op.assemble(dtype).cpu().numpy().astype(np.float64)
        assert rowwise_max_rel_err(csr[0], v, csr[2]) <= tol, dtype
    rng = np.random.default_rng(5)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    ry = oracle.ho_apply(mesh, p, q, prob.kappa, x, beta=beta)
    assert np.abs(y - ry).max() <= 1e-12 * np.abs(ry).max()
    gx, gk = op.apply_backward(t(x), t(gy))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, q, prob.kappa, x, gy, beta=beta)
    assert np.abs(gx.cpu().numpy() - rgx).max() <= 1e-12 * np.abs(rgx).max()
    assert np.abs(gk.cpu().numpy() - rgk.ravel()).max() <= 1e-12 * np.abs(rgk).max()
    op.close()


def test_step_workload_as_a_general_mesh_16x16x16_p4():
    """The step workload handed over in element-restriction form with its
    DOFs and elements randomly renumbered and every element's frame rotated:
    the whole LOR CSR (renumbered) against the oracle's (pattern bit-exact,
    FP64 1e-12, FP32 1e-5), the apply in full, and the Chebyshev-Jacobi
    smoother (staged explicit-CSR kernel) against the oracle's."""
    from paper_2210_12253_gb300 import LOR
    from test_gpu_general import general_from_structured, permuted_csr
    prob = workload("c2_16x16x16_p4")
    p, q = prob.p, prob.q
    mesh = oracle.Mesh(prob.nex, prob.ney, prob.nez, prob.vertices)
    corners, edofs, perm, eperm, rot, kap, to_new, ess, qmaps = general_from_structured(prob, np.random.default_rng(3))
    N = perm.size
    op = LOR.general(p, t(corners), t(edofs), N, t(ess))
    op.set_coefficient(t(kap).reshape(-1), check=True)
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True)
    ref = permuted_csr(*csr, perm)
    rp, ci = op.build_pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref.indptr)
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), ref.indices)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = op.assemble(dtype).cpu().numpy().astype(np.float64)
        assert rowwise_max_rel_err(ref.indptr, v, ref.data) <= tol, dtype
    x = np.random.default_rng(6).standard_normal(N)
    xn = np.empty(N)
    xn[perm] = x
    y = op.apply(t(xn)).cpu().numpy()[perm]
    ry = oracle.ho_apply(mesh, p, q, prob.kappa, x)
    assert np.abs(y - ry).max() <= 1e-12 * np.abs(ry).max()
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    lam = oracle.power_lambda_max(*csr, power_start_vector(N), 20)
    op.precond_setup("cheb", torch.float64, degree=3, lambda_max=lam)
    z = op.precond_apply(t(xn)).cpu().numpy()[perm]
    zr = oracle.chebyshev(*csr, x, 3, lam / 30, 1.1 * lam)
    assert np.abs(z - zr).max() <= 1e-12 * np.abs(zr).max()
    op.close()
