"""The error path of the bounded device-side waits, on the GPU without a
fault: the test hook LOR_TEST_EXPIRE_WAITS makes every CTA of the TMA-staged
SpMV/smoother kernels treat its wait for a bulk copy of matrix values as
expired.  The copy itself still lands and the CTA waits for it before it
exits, so nothing faults or hangs; the CTA records LOR_FLAG_TIMEOUT and skips
its rows, as after a real expiry.  Every call that reads the status word must
then return LOR_ETIMEOUT, and once the hook is cleared (and the status word
read by lor_check) the same context must compute the oracle's results."""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def expect_timeout(fn):
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_ETIMEOUT
    with pytest.raises(LORError) as ei:
        fn()
    assert ei.value.code == LOR_ETIMEOUT, str(ei.value)
    assert "bounded device wait expired" in str(ei.value)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_expired_wait_is_reported_and_the_context_stays_usable(dtype, tol):
    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.lor import LOR_TEST_EXPIRE_WAITS
    dims, p = (3, 3, 4), 3
    prob = make_problem("t", *dims, p, seed=1, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    op = LOR(p, *dims, t(prob.vertices))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    lam = oracle.power_lambda_max(*csr, np.random.default_rng(7).standard_normal(op.ndof), 20)
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    r = np.random.default_rng(8).standard_normal(op.ndof)

    op.set_test_hooks(LOR_TEST_EXPIRE_WAITS)
    op.spmv(t(r), dtype)           # asynchronous: the expiry shows at the next status read
    op.precond_apply(t(r))
    expect_timeout(op.check)       # reports and clears the status word
    expect_timeout(lambda: op.pcg_solve(t(prob.rhs), 1e-10, 2000))
    expect_timeout(op.check)
    expect_timeout(lambda: op.pcg_solve_ir(t(prob.rhs), 1e-10, 1e-4, 2000))
    expect_timeout(op.check)
    expect_timeout(lambda: op.precond_setup("cheb", dtype, degree=3, power_iters=5))
    expect_timeout(op.check)

    op.set_test_hooks(0)
    op.check()
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    z = op.precond_apply(t(r)).cpu().numpy()
    ref = oracle.chebyshev(*csr, r, 3, lam / 30, 1.1 * lam)
    assert np.abs(z - ref).max() <= tol * np.abs(ref).max()
    x, it, rel = op.pcg_solve(t(prob.rhs), 1e-10, 2000)
    xo, ito, relo, _ = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 2000, oracle.PRECOND_CHEB, 3,
                                  lam / 30, 1.1 * lam)
    assert rel <= 1e-10
    if dtype == torch.float64:
        assert abs(it - ito) <= 1
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-8 * np.abs(xo).max()
    op.check()
    op.close()
