"""GPU test of lor_precond_apply_noalloc, the preconditioner entry point for
callers that cannot allocate device memory when they apply it.  It must give
the same z as lor_precond_apply (through the C ABI), on consecutive calls that
share its static scratch array, and refuse sizes beyond that array."""
import numpy as np
import pytest
import torch

from paper_2210_12253_gb300.inputs import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def make_op(dims, p, dtype, kind="cheb", degree=3):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("noalloc", *dims, p, seed=11, kappa="lognormal", rhs="normal")
    op = LOR(p, *dims, torch.tensor(prob.vertices, device="cuda"))
    op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device="cuda"), check=True)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    op.precond_setup(kind, dtype, degree=degree, power_iters=20)
    return op


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("kind,degree", [("cheb", 3), ("cheb", 5), ("jacobi", 1)])
def test_matches_precond_apply_on_consecutive_calls(dtype, tol, kind, degree):
    op = make_op((10, 9, 8), 4, dtype, kind, degree)
    rng = np.random.default_rng(3)
    for _ in range(2):  # the second call reuses the scratch left by the first
        r = torch.tensor(rng.standard_normal(op.ndof), device="cuda")
        z_ref = op.precond_apply(r)
        z = op.precond_apply_noalloc(r, torch.full_like(r, float("nan")))
        torch.cuda.synchronize()
        err = (z - z_ref).abs().max().item()
        assert err <= tol * z_ref.abs().max().item()
    op.close()


def test_rejects_sizes_beyond_the_static_array():
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_EINVAL
    op = make_op((23, 23, 23), 4, torch.float64)  # 804,357 DOFs > 699,050
    r = torch.ones(op.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(LORError) as ei:
        op.precond_apply_noalloc(r, torch.empty_like(r))
    assert ei.value.code == LOR_EINVAL and "static array" in str(ei.value)
    op.assemble_internal(torch.float32)  # FP32 smoother of the same size fits
    op.precond_setup("cheb", torch.float32, degree=3, power_iters=20)
    z = op.precond_apply_noalloc(r, torch.empty_like(r))
    z_ref = op.precond_apply(r)
    assert (z - z_ref).abs().max().item() <= 1e-5 * z_ref.abs().max().item()
    op.close()
