"""GPU test of lor_precond_apply_noalloc, the preconditioner entry point for
callers that cannot allocate device memory when they apply it (a solver loop
whose device memory another allocator reserved up front, or host code where
CUDA allocation calls are not allowed).  Through the C ABI it must give the
same z as lor_precond_apply, bit for bit (the same kernels run), on
consecutive calls that share its static scratch array; leave the device's
free memory unchanged; and refuse sizes beyond that array."""
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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kind,degree", [("cheb", 3), ("cheb", 5), ("jacobi", 1)])
def test_matches_precond_apply_on_consecutive_calls(dtype, kind, degree):
    op = make_op((10, 9, 8), 4, dtype, kind, degree)
    rng = np.random.default_rng(3)
    for _ in range(2):  # the second call reuses the scratch left by the first
        r = torch.tensor(rng.standard_normal(op.ndof), device="cuda")
        z_ref = op.precond_apply(r)
        z = op.precond_apply_noalloc(r, torch.full_like(r, float("nan")))
        torch.cuda.synchronize()
        assert torch.equal(z, z_ref)
    op.close()


def test_allocates_no_device_memory():
    op = make_op((10, 9, 8), 4, torch.float64)
    r = torch.tensor(np.random.default_rng(4).standard_normal(op.ndof), device="cuda")
    z = torch.empty_like(r)
    op.precond_apply_noalloc(r, z)  # first call on the device: looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        op.precond_apply_noalloc(r, z)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
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
    assert torch.equal(z, z_ref)
    op.close()
