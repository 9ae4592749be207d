"""GPU parity of the H(curl) topology of the LOR mesh: the discrete gradient
(Algorithm 1) bit-exact against the oracle, including the 32^3 p = 6 mesh
(21.5M edges), and the deduplicated vertex coordinates."""
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


def make_op(dims, p, seed=1):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("g", *dims, p, seed=seed, jitter=0.1, kappa="one", rhs=None)
    return prob, LOR(p, *dims, torch.tensor(prob.vertices, device=DEV))


@pytest.mark.parametrize("dims,p", [((1, 1, 1), 1), ((3, 2, 4), 2), ((2, 3, 1), 5), ((1, 1, 1), 10),
                                    ((32, 32, 32), 6)])
def test_discrete_gradient_bit_exact(dims, p):
    prob, op = make_op(dims, p)
    rp, ci, v = op.discrete_gradient()
    orp, oci, ov = oracle.discrete_gradient(*dims, p)
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), oci)
    np.testing.assert_array_equal(v.cpu().numpy(), ov)
    op.close()


@pytest.mark.parametrize("dims,p", [((2, 3, 2), 1), ((3, 2, 2), 4), ((2, 2, 2), 7)])
def test_vertex_coordinates(dims, p):
    prob, op = make_op(dims, p)
    xyz = op.vertex_coordinates().cpu().numpy()
    ref = oracle.dof_coordinates(oracle.Mesh(*dims, prob.vertices), p)
    np.testing.assert_allclose(xyz, ref, rtol=0, atol=1e-14)
    op.close()


def test_misaligned_output_rejected():
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_EINVAL, _ptr
    prob, op = make_op((2, 2, 2), 2)
    ne = op.edge_count()
    rp = torch.empty(ne + 1, dtype=torch.int64, device=DEV)
    ci = torch.empty(2 * ne, dtype=torch.int32, device=DEV)
    vals = torch.empty(2 * ne + 1, dtype=torch.float64, device=DEV)[1:]  # 8-byte offset
    with pytest.raises(LORError) as ei:
        op._call("lor_discrete_gradient", _ptr(rp), _ptr(ci), _ptr(vals), None)
    assert ei.value.code == LOR_EINVAL
    op.close()
