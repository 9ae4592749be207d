"""GPU parity of the unstructured LOR assembly (the comparator of the
macro-element algorithm, Section 4.2): the LOR mesh E-vectors against an
independent numpy construction and the oracle's kappa_s binning; the
unstructured assembly on that mesh against the oracle's LOR matrix and the
macro-element assembly; on a randomly renumbered mesh (a general conforming
hex mesh) against the renumbered oracle matrix; and a pattern that lacks a
coupling reported as an error."""
import numpy as np
import pytest
import torch

import oracle
from paper_2210_12253_gb300.inputs import boundary_mask, make_problem

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def setup(dims, p, seed=1, with_beta=False):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("u", *dims, p, seed=seed, jitter=0.1, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    op = LOR(p, *dims, t(prob.vertices))
    op.set_coefficient(t(prob.kappa).reshape(-1), check=True)
    beta = None
    if with_beta:
        beta = np.exp(np.random.default_rng(50 + seed).standard_normal(prob.kappa.shape))
        op.set_reaction(t(beta).reshape(-1), check=True)
    return prob, mesh, op, beta


def rowwise_rel_err(rp, v_gpu, v_ref):
    err = 0.0
    for r in range(len(rp) - 1):
        a, b = rp[r], rp[r + 1]
        err = max(err, np.abs(v_gpu[a:b] - v_ref[a:b]).max() / np.abs(v_ref[a:b]).max())
    return err


@pytest.mark.parametrize("dims,p", [((2, 3, 2), 1), ((2, 2, 1), 3), ((1, 2, 1), 5), ((1, 1, 1), 8)])
def test_lor_mesh_e_vectors(dims, p):
    from meshutil import lor_mesh
    prob, mesh, op, _ = setup(dims, p)
    corners, dofs, ks, _, ess = op.lor_mesh()
    rc, rd = lor_mesh(prob.vertices, *dims, p)
    np.testing.assert_allclose(corners.cpu().numpy(), rc, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(dofs.cpu().numpy(), rd)
    np.testing.assert_allclose(ks.cpu().numpy(), oracle.lor_kappa_sub(p, p + 2, prob.kappa).ravel(), rtol=1e-14)
    np.testing.assert_array_equal(ess.cpu().numpy().astype(bool), boundary_mask(*dims, p))
    op.close()


@pytest.mark.parametrize("with_beta", [False, True])
@pytest.mark.parametrize("dims,p", [((3, 2, 2), 1), ((2, 3, 2), 2), ((2, 2, 3), 4), ((1, 2, 1), 7)])
def test_unstructured_equals_oracle_and_macro(dims, p, with_beta):
    prob, mesh, op, beta = setup(dims, p, with_beta=with_beta)
    rp, ci = op.build_pattern()
    op.build_pattern_internal()
    corners, dofs, ks, bs, ess = op.lor_mesh(with_beta=with_beta)
    orp, _, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True, beta=beta)
    v = op.assemble_unstructured(corners, dofs, ks, rp, ci, op.ndof, beta_sub=bs, ess=ess).cpu().numpy()
    op.check()
    assert rowwise_rel_err(orp, v, ov) <= 1e-12
    vm = op.assemble(torch.float64).cpu().numpy()
    assert rowwise_rel_err(orp, v, vm) <= 1e-12
    v32 = op.assemble_unstructured(corners, dofs, ks, rp, ci, op.ndof, beta_sub=bs, ess=ess,
                                   dtype=torch.float32).cpu().numpy().astype(np.float64)
    assert rowwise_rel_err(orp, v32, ov) <= 1e-5
    op.close()


def test_renumbered_general_mesh():
    """A random permutation of the DOFs and of the sub-hex order turns the
    LOR mesh into a general conforming hex mesh; the unstructured assembly
    must give the permuted oracle matrix."""
    import scipy.sparse as sp
    dims, p = (2, 2, 1), 3
    prob, mesh, op, _ = setup(dims, p)
    corners, dofs, ks, _, ess = op.lor_mesh()
    N = op.ndof
    rng = np.random.default_rng(9)
    perm = rng.permutation(N)          # new id of old DOF i is perm[i]
    order = rng.permutation(ks.numel())
    d_new = perm[dofs.cpu().numpy()][order]
    c_new = corners.cpu().numpy()[order]
    k_new = ks.cpu().numpy()[order]
    e_new = np.zeros(N, np.uint8)
    e_new[perm] = ess.cpu().numpy()
    orp, oci, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    A = sp.csr_matrix((ov, oci, orp), shape=(N, N))
    P = sp.csr_matrix((np.ones(N), (perm, np.arange(N))), shape=(N, N))
    B = (P @ A @ P.T).tocsr()
    B.sort_indices()
    v = op.assemble_unstructured(t(c_new), t(d_new), t(k_new), t(B.indptr.astype(np.int64)),
                                 t(B.indices.astype(np.int32)), N, ess=t(e_new)).cpu().numpy()
    op.check()
    assert rowwise_rel_err(B.indptr, v, B.data) <= 1e-12
    op.close()


def test_missing_coupling_is_reported():
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_EINVAL
    dims, p = (2, 1, 1), 2
    prob, mesh, op, _ = setup(dims, p)
    rp, ci = op.build_pattern()
    corners, dofs, ks, _, _ = op.lor_mesh()
    # drop the last column of row 7 (shift the following rows)
    rp_h, ci_h = rp.cpu().numpy(), ci.cpu().numpy()
    r = 7
    cut = rp_h[r + 1] - 1
    ci2 = np.delete(ci_h, cut)
    rp2 = rp_h.copy()
    rp2[r + 1:] -= 1
    op.assemble_unstructured(corners, dofs, ks, t(rp2), t(ci2), op.ndof)
    with pytest.raises(LORError) as ei:
        op.check()
    assert ei.value.code == LOR_EINVAL and "missing" in str(ei.value)
    op.close()
