"""GPU parity on a general conforming hex mesh that is not a lattice (the
element-restriction path of Step S1.1 / A2 on a mesh whose vertices are not
all shared by 8 hexes): the cube-in-cube mesh of the unit cube (an inner cube
and six hexes joining its faces to the cube's faces, each split into m^3
hexes, interior vertices jittered).  At the inner cube's corners 4 hexes
meet, at the unit cube's corners 3, so the LOR pattern has row lengths that
no lattice produces.  Against the oracle's general-mesh LOR assembly: the
pattern bit-exact, values FP64 1e-12 and FP32 1e-5 of the row maximum;
against the oracle's brute-force dense operator on the same map: the
high-order apply (1e-12) and the PCG solution (FP64 and mixed precision,
1e-8 of the dense solve).  And the pattern builder's device temporaries
count against the context's allocation limit."""
import numpy as np
import pytest
import torch

import oracle
from meshutil import cube_in_cube_corners, eliminate, general_dofs, jitter_interior_vertices

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2210_12253_gb300.build import build
    build()


def t(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def problem(m, p, seed=1):
    rng = np.random.default_rng(seed)
    C = jitter_interior_vertices(cube_in_cube_corners(m), 0.1 * 0.3 / m, rng)
    dofs, N, xyz, ess = general_dofs(C, p)
    q = p + 2
    kap = np.exp(rng.standard_normal((C.shape[0], q ** 3)))
    b = rng.standard_normal(N)
    b[ess.astype(bool)] = 0.0
    return C, dofs, N, ess, kap, b


def make_op(C, dofs, N, ess, kap, p):
    from paper_2210_12253_gb300 import LOR
    op = LOR.general(p, t(C), t(dofs), N, t(ess))
    op.set_coefficient(t(kap).reshape(-1), check=True)
    return op


def rowwise_max_rel_err(rp, v, ref):
    err = np.maximum.reduceat(np.abs(v - ref), rp[:-1])
    scale = np.maximum.reduceat(np.abs(ref), rp[:-1])
    return (err / scale).max()


@pytest.mark.parametrize("m,p", [(1, 1), (1, 2), (1, 4), (1, 7), (2, 3), (2, 5), (3, 2), (3, 4)])
def test_lor_matrix_matches_oracle(m, p):
    C, dofs, N, ess, kap, b = problem(m, p)
    q = p + 2
    op = make_op(C, dofs, N, ess, kap, p)
    rp, ci, ref = oracle.lor_assemble_general(C, dofs, N, p, q, kap, ess, dirichlet=True)
    grp, gci = op.build_pattern()
    grp, gci = grp.cpu().numpy(), gci.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(grp, rp)
    np.testing.assert_array_equal(gci, ci)
    assert set(np.diff(rp).tolist()) - {8, 12, 18, 27}  # row lengths a lattice never has
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = op.assemble(dtype).cpu().numpy().astype(np.float64)
        assert rowwise_max_rel_err(rp, v, ref) <= tol, dtype
    op.close()


@pytest.mark.parametrize("m,p", [(1, 3), (1, 6), (2, 2), (2, 3)])
def test_apply_and_pcg_match_dense_oracle(m, p):
    C, dofs, N, ess, kap, b = problem(m, p)
    q = p + 2
    op = make_op(C, dofs, N, ess, kap, p)
    A = eliminate(oracle.dense_general(C, dofs, kap, p, q, N), ess.astype(bool))
    x = np.random.default_rng(5).standard_normal(N)
    y = op.apply(t(x)).cpu().numpy()
    yref = A @ x
    assert np.abs(y - yref).max() <= 1e-12 * np.abs(yref).max()
    xref = np.linalg.solve(A, b)
    op.build_pattern_internal()
    for dtype in (torch.float64, torch.float32):
        op.assemble_internal(dtype)
        op.precond_setup("cheb", dtype, degree=3, power_iters=20)
        u, it, rel = op.pcg_solve(t(b), 1e-11, 5000)
        assert rel <= 1e-11
        assert np.abs(u.cpu().numpy() - xref).max() <= 1e-8 * np.abs(xref).max(), dtype
    op.close()


def test_pattern_temporaries_count_against_the_allocation_limit(monkeypatch):
    """With LOR_DEVICE_ALLOC_LIMIT just above the context's own buffers, the
    pattern builder's largest temporary (the incidence lists) does not fit:
    lor_create_general reports LOR_ENOMEM; without the limit it succeeds."""
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_ENOMEM
    m, p = 1, 3
    C, dofs, N, ess, kap, b = problem(m, p)
    nel, n3 = C.shape[0], (p + 1) ** 3
    own = 192 * nel + 8 * n3 * nel + N + 16 + 8 * (608 + 16 + 2 * 2048) + 32 + 32 * N
    incidence_lists = 4 * nel * p ** 3 * 64
    limit = own + 24 * (N + 1) + 4096
    assert limit < own + incidence_lists
    monkeypatch.setenv("LOR_DEVICE_ALLOC_LIMIT", str(limit))
    with pytest.raises(LORError) as ei:
        make_op(C, dofs, N, ess, kap, p)
    assert ei.value.code == LOR_ENOMEM and "LOR pattern" in str(ei.value)
    monkeypatch.delenv("LOR_DEVICE_ALLOC_LIMIT")
    op = make_op(C, dofs, N, ess, kap, p)
    assert op.nnz > 0
    op.close()
