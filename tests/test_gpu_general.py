"""GPU parity on general conforming hex meshes (element-restriction form):
a structured problem handed over with its elements and DOFs randomly
renumbered and every element's local frame rotated by a random multiple of
90 degrees about a random axis (a cube rotation maps the reference element,
its GLL nodes and its Gauss points onto themselves, so the operators are
unchanged up to rounding).  The general path must then reproduce the
renumbered oracle results: LOR pattern (bit-exact), LOR values (FP64 1e-12,
FP32 1e-5), apply with and without the reaction term, the kappa gradient,
the load vector and PCG; a tiny mesh is also checked against the oracle's
brute-force dense operator on the general map directly."""
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


# the 24 rotations of the cube as signed axis permutations (det +1):
# new reference coordinate vector xi' maps to old xi = R xi', R[a] = (axis, sign)
def cube_rotations():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            M = np.zeros((3, 3))
            for a in range(3):
                M[a, perm[a]] = signs[a]
            if np.linalg.det(M) > 0:
                out.append(M)
    return out


ROT = cube_rotations()


def index_map(M, n):
    """For a rotation M (old = M new) on the reference cube and n points per
    axis placed symmetrically, the old tensor index of each new index
    (i' + n(j' + n k'))."""
    out = np.empty(n ** 3, np.int64)
    for k in range(n):
        for j in range(n):
            for i in range(n):
                new = np.array([i, j, k])
                c = 2 * new - (n - 1)          # symmetric coordinate
                old = (M @ c + (n - 1)) // 2
                out[i + n * (j + n * k)] = old[0] + n * (old[1] + n * old[2])
    return out


def general_from_structured(prob, rng):
    """(corners, elem_dofs, perm, eperm, rot, kappa_new, beta_rotator) for the
    renumbered and rotated version of a structured problem."""
    p, q = prob.p, prob.q
    n = p + 1
    nex, ney, nez = prob.nex, prob.ney, prob.nez
    nel = nex * ney * nez
    nx, ny = nex * p + 1, ney * p + 1
    N = (nex * p + 1) * (ney * p + 1) * (nez * p + 1)
    V = prob.vertices.reshape(-1, 3)
    perm = rng.permutation(N)
    eperm = rng.permutation(nel)
    rot = rng.integers(0, len(ROT), nel)
    corners = np.empty((nel, 8, 3))
    edofs = np.empty((nel, n ** 3), np.int64)
    kap = np.empty((nel, q ** 3))
    cmaps = [index_map(M, 2) for M in ROT]
    nmaps = [index_map(M, n) for M in ROT]
    qmaps = [index_map(M, q) for M in ROT]
    for new_e in range(nel):
        e = eperm[new_e]
        ex, ey, ez = e % nex, (e // nex) % ney, e // (nex * ney)
        oc = np.array([V[(ex + (c & 1)) + (nex + 1) * ((ey + ((c >> 1) & 1)) + (ney + 1) * (ez + (c >> 2)))]
                       for c in range(8)])
        od = np.array([(ex * p + i) + nx * ((ey * p + j) + ny * (ez * p + k))
                       for k in range(n) for j in range(n) for i in range(n)])
        r = rot[new_e]
        corners[new_e] = oc[cmaps[r]]
        edofs[new_e] = perm[od[nmaps[r]]]
        kap[new_e] = prob.kappa[e][qmaps[r]]
    def to_new_points(a):  # per-point array in the old element order -> new
        return np.stack([a[eperm[k]][qmaps[rot[k]]] for k in range(nel)])
    ess = np.zeros(N, np.uint8)
    ess[perm[boundary_mask(nex, ney, nez, p)]] = 1
    return corners, edofs, perm, eperm, rot, kap, to_new_points, ess, qmaps


def make(dims, p, seed=1, rng_seed=2):
    from paper_2210_12253_gb300 import LOR
    prob = make_problem("gen", *dims, p, seed=seed, jitter=0.12, kappa="lognormal", rhs="normal")
    rng = np.random.default_rng(rng_seed)
    corners, edofs, perm, eperm, rot, kap, to_new, ess, qmaps = general_from_structured(prob, rng)
    N = perm.size
    op = LOR.general(p, t(corners), t(edofs), N, t(ess))
    op.set_coefficient(t(kap).reshape(-1), check=True)
    mesh = oracle.Mesh(*dims, prob.vertices)
    return prob, mesh, op, perm, eperm, rot, to_new, qmaps, corners, edofs, ess, kap


def permuted_csr(rp, ci, v, perm):
    """The CSR matrix renumbered by perm (new id of old DOF i is perm[i]),
    explicit zeros kept (the eliminated rows and columns stay in the
    pattern), columns ascending."""
    from types import SimpleNamespace
    N = rp.size - 1
    inv = np.empty_like(perm)
    inv[perm] = np.arange(N)
    counts = np.diff(rp)[inv]
    indptr = np.zeros(N + 1, np.int64)
    indptr[1:] = np.cumsum(counts)
    indices = np.empty(indptr[-1], np.int64)
    data = np.empty(indptr[-1])
    for r in range(N):
        o = inv[r]
        cols = perm[ci[rp[o]:rp[o + 1]]]
        order = np.argsort(cols)
        indices[indptr[r]:indptr[r + 1]] = cols[order]
        data[indptr[r]:indptr[r + 1]] = v[rp[o]:rp[o + 1]][order]
    return SimpleNamespace(indptr=indptr, indices=indices, data=data, nnz=int(indptr[-1]))


# (3, 3, 3) at p = 2: 27 elements, the FP64 assembly's last four-element CTA three slots short
@pytest.mark.parametrize("dims,p", [((2, 2, 2), 1), ((2, 3, 2), 2), ((3, 3, 3), 2), ((2, 2, 2), 4), ((2, 2, 2), 6)])
def test_general_pattern_and_values(dims, p):
    prob, mesh, op, perm, *_ = make(dims, p)
    rp, ci = op.build_pattern()
    orp, oci, ov = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    B = permuted_csr(orp, oci, ov, perm)
    assert op.nnz == B.nnz
    np.testing.assert_array_equal(rp.cpu().numpy(), B.indptr)
    np.testing.assert_array_equal(ci.cpu().numpy().astype(np.int64), B.indices)
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = op.assemble(dtype).cpu().numpy().astype(np.float64)
        err = max(np.abs(v[a:b] - B.data[a:b]).max() / np.abs(B.data[a:b]).max()
                  for a, b in zip(B.indptr[:-1], B.indptr[1:]))
        assert err <= tol, dtype
    op.close()


@pytest.mark.parametrize("dims,p", [((2, 2, 2), 1), ((3, 2, 2), 3), ((2, 2, 2), 5), ((2, 2, 2), 8)])
def test_general_apply_backward_load(dims, p):
    prob, mesh, op, perm, eperm, rot, to_new, qmaps, *_ = make(dims, p)
    q = p + 2
    rng = np.random.default_rng(7)
    x, gy = rng.standard_normal(op.ndof), rng.standard_normal(op.ndof)
    xn, gyn = np.empty_like(x), np.empty_like(gy)
    xn[perm], gyn[perm] = x, gy
    y = op.apply(t(xn)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, q, prob.kappa, x)
    assert np.abs(y[perm] - ref).max() <= 1e-12 * np.abs(ref).max()
    gx, gk = op.apply_backward(t(xn), t(gyn))
    rgx, rgk = oracle.ho_apply_backward(mesh, p, q, prob.kappa, x, gy)
    assert np.abs(gx.cpu().numpy()[perm] - rgx).max() <= 1e-12 * np.abs(rgx).max()
    gk_ref = to_new(rgk)
    assert np.abs(gk.cpu().numpy().reshape(gk_ref.shape) - gk_ref).max() <= 1e-12 * np.abs(gk_ref).max()
    b = op.load_vector().cpu().numpy()
    bref = oracle.load_vector(mesh, p, q)
    assert np.abs(b[perm] - bref).max() <= 1e-13 * np.abs(bref).max()
    # reaction term
    beta = np.exp(rng.standard_normal(prob.kappa.shape))
    op.set_reaction(t(to_new(beta)).reshape(-1), check=True)
    y = op.apply(t(xn)).cpu().numpy()
    ref = oracle.ho_apply(mesh, p, q, prob.kappa, x, beta=beta)
    assert np.abs(y[perm] - ref).max() <= 1e-12 * np.abs(ref).max()
    op.build_pattern_internal()
    v = op.assemble(torch.float64).cpu().numpy()
    B = permuted_csr(*oracle.lor_assemble(mesh, p, q, prob.kappa, True, beta=beta), perm)
    err = max(np.abs(v[a:b] - B.data[a:b]).max() / np.abs(B.data[a:b]).max() for a, b in zip(B.indptr[:-1], B.indptr[1:]))
    assert err <= 1e-12
    op.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_general_pcg(dtype):
    dims, p = (3, 2, 3), 3
    prob, mesh, op, perm, *_ = make(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    v0 = np.random.default_rng(7).standard_normal(op.ndof)
    lam = oracle.power_lambda_max(*csr, v0, 20)
    v0n = np.empty_like(v0)
    v0n[perm] = v0
    lam_gpu = op.precond_setup("cheb", dtype, degree=3, power_iters=20, v0=t(v0n))
    assert abs(lam_gpu - lam) <= (1e-10 if dtype == torch.float64 else 1e-5) * lam
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    bn = np.empty_like(prob.rhs)
    bn[perm] = prob.rhs
    x, it, rel = op.pcg_solve(t(bn), 1e-10, 2000)
    xo, ito, _, _ = oracle.pcg(mesh, p, p + 2, prob.kappa, csr, prob.rhs, 1e-10, 2000, oracle.PRECOND_CHEB, 3,
                               lam / 30, 1.1 * lam)
    assert rel <= 1e-10
    if dtype == torch.float64:
        assert abs(it - ito) <= 1
    assert np.abs(x.cpu().numpy()[perm] - xo).max() <= 1e-8 * np.abs(xo).max()
    op.close()


def test_general_tiny_mesh_against_dense_brute_force():
    """Directly on the general map: the oracle's dense operator built from
    the same corners, element-to-DOF map and kappa."""
    from meshutil import eliminate
    dims, p = (2, 2, 2), 2
    prob, mesh, op, perm, eperm, rot, to_new, qmaps, corners, edofs, ess, kap = make(dims, p, rng_seed=5)
    A = oracle.dense_general(corners, edofs, kap, p, p + 2, op.ndof)
    Ae = eliminate(A, ess.astype(bool))
    x = np.random.default_rng(3).standard_normal(op.ndof)
    y = op.apply(t(x)).cpu().numpy()
    assert np.abs(y - Ae @ x).max() <= 1e-12 * np.abs(Ae).sum(1).max() * np.abs(x).max()
    op.close()


def test_general_mesh_errors():
    from paper_2210_12253_gb300 import LOR, LORError
    from paper_2210_12253_gb300.lor import LOR_EGEOM, LOR_EINVAL, LOR_ESTATE
    prob = make_problem("gen", 2, 2, 1, 2, seed=1, jitter=0.1, kappa="lognormal", rhs=None)
    corners, edofs, perm, *_ , ess, qmaps = general_from_structured(prob, np.random.default_rng(1))
    N = perm.size
    bad = edofs.copy()
    bad[1, 3] = N  # out of range
    with pytest.raises(LORError) as ei:
        LOR.general(2, t(corners), t(bad), N)
    assert ei.value.code == LOR_EINVAL
    refl = corners.copy()
    refl[0] = refl[0][[1, 0, 3, 2, 5, 4, 7, 6]]  # mirrored element: detJ < 0
    with pytest.raises(LORError) as ei:
        LOR.general(2, t(refl), t(edofs), N)
    assert ei.value.code == LOR_EGEOM
    op = LOR.general(2, t(corners), t(edofs), N, t(ess))
    with pytest.raises(LORError) as ei:
        op.lor_mesh()
    assert ei.value.code == LOR_ESTATE
    op.close()


@pytest.mark.parametrize("dims,p", [((2, 2, 2), 1), ((2, 3, 1), 3), ((2, 2, 2), 6)])
def test_general_discrete_gradient_and_vertices(dims, p):
    """The LOR edges of the renumbered, rotated mesh are the renumbered edges
    of the structured one (each from its lower to its higher DOF, ordered by
    (tail, head)); the vertex coordinates are the renumbered oracle ones."""
    prob, mesh, op, perm, *_ = make(dims, p)
    rp, ci, v = op.discrete_gradient()
    orp, oci, ov = oracle.discrete_gradient(*dims, p)
    a, b = perm[oci[0::2]], perm[oci[1::2]]
    ref = np.stack([np.minimum(a, b), np.maximum(a, b)], 1)
    ref = ref[np.lexsort((ref[:, 1], ref[:, 0]))]
    ne = ref.shape[0]
    assert op.edge_count() == ne
    np.testing.assert_array_equal(rp.cpu().numpy(), 2 * np.arange(ne + 1))
    np.testing.assert_array_equal(ci.cpu().numpy().reshape(-1, 2).astype(np.int64), ref)
    np.testing.assert_array_equal(v.cpu().numpy().reshape(-1, 2), np.tile([-1.0, 1.0], (ne, 1)))
    xyz = op.vertex_coordinates().cpu().numpy()
    oxyz = oracle.dof_coordinates(mesh, p)
    np.testing.assert_allclose(xyz[perm], oxyz, rtol=0, atol=1e-14)
    op.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
def test_general_smoother_and_spmv_staged_and_unstaged(dtype, tol):
    """The explicit-CSR SpMV and Chebyshev-Jacobi smoother (each tile's values
    and columns staged by bulk copies) against the oracle on the renumbered
    matrix; the same kernels reading every tile from global memory (test
    hook) give identical results; the bounded-wait expiry is reported here
    too."""
    from paper_2210_12253_gb300 import LORError
    from paper_2210_12253_gb300.lor import LOR_ETIMEOUT, LOR_TEST_EXPIRE_WAITS, LOR_TEST_UNSTAGED_CSR
    dims, p = (4, 3, 3), 3
    prob, mesh, op, perm, *_ = make(dims, p)
    op.build_pattern_internal()
    op.assemble_internal(dtype)
    csr = oracle.lor_assemble(mesh, p, p + 2, prob.kappa, True)
    N = mesh.ndof(p)
    lam = oracle.power_lambda_max(*csr, np.random.default_rng(7).standard_normal(N), 20)
    op.precond_setup("cheb", dtype, degree=3, lambda_max=lam)
    rng = np.random.default_rng(9)
    r, x = rng.standard_normal(N), rng.standard_normal(N)
    rn, xn = np.empty(N), np.empty(N)
    rn[perm], xn[perm] = r, x
    z = op.precond_apply(t(rn))
    y = op.spmv(t(xn), dtype)
    zref = oracle.chebyshev(*csr, r, 3, lam / 30, 1.1 * lam)
    yref = oracle.csr_spmv(*csr, x)
    assert np.abs(z.cpu().numpy()[perm] - zref).max() <= tol * np.abs(zref).max()
    assert np.abs(y.cpu().numpy()[perm] - yref).max() <= tol * np.abs(yref).max()
    op.set_test_hooks(LOR_TEST_UNSTAGED_CSR)
    assert torch.equal(op.precond_apply(t(rn)), z) and torch.equal(op.spmv(t(xn), dtype), y)
    op.set_test_hooks(LOR_TEST_EXPIRE_WAITS)
    op.precond_apply(t(rn))
    with pytest.raises(LORError) as ei:
        op.check()
    assert ei.value.code == LOR_ETIMEOUT
    op.set_test_hooks(0)
    op.check()
    assert torch.equal(op.precond_apply(t(rn)), z)
    op.close()
