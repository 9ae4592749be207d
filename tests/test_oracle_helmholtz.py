"""Pins of the oracle's reaction (mass) term: the definite Helmholtz
(diffusion-reaction) operator of Section 4.1, -div(kappa grad u) + beta u,
whose mass part uses the basis operator B (x) B (x) B (Section 3, Step S2.1),
and its LOR counterpart (trilinear mass blocks on the sub-hexes, beta_s binned
like kappa_s: reading R16).  Checked against exact polynomial integration,
the brute-force dense operator, the independent p = 1 matrix of the LOR mesh,
volume integrals, and dense solves."""
import numpy as np
import pytest
import scipy.linalg
from numpy.polynomial import polynomial as P

import oracle
from meshutil import (csr_to_dense, element_corners, element_dofs, eliminate, essential_mask, gll_nodes, lor_mesh)
from paper_2210_12253_gb300.inputs import unit_cube_vertices


def jittered(nex, ney, nez, seed=7, jitter=0.2):
    return oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez, jitter, np.random.default_rng(seed)))


def lognormal(rng, shape):
    return np.exp(rng.standard_normal(shape))


def dense(mesh, p, q, kappa, beta):
    C = element_corners(mesh.V, mesh.nex, mesh.ney, mesh.nez)
    Dm = element_dofs(mesh.nex, mesh.ney, mesh.nez, p)
    return oracle.dense_general(C, Dm, kappa, p, q, mesh.ndof(p), beta=beta)


def exact_1d_mass(p):
    """Exact GLL mass matrix on [-1,1] by polynomial algebra."""
    g = gll_nodes(p)
    L = []
    for i in range(p + 1):
        c = P.polyfromroots(np.delete(g, i))
        L.append(c / P.polyval(g[i], c))
    M = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            mij = P.polyint(P.polymul(L[i], L[j]))
            M[i, j] = P.polyval(1, mij) - P.polyval(-1, mij)
    return M


def apply_matrix(mesh, p, q, kappa, beta):
    """The full (no Dirichlet) operator, column by column through ho_apply."""
    N = mesh.ndof(p)
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = oracle.ho_apply(mesh, p, q, kappa, e, dirichlet=False, beta=beta)
    return A


# ------------------------------------------------------------------ HO mass
@pytest.mark.parametrize("p", [1, 2, 3])
def test_undistorted_element_mass_is_kronecker(p):
    """One box element [0,hx]x[0,hy]x[0,hz], beta = 1: the reaction part of
    the operator is Mz (x) My (x) Mx with exact 1D mass matrices (q = p+2
    Gauss points integrate them exactly)."""
    hx, hy, hz = 0.7, 1.3, 0.9
    mesh = oracle.Mesh(1, 1, 1, unit_cube_vertices(1, 1, 1) * np.array([hx, hy, hz]))
    q = p + 2
    kap = lognormal(np.random.default_rng(p), (1, q ** 3))
    M = exact_1d_mass(p)
    ref = np.kron((hz / 2) * M, np.kron((hy / 2) * M, (hx / 2) * M))
    mass = apply_matrix(mesh, p, q, kap, np.ones((1, q ** 3))) - apply_matrix(mesh, p, q, kap, None)
    np.testing.assert_allclose(mass, ref, atol=1e-13 * np.abs(ref).max())
    # a constant beta scales it
    mass3 = apply_matrix(mesh, p, q, kap, 3.0 * np.ones((1, q ** 3))) - apply_matrix(mesh, p, q, kap, None)
    np.testing.assert_allclose(mass3, 3.0 * ref, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sum_factorised_mass_equals_brute_force(p):
    mesh = jittered(2, 2, 2, seed=30 + p)
    q = p + 2
    rng = np.random.default_rng(40 + p)
    kap, bet = lognormal(rng, (mesh.nel, q ** 3)), lognormal(rng, (mesh.nel, q ** 3))
    A = dense(mesh, p, q, kap, bet)
    x = rng.standard_normal(mesh.ndof(p))
    tol = 1e-12 * np.abs(A).sum(1).max() * np.abs(x).max()
    np.testing.assert_allclose(oracle.ho_apply(mesh, p, q, kap, x, dirichlet=False, beta=bet), A @ x, rtol=0, atol=tol)
    ess = essential_mask(mesh.nex, mesh.ney, mesh.nez, p)
    yd = oracle.ho_apply(mesh, p, q, kap, x, dirichlet=True, beta=bet)
    np.testing.assert_allclose(yd, eliminate(A, ess) @ x, rtol=0, atol=tol)
    np.testing.assert_array_equal(yd[ess], x[ess])
    # the mass term really is there: it differs from the diffusion operator
    assert np.abs(A - dense(mesh, p, q, kap, None)).max() > 1e-3 * np.abs(A).max()


@pytest.mark.parametrize("p", [2, 3])
def test_mass_of_constants_is_the_volume(p):
    """Stiffness annihilates constants, so 1^T A 1 = int beta = beta * volume
    (the jittered mesh still fills the unit cube)."""
    mesh = jittered(2, 2, 3, seed=p)
    q = p + 2
    kap = lognormal(np.random.default_rng(p), (mesh.nel, q ** 3))
    one = np.ones(mesh.ndof(p))
    for c in (1.0, 2.5):
        y = oracle.ho_apply(mesh, p, q, kap, one, dirichlet=False, beta=c * np.ones((mesh.nel, q ** 3)))
        assert abs(one @ y - c) <= 1e-13
        rp, ci, v = oracle.lor_assemble(mesh, p, q, kap, dirichlet=False, beta=c * np.ones((mesh.nel, q ** 3)))
        Ah = csr_to_dense(rp, ci, v, mesh.ndof(p))
        assert abs(one @ Ah @ one - c) <= 1e-13


def test_backward_gx_includes_the_mass_term():
    mesh = jittered(2, 2, 2, seed=5)
    p, q = 3, 5
    rng = np.random.default_rng(6)
    kap, bet = lognormal(rng, (mesh.nel, q ** 3)), lognormal(rng, (mesh.nel, q ** 3))
    x, gy = rng.standard_normal(mesh.ndof(p)), rng.standard_normal(mesh.ndof(p))
    gx, gk = oracle.ho_apply_backward(mesh, p, q, kap, x, gy, beta=bet)
    np.testing.assert_allclose(gx, oracle.ho_apply(mesh, p, q, kap, gy, beta=bet), rtol=0, atol=1e-14 * np.abs(gx).max())
    _, gk0 = oracle.ho_apply_backward(mesh, p, q, kap, x, gy)
    np.testing.assert_array_equal(gk, gk0)  # the kappa gradient does not see beta


# ------------------------------------------------------------------ LOR mass
@pytest.mark.parametrize("p,dims", [(1, (2, 2, 2)), (2, (2, 2, 2)), (3, (2, 2, 3)), (4, (2, 2, 2))])
def test_lor_mass_is_q1_mass_of_the_lor_mesh(p, dims):
    """A_h with a reaction term equals the p = 1 stiffness + beta_s mass matrix
    of the LOR mesh integrated by 2x2x2 Gauss (the brute force on the
    sub-hexes with q = 2)."""
    mesh = jittered(*dims, seed=11 + p)
    q = p + 2
    rng = np.random.default_rng(12 + p)
    kap, bet = lognormal(rng, (mesh.nel, q ** 3)), lognormal(rng, (mesh.nel, q ** 3))
    ks = oracle.lor_kappa_sub(p, q, kap).ravel()
    bs = oracle.lor_kappa_sub(p, q, bet).ravel()
    corners, dofs = lor_mesh(mesh.V, mesh.nex, mesh.ney, mesh.nez, p)
    N = mesh.ndof(p)
    ref = oracle.dense_general(corners, dofs, np.repeat(ks[:, None], 8, axis=1), 1, 2, N,
                               beta=np.repeat(bs[:, None], 8, axis=1))
    for dirichlet in (False, True):
        rp, ci, v = oracle.lor_assemble(mesh, p, q, kap, dirichlet, beta=bet)
        A = csr_to_dense(rp, ci, v, N)
        R = eliminate(ref, essential_mask(*dims, p)) if dirichlet else ref
        np.testing.assert_allclose(A, R, atol=1e-13 * np.abs(R).max())
        # rows computed alone agree with the assembly
        rows = np.arange(0, N, max(1, N // 37))
        cnt, cols, vals = oracle.lor_rows(mesh, p, q, kap, rows, dirichlet, beta=bet)
        for k, r in enumerate(rows):
            np.testing.assert_array_equal(cols[k, :cnt[k]], ci[rp[r]:rp[r + 1]])
            np.testing.assert_allclose(vals[k, :cnt[k]], v[rp[r]:rp[r + 1]], atol=1e-14 * np.abs(v).max())


@pytest.mark.parametrize("p", [2, 3, 5])
def test_undistorted_lor_mass_is_kronecker_of_gll_q1_masses(p):
    """Undistorted element, beta = 1: the LOR reaction part is the Kronecker
    product of the 1D Q1 mass matrices on the GLL intervals
    (l/6 [[2, 1], [1, 2]] per interval of length l)."""
    h = np.array([0.6, 1.1, 0.8])
    mesh = oracle.Mesh(1, 1, 1, unit_cube_vertices(1, 1, 1) * h)
    q = p + 2
    kap = lognormal(np.random.default_rng(p), (1, q ** 3))
    g = gll_nodes(p)

    def m1(scale):
        M = np.zeros((p + 1, p + 1))
        for t in range(p):
            l = scale * (g[t + 1] - g[t])
            M[t:t + 2, t:t + 2] += l * np.array([[2.0, 1.0], [1.0, 2.0]]) / 6
        return M

    ref = np.kron(m1(h[2] / 2), np.kron(m1(h[1] / 2), m1(h[0] / 2)))
    N = mesh.ndof(p)
    with_m = csr_to_dense(*oracle.lor_assemble(mesh, p, q, kap, False, beta=np.ones((1, q ** 3))), N)
    without = csr_to_dense(*oracle.lor_assemble(mesh, p, q, kap, False), N)
    np.testing.assert_allclose(with_m - without, ref, atol=1e-14 * np.abs(ref).max())


def test_p1_lor_equals_ho_with_mass_on_affine_mesh():
    """p = 1, affine mesh, element-wise constant kappa and beta: the LOR
    matrix is the high-order Q1 diffusion-reaction matrix."""
    rng = np.random.default_rng(2)
    Am = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
    if np.linalg.det(Am) < 0:
        Am[:, 0] *= -1
    dims = (2, 3, 2)
    mesh = oracle.Mesh(*dims, unit_cube_vertices(*dims) @ Am.T)
    q = 3
    kap = np.repeat(lognormal(rng, (mesh.nel, 1)), q ** 3, axis=1)
    bet = np.repeat(lognormal(rng, (mesh.nel, 1)), q ** 3, axis=1)
    N = mesh.ndof(1)
    A = csr_to_dense(*oracle.lor_assemble(mesh, 1, q, kap, True, beta=bet), N)
    Ah = eliminate(dense(mesh, 1, q, kap, bet), essential_mask(*dims, 1))
    np.testing.assert_allclose(A, Ah, atol=1e-13 * np.abs(Ah).max())


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_helmholtz_spectral_equivalence_within_tensor_bounds(p):
    """(K + M)_p against (K + M)_h on the free DOFs of an undistorted mesh:
    the generalised eigenvalues lie between the smaller of the stiffness and
    mass lower bounds (lk_min lm_min^2, lm_min^3) and the larger of their
    upper bounds, products of the bounded 1D constants."""
    from test_oracle_lor import one_d_pair
    ne = 2 if p <= 4 else 1
    dims = (ne, ne, ne)
    mesh = oracle.Mesh(*dims, unit_cube_vertices(*dims))
    q = p + 2
    one = np.ones((mesh.nel, q ** 3))
    N = mesh.ndof(p)
    Ah = csr_to_dense(*oracle.lor_assemble(mesh, p, q, one, False, beta=one), N)
    Ap = dense(mesh, p, q, one, one)
    free = ~essential_mask(*dims, p)
    lam = scipy.linalg.eigh(Ap[np.ix_(free, free)], Ah[np.ix_(free, free)], eigvals_only=True)
    Kp, Mp, Kh, Mh = one_d_pair(p, ne)
    lk = scipy.linalg.eigh(Kp, Kh, eigvals_only=True)
    lm = scipy.linalg.eigh(Mp, Mh, eigvals_only=True)
    lo = min(lk.min() * lm.min() ** 2, lm.min() ** 3)
    hi = max(lk.max() * lm.max() ** 2, lm.max() ** 3)
    assert lam.min() >= lo * (1 - 1e-10) and lam.max() <= hi * (1 + 1e-10)
    if p == 1:
        np.testing.assert_allclose(lam, 1.0, atol=1e-12)


# ------------------------------------------------------------------ solve
@pytest.mark.parametrize("precond", [oracle.PRECOND_JACOBI, oracle.PRECOND_CHEB])
def test_helmholtz_pcg_matches_dense_solve(precond):
    mesh = jittered(2, 2, 2, seed=8)
    p, q = 3, 5
    rng = np.random.default_rng(9)
    kap, bet = lognormal(rng, (mesh.nel, q ** 3)), 50.0 * lognormal(rng, (mesh.nel, q ** 3))
    N = mesh.ndof(p)
    ess = essential_mask(*(2, 2, 2), p)
    b = rng.standard_normal(N)
    b[ess] = 0.0
    csr = oracle.lor_assemble(mesh, p, q, kap, True, beta=bet)
    lam = oracle.power_lambda_max(*csr, np.ones(N), 50)
    x, it, rel, rc = oracle.pcg(mesh, p, q, kap, csr, b, 1e-12, 500, precond=precond, cheb_k=3,
                                lo=lam / 30, hi=1.1 * lam, beta=bet)
    A = eliminate(dense(mesh, p, q, kap, bet), ess)
    ref = np.linalg.solve(A, b)
    assert rc == oracle.OK and rel <= 1e-12
    np.testing.assert_allclose(x, ref, atol=1e-9 * np.abs(ref).max())
    # the reaction term changes the solution
    x0 = np.linalg.solve(eliminate(dense(mesh, p, q, kap, None), ess), b)
    assert np.abs(x0 - ref).max() > 1e-2 * np.abs(ref).max()
