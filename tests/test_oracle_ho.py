"""Pins of the oracle's geometry (Step S1.1) and high-order operator
(Step S2.1, Eq. (4)) against closed forms, brute force and invariants."""
import numpy as np
import pytest
from numpy.polynomial import polynomial as P

import oracle
from meshutil import (element_corners, element_dofs, eliminate, essential_mask, gll_nodes, gll_weights)
from paper_2210_12253_gb300.inputs import unit_cube_vertices


def jittered(nex, ney, nez, seed=7, jitter=0.2):
    return oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez, jitter, np.random.default_rng(seed)))


def dense_ho(mesh, p, q, kappa):
    C = element_corners(mesh.V, mesh.nex, mesh.ney, mesh.nez)
    Dm = element_dofs(mesh.nex, mesh.ney, mesh.nez, p)
    return oracle.dense_general(C, Dm, kappa, p, q, mesh.ndof(p))


# ------------------------------------------------------------------ geometry
def test_geometry_undistorted_box():
    nex, ney, nez, q = 3, 2, 4, 4
    mesh = oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez))
    detJ, G = oracle.geometry(mesh, q)
    h = np.array([1 / nex, 1 / ney, 1 / nez])
    np.testing.assert_allclose(detJ, np.prod(h / 2), rtol=1e-14)
    _, w = oracle.gauss_legendre(q)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    for a, idx in enumerate((0, 3, 5)):
        np.testing.assert_allclose(G[:, :, idx], np.broadcast_to(W[None, :] * np.prod(h / 2) * (2 / h[a]) ** 2, G[:, :, idx].shape), rtol=1e-14)
    np.testing.assert_allclose(G[:, :, [1, 2, 4]], 0.0, atol=1e-16)


def test_geometry_global_affine_map():
    """x -> A x + c maps every element affinely: J = A diag(h/2) everywhere."""
    rng = np.random.default_rng(3)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    nex, ney, nez, q = 2, 3, 2, 3
    V = unit_cube_vertices(nex, ney, nez) @ A.T + np.array([0.1, -0.2, 0.3])
    detJ, G = oracle.geometry(oracle.Mesh(nex, ney, nez, V), q)
    h = np.array([1 / nex, 1 / ney, 1 / nez])
    J = A @ np.diag(h / 2)
    Ji = np.linalg.inv(J)
    M = np.linalg.det(J) * Ji @ Ji.T
    _, w = oracle.gauss_legendre(q)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    np.testing.assert_allclose(detJ, np.linalg.det(J), rtol=1e-13)
    for idx, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        np.testing.assert_allclose(G[:, :, idx], np.broadcast_to(W[None, :] * M[a, b], G[:, :, idx].shape), rtol=1e-12, atol=1e-15)


def test_geometry_volume_of_jittered_cube():
    mesh = jittered(4, 3, 5)
    q = 3
    detJ, _ = oracle.geometry(mesh, q)
    _, w = oracle.gauss_legendre(q)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    assert abs((detJ * W[None, :]).sum() - 1.0) < 1e-14


def test_geometry_rejects_inverted_element():
    nex = ney = nez = 2
    V = unit_cube_vertices(nex, ney, nez)
    c = 1 + 3 * (1 + 3 * 1)  # the centre vertex, pushed through a face
    V[c] = [0.5, 0.5, 1.2]
    with pytest.raises(oracle.OracleError) as ei:
        oracle.geometry(oracle.Mesh(nex, ney, nez, V), 3)
    assert ei.value.code == oracle.EGEOM


def test_dof_coordinates_undistorted():
    nex, ney, nez, p = 2, 3, 1, 3
    xyz = oracle.dof_coordinates(oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez)), p)
    g = gll_nodes(p)
    def axis(ne):
        pts = [0.0]
        for e in range(ne):
            pts += list(e / ne + (g[1:] + 1) / (2 * ne))
        return np.array(pts)
    X, Y, Z = axis(nex), axis(ney), axis(nez)
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    np.testing.assert_allclose(xyz, np.stack([Xg.ravel(), Yg.ravel(), Zg.ravel()], 1), atol=1e-15)


# ------------------------------------------------------------------ HO operator
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_sum_factorisation_equals_brute_force(p):
    mesh = jittered(2, 2, 2, seed=p)  # one interior vertex: a genuinely distorted mesh
    q = p + 2
    kappa = np.exp(np.random.default_rng(10 + p).standard_normal((mesh.nel, q ** 3)))
    A = dense_ho(mesh, p, q, kappa)
    x = np.random.default_rng(20 + p).standard_normal(mesh.ndof(p))
    y = oracle.ho_apply(mesh, p, q, kappa, x, dirichlet=False)
    np.testing.assert_allclose(y, A @ x, rtol=0, atol=1e-12 * np.abs(A).sum(1).max() * np.abs(x).max())
    ess = essential_mask(mesh.nex, mesh.ney, mesh.nez, p)
    yd = oracle.ho_apply(mesh, p, q, kappa, x, dirichlet=True)
    np.testing.assert_allclose(yd, eliminate(A, ess) @ x, rtol=0, atol=1e-12 * np.abs(A).sum(1).max() * np.abs(x).max())
    np.testing.assert_array_equal(yd[ess], x[ess])


def exact_1d_matrices(p):
    """Exact GLL stiffness and mass matrices on [-1,1] by polynomial algebra."""
    g = gll_nodes(p)
    L = []
    for i in range(p + 1):
        c = P.polyfromroots(np.delete(g, i))
        L.append(c / P.polyval(g[i], c))
    K = np.zeros((p + 1, p + 1))
    M = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            kij = P.polyint(P.polymul(P.polyder(L[i]), P.polyder(L[j])))
            mij = P.polyint(P.polymul(L[i], L[j]))
            K[i, j] = P.polyval(1, kij) - P.polyval(-1, kij)
            M[i, j] = P.polyval(1, mij) - P.polyval(-1, mij)
    return K, M


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_undistorted_element_matrix_is_kronecker_sum(p):
    """One box element [0,hx]x[0,hy]x[0,hz], kappa = 1: A = Kx(x)My(x)Mz + ...
    with exact 1D matrices (q = p+2 Gauss points integrate them exactly)."""
    hx, hy, hz = 0.7, 1.3, 0.9
    V = unit_cube_vertices(1, 1, 1) * np.array([hx, hy, hz])
    mesh = oracle.Mesh(1, 1, 1, V)
    q = p + 2
    A = dense_ho(mesh, p, q, np.ones((1, q ** 3)))
    K, M = exact_1d_matrices(p)
    Kx, Ky, Kz = (2 / hx) * K, (2 / hy) * K, (2 / hz) * K
    Mx, My, Mz = (hx / 2) * M, (hy / 2) * M, (hz / 2) * M
    ref = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    np.testing.assert_allclose(A, ref, atol=1e-12 * np.abs(ref).max())
    x = np.random.default_rng(1).standard_normal(A.shape[0])
    np.testing.assert_allclose(oracle.ho_apply(mesh, p, q, np.ones((1, q ** 3)), x, dirichlet=False), ref @ x,
                               atol=1e-12 * np.abs(ref).sum(1).max() * np.abs(x).max())


@pytest.mark.parametrize("p", [2, 3, 4])
def test_bubble_energy_is_one_over_900(p):
    """u = x(1-x) y(1-y) z(1-z) lies in Q_p (p >= 2): u^T A u = 3 (1/3)(1/30)^2."""
    nex, ney, nez = 2, 3, 2
    mesh = oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez))
    q = p + 2
    xyz = oracle.dof_coordinates(mesh, p)
    u = np.prod(xyz * (1 - xyz), axis=1)
    k1 = np.ones((mesh.nel, q ** 3))
    for dirichlet in (False, True):
        y = oracle.ho_apply(mesh, p, q, k1, u, dirichlet=dirichlet)
        assert abs(u @ y - 1.0 / 900.0) < 1e-15


@pytest.mark.parametrize("p", [1, 2, 4])
def test_patch_test_on_jittered_mesh(p):
    """Linear u = a.x: u^T A u = sum_g kappa w detJ |a|^2 (= |a|^2 for kappa = 1),
    and the interior rows of A u vanish for kappa = 1 (exact quadrature)."""
    mesh = jittered(3, 2, 2, seed=11)
    q = p + 2
    xyz = oracle.dof_coordinates(mesh, p)
    a = np.array([0.3, -1.1, 0.7])
    u = xyz @ a
    k1 = np.ones((mesh.nel, q ** 3))
    y = oracle.ho_apply(mesh, p, q, k1, u, dirichlet=False)
    assert abs(u @ y - a @ a) < 1e-13
    ess = essential_mask(mesh.nex, mesh.ney, mesh.nez, p)
    assert np.abs(y[~ess]).max() < 1e-13
    kap = np.exp(np.random.default_rng(2).standard_normal((mesh.nel, q ** 3)))
    detJ, _ = oracle.geometry(mesh, q)
    _, w = oracle.gauss_legendre(q)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    yk = oracle.ho_apply(mesh, p, q, kap, u, dirichlet=False)
    assert abs(u @ yk - (kap * detJ * W).sum() * (a @ a)) < 1e-12


def test_constants_in_kernel_and_symmetry():
    mesh = jittered(2, 2, 3, seed=5)
    p, q = 3, 5
    kap = np.exp(np.random.default_rng(4).standard_normal((mesh.nel, q ** 3)))
    one = np.ones(mesh.ndof(p))
    assert np.abs(oracle.ho_apply(mesh, p, q, kap, one, dirichlet=False)).max() < 1e-13
    rng = np.random.default_rng(6)
    x, z = rng.standard_normal(mesh.ndof(p)), rng.standard_normal(mesh.ndof(p))
    for d in (False, True):
        ax = oracle.ho_apply(mesh, p, q, kap, x, dirichlet=d)
        az = oracle.ho_apply(mesh, p, q, kap, z, dirichlet=d)
        assert abs(z @ ax - x @ az) < 1e-12 * abs(z @ ax)


def test_backward_against_brute_force():
    """gx = A gy and <gkappa, dk> = gy^T A(dk) x with x, gy masked on the
    boundary, A(dk) the brute-force matrix with coefficient dk."""
    mesh = jittered(2, 2, 2, seed=9)  # distorted: the metric has off-diagonal entries
    p, q = 3, 5
    rng = np.random.default_rng(8)
    kap = np.exp(rng.standard_normal((mesh.nel, q ** 3)))
    x, gy = rng.standard_normal(mesh.ndof(p)), rng.standard_normal(mesh.ndof(p))
    gx, gk = oracle.ho_apply_backward(mesh, p, q, kap, x, gy)
    np.testing.assert_allclose(gx, oracle.ho_apply(mesh, p, q, kap, gy), atol=1e-14)
    ess = essential_mask(mesh.nex, mesh.ney, mesh.nez, p)
    xm, gm = x.copy(), gy.copy()
    xm[ess] = 0
    gm[ess] = 0
    for t in range(3):
        dk = rng.standard_normal((mesh.nel, q ** 3))
        lhs = (gk * dk).sum()
        rhs = gm @ dense_ho(mesh, p, q, dk) @ xm
        assert abs(lhs - rhs) < 1e-11 * (np.abs(gk).sum())
    # single-point derivative: gkappa[e,g] = d/dk (gy^T A x) by a unit perturbation
    e, g = 1, 17
    dk = np.zeros((mesh.nel, q ** 3))
    dk[e, g] = 1.0
    assert abs(gk[e, g] - gm @ dense_ho(mesh, p, q, dk) @ xm) < 1e-12 * max(1.0, abs(gk[e, g]))


@pytest.mark.parametrize("p", [2, 4])
def test_load_vector_variable_source_closed_form(p):
    """f = x at the Gauss points of the unit cube and u = x(1-x)y(1-y)z(1-z)
    interpolated at the GLL nodes (exact for p >= 2, zero on the boundary):
    sum_i b_i u_i = int f u = (1/12)(1/6)(1/6) = 1/432, exact at q = p+2."""
    nex, ney, nez = 2, 3, 2
    q = p + 2
    mesh = oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez))
    xg, _ = np.polynomial.legendre.leggauss(q)
    f = np.zeros((mesh.nel, q ** 3))
    for ez in range(nez):
        for ey in range(ney):
            for ex in range(nex):
                e = ex + nex * (ey + ney * ez)
                for g in range(q ** 3):
                    f[e, g] = (ex + 0.5 * (xg[g % q] + 1.0)) / nex
    b = oracle.load_vector(mesh, p, q, f)
    t = gll_nodes(p)
    def coords(ne):
        c = np.zeros(ne * p + 1)
        for e in range(ne):
            c[e * p:e * p + p + 1] = (e + 0.5 * (t + 1.0)) / ne
        return c
    X, Y, Z = coords(nex), coords(ney), coords(nez)
    u = np.einsum("k,j,i->kji", Z * (1 - Z), Y * (1 - Y), X * (1 - X)).ravel()
    assert abs(b @ u - 1.0 / 432.0) < 1e-14


@pytest.mark.parametrize("p", [1, 3])
def test_load_vector_unit_source_closed_form(p):
    """f = 1 on box elements: b_i = prod_d (sum over elements of (h_d/2) w_i^GLL)."""
    nex, ney, nez = 2, 3, 2
    mesh = oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez))
    b = oracle.load_vector(mesh, p, p + 2)
    w = gll_weights(p)
    def one_d(ne):
        v = np.zeros(ne * p + 1)
        for e in range(ne):
            v[e * p:e * p + p + 1] += w / (2 * ne)
        return v
    ref = np.einsum("k,j,i->kji", one_d(nez), one_d(ney), one_d(nex)).ravel()
    ref[essential_mask(nex, ney, nez, p)] = 0
    np.testing.assert_allclose(b, ref, atol=1e-16)
