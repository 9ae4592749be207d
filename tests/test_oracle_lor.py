"""Pins of the oracle's LOR matrix (Sections 2.1-2.2, Step S1.2 A1-A4 and
the readings R1, R2, R4) against closed forms, an independent brute force on
the LOR mesh, and invariants."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
import scipy.linalg

import oracle
from meshutil import (csr_to_dense, element_corners, element_dofs, eliminate, essential_mask, gll_nodes, lor_mesh)
from paper_2210_12253_gb300.inputs import unit_cube_vertices


def jittered(nex, ney, nez, seed=7, jitter=0.2):
    return oracle.Mesh(nex, ney, nez, unit_cube_vertices(nex, ney, nez, jitter, np.random.default_rng(seed)))


def lor_dense(mesh, p, q, kappa, dirichlet):
    rp, ci, v = oracle.lor_assemble(mesh, p, q, kappa, dirichlet)
    return csr_to_dense(rp, ci, v, mesh.ndof(p)), (rp, ci, v)


# ------------------------------------------------------------ kappa binning (R1)
def bin_of(p, q):
    """Sub-interval of each Gauss-Legendre point along one axis: the GLL
    interval [x_a, x_{a+1}] that contains it (from numpy's nodes alone)."""
    xg, _ = npleg.leggauss(q)
    return np.clip(np.searchsorted(gll_nodes(p), xg, side="left") - 1, 0, p - 1)


@pytest.mark.parametrize("p", range(1, 11))
def test_kappa_sub_of_a_coefficient_constant_on_each_sub_hex(p):
    """kappa constant on each sub-hex's set of Gauss points (the value c_s
    drawn per sub-hex) gives kappa_s = c_s exactly, whatever the weights:
    this fixes which high-order points belong to which sub-hex."""
    q = p + 2
    rng = np.random.default_rng(100 + p)
    c = np.exp(rng.standard_normal((2, p ** 3)))
    b = bin_of(p, q)
    g0, g1, g2 = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    sub = (b[g0] + p * (b[g1] + p * b[g2]))          # [g0, g1, g2] -> sub-hex index
    kap = np.zeros((2, q ** 3))
    kap[:, (g0 + q * (g1 + q * g2)).ravel()] = c[:, sub.ravel()]
    np.testing.assert_allclose(oracle.lor_kappa_sub(p, q, kap), c, rtol=1e-15, atol=0)


def test_kappa_sub_of_a_linear_coefficient_p2():
    """p = 2 (GLL nodes -1, 0, 1), q = 4 Gauss points
    +-x1 = +-sqrt(3/7 - (2/7) sqrt(6/5)), weight (18 + sqrt 30)/36, and
    +-x2 = +-sqrt(3/7 + (2/7) sqrt(6/5)), weight (18 - sqrt 30)/36.
    For kappa = 2 + xi_d the weighted bin average is 2 -+ (w1 x1 + w2 x2) / (w1 + w2)
    on the lower / upper half of axis d (the other axes' weights cancel),
    with w1 + w2 = 1."""
    x1 = np.sqrt(3 / 7 - 2 / 7 * np.sqrt(6 / 5))
    x2 = np.sqrt(3 / 7 + 2 / 7 * np.sqrt(6 / 5))
    w1, w2 = (18 + np.sqrt(30)) / 36, (18 - np.sqrt(30)) / 36
    S = (w1 * x1 + w2 * x2) / (w1 + w2)
    xs = np.array([-x2, -x1, x1, x2])                 # ascending Gauss points
    p, q = 2, 4
    for d in range(3):
        g = np.stack(np.meshgrid(np.arange(q), np.arange(q), np.arange(q), indexing="ij"), 0)
        kap = np.zeros(q ** 3)
        kap[(g[0] + q * (g[1] + q * g[2])).ravel()] = (2.0 + xs[g[d]]).ravel()
        ks = oracle.lor_kappa_sub(p, q, kap[None])[0]
        for s in range(p ** 3):
            a = (s, s // p, s // (p * p))[d] % p
            assert abs(ks[s] - (2.0 - S if a == 0 else 2.0 + S)) < 2e-15  # a few ulps of 2.5


# ------------------------------------------------------------ closed forms
def test_p1_undistorted_interior_stencil():
    """p = 1, cube elements of side h, kappa = 1: the Q1 stencil
    8h/3 (centre), 0 (face), -h/6 (edge), -h/12 (corner)."""
    ne = 4
    h = 1.0 / ne
    mesh = oracle.Mesh(ne, ne, ne, unit_cube_vertices(ne, ne, ne))
    A, _ = lor_dense(mesh, 1, 3, np.ones((mesh.nel, 27)), dirichlet=False)
    n = ne + 1
    r = 2 + n * (2 + n * 2)
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                m = abs(di) + abs(dj) + abs(dk)
                ref = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[m]
                assert abs(A[r, r + di + n * (dj + n * dk)] - ref) < 1e-15


@pytest.mark.parametrize("p", [2, 3, 5])
def test_undistorted_subhex_blocks_are_kronecker(p):
    """Box element, kappa = 1: each sub-hex block is Kx(x)My(x)Mz + ... with
    K = [[1,-1],[-1,1]]/h and M = h [[2,1],[1,2]]/6 on the GLL spacings."""
    hx, hy, hz = 0.6, 1.1, 0.8
    mesh = oracle.Mesh(1, 1, 1, unit_cube_vertices(1, 1, 1) * np.array([hx, hy, hz]))
    q = p + 2
    A, _ = lor_dense(mesh, p, q, np.ones((1, q ** 3)), dirichlet=False)
    g = gll_nodes(p)
    n = p + 1
    ref = np.zeros_like(A)
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6
    for c in range(p):
        for b in range(p):
            for a in range(p):
                lx, ly, lz = (g[a + 1] - g[a]) * hx / 2, (g[b + 1] - g[b]) * hy / 2, (g[c + 1] - g[c]) * hz / 2
                blk = (np.kron(lz * M1, np.kron(ly * M1, K1 / lx)) + np.kron(lz * M1, np.kron(K1 / ly, lx * M1))
                       + np.kron(K1 / lz, np.kron(ly * M1, lx * M1)))
                idx = [(a + (r & 1)) + n * ((b + ((r >> 1) & 1)) + n * (c + ((r >> 2) & 1))) for r in range(8)]
                ref[np.ix_(idx, idx)] += blk
    np.testing.assert_allclose(A, ref, atol=1e-14 * np.abs(ref).max())


# ------------------------------------------------------------ brute force on the LOR mesh
@pytest.mark.parametrize("p,dims", [(1, (2, 3, 2)), (2, (2, 2, 2)), (3, (2, 2, 3)), (4, (2, 2, 2))])
def test_lor_is_q1_matrix_of_the_lor_mesh(p, dims):
    """A_h equals the p = 1 stiffness matrix of the LOR mesh (sub-hexes with
    vertices T_e(GLL points)) integrated by 2x2x2 Gauss with kappa_s."""
    mesh = jittered(*dims, seed=3 + p)
    q = p + 2
    kap = np.exp(np.random.default_rng(p).standard_normal((mesh.nel, q ** 3)))
    ks = oracle.lor_kappa_sub(p, q, kap).ravel()
    corners, dofs = lor_mesh(mesh.V, mesh.nex, mesh.ney, mesh.nez, p)
    N = mesh.ndof(p)
    ref = oracle.dense_general(corners, dofs, np.repeat(ks[:, None], 8, axis=1), 1, 2, N)
    for dirichlet in (False, True):
        A, _ = lor_dense(mesh, p, q, kap, dirichlet)
        R = eliminate(ref, essential_mask(*dims, p)) if dirichlet else ref
        np.testing.assert_allclose(A, R, atol=1e-13 * np.abs(R).max())


def test_p1_lor_equals_ho_on_affine_mesh():
    """p = 1 on an affinely mapped mesh with element-wise constant kappa: the
    LOR matrix is the high-order (Q1) matrix itself."""
    rng = np.random.default_rng(1)
    Am = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
    if np.linalg.det(Am) < 0:
        Am[:, 0] *= -1
    dims = (3, 2, 2)
    mesh = oracle.Mesh(*dims, unit_cube_vertices(*dims) @ Am.T)
    q = 3
    kap = np.repeat(np.exp(rng.standard_normal((mesh.nel, 1))), q ** 3, axis=1)
    A, _ = lor_dense(mesh, 1, q, kap, dirichlet=True)
    Ah = eliminate(oracle.dense_general(element_corners(mesh.V, *dims), element_dofs(*dims, 1), kap, 1, q,
                                        mesh.ndof(1)), essential_mask(*dims, 1))
    np.testing.assert_allclose(A, Ah, atol=1e-13 * np.abs(Ah).max())


# ------------------------------------------------------------ invariants
@pytest.mark.parametrize("p", [2, 4])
def test_row_sums_symmetry_and_patch(p):
    mesh = jittered(2, 3, 2, seed=p)
    q = p + 2
    kap = np.exp(np.random.default_rng(5).standard_normal((mesh.nel, q ** 3)))
    A, _ = lor_dense(mesh, p, q, kap, dirichlet=False)
    assert np.abs(A.sum(axis=1)).max() < 1e-13 * np.abs(A).max()
    np.testing.assert_allclose(A, A.T, atol=1e-15 * np.abs(A).max())
    xyz = oracle.dof_coordinates(mesh, p)
    a = np.array([0.4, 1.2, -0.5])
    u = xyz @ a
    A1, _ = lor_dense(mesh, p, q, np.ones_like(kap), dirichlet=False)
    assert abs(u @ A1 @ u - a @ a) < 1e-13
    ess = essential_mask(mesh.nex, mesh.ney, mesh.nez, p)
    assert np.abs((A1 @ u)[~ess]).max() < 1e-13


@pytest.mark.parametrize("dims,p", [((3, 3, 3), 2), ((2, 3, 4), 3), ((1, 1, 1), 1), ((4, 4, 4), 3)])
def test_sparsity_pattern(dims, p):
    mesh = jittered(*dims, seed=1)
    q = p + 2
    rp, ci, v = oracle.lor_assemble(mesh, p, q, np.ones((mesh.nel, q ** 3)), True)
    nx, ny, nz = (d * p + 1 for d in dims)
    assert rp[-1] == (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2)
    for r in range(nx * ny * nz):
        I, J, K = r % nx, (r // nx) % ny, r // (nx * ny)
        expect = sorted((I + di) + nx * ((J + dj) + ny * (K + dk))
                        for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)
                        if 0 <= I + di < nx and 0 <= J + dj < ny and 0 <= K + dk < nz)
        assert ci[rp[r]:rp[r + 1]].tolist() == expect


def test_paper_3d_problem_size():
    """Section 4.1: 32^3 elements, p = 6 -> 7,189,057 DOFs and 192,100,033 LOR nonzeros."""
    n = 32 * 6 + 1
    assert n ** 3 == 7189057
    assert (3 * n - 2) ** 3 == 192100033


def test_dirichlet_rows_and_columns():
    dims, p = (2, 2, 3), 3
    mesh = jittered(*dims, seed=2)
    q = p + 2
    kap = np.exp(np.random.default_rng(0).standard_normal((mesh.nel, q ** 3)))
    A, _ = lor_dense(mesh, p, q, kap, dirichlet=True)
    Af, _ = lor_dense(mesh, p, q, kap, dirichlet=False)
    ess = essential_mask(*dims, p)
    np.testing.assert_array_equal(A[ess][:, ess], np.eye(ess.sum()))
    assert not A[ess][:, ~ess].any() and not A[~ess][:, ess].any()
    np.testing.assert_array_equal(A[~ess][:, ~ess], Af[~ess][:, ~ess])


def test_rows_computed_alone_match_assembly():
    dims, p = (3, 2, 2), 3
    mesh = jittered(*dims, seed=4)
    q = p + 2
    kap = np.exp(np.random.default_rng(3).standard_normal((mesh.nel, q ** 3)))
    for dirichlet in (False, True):
        rp, ci, v = oracle.lor_assemble(mesh, p, q, kap, dirichlet)
        rows = np.arange(mesh.ndof(p))
        cnt, cols, vals = oracle.lor_rows(mesh, p, q, kap, rows, dirichlet)
        for r in rows:
            assert cnt[r] == rp[r + 1] - rp[r]
            assert cols[r, :cnt[r]].tolist() == ci[rp[r]:rp[r + 1]].tolist()
            np.testing.assert_allclose(vals[r, :cnt[r]], v[rp[r]:rp[r + 1]], rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------ spectral equivalence (Section 2.2)
def one_d_pair(p, ne):
    """Assembled 1D stiffness/mass on ne unit-length/ne elements: high order
    (exact, GLL Lagrange) and LOR (P1 on the GLL sub-mesh)."""
    from test_oracle_ho import exact_1d_matrices
    K, M = exact_1d_matrices(p)
    g = gll_nodes(p)
    n = ne * p + 1
    h = 1.0 / ne
    Kp, Mp, Kh, Mh = (np.zeros((n, n)) for _ in range(4))
    for e in range(ne):
        s = slice(e * p, e * p + p + 1)
        Kp[s, s] += (2 / h) * K
        Mp[s, s] += (h / 2) * M
        for a in range(p):
            l = (g[a + 1] - g[a]) * h / 2
            t = slice(e * p + a, e * p + a + 2)
            Kh[t, t] += np.array([[1.0, -1.0], [-1.0, 1.0]]) / l
            Mh[t, t] += l * np.array([[2.0, 1.0], [1.0, 2.0]]) / 6
    f = slice(1, n - 1)
    return Kp[f, f], Mp[f, f], Kh[f, f], Mh[f, f]


@pytest.mark.parametrize("p", range(1, 17))
def test_one_d_equivalence_constants_bounded(p):
    Kp, Mp, Kh, Mh = one_d_pair(p, 1 if p > 1 else 3)
    lk = scipy.linalg.eigh(Kp, Kh, eigvals_only=True)
    lm = scipy.linalg.eigh(Mp, Mh, eigvals_only=True)
    assert 1.0 - 1e-12 <= lk.min() and lk.max() <= np.pi ** 2 / 4
    assert 0.5 <= lm.min() and lm.max() <= 3.0


@pytest.mark.parametrize("p", range(1, 9))
def test_spectral_equivalence_within_tensor_bounds(p):
    """Generalised eigenvalues of (A_p, A_h) on the free DOFs of an
    undistorted mesh lie in [lk_min lm_min^2, lk_max lm_max^2], the products
    of the 1D stiffness/mass equivalence constants, which stay bounded in p
    (previous test).  The paper gives no 3D constant: beyond this property
    the constant itself is not pinned."""
    ne = 2 if p <= 4 else 1
    dims = (ne, ne, ne)
    mesh = oracle.Mesh(*dims, unit_cube_vertices(*dims))
    q = p + 2
    k1 = np.ones((mesh.nel, q ** 3))
    Ah, _ = lor_dense(mesh, p, q, k1, dirichlet=False)
    Ap = oracle.dense_general(element_corners(mesh.V, *dims), element_dofs(*dims, p), k1, p, q, mesh.ndof(p))
    free = ~essential_mask(*dims, p)
    lam = scipy.linalg.eigh(Ap[np.ix_(free, free)], Ah[np.ix_(free, free)], eigvals_only=True)
    Kp, Mp, Kh, Mh = one_d_pair(p, ne)
    lk = scipy.linalg.eigh(Kp, Kh, eigvals_only=True)
    lm = scipy.linalg.eigh(Mp, Mh, eigvals_only=True)
    lo, hi = lk.min() * lm.min() ** 2, lk.max() * lm.max() ** 2
    assert lam.min() >= lo * (1 - 1e-10) and lam.max() <= hi * (1 + 1e-10)
    if p == 1:
        np.testing.assert_allclose(lam, 1.0, atol=1e-12)
    assert hi <= (np.pi ** 2 / 4) * 9.0


def element_bounds(X, p):
    """Extreme generalised eigenvalues of one element's high-order and LOR
    stiffness matrices (kappa = 1, no boundary conditions) on the complement
    of the constants, the common kernel of both."""
    q = p + 2
    n = (p + 1) ** 3
    k1 = np.ones((1, q ** 3))
    Ah, _ = lor_dense(oracle.Mesh(1, 1, 1, X.copy()), p, q, k1, dirichlet=False)
    Ap = oracle.dense_general(X[None], element_dofs(1, 1, 1, p), k1, p, q, n)
    Z = scipy.linalg.null_space(np.ones((1, n)))
    lam = scipy.linalg.eigh(Z.T @ Ap @ Z, Z.T @ Ah @ Z, eigvals_only=True)
    return lam.min(), lam.max()


@pytest.mark.parametrize("p", range(1, 8))
def test_spectral_equivalence_jittered_mesh_lognormal_kappa(p):
    """Jittered mesh, kappa lognormal and constant on each element: both
    operators are sums of kappa_e times element matrices (kappa_s = kappa_e by
    R1), so the generalised eigenvalues of (A_p, A_h) on the free DOFs lie in
    [min_e mu_lo(e), max_e mu_hi(e)] of the elements' own kappa = 1 bounds,
    independent of the coefficient's contrast; and those bounds stay within
    the undistorted tensor-product range (1D stiffness at most pi^2/4, 1D mass
    in [1/2, 3]) as p grows."""
    dims = (2, 2, 2) if p <= 5 else (2, 1, 1)
    mesh = jittered(*dims, seed=p, jitter=0.2)
    q = p + 2
    kap = np.repeat(np.exp(np.random.default_rng(20 + p).standard_normal((mesh.nel, 1))), q ** 3, axis=1)
    Ah, _ = lor_dense(mesh, p, q, kap, dirichlet=False)
    C = element_corners(mesh.V, *dims)
    Ap = oracle.dense_general(C, element_dofs(*dims, p), kap, p, q, mesh.ndof(p))
    free = ~essential_mask(*dims, p)
    lam = scipy.linalg.eigh(Ap[np.ix_(free, free)], Ah[np.ix_(free, free)], eigvals_only=True)
    b = [element_bounds(C[e], p) for e in range(mesh.nel)]
    lo, hi = min(x[0] for x in b), max(x[1] for x in b)
    assert lam.min() >= lo * (1 - 1e-10) and lam.max() <= hi * (1 + 1e-10)
    assert lo >= 0.25 and hi <= 9.0 * np.pi ** 2 / 4


# ------------------------------------------------------------ general (element-restriction) meshes
def cube_in_cube(m, p, seed=1):
    from meshutil import cube_in_cube_corners, general_dofs, jitter_interior_vertices
    C = jitter_interior_vertices(cube_in_cube_corners(m), 0.1 * 0.3 / m, np.random.default_rng(seed))
    dofs, N, xyz, ess = general_dofs(C, p)
    return C, dofs, N, xyz, ess


@pytest.mark.parametrize("p,dims", [(1, (2, 3, 2)), (2, (2, 2, 3)), (4, (2, 2, 2))])
def test_general_lor_on_a_lattice_is_the_structured_lor(p, dims):
    """A structured mesh handed over in element-restriction form (natural
    numbering) gives the structured routine's matrix (same sub-hex blocks;
    only the summation order of the merged triplets may differ)."""
    mesh = jittered(*dims, seed=p)
    q = p + 2
    kap = np.exp(np.random.default_rng(p).standard_normal((mesh.nel, q ** 3)))
    ess = essential_mask(*dims, p).astype(np.uint8)
    for dirichlet in (False, True):
        rp, ci, v = oracle.lor_assemble(mesh, p, q, kap, dirichlet)
        g = oracle.lor_assemble_general(element_corners(mesh.V, *dims), element_dofs(*dims, p), mesh.ndof(p), p, q,
                                        kap, ess, dirichlet)
        np.testing.assert_array_equal(g[0], rp)
        np.testing.assert_array_equal(g[1], ci)
        np.testing.assert_allclose(g[2], v, rtol=0, atol=1e-14 * np.abs(v).max())


@pytest.mark.parametrize("m,p", [(1, 1), (1, 2), (1, 3), (2, 2)])
def test_general_lor_on_cube_in_cube_is_q1_matrix_of_its_lor_mesh(m, p):
    """On the non-lattice cube-in-cube mesh (vertex valences 3 and 4 at the
    special corners), A_h equals the brute-force p = 1 stiffness matrix of the
    LOR mesh (sub-hexes T_e(GLL boxes), 2x2x2 Gauss, kappa_s per sub-hex);
    the pattern is the union of the sub-hexes' 8 x 8 couplings; zero row
    sums and symmetry hold; with the boundary mask the essential rows and
    columns become the identity and the free block is unchanged."""
    from meshutil import general_lor_mesh
    C, dofs, N, xyz, ess = cube_in_cube(m, p)
    q = p + 2
    kap = np.exp(np.random.default_rng(3).standard_normal((C.shape[0], q ** 3)))
    ks = oracle.lor_kappa_sub(p, q, kap).ravel()
    sc, sd = general_lor_mesh(C, dofs, p)
    ref = oracle.dense_general(sc, sd, np.repeat(ks[:, None], 8, axis=1), 1, 2, N)
    rp, ci, v = oracle.lor_assemble_general(C, dofs, N, p, q, kap, ess, dirichlet=False)
    A = csr_to_dense(rp, ci, v, N)
    np.testing.assert_allclose(A, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    pattern = np.zeros((N, N), bool)
    for s in range(sd.shape[0]):
        pattern[np.ix_(sd[s], sd[s])] = True
    assert rp[-1] == pattern.sum()
    for r in range(N):
        assert ci[rp[r]:rp[r + 1]].tolist() == np.nonzero(pattern[r])[0].tolist()
    lengths = set(np.diff(rp).tolist())
    assert lengths - {8, 12, 18, 27}, lengths  # row lengths a lattice never has
    assert np.abs(A.sum(axis=1)).max() < 1e-13 * np.abs(A).max()
    np.testing.assert_allclose(A, A.T, atol=1e-15 * np.abs(A).max())
    rp2, ci2, v2 = oracle.lor_assemble_general(C, dofs, N, p, q, kap, ess, dirichlet=True)
    np.testing.assert_array_equal(rp2, rp)
    np.testing.assert_array_equal(ci2, ci)
    np.testing.assert_allclose(csr_to_dense(rp2, ci2, v2, N), eliminate(A, ess.astype(bool)), rtol=0, atol=0)


@pytest.mark.parametrize("p", range(2, 11))
def test_each_lor_interval_holds_one_or_two_gauss_points(p):
    """The FP64 LOR assembly from p = 2 gives each high-order Gauss point of
    a sub-hex's kappa_s average a lane of an 8-lane group, so every LOR
    interval must hold one or two of the q = p + 2 Gauss-Legendre points per
    axis (a point on a GLL node belongs to the lower interval); its launcher
    returns an error otherwise.  p = 1 (three points in its one interval)
    uses the one-thread kernel."""
    gx, _ = oracle.gauss_legendre(p + 2)
    gll = oracle.gauss_lobatto(p)
    counts = np.bincount([int(np.sum(gll[1:p] < x)) for x in gx], minlength=p)
    assert counts.min() >= 1 and counts.max() <= 2, counts
    # the same count from the oracle's kappa_s: a coefficient that is 1 at
    # one Gauss point (and 0 elsewhere) reaches exactly one sub-hex per axis
    q = p + 2
    for g in range(q):
        kappa = np.zeros((1, q, q, q))
        kappa[0, 0, 0, g] = 1.0  # Gauss point (g, 0, 0), the first index fastest
        ks = oracle.lor_kappa_sub(p, q, kappa).reshape(p, p, p)  # [c][b][a]
        hit = np.nonzero(ks[0, 0, :])[0]
        assert len(hit) == 1 and hit[0] == int(np.sum(gll[1:p] < gx[g]))
