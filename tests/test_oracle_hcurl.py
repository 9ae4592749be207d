"""Pins of the oracle's discrete gradient of the LOR mesh (the vertex-to-edge
incidence matrix Algorithm 1 builds for the H(curl) solver, Section 3, with
the edge numbering of reading R17): closed forms and invariants."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle


def path_laplacian(n):
    """Graph Laplacian of a path with n vertices (degree on the diagonal)."""
    L = np.zeros((n, n))
    for i in range(n - 1):
        L[i, i] += 1
        L[i + 1, i + 1] += 1
        L[i, i + 1] -= 1
        L[i + 1, i] -= 1
    return L


@pytest.mark.parametrize("dims,p", [((1, 1, 1), 1), ((2, 1, 3), 2), ((1, 2, 1), 4), ((2, 2, 2), 3)])
def test_gradient_structure_and_graph_laplacian(dims, p):
    nx, ny, nz = (d * p + 1 for d in dims)
    rp, ci, v = oracle.discrete_gradient(*dims, p)
    ne = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert rp.size == ne + 1 and ci.size == 2 * ne
    np.testing.assert_array_equal(rp, 2 * np.arange(ne + 1))
    np.testing.assert_array_equal(v.reshape(-1, 2), np.tile([-1.0, 1.0], (ne, 1)))
    assert np.all(ci[1::2] > ci[0::2])
    N = nx * ny * nz
    G = sp.csr_matrix((v, ci, rp), shape=(ne, N)).toarray()
    # G^T G is the Laplacian of the grid graph: a Kronecker sum of path Laplacians
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    ref = (np.kron(Iz, np.kron(Iy, path_laplacian(nx))) + np.kron(Iz, np.kron(path_laplacian(ny), Ix)) +
           np.kron(path_laplacian(nz), np.kron(Iy, Ix)))
    np.testing.assert_array_equal(G.T @ G, ref)
    # gradients of constants vanish; of the grid index functions they are the
    # indicator of the edges along that axis (x-, then y-, then z-edges)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    np.testing.assert_array_equal(G @ np.ones(N), 0.0)
    nxe, nye = (nx - 1) * ny * nz, nx * (ny - 1) * nz
    for f, lo, hi in ((I, 0, nxe), (J, nxe, nxe + nye), (K, nxe + nye, ne)):
        g = G @ f.ravel().astype(float)
        expect = np.zeros(ne)
        expect[lo:hi] = 1.0
        np.testing.assert_array_equal(g, expect)


def test_edges_are_the_lor_mesh_edges():
    """Each edge joins two vertices of one sub-hex differing in one index by
    one, and every such pair appears exactly once."""
    dims, p = (2, 1, 2), 3
    nx, ny, nz = (d * p + 1 for d in dims)
    rp, ci, v = oracle.discrete_gradient(*dims, p)
    pairs = set(zip(ci[0::2].tolist(), ci[1::2].tolist()))
    assert len(pairs) == len(ci) // 2
    ref = set()
    for K in range(nz):
        for J in range(ny):
            for I in range(nx):
                a = I + nx * (J + ny * K)
                if I + 1 < nx:
                    ref.add((a, a + 1))
                if J + 1 < ny:
                    ref.add((a, a + nx))
                if K + 1 < nz:
                    ref.add((a, a + nx * ny))
    assert pairs == ref
