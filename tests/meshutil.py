"""Test helpers that rebuild mesh data with numpy alone (independent of the
oracle's C code), so that the oracle's structured routines can be checked
against its brute-force general-mesh routine and against closed forms."""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes(p):
    """Gauss-Lobatto nodes from numpy: +-1 and the roots of P_p'."""
    if p == 1:
        return np.array([-1.0, 1.0])
    inner = npleg.Legendre.basis(p).deriv().roots()
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def gll_weights(p):
    """Closed-form GLL weights 2 / (p (p+1) P_p(x_i)^2)."""
    x = gll_nodes(p)
    return 2.0 / (p * (p + 1) * npleg.legval(x, [0] * p + [1]) ** 2)


def trilinear(X, xi):
    """x(xi) = sum_c X_c prod_k l_{c_k}(xi_k) for corners X[8,3] (c = c0+2c1+4c2)."""
    x = np.zeros(3)
    for c in range(8):
        ck = (c & 1, (c >> 1) & 1, (c >> 2) & 1)
        w = 1.0
        for k in range(3):
            w *= 0.5 * (1 + xi[k]) if ck[k] else 0.5 * (1 - xi[k])
        x += w * X[c]
    return x


def vid(a, b, c, nex, ney):
    return a + (nex + 1) * (b + (ney + 1) * c)


def element_corners(V, nex, ney, nez):
    out = np.zeros((nex * ney * nez, 8, 3))
    e = 0
    for ez in range(nez):
        for ey in range(ney):
            for ex in range(nex):
                for c in range(8):
                    out[e, c] = V[vid(ex + (c & 1), ey + ((c >> 1) & 1), ez + ((c >> 2) & 1), nex, ney)]
                e += 1
    return out


def element_dofs(nex, ney, nez, p):
    n = p + 1
    nx, ny = nex * p + 1, ney * p + 1
    out = np.zeros((nex * ney * nez, n ** 3), np.int64)
    e = 0
    for ez in range(nez):
        for ey in range(ney):
            for ex in range(nex):
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            out[e, i + n * (j + n * k)] = (ex * p + i) + nx * ((ey * p + j) + ny * (ez * p + k))
                e += 1
    return out


def lor_mesh(V, nex, ney, nez, p):
    """The LOR mesh as a general p=1 hex mesh: sub-hex (a,b,c) of each element
    (element-major, sub-hex a + p(b + p c)) with corners T_e(GLL points)."""
    g = gll_nodes(p)
    EC = element_corners(V, nex, ney, nez)
    nx, ny = nex * p + 1, ney * p + 1
    nel = nex * ney * nez
    corners = np.zeros((nel * p ** 3, 8, 3))
    dofs = np.zeros((nel * p ** 3, 8), np.int64)
    e = 0
    s = 0
    for ez in range(nez):
        for ey in range(ney):
            for ex in range(nex):
                for c in range(p):
                    for b in range(p):
                        for a in range(p):
                            for r in range(8):
                                r0, r1, r2 = r & 1, (r >> 1) & 1, (r >> 2) & 1
                                corners[s, r] = trilinear(EC[e], (g[a + r0], g[b + r1], g[c + r2]))
                                dofs[s, r] = (ex * p + a + r0) + nx * ((ey * p + b + r1) + ny * (ez * p + c + r2))
                            s += 1
                e += 1
    return corners, dofs


def essential_mask(nex, ney, nez, p):
    nx, ny, nz = nex * p + 1, ney * p + 1, nez * p + 1
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((I == 0) | (I == nx - 1) | (J == 0) | (J == ny - 1) | (K == 0) | (K == nz - 1)).ravel()


def eliminate(A, ess):
    """Dirichlet elimination keeping the pattern: zero rows/cols, unit diagonal."""
    A = A.copy()
    A[ess, :] = 0.0
    A[:, ess] = 0.0
    A[ess, ess] = 1.0
    return A


def csr_to_dense(rowptr, colidx, values, n):
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(rowptr[i], rowptr[i + 1]):
            A[i, colidx[j]] += values[j]
    return A


# ------------------------------------------------------------------ general (non-lattice) meshes
def cube_in_cube_corners(m, inner=(0.3, 0.7)):
    """A conforming hex mesh of the unit cube that is not a lattice: an inner
    cube [lo, hi]^3 and six hexes joining each of its faces to the matching
    face of the unit cube (7 macro hexes), each split into m^3 hexes.  The 8
    corners of the inner cube are shared by 4 hexes of the macro mesh and the
    8 corners of the unit cube by 3 (8 in a lattice).  Corners per element in
    the order c0 + 2 c1 + 4 c2, every map positively oriented (the local axes
    follow the global ones)."""
    lo, hi = inner
    I = np.array([[lo + (hi - lo) * (c & 1), lo + (hi - lo) * ((c >> 1) & 1), lo + (hi - lo) * (c >> 2)]
                  for c in range(8)])
    O = np.array([[c & 1, (c >> 1) & 1, c >> 2] for c in range(8)], dtype=float)
    macros = [I]
    for d in range(3):
        for side in (0, 1):
            X = np.zeros((8, 3))
            for c in range(8):
                cd = (c >> d) & 1
                src = (c & ~(1 << d)) | (side << d)   # the corner on this face of the inner/outer cube
                if side == 1:
                    X[c] = O[src] if cd else I[src]
                else:
                    X[c] = I[src] if cd else O[src]
            macros.append(X)
    out = []
    for X in macros:
        for k in range(m):
            for j in range(m):
                for i in range(m):
                    out.append([trilinear(X, (2.0 * (i + (c & 1)) / m - 1, 2.0 * (j + ((c >> 1) & 1)) / m - 1,
                                              2.0 * (k + (c >> 2)) / m - 1)) for c in range(8)])
    return np.array(out)


def merge_points(P, tol=1e-9):
    """Ids of points (rows of P) with points closer than tol merged, numbered
    in order of first appearance."""
    from scipy.spatial import cKDTree
    parent = np.arange(len(P))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for a, b in cKDTree(P).query_pairs(tol):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(len(P))])
    _, first, inv = np.unique(roots, return_index=True, return_inverse=True)
    order = np.argsort(np.argsort(first))
    return order[inv]


def jitter_interior_vertices(corners, amount, rng):
    """Move every vertex not on the unit cube's boundary by U(-amount, amount)
    per coordinate (shared vertices move together)."""
    P = corners.reshape(-1, 3)
    vid = merge_points(P)
    V = np.zeros((vid.max() + 1, 3))
    V[vid] = P
    on_bnd = np.any((np.abs(V) < 1e-12) | (np.abs(V - 1) < 1e-12), axis=1)
    V[~on_bnd] += rng.uniform(-amount, amount, (int((~on_bnd).sum()), 3))
    return V[vid].reshape(corners.shape)


def general_dofs(corners, p):
    """Element-to-DOF map of the order-p space on a conforming hex mesh:
    GLL nodes T_e(gll_i, gll_j, gll_k) of all elements, coinciding nodes
    merged.  Returns (dofs [nel][(p+1)^3], N, xyz [N][3], essential mask of
    the unit cube's boundary uint8[N])."""
    g = gll_nodes(p)
    n = p + 1
    nel = corners.shape[0]
    P = np.zeros((nel, n ** 3, 3))
    for e in range(nel):
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    P[e, i + n * (j + n * k)] = trilinear(corners[e], (g[i], g[j], g[k]))
    ids = merge_points(P.reshape(-1, 3))
    N = int(ids.max()) + 1
    xyz = np.zeros((N, 3))
    xyz[ids] = P.reshape(-1, 3)
    ess = np.any((np.abs(xyz) < 1e-12) | (np.abs(xyz - 1) < 1e-12), axis=1).astype(np.uint8)
    return ids.reshape(nel, n ** 3).astype(np.int64), N, xyz, ess


def general_lor_mesh(corners, dofs, p):
    """The LOR mesh of a general mesh as a p = 1 hex mesh: sub-hex (a,b,c) of
    each element (element-major, a + p(b + p c)), corners T_e(GLL points),
    DOFs through the element-to-DOF map."""
    g = gll_nodes(p)
    n = p + 1
    nel = corners.shape[0]
    sc = np.zeros((nel * p ** 3, 8, 3))
    sd = np.zeros((nel * p ** 3, 8), np.int64)
    s = 0
    for e in range(nel):
        for c in range(p):
            for b in range(p):
                for a in range(p):
                    for r in range(8):
                        i, j, k = a + (r & 1), b + ((r >> 1) & 1), c + (r >> 2)
                        sc[s, r] = trilinear(corners[e], (g[i], g[j], g[k]))
                        sd[s, r] = dofs[e, i + n * (j + n * k)]
                    s += 1
    return sc, sd
