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
