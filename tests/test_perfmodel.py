"""Pins of the roofline numerators in paper_2210_12253_gb300/perfmodel.py.

Each flop count there is the cost of a formula as the kernel evaluates it.
Here that formula is evaluated once, on one element, with a scalar type that
records every +, -, * and / as a node of an expression graph; the count is
the number of nodes the outputs depend on (work whose result is never used
is not counted, as a compiler drops it), and the evaluation is checked
against the oracle on the same element, so the counted work is shown to
compute the right thing.  Plain floats stand for compile-time constants
(they combine for free); values a kernel reads from a table or computes at
run time are graph leaves.

Conventions (those of the counts): a sum of k products accumulated from
zero costs 2k (one FMA each), the 3x3 metric product and the dot products of
the geometry start from their first product.
"""
import math
import operator

import numpy as np
import pytest

import oracle
from paper_2210_12253_gb300 import perfmodel as pm


class Flop:
    __slots__ = ("v", "args")

    def __init__(self, v, args=None):
        self.v = v
        self.args = args  # None: a leaf

    def _op(self, o, f, swap=False):
        ov = o.v if isinstance(o, Flop) else o
        v = f(ov, self.v) if swap else f(self.v, ov)
        return Flop(v, (self, o) if isinstance(o, Flop) else (self,))

    def __add__(self, o): return self._op(o, operator.add)
    def __radd__(self, o): return self._op(o, operator.add, True)
    def __sub__(self, o): return self._op(o, operator.sub)
    def __rsub__(self, o): return self._op(o, operator.sub, True)
    def __mul__(self, o): return self._op(o, operator.mul)
    def __rmul__(self, o): return self._op(o, operator.mul, True)
    def __truediv__(self, o): return self._op(o, operator.truediv)
    def __rtruediv__(self, o): return self._op(o, operator.truediv, True)


def rsqrt(x):
    """1/sqrt(x) as one operation (like a division)."""
    return Flop(1.0 / math.sqrt(x.v), (x,))


def leaves(a):
    return [Flop(float(v)) for v in np.asarray(a, dtype=float).ravel()]


def count(outputs):
    seen, stack, n = set(), list(outputs), 0
    while stack:
        x = stack.pop()
        if not isinstance(x, Flop) or x.args is None or id(x) in seen:
            continue
        seen.add(id(x))
        n += 1
        stack.extend(x.args)
    return n


def val(a):
    return np.array([x.v for x in a])


def acc(coefs, vals):
    """Sum of products from zero: one FMA (2 flops) per term."""
    s = 0.0
    for c, v in zip(coefs, vals):
        s = s + c * v
    return s


def one_element(p, seed):
    """One trilinear, non-affine hex (the unit cube with every corner moved)."""
    rng = np.random.default_rng(seed)
    corners = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], float)
    corners += rng.uniform(-0.12, 0.12, corners.shape)
    q = p + 2
    kappa = np.exp(rng.standard_normal(q ** 3))
    return oracle.Mesh(1, 1, 1, corners), corners, kappa, rng


# ---------------------------------------------------------------------------
# Sum factorisation (the HO apply and its backward).
# u is indexed i + n (j + n k), points qx + q (qy + q qz).
# ---------------------------------------------------------------------------
def grad_ref(u, B, D, want_bb=False):
    q, n = B.shape
    U = lambda i, j, k: u[i + n * (j + n * k)]
    Bu = {(k, j, a): acc(B[a], [U(i, j, k) for i in range(n)]) for k in range(n) for j in range(n) for a in range(q)}
    Du = {(k, j, a): acc(D[a], [U(i, j, k) for i in range(n)]) for k in range(n) for j in range(n) for a in range(q)}
    BB, DB, BD = {}, {}, {}
    for k in range(n):
        for b in range(q):
            for a in range(q):
                cb = [Bu[k, j, a] for j in range(n)]
                BB[k, b, a] = acc(B[b], cb)
                DB[k, b, a] = acc(D[b], cb)
                BD[k, b, a] = acc(B[b], [Du[k, j, a] for j in range(n)])
    gx, gy, gz = [], [], []
    for c in range(q):
        for b in range(q):
            for a in range(q):
                gx.append(acc(B[c], [BD[k, b, a] for k in range(n)]))
                gy.append(acc(B[c], [DB[k, b, a] for k in range(n)]))
                gz.append(acc(D[c], [BB[k, b, a] for k in range(n)]))
    return (gx, gy, gz, BB) if want_bb else (gx, gy, gz)


def grad_ref_t(vx, vy, vz, B, D, vm=None):
    """The transposed pass; vm (reaction term): values at the points that
    B_z^T adds into the same slot as the z-derivative part."""
    q, n = B.shape
    P = lambda a, b, c: a + q * (b + q * c)
    tx, ty, tz = {}, {}, {}
    for k in range(n):
        for b in range(q):
            for a in range(q):
                tx[k, b, a] = acc(B[:, k], [vx[P(a, b, c)] for c in range(q)])
                ty[k, b, a] = acc(B[:, k], [vy[P(a, b, c)] for c in range(q)])
                if vm is None:
                    tz[k, b, a] = acc(D[:, k], [vz[P(a, b, c)] for c in range(q)])
                else:
                    tz[k, b, a] = acc(list(D[:, k]) + list(B[:, k]),
                                      [vz[P(a, b, c)] for c in range(q)] + [vm[P(a, b, c)] for c in range(q)])
    sB, sD = {}, {}
    for k in range(n):
        for j in range(n):
            for a in range(q):
                sB[k, j, a] = acc(list(B[:, j]) + list(D[:, j]),
                                  [tz[k, b, a] for b in range(q)] + [ty[k, b, a] for b in range(q)])
                sD[k, j, a] = acc(B[:, j], [tx[k, b, a] for b in range(q)])
    return [acc(list(B[:, i]) + list(D[:, i]), [sB[k, j, a] for a in range(q)] + [sD[k, j, a] for a in range(q)])
            for k in range(n) for j in range(n) for i in range(n)]


def metric_product(d, g):
    """v = D g with D symmetric (00, 01, 02, 11, 12, 22): 15 flops."""
    d00, d01, d02, d11, d12, d22 = d
    a, b, c = g
    return (d00 * a + d01 * b + d02 * c, d01 * a + d11 * b + d12 * c, d02 * a + d12 * b + d22 * c)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_sumfact_fma_counts_a_correct_reference_gradient(p):
    q, n = p + 2, p + 1
    B, D = oracle.basis_1d(p, q)
    u = np.random.default_rng(p).standard_normal(n ** 3)
    g = grad_ref(leaves(u), B, D)
    assert count(g[0] + g[1] + g[2]) == 2 * pm.sumfact_fma(p)
    U = u.reshape(n, n, n)  # [k, j, i]
    for got, (bz, by, bx) in zip(g, [(B, B, D), (B, D, B), (D, B, B)]):
        ref = np.einsum("ck,bj,ai,kji->cba", bz, by, bx, U).ravel()
        np.testing.assert_allclose(val(got), ref, rtol=1e-13, atol=1e-13)
    # the transposed pass costs the same and is the adjoint
    v = [np.random.default_rng(10 + i).standard_normal(q ** 3) for i in range(3)]
    ut = grad_ref_t(*(leaves(x) for x in v), B, D)
    assert count(ut) == 2 * pm.sumfact_fma(p)
    lhs = sum(float(val(gi) @ vi) for gi, vi in zip(g, v))
    assert abs(lhs - float(u @ val(ut))) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_apply_flops_evaluate_the_oracle_apply(p):
    q, n = p + 2, p + 1
    mesh, _, kappa, rng = one_element(p, 20 + p)
    B, D = oracle.basis_1d(p, q)
    _, G = oracle.geometry(mesh, q)
    Dq = kappa[:, None] * G[0]
    x = rng.standard_normal(n ** 3)
    gx, gy, gz = grad_ref(leaves(x), B, D)
    v = [metric_product(Dq[pt], (gx[pt], gy[pt], gz[pt])) for pt in range(q ** 3)]
    y = grad_ref_t([t[0] for t in v], [t[1] for t in v], [t[2] for t in v], B, D)
    assert count(y) == pm.apply_flops_per_element(p)
    ref = oracle.ho_apply(mesh, p, q, kappa, x, dirichlet=False)
    np.testing.assert_allclose(val(y), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("p", [1, 3])
def test_apply_reaction_flops_evaluate_the_oracle_apply(p):
    """The reaction term's share: B_z on the BB lines the forward pass already
    holds, the scaling by M = beta w detJ, B_z^T into the transposed pass."""
    q, n = p + 2, p + 1
    mesh, _, kappa, rng = one_element(p, 70 + p)
    beta = np.exp(rng.standard_normal(q ** 3))
    B, D = oracle.basis_1d(p, q)
    detJ, G = oracle.geometry(mesh, q)
    _, wg = oracle.gauss_legendre(q)
    Dq = kappa[:, None] * G[0]
    M = beta * np.einsum("c,b,a->cba", wg, wg, wg).ravel() * detJ[0]
    x = rng.standard_normal(n ** 3)
    gx, gy, gz, BB = grad_ref(leaves(x), B, D, want_bb=True)
    v = [metric_product(Dq[pt], (gx[pt], gy[pt], gz[pt])) for pt in range(q ** 3)]
    um = [acc(B[c], [BB[k, b, a] for k in range(n)]) * M[a + q * (b + q * c)]
          for c in range(q) for b in range(q) for a in range(q)]
    y = grad_ref_t([t[0] for t in v], [t[1] for t in v], [t[2] for t in v], B, D, vm=um)
    assert count(y) == pm.apply_flops_per_element(p) + pm.reaction_extra_apply_flops_per_element(p)
    ref = oracle.ho_apply(mesh, p, q, kappa, x, dirichlet=False, beta=beta)
    np.testing.assert_allclose(val(y), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("p", [2, 3])
def test_backward_flops_evaluate_the_oracle_backward(p):
    q, n = p + 2, p + 1
    mesh, _, kappa, rng = one_element(p, 30 + p)
    B, D = oracle.basis_1d(p, q)
    _, G = oracle.geometry(mesh, q)
    Dq = kappa[:, None] * G[0]
    # the oracle's backward holds essential DOFs at zero: on one element only
    # the interior ones are free (zeros stay leaves: the kernel reads them)
    I, J, K = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    inner = ((I > 0) & (I < p) & (J > 0) & (J < p) & (K > 0) & (K < p)).transpose(2, 1, 0).ravel()
    x = np.where(inner, rng.standard_normal(n ** 3), 0.0)
    gyv = np.where(inner, rng.standard_normal(n ** 3), 0.0)
    ax = grad_ref(leaves(x), B, D)
    ay = grad_ref(leaves(gyv), B, D)
    gk, t = [], []
    for pt in range(q ** 3):
        t0, t1, t2 = metric_product(Dq[pt], (ay[0][pt], ay[1][pt], ay[2][pt]))
        gk.append((ax[0][pt] * t0 + ax[1][pt] * t1 + ax[2][pt] * t2) / kappa[pt])
        t.append((t0, t1, t2))
    gx = grad_ref_t([s[0] for s in t], [s[1] for s in t], [s[2] for s in t], B, D)
    assert count(gk + gx) == pm.backward_flops_per_element(p)
    rgx, rgk = oracle.ho_apply_backward(mesh, p, q, kappa, x, gyv)
    np.testing.assert_allclose(val(gk), rgk[0], rtol=0, atol=1e-12 * np.abs(rgk).max())
    np.testing.assert_allclose(val(gx)[inner], rgx[inner], rtol=0, atol=1e-12 * np.abs(rgx).max())


# ---------------------------------------------------------------------------
# Geometry: Jacobian columns of the trilinear map per element, then the
# adjugate rows a_i and det at each point (as the setup and the assembly
# evaluate them).
# ---------------------------------------------------------------------------
def jacobian_columns(X, w0, w1):
    """col[d][(u, v)] = d x / d xi_d at the coordinates (u, v) of the two
    other axes (in increasing axis order), bilinear in them."""
    L = len(w0)
    E = {}
    for d in range(3):
        for o1 in (0, 1):
            for o0 in (0, 1):
                lo = [0 + 2 * o0 + 4 * o1, o0 + 0 + 4 * o1, o0 + 2 * o1 + 0][d]
                hi = lo + (1 << d)
                E[d, o0 + 2 * o1] = [0.5 * (X[hi][c] - X[lo][c]) for c in range(3)]
    col = [dict() for _ in range(3)]
    for d in range(3):
        for u in range(L):
            a = [w0[u] * E[d, 0][c] + w1[u] * E[d, 1][c] for c in range(3)]
            b = [w0[u] * E[d, 2][c] + w1[u] * E[d, 3][c] for c in range(3)]
            for v in range(L):
                col[d][u, v] = [w0[v] * a[c] + w1[v] * b[c] for c in range(3)]
    return col


def cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def dot3(u, v):
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]


PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def corner_leaves(corners):
    return [leaves(c) for c in corners]


@pytest.mark.parametrize("p", [1, 3, 4])
def test_setup_flops_evaluate_the_oracle_metric(p):
    q = p + 2
    mesh, corners, kappa, _ = one_element(p, 40 + p)
    xg, wg = oracle.gauss_legendre(q)
    w0, w1 = (1 - xg) / 2, (1 + xg) / 2
    col = jacobian_columns(corner_leaves(corners), w0, w1)
    sw = leaves(wg)  # weights are read from a table and multiplied at run time
    out = []
    for g2 in range(q):
        for g1 in range(q):
            for g0 in range(q):
                c0, c1, c2 = col[0][g1, g2], col[1][g0, g2], col[2][g0, g1]
                R = [cross(c1, c2), cross(c2, c0), cross(c0, c1)]  # adjugate rows of J
                dj = dot3(c0, R[0])
                detM = dj * dj
                adj = [dot3(R[i], R[j]) for i, j in PAIRS]
                k = Flop(kappa[g0 + q * (g1 + q * g2)])
                s = k * (sw[g0] * sw[g1] * sw[g2]) * rsqrt(detM)
                out.append([s * a for a in adj])
    flat = [x for d in out for x in d]
    assert count(flat) == pm.setup_flops_per_element(p)
    _, G = oracle.geometry(mesh, q)
    ref = kappa[:, None] * G[0]
    np.testing.assert_allclose(val(flat).reshape(-1, 6), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# ---------------------------------------------------------------------------
# LOR assembly: the modal (Walsh-Hadamard) form of the sub-hex block.
# ---------------------------------------------------------------------------
def popc(m):
    return bin(m).count("1")


def sym(i, j):
    return (i, j) if i <= j else (j, i)


def walsh8(v, first):
    for k in [first] + [k for k in range(3) if k != first]:
        for g in range(8):
            if not (g >> k) & 1:
                lo, hi = v[g], v[g | 1 << k]
                v[g], v[g | 1 << k] = lo + hi, hi - lo


def hadamard_axis(K, k):
    bit, out = 1 << k, {}
    for i0 in range(8):
        if i0 & bit:
            continue
        for j0 in range(i0, 8):
            if j0 & bit:
                continue
            i1, j1 = i0 | bit, j0 | bit
            if i0 == j0:
                a, b, d = K[i0, i0], K[i0, i1], K[i1, i1]
                t = a + d
                out[i0, i0], out[i1, i1], out[i0, i1] = t - 2.0 * b, t + 2.0 * b, a - d
            else:
                a, b, c, d = K[sym(i0, j0)], K[sym(i0, j1)], K[sym(i1, j0)], K[sym(i1, j1)]
                u0, u1, v0, v1 = a - c, a + c, b - d, b + d
                out[sym(i0, j0)], out[sym(i0, j1)] = u0 - v0, u0 + v0
                out[sym(i1, j0)], out[sym(i1, j1)] = u1 - v1, u1 + v1
    return out


def modal_block(G, W=None, sums=False):
    """Nodal 8x8 block (36 symmetric entries) from the scaled metric G[ab][g]
    (1/64 folded in) and, for the reaction term, W(g) = beta_s detJ_sub / 64:
    Walsh transforms, modal block, Hadamard sandwich on each axis.  sums:
    each modal entry as the FP64 kernel forms it, the plain sum of its
    transformed terms times its factor 3^(-(|m|+|n|-2)/2) (when not 1);
    otherwise as the FP32 kernel does, one FMA per term with the factor."""
    for ab, first in enumerate([0, 0, 0, 1, 0, 2]):
        walsh8(G[ab], first)
    K = {(0, n): Flop(0.0) for n in range(8)}  # psi_0 has no gradient
    for m in range(1, 8):
        for n in range(m, 8):
            terms = [PAIRS.index(sym(x, y)) for x in range(3) if (m >> x) & 1 for y in range(3) if (n >> y) & 1]
            ws = [(m & ~(1 << x)) ^ (n & ~(1 << y)) for x in range(3) if (m >> x) & 1 for y in range(3)
                  if (n >> y) & 1]
            cf = 3.0 ** (-(popc(m) + popc(n) - 2) / 2)
            if sums:
                t = [G[t][w] for t, w in zip(terms, ws)]
                s = t[0]
                for x in t[1:]:
                    s = s + x
                K[m, n] = s * cf if popc(m) + popc(n) > 2 else s
            else:
                K[m, n] = acc([cf] * len(terms), [G[t][w] for t, w in zip(terms, ws)])
    if W is not None:
        walsh8(W, 0)
        for m in range(8):
            for n in range(m, 8):
                cw = 3.0 ** (-(popc(m) + popc(n)) / 2)
                K[m, n] = K[m, n] + (cw * W[m ^ n] if popc(m) + popc(n) > 0 else W[m ^ n])
    for k in range(3):
        K = hadamard_axis(K, k)
    return K


def nodal_block(G):
    """The same block evaluated directly: at each Gauss point v_j = G grad(phi_j)
    (8 x 3 sums of 3 products) and K_ij += grad(phi_i) . v_j on the 36
    symmetric entries; grad(phi) at the points are constants."""
    t = 1.0 / math.sqrt(3.0)
    lin = lambda i, x: (1 + x) / 2 if i else (1 - x) / 2
    K = {}
    for g in range(8):
        tau = [t if (g >> k) & 1 else -t for k in range(3)]
        grad = [[(0.5 if (i >> a) & 1 else -0.5) * math.prod(lin((i >> k) & 1, tau[k]) for k in range(3) if k != a)
                 for a in range(3)] for i in range(8)]
        Gm = [[G[PAIRS.index(sym(a, b))][g] for b in range(3)] for a in range(3)]
        v = [[acc(Gm[a], grad[j]) for a in range(3)] for j in range(8)]
        for i in range(8):
            for j in range(i, 8):
                s = K.get((i, j), 0.0)
                for c in range(3):
                    s = s + grad[i][c] * v[j][c]
                K[i, j] = s
    return K


def test_modal_block_equals_the_direct_nodal_block_and_costs_less():
    rng = np.random.default_rng(7)
    Gv = np.empty((6, 8))
    for g in range(8):
        M = rng.standard_normal((3, 3))
        S = M @ M.T + 3 * np.eye(3)
        Gv[:, g] = [S[i, j] for i, j in PAIRS]
    Km = modal_block([leaves(Gv[ab] / 64.0) for ab in range(6)])
    Kn = nodal_block([leaves(Gv[ab]) for ab in range(6)])
    assert count(Km.values()) == 108 + 168 + 216
    assert count(Kn.values()) == 8 * (144 + 216)
    for ij in Kn:
        assert abs(Km[ij].v - Kn[ij].v) <= 1e-13 * max(abs(x.v) for x in Kn.values())
    # a block of the p = 1 stiffness: rows sum to zero
    assert all(abs(sum(Kn[sym(i, j)].v for j in range(8))) <= 1e-12 * abs(Kn[i, i].v) for i in range(8))


def lor_element_modal(p, corners, kappa, beta=None, fp64=True):
    """The LOR blocks of one element, each sub-hex's 8x8 block by 2x2x2 Gauss
    in the modal form: metric at the 8 points, its Walsh transforms, the modal
    block, the Hadamard sandwich.  fp64: the metric as the FP64 kernel forms
    it, adj(M) / sqrt(det M) with adj(M)_ab = r_a . r_b for the adjugate rows
    r_a of J and det M = (c_0 . r_0)^2; otherwise from the adjugate rows and
    1/det (the FP32 kernel).  Returns (blocks {(a, b, c): {(i, j): K_ij}}, all outputs)."""
    q, L = p + 2, 2 * p
    gll = oracle.gauss_lobatto(p)
    xg, wg = oracle.gauss_legendre(q)
    r = (gll[1:] - gll[:-1]) / 2
    mid = (gll[1:] + gll[:-1]) / 2
    xi = np.array([mid[a] + s * r[a] / math.sqrt(3.0) for a in range(p) for s in (-1, 1)])
    col = jacobian_columns(corner_leaves(corners), (1 - xi) / 2, (1 + xi) / 2)
    binof = np.array([int(np.sum(gll[1:-1] < x)) for x in xg])
    wn = np.array([wg[g] / wg[binof == binof[g]].sum() for g in range(q)])
    bw = leaves(wn)  # normalised Gauss weights per axis bin, read from a table
    bins = [[g for g in range(q) if binof[g] == a] for a in range(p)]
    kap = leaves(kappa)
    bet = leaves(beta) if beta is not None else None
    blocks, outs = {}, []
    for c in range(p):
        for b in range(p):
            for a in range(p):
                ks, bs = 0.0, 0.0
                for g2 in bins[c]:
                    for g1 in bins[b]:
                        w12 = bw[g1] * bw[g2]
                        for g0 in bins[a]:
                            w = w12 * bw[g0]
                            pt = g0 + q * (g1 + q * g2)
                            ks = ks + w * kap[pt]
                            if bet is not None:
                                bs = bs + w * bet[pt]
                k64 = ks * (1.0 / 64.0)
                ra, rb, rc = r[a], r[b], r[c]
                F = [k64 * rb * rc * (1 / ra), k64 * rc, k64 * rb, k64 * ra * rc * (1 / rb), k64 * ra,
                     k64 * ra * rb * (1 / rc)]
                bR = bs * (1.0 / 64.0) * ra * rb * rc if bet is not None else None
                G = [[None] * 8 for _ in range(6)]
                W = [None] * 8
                for g in range(8):
                    u0, u1, u2 = 2 * a + (g & 1), 2 * b + ((g >> 1) & 1), 2 * c + (g >> 2)
                    c0, c1, c2 = col[0][u1, u2], col[1][u0, u2], col[2][u0, u1]
                    if fp64:
                        R = [cross(c1, c2), cross(c2, c0), cross(c0, c1)]
                        dj = dot3(c0, R[0])
                        detM = dj * dj
                        adj = [dot3(R[i], R[j]) for i, j in PAIRS]
                        rr = rsqrt(detM)
                        if bR is not None:
                            W[g] = bR * (detM * rr)
                        for ab in range(6):
                            G[ab][g] = (F[ab] * rr) * adj[ab]
                    else:
                        A = [cross(c1, c2), cross(c2, c0), cross(c0, c1)]
                        det = dot3(c0, A[0])
                        rr = 1.0 / det
                        if bR is not None:
                            W[g] = bR * det
                        for ab, (i, j) in enumerate(PAIRS):
                            G[ab][g] = (F[ab] * rr) * dot3(A[i], A[j])
                K = modal_block(G, W if bR is not None else None, sums=fp64)
                blocks[a, b, c] = K
                outs.extend(K.values())
    return blocks, outs


def scatter(p, blocks):
    n = p + 1
    A = np.zeros((n ** 3, n ** 3))
    dof = lambda a, b, c, r: (a + (r & 1)) + n * ((b + ((r >> 1) & 1)) + n * (c + (r >> 2)))
    for (a, b, c), K in blocks.items():
        for i in range(8):
            for j in range(8):
                A[dof(a, b, c, i), dof(a, b, c, j)] += K[sym(i, j)].v
    return A


def dense(csr, n):
    rowptr, colidx, values = csr
    A = np.zeros((n, n))
    for i in range(n):
        A[i, colidx[rowptr[i]:rowptr[i + 1]]] = values[rowptr[i]:rowptr[i + 1]]
    return A


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_assemble_flops_evaluate_the_oracle_lor_matrix(p, fp64):
    q, n = p + 2, p + 1
    mesh, corners, kappa, _ = one_element(p, 50 + p)
    blocks, outs = lor_element_modal(p, corners, kappa, fp64=fp64)
    want = pm.assemble_flops_per_element(p) if fp64 else pm.assemble_f32_flops_per_element(p)
    assert count(outs) == want
    ref = dense(oracle.lor_assemble(mesh, p, q, kappa, dirichlet=False), n ** 3)
    np.testing.assert_allclose(scatter(p, blocks), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("p", [2, 3])
def test_assemble_reaction_flops_evaluate_the_oracle_lor_matrix(p, fp64):
    q, n = p + 2, p + 1
    mesh, corners, kappa, rng = one_element(p, 60 + p)
    beta = np.exp(rng.standard_normal(q ** 3))
    blocks, outs = lor_element_modal(p, corners, kappa, beta, fp64=fp64)
    if fp64:
        want = pm.assemble_flops_per_element(p) + pm.reaction_extra_assemble_flops_per_element(p)
    else:
        want = pm.assemble_f32_flops_per_element(p) + pm.reaction_extra_assemble_f32_flops_per_element(p)
    assert count(outs) == want
    ref = dense(oracle.lor_assemble(mesh, p, q, kappa, dirichlet=False, beta=beta), n ** 3)
    np.testing.assert_allclose(scatter(p, blocks), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_kernel_work_uses_the_per_element_counts():
    p, nel, ndof, nnz = 4, 10, 1000, 27000
    q = p + 2
    assert pm.kernel_work("setup", p, ndof, nel, nnz)[0] == nel * pm.setup_flops_per_element(p)
    assert pm.kernel_work("assemble", p, ndof, nel, nnz)[0] == nel * pm.assemble_flops_per_element(p)
    # x in, y read and written; D (48 bytes and a 4-byte scale) per Gauss point
    assert pm.kernel_work("apply", p, ndof, nel, nnz) == (nel * pm.apply_flops_per_element(p),
                                                           16 * ndof + 52 * nel * q ** 3)
    assert pm.kernel_work("backward", p, ndof, nel, nnz)[0] == nel * pm.backward_flops_per_element(p)
    # bytes: values once per nonzero and kappa once per Gauss point
    assert pm.kernel_work("assemble", p, ndof, nel, nnz, vbytes=4) == (nel * pm.assemble_f32_flops_per_element(p),
                                                                       4 * nnz + 8 * nel * q ** 3)


def _folded_forward(C, u, odd_table):
    """Even-odd folded y = C u for a table with C[q-1-g][n-1-i] = +-C[g][i]
    (+ for B_1D, - for d_1D), counting multiply-adds as the fixed-point
    kernels do."""
    q, n = C.shape
    nh, qh = n // 2, q // 2
    e = [u[i] + u[n - 1 - i] for i in range(nh)]
    o = [u[i] - u[n - 1 - i] for i in range(nh)]
    CE = [[(C[g][i] + C[g][n - 1 - i]) / 2 for i in range(nh)] for g in range(q)]
    CO = [[(C[g][i] - C[g][n - 1 - i]) / 2 for i in range(nh)] for g in range(q)]
    y, macs = np.zeros(q), 0
    for g in range(qh):
        a = 0.0
        if n & 1:
            a += C[g][n // 2] * u[n // 2]
            macs += 1
        a += sum(CE[g][i] * e[i] for i in range(nh))
        b = sum(CO[g][i] * o[i] for i in range(nh))
        macs += 2 * nh
        y[g], y[q - 1 - g] = (b + a, b - a) if odd_table else (a + b, a - b)
    if q & 1:
        y[q // 2] = sum((CO if odd_table else CE)[q // 2][i] * (o if odd_table else e)[i] for i in range(nh))
        macs += nh
    return y, macs


def _folded_transpose(C, v, odd_table):
    """y = C^T v, folded over the q points, with its multiply-add count."""
    q, n = C.shape
    nh, qh = n // 2, q // 2
    e = [v[g] + v[q - 1 - g] for g in range(qh)]
    o = [v[g] - v[q - 1 - g] for g in range(qh)]
    CE = [[(C[g][i] + C[g][n - 1 - i]) / 2 for i in range(n)] for g in range(q)]
    CO = [[(C[g][i] - C[g][n - 1 - i]) / 2 for i in range(n)] for g in range(q)]
    y, macs = np.zeros(n), 0
    for i in range(nh):
        a1 = a2 = 0.0
        if q & 1:
            if odd_table:
                a2 += C[q // 2][i] * v[q // 2]
            else:
                a1 += C[q // 2][i] * v[q // 2]
            macs += 1
        for g in range(qh):
            if odd_table:
                a1 += CE[g][i] * o[g]
                a2 += CO[g][i] * e[g]
            else:
                a1 += CE[g][i] * e[g]
                a2 += CO[g][i] * o[g]
            macs += 2
        y[i], y[n - 1 - i] = a1 + a2, a1 - a2
    if n & 1:
        y[n // 2] = sum(C[g][n // 2] * (o if odd_table else e)[g] for g in range(qh))
        macs += qh
    return y, macs


@pytest.mark.parametrize("p", range(1, 11))
def test_folded_contraction_counts(p):
    """The fixed-point kernels' multiply-add counts per 1D contraction: an
    emulation of the folded contraction reproduces the dense product with
    B_1D- and d_1D-symmetric tables and takes exactly the counted
    multiply-adds."""
    n, q = p + 1, p + 2
    rng = np.random.default_rng(p)
    R = rng.standard_normal((q, n))
    Bt = R + R[::-1, ::-1]  # B[q-1-g][n-1-i] = B[g][i]
    Dt = R - R[::-1, ::-1]  # d[q-1-g][n-1-i] = -d[g][i]
    u, v = rng.standard_normal(n), rng.standard_normal(q)
    for C, odd in ((Bt, False), (Dt, True)):
        y, macs = _folded_forward(C, u, odd)
        np.testing.assert_allclose(y, C @ u, rtol=0, atol=1e-12)
        assert macs == pm.folded_forward_macs(p)
        y, macs = _folded_transpose(C, v, odd)
        np.testing.assert_allclose(y, C.T @ v, rtol=0, atol=1e-12)
        assert macs == pm.folded_transpose_macs(p, 1)
    assert pm.folded_transpose_macs(p, 2) == 2 * pm.folded_transpose_macs(p, 1)
    # per element: the stages' line counts times these, plus 9 (10) per Gauss point
    f, t1, t2 = pm.folded_forward_macs(p), pm.folded_transpose_macs(p, 1), pm.folded_transpose_macs(p, 2)
    fwd = 2 * n * n * f + 3 * n * q * f + 3 * q * q * f
    tr = q * q * 3 * t1 + n * q * (t1 + t2) + n * n * t2
    assert pm.apply_fixed_macs_per_element(p) == fwd + 9 * q ** 3 + tr
    assert pm.backward_fixed_macs_per_element(p) == 2 * fwd + 12 * q ** 3 + tr
    assert pm.apply_fixed_macs_per_element(p, mass=True) == fwd + q * q * f + 10 * q ** 3 + tr - q * q * t1 + q * q * t2
