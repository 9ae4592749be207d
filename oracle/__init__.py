"""FP64 CPU oracle for LOR preconditioning of high-order H1 diffusion.

TEST INFRASTRUCTURE ONLY.  This package is the correctness reference for the
CUDA library in ``paper_2210_12253_gb300``; only ``tests/``, the smoke check
in ``__graft_entry__.py`` and the ``cpu_baseline`` / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA path.  Every
routine is a thin numpy/ctypes wrapper around ``lor_oracle.c``, which
computes each quantity from its plain definition (see that file's header for
the conventions and the readings R1-R7 of the paper).

Parity status: every function is pinned by tests/test_oracle_*.py except the
3D spectral-equivalence constant, for which the paper gives no number (the
tests check only that it stays bounded as p grows: "parity unpinned" beyond
that property).
"""
import ctypes as C
import os

import numpy as np

from .build import build_oracle

_lib = None


def lib():
    """The oracle library; LOR_ORACLE_LIB names another build of the same
    source (the mutation tests load deliberately broken copies this way)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("LOR_ORACLE_LIB") or build_oracle())
        _declare(_lib)
    return _lib


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _declare(L):
    i, i64, d, vp = C.c_int, C.c_int64, C.c_double, C.c_void_p
    sig = {
        "orc_gauss_legendre": (i, [i, _dp, _dp]),
        "orc_gauss_lobatto": (i, [i, _dp]),
        "orc_lagrange": (None, [i, _dp, d, _dp, _dp]),
        "orc_basis_1d": (i, [i, i, _dp, _dp]),
        "orc_geometry": (i, [i, i, i, _dp, i, _dp, _dp]),
        "orc_dof_coordinates": (i, [i, i, i, _dp, i, _dp]),
        "orc_ho_apply": (i, [i, i, i, _dp, i, i, _dp, vp, _dp, _dp, i]),
        "orc_ho_apply_backward": (i, [i, i, i, _dp, i, i, _dp, vp, _dp, _dp, vp, vp]),
        "orc_load_vector": (i, [i, i, i, _dp, i, i, vp, _dp]),
        "orc_dense_general": (i, [i64, i, i, _dp, _i64p, _dp, vp, i64, _dp]),
        "orc_lor_kappa_sub": (i, [i, i, i64, _dp, _dp]),
        "orc_lor_assemble": (vp, [i, i, i, _dp, i, i, _dp, vp, i, C.POINTER(i)]),
        "orc_lor_assemble_general": (vp, [i64, i, i, _dp, _i64p, i64, vp, _dp, vp, i, C.POINTER(i)]),
        "orc_csr_nnz": (i64, [vp]),
        "orc_csr_n": (i64, [vp]),
        "orc_csr_copy": (None, [vp, _i64p, _i64p, _dp]),
        "orc_csr_free": (None, [vp]),
        "orc_lor_rows": (i, [i, i, i, _dp, i, i, _dp, vp, i, i64, _i64p, i, _i32p, _i64p, _dp]),
        "orc_lor_edge_count": (i64, [i, i, i, i]),
        "orc_discrete_gradient": (i, [i, i, i, i, _i64p, _i64p, _dp]),
        "orc_csr_spmv": (None, [i64, _i64p, _i64p, _dp, _dp, _dp]),
        "orc_csr_diagonal": (None, [i64, _i64p, _i64p, _dp, _dp]),
        "orc_power_lambda_max": (d, [i64, _i64p, _i64p, _dp, _dp, i]),
        "orc_chebyshev": (None, [i64, _i64p, _i64p, _dp, vp, i, d, d, _dp, _dp]),
        "orc_pcg": (i, [i, i, i, _dp, i, i, _dp, vp, _i64p, _i64p, _dp, i, i, d, d,
                        _dp, _dp, d, i, C.POINTER(i), C.POINTER(d)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


OK, EINVAL, EGEOM, ENOMEM, ENOCONV = 0, 1, 2, 3, 5


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("oracle %s failed with status %d" % (what, code))
        self.code = code


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _opt(a, n=None):
    """Optional coefficient array (None stays None): contiguous f64, flattened."""
    if a is None:
        return None
    a = _f64(a).ravel()
    if n is not None:
        assert a.size == n
    return a


# ---------------------------------------------------------------- 1D rules
def gauss_legendre(q):
    x, w = np.zeros(q), np.zeros(q)
    _check(lib().orc_gauss_legendre(q, x, w), "gauss_legendre")
    return x, w


def gauss_lobatto(p):
    x = np.zeros(p + 1)
    _check(lib().orc_gauss_lobatto(p, x), "gauss_lobatto")
    return x


def lagrange(nodes, t):
    nodes = _f64(nodes)
    phi, dphi = np.zeros(len(nodes)), np.zeros(len(nodes))
    lib().orc_lagrange(len(nodes), nodes, float(t), phi, dphi)
    return phi, dphi


def basis_1d(p, q):
    B, D = np.zeros((q, p + 1)), np.zeros((q, p + 1))
    _check(lib().orc_basis_1d(p, q, B, D), "basis_1d")
    return B, D


# ---------------------------------------------------------------- mesh
class Mesh:
    """Structured hex mesh of the unit cube: nex x ney x nez elements with
    vertex coordinates V[(nex+1)(ney+1)(nez+1), 3] (lexicographic, x fastest)."""

    def __init__(self, nex, ney, nez, V):
        self.nex, self.ney, self.nez = int(nex), int(ney), int(nez)
        self.V = _f64(V).reshape(-1, 3)
        assert self.V.shape[0] == (nex + 1) * (ney + 1) * (nez + 1)

    @property
    def nel(self):
        return self.nex * self.ney * self.nez

    def ndof(self, p):
        return (self.nex * p + 1) * (self.ney * p + 1) * (self.nez * p + 1)

    def args(self):
        return (self.nex, self.ney, self.nez, self.V)


def geometry(mesh, q):
    nq3 = q ** 3
    detJ = np.zeros((mesh.nel, nq3))
    G = np.zeros((mesh.nel, nq3, 6))
    _check(lib().orc_geometry(*mesh.args(), q, detJ, G), "geometry")
    return detJ, G


def dof_coordinates(mesh, p):
    xyz = np.zeros((mesh.ndof(p), 3))
    _check(lib().orc_dof_coordinates(*mesh.args(), p, xyz), "dof_coordinates")
    return xyz


# ---------------------------------------------------------------- HO operator
def ho_apply(mesh, p, q, kappa, x, dirichlet=True, beta=None):
    """y = A_p x; beta (reaction coefficient at the Gauss points) adds the mass term."""
    y = np.zeros(mesh.ndof(p))
    b = _opt(beta, mesh.nel * q ** 3)
    _check(lib().orc_ho_apply(*mesh.args(), p, q, _f64(kappa).ravel(), _ptr(b), _f64(x), y, int(dirichlet)),
           "ho_apply")
    return y


def ho_apply_backward(mesh, p, q, kappa, x, gy, want_gx=True, want_gkappa=True, beta=None):
    gx = np.zeros(mesh.ndof(p)) if want_gx else None
    gk = np.zeros((mesh.nel, q ** 3)) if want_gkappa else None
    b = _opt(beta, mesh.nel * q ** 3)
    _check(lib().orc_ho_apply_backward(*mesh.args(), p, q, _f64(kappa).ravel(), _ptr(b), _f64(x), _f64(gy),
                                       _ptr(gx), _ptr(gk)), "ho_apply_backward")
    return gx, gk


def load_vector(mesh, p, q, f=None):
    b = np.zeros(mesh.ndof(p))
    fa = None if f is None else _f64(f).ravel()
    _check(lib().orc_load_vector(*mesh.args(), p, q, _ptr(fa), b), "load_vector")
    return b


def dense_general(corners, dofs, kappa, p, q, N, beta=None):
    """Brute-force dense stiffness (+ beta-weighted mass) matrix on a general hex mesh."""
    corners = _f64(corners).reshape(-1, 8, 3)
    nel = corners.shape[0]
    dofs = np.ascontiguousarray(dofs, dtype=np.int64).reshape(nel, (p + 1) ** 3)
    kappa = _f64(kappa).reshape(nel, q ** 3)
    b = _opt(beta, nel * q ** 3)
    A = np.zeros((N, N))
    _check(lib().orc_dense_general(nel, p, q, corners, dofs, kappa, _ptr(b), N, A), "dense_general")
    return A


# ---------------------------------------------------------------- LOR
def lor_kappa_sub(p, q, kappa):
    kappa = _f64(kappa)
    nel = kappa.size // q ** 3
    ks = np.zeros((nel, p ** 3))
    _check(lib().orc_lor_kappa_sub(p, q, nel, kappa.ravel(), ks), "lor_kappa_sub")
    return ks


def lor_assemble(mesh, p, q, kappa, dirichlet=True, beta=None):
    """Full LOR CSR (rowptr int64, colidx int64, values f64); beta adds the LOR mass blocks."""
    st = C.c_int(0)
    b = _opt(beta, mesh.nel * q ** 3)
    h = lib().orc_lor_assemble(*mesh.args(), p, q, _f64(kappa).ravel(), _ptr(b), int(dirichlet), C.byref(st))
    if not h:
        raise OracleError(st.value, "lor_assemble")
    try:
        _check(st.value, "lor_assemble")
        n, nnz = lib().orc_csr_n(h), lib().orc_csr_nnz(h)
        rowptr, colidx, values = np.zeros(n + 1, np.int64), np.zeros(nnz, np.int64), np.zeros(nnz)
        lib().orc_csr_copy(h, rowptr, colidx, values)
    finally:
        lib().orc_csr_free(h)
    return rowptr, colidx, values


def _csr_from_handle(h, st, what):
    if not h:
        raise OracleError(st.value, what)
    try:
        _check(st.value, what)
        n, nnz = lib().orc_csr_n(h), lib().orc_csr_nnz(h)
        rowptr, colidx, values = np.zeros(n + 1, np.int64), np.zeros(nnz, np.int64), np.zeros(nnz)
        lib().orc_csr_copy(h, rowptr, colidx, values)
    finally:
        lib().orc_csr_free(h)
    return rowptr, colidx, values


def lor_assemble_general(corners, dofs, N, p, q, kappa, ess=None, dirichlet=True, beta=None):
    """Full LOR CSR of a general conforming hex mesh (corners [nel][8][3],
    element-to-DOF map [nel][(p+1)^3], essential mask uint8[N] or None)."""
    corners = _f64(corners).reshape(-1, 8, 3)
    nel = corners.shape[0]
    dofs = np.ascontiguousarray(dofs, dtype=np.int64).reshape(nel, (p + 1) ** 3)
    e = None if ess is None else np.ascontiguousarray(ess, dtype=np.uint8).reshape(N)
    b = _opt(beta, nel * q ** 3)
    st = C.c_int(0)
    h = lib().orc_lor_assemble_general(nel, p, q, corners, dofs, N, None if e is None else e.ctypes.data_as(C.c_void_p),
                                       _f64(kappa).ravel(), _ptr(b), int(dirichlet), C.byref(st))
    return _csr_from_handle(h, st, "lor_assemble_general")


def lor_rows(mesh, p, q, kappa, rows, dirichlet=True, cap=64, beta=None):
    """Selected rows of the LOR matrix, each computed from its own sub-hexes.
    Returns (counts int32[n], cols int64[n, cap], vals f64[n, cap])."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = rows.size
    counts = np.zeros(n, np.int32)
    cols = np.zeros((n, cap), np.int64)
    vals = np.zeros((n, cap))
    b = _opt(beta, mesh.nel * q ** 3)
    _check(lib().orc_lor_rows(*mesh.args(), p, q, _f64(kappa).ravel(), _ptr(b), int(dirichlet), n, rows, cap,
                              counts, cols, vals), "lor_rows")
    return counts, cols, vals


# ---------------------------------------------------------------- H(curl) topology
def discrete_gradient(nex, ney, nez, p):
    """LOR vertex-to-edge discrete gradient as CSR (rowptr, colidx int64, values)."""
    ne = lib().orc_lor_edge_count(nex, ney, nez, p)
    rowptr, colidx, values = np.zeros(ne + 1, np.int64), np.zeros(2 * ne, np.int64), np.zeros(2 * ne)
    _check(lib().orc_discrete_gradient(nex, ney, nez, p, rowptr, colidx, values), "discrete_gradient")
    return rowptr, colidx, values


# ---------------------------------------------------------------- sparse / solver
def _csr(rowptr, colidx, values):
    return (np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(colidx, np.int64), _f64(values))


def csr_spmv(rowptr, colidx, values, x):
    rp, ci, v = _csr(rowptr, colidx, values)
    y = np.zeros(rp.size - 1)
    lib().orc_csr_spmv(rp.size - 1, rp, ci, v, _f64(x), y)
    return y


def csr_diagonal(rowptr, colidx, values):
    rp, ci, v = _csr(rowptr, colidx, values)
    d = np.zeros(rp.size - 1)
    lib().orc_csr_diagonal(rp.size - 1, rp, ci, v, d)
    return d


def power_lambda_max(rowptr, colidx, values, v0, iters):
    rp, ci, v = _csr(rowptr, colidx, values)
    return lib().orc_power_lambda_max(rp.size - 1, rp, ci, v, _f64(v0), int(iters))


def chebyshev(rowptr, colidx, values, r, k, lo, hi, diag=None):
    rp, ci, v = _csr(rowptr, colidx, values)
    z = np.zeros(rp.size - 1)
    dg = None if diag is None else _f64(diag)
    lib().orc_chebyshev(rp.size - 1, rp, ci, v, _ptr(dg), int(k), float(lo), float(hi), _f64(r), z)
    return z


PRECOND_NONE, PRECOND_JACOBI, PRECOND_CHEB = 0, 1, 2


def pcg(mesh, p, q, kappa, csr, b, rtol, maxit, precond=PRECOND_CHEB, cheb_k=3, lo=0.0, hi=1.0,
        raise_on_noconv=True, beta=None):
    """Returns (x, iterations, final relative residual, status)."""
    rp, ci, v = _csr(*csr)
    x = np.zeros(mesh.ndof(p))
    it, rel = C.c_int(0), C.c_double(0.0)
    bt = _opt(beta, mesh.nel * q ** 3)
    rc = lib().orc_pcg(*mesh.args(), p, q, _f64(kappa).ravel(), _ptr(bt), rp, ci, v, int(precond), int(cheb_k),
                       float(lo), float(hi), _f64(b), x, float(rtol), int(maxit), C.byref(it), C.byref(rel))
    if rc not in (OK, ENOCONV) or (raise_on_noconv and rc != OK):
        raise OracleError(rc, "pcg")
    return x, it.value, rel.value, rc
