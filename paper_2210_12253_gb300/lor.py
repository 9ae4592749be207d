"""Thin Python binding of liblor (include/lor.h).

Argument marshalling only: every step runs in the CUDA library.  Tensors are
PyTorch CUDA tensors (device memory); the stream is PyTorch's current stream.
There is no CPU fallback: if liblor.so is missing or no GPU is present the
calls raise.
"""
import ctypes as C
import os

import torch

from .build import LIB

LOR_OK, LOR_EINVAL, LOR_EGEOM, LOR_ENOMEM, LOR_ECUDA, LOR_ENOCONV, LOR_ETIMEOUT, LOR_ESTATE = 0, 1, 2, 3, 4, 5, 6, 7
LOR_F64, LOR_F32 = 0, 1
LOR_PRECOND_NONE, LOR_PRECOND_JACOBI, LOR_PRECOND_CHEB = 0, 1, 2
LOR_IR_RESTART, LOR_IR_REPLACE = 0, 1
LOR_MAX_P = 10
LOR_TEST_EXPIRE_WAITS, LOR_TEST_UNSTAGED_CSR = 1, 2

EXPORTED = [
    "lor_last_error", "lor_create", "lor_destroy", "lor_sizes", "lor_set_coefficient", "lor_check",
    "lor_build_pattern", "lor_assemble", "lor_apply", "lor_apply_backward", "lor_load_vector", "lor_spmv",
    "lor_precond_setup", "lor_precond_apply", "lor_pcg_solve", "lor_launch_count",
    "lor_precond_apply_noalloc", "lor_set_reaction", "lor_lor_mesh", "lor_assemble_unstructured",
    "lor_discrete_gradient", "lor_vertex_coordinates", "lor_create_general", "lor_apply_f32",
    "lor_pcg_solve_ir", "lor_set_test_hooks",
]


class lor_config(C.Structure):
    _fields_ = [("p", C.c_int32), ("nex", C.c_int32), ("ney", C.c_int32), ("nez", C.c_int32)]


class LORError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("liblor error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load_library(path=LIB):
    """Load liblor.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblor.so not found at %s: build it with paper_2210_12253_gb300.build.build() "
                           "(there is no CPU fallback)" % path)
    L = C.CDLL(path)
    vp, i, d, i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    L.lor_last_error.restype = C.c_char_p
    L.lor_last_error.argtypes = [vp]
    L.lor_create.restype = i
    L.lor_create.argtypes = [C.POINTER(vp), C.POINTER(lor_config), vp, vp]
    L.lor_create_general.restype = i
    L.lor_create_general.argtypes = [C.POINTER(vp), i, i64, i64, vp, vp, vp, vp]
    L.lor_destroy.restype = i
    L.lor_destroy.argtypes = [vp]
    L.lor_sizes.restype = i
    L.lor_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    L.lor_set_coefficient.restype = i
    L.lor_set_coefficient.argtypes = [vp, vp, vp]
    L.lor_set_reaction.restype = i
    L.lor_set_reaction.argtypes = [vp, vp, vp]
    L.lor_discrete_gradient.restype = i
    L.lor_discrete_gradient.argtypes = [vp, vp, vp, vp, C.POINTER(i64), vp]
    L.lor_vertex_coordinates.restype = i
    L.lor_vertex_coordinates.argtypes = [vp, vp, vp]
    L.lor_lor_mesh.restype = i
    L.lor_lor_mesh.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.lor_assemble_unstructured.restype = i
    L.lor_assemble_unstructured.argtypes = [vp, i64, vp, vp, vp, vp, i64, i64, vp, vp, vp, vp, i, vp]
    L.lor_check.restype = i
    L.lor_check.argtypes = [vp, vp]
    L.lor_set_test_hooks.restype = i
    L.lor_set_test_hooks.argtypes = [vp, C.c_uint]
    L.lor_build_pattern.restype = i
    L.lor_build_pattern.argtypes = [vp, vp, vp, vp]
    L.lor_assemble.restype = i
    L.lor_assemble.argtypes = [vp, vp, i, vp]
    L.lor_apply.restype = i
    L.lor_apply.argtypes = [vp, vp, vp, vp]
    L.lor_apply_f32.restype = i
    L.lor_apply_f32.argtypes = [vp, vp, vp, vp]
    L.lor_pcg_solve_ir.restype = i
    L.lor_pcg_solve_ir.argtypes = [vp, vp, vp, d, d, i, i, C.POINTER(i), C.POINTER(i), C.POINTER(d), vp]
    L.lor_apply_backward.restype = i
    L.lor_apply_backward.argtypes = [vp, vp, vp, vp, vp, vp]
    L.lor_load_vector.restype = i
    L.lor_load_vector.argtypes = [vp, vp, vp, vp]
    L.lor_spmv.restype = i
    L.lor_spmv.argtypes = [vp, i, vp, vp, vp]
    L.lor_precond_setup.restype = i
    L.lor_precond_setup.argtypes = [vp, i, i, i, d, d, d, i, vp, C.POINTER(d), vp]
    L.lor_precond_apply.restype = i
    L.lor_precond_apply.argtypes = [vp, vp, vp, vp]
    L.lor_precond_apply_noalloc.restype = i
    L.lor_precond_apply_noalloc.argtypes = [vp, vp, vp, vp]
    L.lor_launch_count.restype = i
    L.lor_launch_count.argtypes = [C.POINTER(i64)]
    L.lor_pcg_solve.restype = i
    L.lor_pcg_solve.argtypes = [vp, vp, vp, d, i, C.POINTER(i), C.POINTER(d), vp]
    _lib = L
    return L


def launch_count():
    """Kernels liblor has launched in this process."""
    n = C.c_int64(0)
    load_library().lor_launch_count(C.byref(n))
    return n.value


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype, numel, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    return t


def _dtype_code(dtype):
    if dtype in (torch.float64, "f64", LOR_F64):
        return LOR_F64, torch.float64
    if dtype in (torch.float32, "f32", LOR_F32):
        return LOR_F32, torch.float32
    raise ValueError("dtype must be float64 or float32")


class LOR:
    """One LOR discretisation: order-p H1 space on a structured hex mesh of
    the unit cube (nex x ney x nez trilinear elements, vertices given), its
    high-order operator, LOR matrix, preconditioner and PCG solver."""

    def __init__(self, p, nex, ney, nez, vertices):
        self._lib = load_library()
        self.p, self.nex, self.ney, self.nez = int(p), int(nex), int(ney), int(nez)
        nv = (nex + 1) * (ney + 1) * (nez + 1)
        _dev(vertices, torch.float64, 3 * nv, "vertices")
        self.device = vertices.device
        cfg = lor_config(self.p, self.nex, self.ney, self.nez)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.lor_create(C.byref(h), C.byref(cfg), _ptr(vertices), _stream())
        if rc != LOR_OK:
            raise LORError(rc, self._lib.lor_last_error(None).decode())
        self._h = h
        self._sizes()

    def _sizes(self):
        n, z, e, q = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        self._call("lor_sizes", C.byref(n), C.byref(z), C.byref(e), C.byref(q), stream=False)
        self.ndof, self.nnz, self.nel, self.nqpt = n.value, z.value, e.value, q.value
        self.q = self.p + 2
        self._kappa_key = None

    @classmethod
    def general(cls, p, corners, elem_dofs, ndof, ess=None):
        """A context on a general conforming hex mesh in element-restriction
        form: corners [nel, 8, 3] f64, elem_dofs [nel, (p+1)^3] int64 (local
        node i + n(j + n k) -> global DOF), ess uint8[ndof] or None."""
        self = cls.__new__(cls)
        self._lib = load_library()
        self._h = None
        self.p = int(p)
        nel = int(corners.numel() // 24)
        self.nex = self.ney = self.nez = None
        _dev(corners, torch.float64, 24 * nel, "corners")
        _dev(elem_dofs, torch.int64, nel * (self.p + 1) ** 3, "elem_dofs")
        if ess is not None:
            _dev(ess, torch.uint8, int(ndof), "ess")
        self.device = corners.device
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.lor_create_general(C.byref(h), self.p, nel, int(ndof), _ptr(corners), _ptr(elem_dofs),
                                              _ptr(ess), _stream())
        if rc != LOR_OK:
            raise LORError(rc, self._lib.lor_last_error(None).decode())
        self._h = h
        self._sizes()
        return self

    # ------------------------------------------------------------------ plumbing
    def _call(self, name, *args, stream=True):
        if self._h is None:
            raise RuntimeError("LOR context already destroyed")
        extra = (_stream(),) if stream else ()
        rc = getattr(self._lib, name)(self._h, *args, *extra)
        if rc != LOR_OK:
            raise LORError(rc, self._lib.lor_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.lor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new(self, n, dtype=torch.float64):
        return torch.empty(n, dtype=dtype, device=self.device)

    # ------------------------------------------------------------------ steps
    def set_coefficient(self, kappa, check=False):
        """Step S1.1: D = kappa w detJ J^-1 J^-T at every Gauss point."""
        _dev(kappa, torch.float64, self.nqpt, "kappa")
        self._call("lor_set_coefficient", _ptr(kappa))
        self._kappa_key = (kappa.data_ptr(), kappa._version)
        if check:
            self.check()

    def set_reaction(self, beta, check=False):
        """Reaction term beta u of the definite Helmholtz operator (beta at
        the Gauss points, like kappa); None switches it off.  Re-assemble the
        LOR matrix (and the preconditioner) afterwards."""
        if beta is not None:
            _dev(beta, torch.float64, self.nqpt, "beta")
        self._call("lor_set_reaction", _ptr(beta))
        if check:
            self.check()

    def check(self):
        self._call("lor_check")

    def set_test_hooks(self, flags):
        """Test hooks (LOR_TEST_EXPIRE_WAITS: the TMA-staged kernels treat
        their first bounded wait as expired; LOR_TEST_UNSTAGED_CSR: the
        explicit-CSR kernel reads every tile from global memory); 0 clears
        them."""
        self._call("lor_set_test_hooks", C.c_uint(flags), stream=False)

    def build_pattern(self, rowptr=None, colidx=None):
        """Step S1.2 A2: CSR pattern (rowptr int64[N+1], colidx int32[nnz])."""
        if rowptr is None:
            rowptr = self._new(self.ndof + 1, torch.int64)
            colidx = self._new(self.nnz, torch.int32)
        _dev(rowptr, torch.int64, self.ndof + 1, "rowptr")
        _dev(colidx, torch.int32, self.nnz, "colidx")
        self._call("lor_build_pattern", _ptr(rowptr), _ptr(colidx))
        return rowptr, colidx

    def build_pattern_internal(self):
        self._call("lor_build_pattern", None, None)

    def assemble(self, dtype=torch.float64, out=None):
        """Step S1.2 A1+A4: LOR matrix values in `dtype` into `out` (new tensor if None)."""
        code, tdt = _dtype_code(dtype)
        if out is None:
            out = self._new(self.nnz, tdt)
        _dev(out, tdt, self.nnz, "values")
        self._call("lor_assemble", _ptr(out), code)
        return out

    def assemble_internal(self, dtype=torch.float64):
        """Assemble into the context's own matrix (used by the preconditioner)."""
        code, _ = _dtype_code(dtype)
        self._call("lor_assemble", None, code)

    def edge_count(self):
        ne = C.c_int64(0)
        self._call("lor_discrete_gradient", None, None, None, C.byref(ne))
        return ne.value

    def discrete_gradient(self):
        """LOR vertex-to-edge discrete gradient (Algorithm 1): (rowptr int64,
        colidx int32, values f64) CSR with two entries per edge."""
        ne = self.edge_count()
        rowptr = torch.empty(ne + 1, dtype=torch.int64, device=self.device)
        colidx = torch.empty(2 * ne, dtype=torch.int32, device=self.device)
        values = self._new(2 * ne)
        self._call("lor_discrete_gradient", _ptr(rowptr), _ptr(colidx), _ptr(values), None)
        return rowptr, colidx, values

    def vertex_coordinates(self):
        """Deduplicated LOR vertex coordinates [N, 3]."""
        xyz = self._new(3 * self.ndof).reshape(self.ndof, 3)
        self._call("lor_vertex_coordinates", _ptr(xyz))
        return xyz

    def lor_mesh(self, with_beta=False):
        """The LOR mesh as a general hex mesh: (corners [nsub, 8, 3] f64,
        dofs [nsub, 8] int64, kappa_s [nsub], beta_s [nsub] or None,
        essential mask uint8[N])."""
        nsub = self.nel * self.p ** 3
        corners = self._new(nsub * 24).reshape(nsub, 8, 3)
        dofs = torch.empty((nsub, 8), dtype=torch.int64, device=self.device)
        ks = self._new(nsub)
        bs = self._new(nsub) if with_beta else None
        ess = torch.empty(self.ndof, dtype=torch.uint8, device=self.device)
        self._call("lor_lor_mesh", _ptr(corners), _ptr(dofs), _ptr(ks), _ptr(bs), _ptr(ess))
        return corners, dofs, ks, bs, ess

    def assemble_unstructured(self, corners, dofs, kappa_sub, rowptr, colidx, n, beta_sub=None, ess=None,
                              dtype=torch.float64, out=None):
        """Unstructured Q1 assembly of a general hex mesh (E-vectors) into the
        CSR pattern (rowptr int64[n+1], colidx int32[nnz]); the comparator of
        the macro-element assembly."""
        code, tdt = _dtype_code(dtype)
        nsub = int(kappa_sub.numel())
        nnz = int(colidx.numel())
        _dev(corners, torch.float64, nsub * 24, "corners")
        _dev(dofs, torch.int64, nsub * 8, "dofs")
        _dev(kappa_sub, torch.float64, nsub, "kappa_sub")
        if beta_sub is not None:
            _dev(beta_sub, torch.float64, nsub, "beta_sub")
        _dev(rowptr, torch.int64, n + 1, "rowptr")
        _dev(colidx, torch.int32, nnz, "colidx")
        if ess is not None:
            _dev(ess, torch.uint8, n, "ess")
        if out is None:
            out = self._new(nnz, tdt)
        _dev(out, tdt, nnz, "values")
        self._call("lor_assemble_unstructured", nsub, _ptr(corners), _ptr(dofs), _ptr(kappa_sub), _ptr(beta_sub),
                   n, nnz, _ptr(rowptr), _ptr(colidx), _ptr(ess), _ptr(out), code)
        return out

    def apply(self, x, out=None):
        """Step S2.1: y = A_p x (FP64, Dirichlet rows return x)."""
        _dev(x, torch.float64, self.ndof, "x")
        y = self._new(self.ndof) if out is None else _dev(out, torch.float64, self.ndof, "out")
        self._call("lor_apply", _ptr(x), _ptr(y))
        return y

    def apply_f32(self, x, out=None):
        """y = A_p x with FP32 arithmetic inside the kernel (FP64 x and y); the
        operator of the refinement's inner solves."""
        _dev(x, torch.float64, self.ndof, "x")
        y = self._new(self.ndof) if out is None else _dev(out, torch.float64, self.ndof, "out")
        self._call("lor_apply_f32", _ptr(x), _ptr(y))
        return y

    def apply_backward(self, x, gy, want_gx=True, want_gkappa=True, gx_out=None, gk_out=None):
        """(A_p gy, d(gy^T A_p x)/d kappa)."""
        _dev(gy, torch.float64, self.ndof, "gy")
        if want_gkappa:
            _dev(x, torch.float64, self.ndof, "x")
        gx = gk = None
        if want_gx:
            gx = self._new(self.ndof) if gx_out is None else _dev(gx_out, torch.float64, self.ndof, "gx_out")
        if want_gkappa:
            gk = self._new(self.nqpt) if gk_out is None else _dev(gk_out, torch.float64, self.nqpt, "gk_out")
        self._call("lor_apply_backward", _ptr(x if want_gkappa else None), _ptr(gy), _ptr(gx), _ptr(gk))
        return gx, gk

    def load_vector(self, f=None):
        """b_i = int f phi_i (f at Gauss points, or f = 1); b = 0 on the boundary."""
        if f is not None:
            _dev(f, torch.float64, self.nqpt, "f")
        b = self._new(self.ndof)
        self._call("lor_load_vector", _ptr(f), _ptr(b))
        return b

    def spmv(self, x, dtype=torch.float64):
        code, _ = _dtype_code(dtype)
        _dev(x, torch.float64, self.ndof, "x")
        y = self._new(self.ndof)
        self._call("lor_spmv", code, _ptr(x), _ptr(y))
        return y

    def precond_setup(self, kind="cheb", dtype=torch.float32, degree=3, lo_ratio=1.0 / 30.0, hi_ratio=1.1,
                      lambda_max=None, power_iters=20, v0=None):
        """Preconditioner B_h on the context's LOR matrix; returns lambda_max."""
        k = {"none": LOR_PRECOND_NONE, "jacobi": LOR_PRECOND_JACOBI, "cheb": LOR_PRECOND_CHEB}[kind]
        code, _ = _dtype_code(dtype)
        if v0 is not None:
            _dev(v0, torch.float64, self.ndof, "v0")
        lam = C.c_double(0.0)
        self._call("lor_precond_setup", k, code, int(degree), float(lo_ratio), float(hi_ratio),
                   float(lambda_max) if lambda_max else 0.0, int(power_iters), _ptr(v0), C.byref(lam))
        return lam.value

    def precond_apply(self, r, out=None):
        _dev(r, torch.float64, self.ndof, "r")
        z = self._new(self.ndof) if out is None else _dev(out, torch.float64, self.ndof, "out")
        self._call("lor_precond_apply", _ptr(r), _ptr(z))
        return z

    def precond_apply_noalloc(self, r, out):
        """z = B_h r like precond_apply, with no device allocation in the call:
        the output must be given and the smoother's work vectors come from a
        static device array inside the library (see include/lor.h)."""
        _dev(r, torch.float64, self.ndof, "r")
        _dev(out, torch.float64, self.ndof, "out")
        self._call("lor_precond_apply_noalloc", _ptr(r), _ptr(out))
        return out

    def pcg_solve(self, b, rtol=1e-8, maxit=1000, x=None, raise_on_noconv=True):
        """Section 3 step S2: PCG for A_p x = b.  Returns (x, iterations, rel. residual)."""
        _dev(b, torch.float64, self.ndof, "b")
        x = self._new(self.ndof) if x is None else _dev(x, torch.float64, self.ndof, "x")
        it, rel = C.c_int(0), C.c_double(0.0)
        rc = self._lib.lor_pcg_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), C.byref(it),
                                     C.byref(rel), _stream())
        if rc != LOR_OK and (rc != LOR_ENOCONV or raise_on_noconv):
            raise LORError(rc, self._lib.lor_last_error(self._h).decode())
        return x, it.value, rel.value

    def pcg_solve_ir(self, b, rtol=1e-8, inner_rtol=1e-4, maxit=20000, x=None, raise_on_noconv=True,
                     scheme="replace"):
        """Mixed-precision iterative refinement: FP64 outer residuals, inner PCG
        iterations with the FP32 operator; scheme "restart" (a fresh PCG per
        correction, to inner_rtol) or "replace" (one PCG whose residual is
        replaced by the FP64 one after each inner_rtol reduction).  Returns
        (x, outer steps, inner iterations, FP64 relative residual)."""
        _dev(b, torch.float64, self.ndof, "b")
        x = self._new(self.ndof) if x is None else _dev(x, torch.float64, self.ndof, "x")
        code = {"restart": LOR_IR_RESTART, "replace": LOR_IR_REPLACE}[scheme]
        no, ni, rel = C.c_int(0), C.c_int(0), C.c_double(0.0)
        rc = self._lib.lor_pcg_solve_ir(self._h, _ptr(b), _ptr(x), float(rtol), float(inner_rtol), int(maxit), code,
                                        C.byref(no), C.byref(ni), C.byref(rel), _stream())
        if rc != LOR_OK and (rc != LOR_ENOCONV or raise_on_noconv):
            raise LORError(rc, self._lib.lor_last_error(self._h).decode())
        return x, no.value, ni.value, rel.value

    # ------------------------------------------------------------------ autograd glue
    def ensure_coefficient(self, kappa):
        if self._kappa_key != (kappa.data_ptr(), kappa._version):
            self.set_coefficient(kappa)


class LORApply(torch.autograd.Function):
    """y = A_p(kappa) x with the hand-written backward kernel:
    dL/dx = A_p (dL/dy), dL/dkappa = grad(x)^T G grad(dL/dy) at Gauss points."""

    @staticmethod
    def forward(ctx, op, kappa, x):
        op.set_coefficient(kappa)
        ctx.op = op
        ctx.save_for_backward(kappa, x)
        return op.apply(x.contiguous())

    @staticmethod
    def backward(ctx, gy):
        kappa, x = ctx.saved_tensors
        op = ctx.op
        op.ensure_coefficient(kappa)
        gx, gk = op.apply_backward(x, gy.contiguous(), want_gx=ctx.needs_input_grad[2],
                                   want_gkappa=ctx.needs_input_grad[1])
        return None, (gk.view_as(kappa) if gk is not None else None), gx


class LORSolve(torch.autograd.Function):
    """u = A_p(kappa)^-1 b by LOR-preconditioned CG; backward is the adjoint
    solve A_p lambda = dL/du with the same preconditioner, giving
    dL/db = lambda and dL/dkappa = -grad(u)^T G grad(lambda)."""

    @staticmethod
    def forward(ctx, op, kappa, b, opts):
        op.set_coefficient(kappa)
        op.build_pattern_internal()
        op.assemble_internal(opts.get("dtype", torch.float64))
        op.precond_setup(kind=opts.get("precond", "cheb"), dtype=opts.get("dtype", torch.float64),
                         degree=opts.get("degree", 3), power_iters=opts.get("power_iters", 20),
                         v0=opts.get("v0"))
        u, it, rel = op.pcg_solve(b.contiguous(), opts.get("rtol", 1e-10), opts.get("maxit", 5000))
        ctx.op, ctx.opts = op, opts
        ctx.info = (it, rel)
        ctx.save_for_backward(kappa, u)
        return u

    @staticmethod
    def backward(ctx, gu):
        kappa, u = ctx.saved_tensors
        op, opts = ctx.op, ctx.opts
        op.ensure_coefficient(kappa)
        lam, _, _ = op.pcg_solve(gu.contiguous(), opts.get("rtol", 1e-10), opts.get("maxit", 5000))
        _, gk = op.apply_backward(u, lam, want_gx=False, want_gkappa=True)
        return None, (-gk).view_as(kappa), lam, None


def solve(op, kappa, b, **opts):
    """Differentiable solve u(kappa, b) (see LORSolve)."""
    return LORSolve.apply(op, kappa, b, opts)


def solve_with_adjoint(op, theta, b, u_star, **opts):
    """J(theta) = 1/2 |u - u*|^2 with A_p(e^theta) u = b; returns (J, dJ/dtheta)
    computed by one forward and one adjoint PCG solve and the backward kernel."""
    th = theta.detach().clone().requires_grad_(True)
    u = solve(op, torch.exp(th), b, **opts)
    J = 0.5 * torch.sum((u - u_star) ** 2)
    J.backward()
    return J.detach(), th.grad
