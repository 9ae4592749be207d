"""Algorithmic work per launch of each liblor kernel (roofline numerators).

Flops are FP64 (an FMA counts 2), counted from the formulas each kernel
evaluates, not from what the hardware issues; bytes are the minimum HBM
traffic (every input read once, every output written once).  N = DOFs,
E = elements, nq = E (p+2)^3 Gauss points, S = E p^3 LOR sub-hexes.

Peaks: FP64 has no entry in MEASURED_PEAKS.json, so the FP64 peak is derived
from unit counts and clock: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz =
1.2586 TFLOP/s (an own DFMA loop measured 1.19 TFLOP/s, 1.90 DFMA/clk/SM);
likewise FP32: 152 x 128 FFMA/clk/SM x 2 x 2.07 GHz = 80.55 TFLOP/s.
The HBM peak is MEASURED_PEAKS.json's copy bandwidth.
"""
import json
import os

SMS, DFMA_PER_CLK_SM, FFMA_PER_CLK_SM, IMAD_PER_CLK_SM, MAX_SM_GHZ = 152, 2, 128, 64, 2.07
FP64_PEAK_TFLOPS = SMS * DFMA_PER_CLK_SM * 2 * MAX_SM_GHZ / 1e3  # 1.2586
FP32_PEAK_TFLOPS = SMS * FFMA_PER_CLK_SM * 2 * MAX_SM_GHZ / 1e3  # 80.55 (an own FFMA loop: 74.6)
# 32 x 32 -> 64 bit integer multiply-adds (mad.wide.s32), lanes per second:
# 152 x 64 x 2.07 GHz = 20.14 T (an own loop: 59.4 lanes/clk/SM)
INT_MAD_PEAK_TOPS = SMS * IMAD_PER_CLK_SM * MAX_SM_GHZ / 1e3
# the FP64 operator and its backward run in 64-bit fixed point on the integer
# pipe; each fixed-point multiply-add is three 32 x 32 -> 64 bit ones
FIXED_POINT_KINDS = ("apply", "backward", "apply_helmholtz", "backward_helmholtz")
MAD_WIDE_PER_FIXED_MAC = 3
HBM_FALLBACK_GBS = 6800.0


def hbm_peak_gbs():
    """(GB/s, source) from MEASURED_PEAKS.json, else the recipe's fallback."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def sumfact_fma(p):
    """FMAs of one forward pass grad_ref(u) at the Gauss points of an element:
    x-stage 2 q n^3, y-stage 3 q^2 n^2, z-stage 3 q^3 n (n = p+1, q = p+2)."""
    q, n = p + 2, p + 1
    return 2 * q * n ** 3 + 3 * q * q * n * n + 3 * q ** 3 * n


def jacobian_columns_flops(L):
    """Per element, the three Jacobian columns of the trilinear map at L x L
    coordinate pairs (each column is bilinear in the two other coordinates):
    36 half edge vectors (2 each), then per column, component and first
    coordinate two edge interpolations (6) and L second-coordinate ones (3)."""
    return 72 + 9 * L * (6 + 3 * L)


def setup_flops_per_element(p):
    """Jacobian columns at the q x q Gauss pairs; per Gauss point the
    adjugate rows r_a = c_b x c_c (27), det J = c_0 . r_0 (5), det M =
    (det J)^2 (1), 1/sqrt(det M) (1), the weight product (2), kappa w /
    sqrt(det M) (2), adj(M)_ab = r_a . r_b (30) and the six scaled cofactors
    (6): 74."""
    q = p + 2
    return jacobian_columns_flops(q) + 74 * q ** 3


def assemble_flops_per_element(p):
    """FP64 LOR assembly as the kernel evaluates it: per element the Jacobian
    columns at the 2p x 2p sub-hex Gauss pairs; per sub-hex, one 8x8 block by
    2x2x2 Gauss in the modal (Walsh-Hadamard) form: per Gauss point the
    adjugate rows r_a = c_b x c_c (27), det J = c_0 . r_0 (5), det M (1),
    1/sqrt(det M) (1), adj(M)_ab = r_a . r_b (30), the six metric entries
    (F_ab / sqrt(det M)) adj(M)_ab (12) = 76 x 8; six 8-point Walsh transforms, 24 additions
    each less the 12 whose outputs the diagonal entries never use (108); the
    modal block, 28 sums of the |m||n| transformed entries (56 additions) and
    their 22 factors 3^(-(|m|+|n|-2)/2) other than 1 (78); the
    modal-to-nodal transform per axis, 8 additions for each of the 6
    off-diagonal 2x2 blocks and 6 flops for each of the 4 diagonal ones
    (3 x 72 = 216); the six scales F_ab (13).  Per element the kappa_s
    averages: 3 per high-order Gauss point and one weight product per (y, z)
    point pair of each sub-hex column (p q^2).  (The kernel executes the
    additions of the transforms, the modal sums and the sandwich as exact
    64-bit integer additions; they are counted here as the flops they are.)"""
    q, L = p + 2, 2 * p
    return jacobian_columns_flops(L) + p ** 3 * (8 * 76 + 108 + 78 + 216 + 13) + 3 * q ** 3 + p * q * q


def assemble_f32_flops_per_element(p):
    """The FP32 LOR assembly (the values of the mixed-precision smoother) as
    that kernel evaluates it: Jacobian columns at the sub-hex Gauss pairs;
    per Gauss point adjugate rows (27), det (5), 1/det (1), the six scaled
    metric entries (42) = 75 x 8; the Walsh transforms (108); the 84-term
    modal block (168); the sandwich (216); the scales F_ab (13); per element
    the kappa_s averages.  (Evaluated directly, G grad(phi_j) and 36 dot
    products at each Gauss point, the block costs 8 x (144 + 216) = 2,880
    flops instead of the 492 of the transforms, the modal block and the
    sandwich.)"""
    q = p + 2
    return jacobian_columns_flops(2 * p) + p ** 3 * (8 * 75 + 108 + 168 + 216 + 13) + 3 * q ** 3 + p * q * q


def apply_flops_per_element(p):
    """Forward and transpose sum factorisation (2 flops per FMA each) plus the
    symmetric 3x3 D product (15 flops) per Gauss point."""
    return 4 * sumfact_fma(p) + 15 * (p + 2) ** 3


def backward_flops_per_element(p):
    """Two forward passes (x and gy), one transpose pass, and per point the
    D product (15, shared by gx and gkappa) and gkappa = grad(x) . (D grad(gy))
    / kappa (6)."""
    return 6 * sumfact_fma(p) + 21 * (p + 2) ** 3


def folded_forward_macs(p):
    """Multiply-adds of one even-odd folded 1D contraction n -> q (B_1D or
    d_1D): per output pair the even part (n/2 entries, plus the middle node
    when n is odd) and the odd part (n/2); the middle output (q odd) takes
    the even or the odd part alone."""
    n, q = p + 1, p + 2
    return (q // 2) * ((n & 1) + 2 * (n // 2)) + (q & 1) * (n // 2)


def folded_transpose_macs(p, parts=1):
    """Multiply-adds of one folded transposed contraction q -> n with `parts`
    tables summed (B^T v1, or B^T v1 + d^T v2)."""
    n, q = p + 1, p + 2
    return parts * ((n // 2) * ((q & 1) + 2 * (q // 2)) + (n & 1) * (q // 2))


def apply_fixed_macs_per_element(p, mass=False):
    """Fixed-point multiply-adds per element of the FP64 apply as the kernel
    runs it: x stage (B and d on n^2 lines), y stage (3 contractions on n q
    lines), z stage (3, with the reaction term 4, on q^2 lines), the 3 x 3
    D product (9 per Gauss point, the reaction's M 1 more), the transposed z
    (B^T, B^T, d^T or B^T + d^T), y (B^T and B^T + d^T) and x (B^T + d^T)
    stages."""
    n, q = p + 1, p + 2
    f, t1, t2 = folded_forward_macs(p), folded_transpose_macs(p, 1), folded_transpose_macs(p, 2)
    return (n * n * 2 * f + n * q * 3 * f + q * q * (4 if mass else 3) * f
            + q ** 3 * (10 if mass else 9)
            + q * q * (2 * t1 + (t2 if mass else t1)) + n * q * (t1 + t2) + n * n * t2)


def backward_fixed_macs_per_element(p, mass=False):
    """The apply's multiply-adds plus the second field's forward pass (x, y
    and z stages) and grad(x) . (D grad(gy)) (3 per Gauss point)."""
    n, q = p + 1, p + 2
    f = folded_forward_macs(p)
    return apply_fixed_macs_per_element(p, mass) + n * n * 2 * f + n * q * 3 * f + q * q * 3 * f + 3 * q ** 3


def fixed_macs(kind, p, nel):
    """Fixed-point multiply-adds of one launch of a FIXED_POINT_KINDS kernel."""
    mass = kind.endswith("helmholtz")
    per = backward_fixed_macs_per_element(p, mass) if kind.startswith("backward") else \
        apply_fixed_macs_per_element(p, mass)
    return per * nel


def reaction_extra_apply_flops_per_element(p):
    """The reaction term's share of the apply: B_z on the q^2 BB lines and its
    transpose (q^3 n FMAs each) and the scaling by beta w detJ (q^3)."""
    q, n = p + 2, p + 1
    return 4 * q ** 3 * n + q ** 3


def reaction_extra_assemble_flops_per_element(p):
    """FP64, per sub-hex: the scale beta_s r_a r_b r_c / 64 (4), W(g) = that
    scale times det J_e = det M / sqrt(det M) (16), its Walsh transform (24),
    the 36 modal mass terms 3^(-(|m|+|n|)/2) What(m xor n) added to the block
    (35 products, 36 additions); per element the beta_s averages (2 per
    high-order Gauss point, sharing the kappa_s weights)."""
    return p ** 3 * (4 + 16 + 24 + 71) + 2 * (p + 2) ** 3


def reaction_extra_assemble_f32_flops_per_element(p):
    """FP32: the scale (4), W(g) (8), its Walsh transform (24), the 36 modal
    mass terms added to the block (35 products, 36 additions); per element
    the beta_s averages."""
    return p ** 3 * (4 + 8 + 24 + 71) + 2 * (p + 2) ** 3


def kernel_work(kind, p, ndof, nel, nnz, vbytes=8, degree=3):
    """(flops, bytes) of one launch of `kind` on the given sizes."""
    q = p + 2
    nq = nel * q ** 3
    nsub = nel * p ** 3
    if kind == "setup":
        # kappa in, D (48 + a 4-byte scale per point) and the kappa copy out
        return setup_flops_per_element(p) * nel, 68 * nq
    if kind == "assemble":
        f = assemble_flops_per_element(p) if vbytes == 8 else assemble_f32_flops_per_element(p)
        return f * nel, vbytes * nnz + 8 * nq
    if kind == "apply":
        return apply_flops_per_element(p) * nel, 16 * ndof + 52 * nq
    if kind == "apply_f32":
        # the same contractions in FP32 (flops are FP32 here); D read as FP32
        return apply_flops_per_element(p) * nel, 16 * ndof + 24 * nq
    if kind == "backward":
        return backward_flops_per_element(p) * nel, 24 * ndof + 68 * nq
    if kind == "reaction_setup":
        # det (3 cross-product terms, 5) and beta w detJ (3); beta in, beta copy and M out
        return 8 * nq, 24 * nq
    if kind == "assemble_helmholtz":
        f, b = kernel_work("assemble", p, ndof, nel, nnz, vbytes)
        extra = reaction_extra_assemble_flops_per_element(p) if vbytes == 8 else \
            reaction_extra_assemble_f32_flops_per_element(p)
        return f + extra * nel, b + 8 * nq
    if kind == "apply_helmholtz":
        f, b = kernel_work("apply", p, ndof, nel, nnz, vbytes)
        return f + reaction_extra_apply_flops_per_element(p) * nel, b + 8 * nq
    if kind == "backward_helmholtz":
        f, b = kernel_work("backward", p, ndof, nel, nnz, vbytes)
        return f + reaction_extra_apply_flops_per_element(p) * nel, b + 8 * nq
    if kind == "precond":
        # degree-1 SpMV passes over the matrix values (the pattern-implicit
        # SpMV reads no column indices or row pointers: they are the closed
        # form of the 27-point pattern) and ~6 vector streams per step
        spmv = nnz * vbytes
        return 2 * nnz * (degree - 1), (degree - 1) * (spmv + 6 * vbytes * ndof) + 3 * 8 * ndof
    raise KeyError(kind)
