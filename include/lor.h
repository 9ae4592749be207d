/*
 * lor.h -- C ABI of liblor, a GB300 (sm_103a) implementation of
 * low-order-refined (LOR) preconditioning for high-order H1 diffusion,
 *   -div(kappa grad u) = f  on hexahedral meshes, u = 0 on the boundary,
 * after W. Pazner, Tz. Kolev, J.-S. Camier, "End-to-end GPU acceleration of
 * low-order-refined preconditioning for high-order finite element
 * discretizations" (arXiv 2210.12253).
 *
 * The paper's pipeline (Section 3) is: S1.1 high-order operator setup
 * (partial assembly of D at quadrature points), S1.2 LOR matrix assembly
 * (A1 macro-element batching, A2 local CSR, A4 boundary elimination),
 * S1.3 preconditioner setup, S2 preconditioned CG whose iterations apply the
 * high-order operator A_p = P^T G^T B^T D B G P matrix-free (Eq. (4),
 * Step S2.1) and the LOR-based preconditioner B_h (Step S2.2).  This library
 * implements that pipeline on one GPU for structured meshes of the unit cube
 * (nex x ney x nez trilinear hexes with arbitrary interior vertex positions,
 * lor_create) and for general conforming hex meshes given by element corners
 * and an element-to-DOF map (lor_create_general), with B_h a Chebyshev-Jacobi
 * smoother on the assembled LOR matrix.  Optional parts: the reaction term
 * of the definite Helmholtz problem of Section 4.1 (lor_set_reaction), the
 * gradients of the operator with respect to x and kappa, the unstructured
 * LOR assembly the paper compares against (lor_assemble_unstructured), and
 * the discrete gradient of the LOR mesh (Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every call returns LOR_OK (0) or a positive LOR_E* code;
 *    lor_last_error() gives a message.  A failed call leaves the context
 *    usable unless it returns LOR_ECUDA.
 *  - Pointers named d_* are DEVICE pointers owned by the caller and borrowed
 *    for the duration of the call (for asynchronous calls: until the work
 *    enqueued on the stream has run).  Host scalars are returned through
 *    plain host pointers.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Work is enqueued on it in order; no call synchronises
 *    the device except those documented as returning a host scalar.
 *  - Layouts (x fastest everywhere):
 *      vertex (a,b,c)      -> a + (nex+1)(b + (ney+1) c), 3 f64 (x,y,z)
 *      element (ex,ey,ez)  -> ex + nex (ey + ney ez)
 *      DOF (I,J,K)         -> I + nx (J + ny K), nx = nex p + 1, etc.;
 *                             element node (i,j,k) is DOF (ex p+i, ey p+j, ez p+k)
 *      quadrature point    -> g0 + q (g1 + q g2), q = p + 2 Gauss-Legendre
 *                             points per axis; kappa is [nel][q^3] f64
 *      LOR CSR             -> rowptr int64[N+1], colidx int32[nnz] (sorted),
 *                             values f64 or f32 [nnz]; full symmetric matrix
 *                             with the 27-point pattern of the LOR mesh.
 *  - Essential DOFs are all DOFs on the boundary of the unit cube.  Their rows
 *    and columns are eliminated with the sparsity pattern kept and the
 *    diagonal set to 1 (Step S1.2, A4); the high-order apply returns
 *    y_ess = x_ess and ignores x_ess elsewhere.
 */
#ifndef LOR_H
#define LOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LOR_MAX_P 10 /* largest supported polynomial degree */

enum lor_status {
  LOR_OK = 0,
  LOR_EINVAL = 1,   /* bad argument (size, pointer, degree, coefficient <= 0 or NaN) */
  LOR_EGEOM = 2,    /* a Jacobian determinant <= 0 (inverted or degenerate element) */
  LOR_ENOMEM = 3,   /* device allocation failed (also injected on the host: an environment
                       variable LOR_DEVICE_ALLOC_LIMIT=<bytes> caps the device memory a
                       context's own buffers may hold) */
  LOR_ECUDA = 4,    /* CUDA runtime error (message in lor_last_error) */
  LOR_ENOCONV = 5,  /* PCG hit maxit before reaching the tolerance */
  LOR_ETIMEOUT = 6, /* a bounded device-side wait expired (a bulk copy into shared
                       memory did not complete within 1 s); results of the
                       calls since the last check are invalid */
  LOR_ESTATE = 7    /* call out of order (e.g. apply before set_coefficient) */
};

enum lor_dtype { LOR_F64 = 0, LOR_F32 = 1 };

enum lor_precond { LOR_PRECOND_NONE = 0, LOR_PRECOND_JACOBI = 1, LOR_PRECOND_CHEB = 2 };
/* Schemes of lor_pcg_solve_ir. */
enum lor_ir_scheme { LOR_IR_RESTART = 0, LOR_IR_REPLACE = 1 };

typedef struct lor_ctx lor_ctx;

typedef struct lor_config {
  int32_t p;   /* polynomial degree, 1 <= p <= LOR_MAX_P */
  int32_t nex; /* elements along x, y, z (>= 1 each) */
  int32_t ney;
  int32_t nez;
} lor_config;

/* Message for the last failed call on ctx (or, for ctx == NULL, the last
 * failed lor_create on this thread).  Valid until the next call.  Plumbing
 * (no passage of the paper).  Never fails: an empty string when nothing
 * has failed. */
const char* lor_last_error(const lor_ctx* ctx);

/* Create a context for the order-p space on the structured hex mesh with
 * vertex coordinates d_vertices [(nex+1)(ney+1)(nez+1)][3] f64 (device,
 * copied).  Element maps are the trilinear maps through the 8 element
 * vertices (p_g = 1); the LOR mesh (Section 2.1) splits each element at the
 * Gauss-Lobatto points into p^3 sub-hexes.  Checks every Jacobian at the
 * Gauss points used by the high-order operator and by the LOR assembly and
 * returns LOR_EGEOM if one is <= 0.  LOR_EINVAL for p outside [1, LOR_MAX_P],
 * an empty mesh or 2^31 or more DOFs (the CSR column indices are int32).
 * Synchronises the stream.  *out receives the context (NULL on failure). */
int lor_create(lor_ctx** out, const lor_config* cfg, const double* d_vertices, void* stream);

/* Create a context on a general conforming hex mesh given in the
 * element-restriction form of Step S1.1 (the maps G of Eq. (4)): nel
 * trilinear elements with corners d_corners [nel][8][3] f64 (corner
 * c0 + 2 c1 + 4 c2 at reference vertex (2 c0 - 1, 2 c1 - 1, 2 c2 - 1)), the
 * element-to-DOF map d_elem_dofs [nel][(p+1)^3] int64 (local GLL node
 * i + n(j + n k), n = p+1, to a global DOF in [0, ndof); nodes shared by
 * elements share their DOF) and the essential-DOF mask d_ess uint8[ndof]
 * (NULL: none).  kappa, beta, x, y and every per-point array use the element
 * order and the same local node / Gauss point order as on the structured
 * mesh.  The LOR pattern is built here from the map (the sub-hexes' 8-DOF
 * couplings, sorted and de-duplicated per row; vertex valence up to 64) and
 * the LOR assembly finds CSR positions by binary search; lor_spmv and the
 * smoother read the explicit pattern.  lor_lor_mesh is for structured meshes
 * only (LOR_ESTATE); lor_discrete_gradient numbers the LOR edges of a general
 * mesh itself (see there).
 * LOR_EINVAL for a map entry out of range, 2^31 or more DOFs or more than
 * 8.7e14 elements (the byte sizes of the element arrays would overflow
 * int64), LOR_EGEOM for detJ <= 0.  All
 * input arrays are device memory, copied.  Synchronises the stream. */
int lor_create_general(lor_ctx** out, int p, int64_t nel, int64_t ndof, const double* d_corners,
                       const int64_t* d_elem_dofs, const uint8_t* d_ess, void* stream);

/* Free the context and every device buffer it owns.  Synchronises the device
 * work of the context first.  Plumbing.  Always LOR_OK (NULL is accepted). */
int lor_destroy(lor_ctx* ctx);

/* Number of CUDA kernels liblor has launched in this process so far (all
 * contexts, all threads).  Host-only; for instrumentation (no passage).
 * Errors: LOR_EINVAL if count is NULL. */
int lor_launch_count(int64_t* count);

/* Sizes: DOFs N = nx ny nz, LOR nonzeros (3nx-2)(3ny-2)(3nz-2) (the count
 * behind the sizes of Section 4.1), elements, quadrature points nel q^3.  Any
 * output pointer may be NULL.  Errors: LOR_EINVAL for a NULL ctx. */
int lor_sizes(const lor_ctx* ctx, int64_t* ndof, int64_t* nnz, int64_t* nel, int64_t* nqpt);

/* Step S1.1 (high-order operator setup, partial assembly): from the mesh and
 * kappa [nel][q^3] (device, f64) compute at every Gauss point
 *   D_g = kappa_g w_g detJ_g J_g^-1 J_g^-T
 * in FP64 and keep it (and a copy of kappa) in the context.  kappa must be
 * finite and > 0; a violation is recorded on the device and reported by the
 * next lor_check (the call itself does not synchronise).  Errors: LOR_EINVAL
 * for a NULL ctx or d_kappa, LOR_ENOMEM, LOR_ECUDA. */
int lor_set_coefficient(lor_ctx* ctx, const double* d_kappa, void* stream);

/* Reaction term of the definite Helmholtz (diffusion-reaction) operator
 * -div(kappa grad u) + beta u that Section 4.1 solves: beta [nel][q^3]
 * (device, f64, finite and > 0, same layout as kappa) at the Gauss points.
 * The context keeps a copy and M_g = beta_g w_g detJ_g (FP64); from then on
 * lor_apply, lor_apply_backward (gx), lor_assemble and lor_pcg_solve include
 * the mass term: B_m^T M B_m with B_m = B(x)B(x)B (Step S2.1's Kronecker
 * basis operator) in the high-order operator, and beta_s times the trilinear
 * mass matrix of every sub-hex (2x2x2 Gauss, beta_s the Gauss-weight average
 * of beta over the sub-hex like kappa_s) in the LOR matrix.  d_beta == NULL
 * switches the term off.  Re-assemble (lor_assemble, lor_precond_setup) after
 * changing it.  A bad beta is reported by the next lor_check.  Does not
 * synchronise.  Errors: LOR_EINVAL for a NULL ctx, LOR_ENOMEM, LOR_ECUDA. */
int lor_set_reaction(lor_ctx* ctx, const double* d_beta, void* stream);

/* Synchronise the stream and report any error recorded by earlier device
 * work of this context, then clear it.  Plumbing (no passage).  Errors:
 * LOR_EINVAL for a NULL ctx, a bad coefficient or a coupling missing from
 * the pattern given to lor_assemble_unstructured; LOR_EGEOM for a detJ <= 0
 * met there; LOR_ETIMEOUT when an SpMV-type kernel gave up waiting for its
 * bulk copy of matrix values (lor_precond_setup and the solvers check that
 * themselves); LOR_ECUDA. */
int lor_check(lor_ctx* ctx, void* stream);

/* Bits of lor_set_test_hooks. */
#define LOR_TEST_EXPIRE_WAITS 1u
#define LOR_TEST_UNSTAGED_CSR 2u

/* Test hooks (no passage: the paper has no counterpart; a way for tests to exercise the
 * error paths of device-side waits without a fault).  flags is a bit mask:
 *   LOR_TEST_EXPIRE_WAITS  every CTA of the TMA-staged SpMV/smoother kernels
 *                          treats its first bounded wait for a bulk copy as
 *                          expired: it records
 *                          LOR_FLAG_TIMEOUT in the context's status word, lets
 *                          every copy it issued land (waits at the normal
 *                          bound) and exits without writing its rows, exactly
 *                          as after a real expiry.  lor_check, lor_precond_setup
 *                          and the solvers then return LOR_ETIMEOUT.
 *   LOR_TEST_UNSTAGED_CSR  the explicit-CSR SpMV/smoother kernel (general
 *                          meshes) reads every tile from global memory, the
 *                          path it otherwise takes only for tiles whose rows
 *                          do not fit its shared-memory buffers (same result).
 * 0 clears the hooks; a cleared context computes as before (clear the status
 * word with lor_check first).  Host only, does not synchronise.  Errors:
 * LOR_EINVAL for a NULL ctx or an unknown flag. */
int lor_set_test_hooks(lor_ctx* ctx, unsigned flags);

/* Step S1.2 / A2: build the CSR sparsity of the LOR matrix (27-point graph of
 * the LOR mesh, columns ascending, Dirichlet rows included) inside the
 * context.  If d_rowptr (int64[N+1]) and d_colidx (int32[nnz]) are non-NULL
 * the pattern is also written there.  Idempotent.  Errors: LOR_EINVAL for a
 * NULL ctx or when only one of the two arrays is given, LOR_ENOMEM,
 * LOR_ECUDA. */
int lor_build_pattern(lor_ctx* ctx, int64_t* d_rowptr, int32_t* d_colidx, void* stream);

/* Step S1.2 / A1 + A4: assemble the values of the LOR matrix A_h for the
 * current coefficient (the p = 1 stiffness matrix of the LOR mesh; each
 * sub-hex block integrated by 2x2x2 Gauss on the sub-hex's trilinear map with
 * kappa averaged over the high-order Gauss points inside the sub-hex), then
 * eliminate the essential rows and columns.  Geometry (Jacobians,
 * determinants) is always FP64; dtype selects the arithmetic and storage of
 * the block entries (LOR_F64 or LOR_F32).  d_values: nnz entries of dtype in
 * the order of lor_build_pattern, or NULL to assemble into the context's own
 * matrix of that dtype (the one lor_precond_setup uses).  Requires
 * lor_build_pattern and lor_set_coefficient.  Errors: LOR_EINVAL for a NULL
 * ctx or a bad dtype, LOR_ESTATE before those two calls, LOR_ENOMEM,
 * LOR_ECUDA. */
int lor_assemble(lor_ctx* ctx, void* d_values, int dtype, void* stream);

/* The LOR mesh as a general hex mesh (E-vectors: the input of the
 * unstructured assembly of Section 4.2, below): for every sub-hex s = a + p(b + p c) of every
 * element e (index e p^3 + s), its 8 vertices T_e(GLL tensor points)
 * d_corners [nsub][8][3] f64 (local vertex r = r0 + 2 r1 + 4 r2), their global
 * DOF ids d_dofs [nsub][8] int64, kappa_s d_kappa_sub [nsub] f64 (the same
 * Gauss-weight binning the macro-element assembly uses) and, if d_beta_sub is
 * not NULL, beta_s [nsub] (requires lor_set_reaction).  d_ess (uint8[N], may
 * be NULL) receives 1 on essential (boundary) DOFs.  nsub = nel p^3.  All
 * arrays are caller-owned device memory.  Requires lor_set_coefficient.
 * Errors: LOR_EINVAL for a NULL ctx or output array, LOR_ESTATE on a general
 * mesh (lor_create_general), before lor_set_coefficient, or for d_beta_sub
 * without lor_set_reaction; LOR_ECUDA. */
int lor_lor_mesh(lor_ctx* ctx, double* d_corners, int64_t* d_dofs, double* d_kappa_sub, double* d_beta_sub,
                 uint8_t* d_ess, void* stream);

/* Unstructured Q1 assembly, the comparator of the macro-element algorithm
 * in Section 4.2 (one thread per degree of freedom of a sub-element, global
 * CSR positions found by search): for any conforming hex mesh given as
 * E-vectors (d_corners, d_dofs as above, one coefficient per element in
 * d_kappa_sub, optional reaction coefficient d_beta_sub), adds each element's
 * 8x8 block
 *   K_rc = sum over the 2x2x2 Gauss points of kappa_s grad phi_r . grad phi_c
 *          detJ (+ beta_s phi_r phi_c detJ)
 * into d_values (f64 or f32 per dtype, nnz entries, zeroed first) of the CSR
 * pattern d_rowptr int64[n+1] / d_colidx int32[nnz] (columns ascending per
 * row), the position of each coupling found by binary search in its row.
 * Rows and columns with d_ess[i] != 0 (may be NULL) are eliminated, their
 * diagonal set to 1.  The context only carries the error state.  A coupling
 * missing from the pattern or a detJ <= 0 is reported by the next
 * lor_check.  Does not synchronise.  Errors: LOR_EINVAL for a NULL ctx, a bad
 * dtype, a negative size or a missing array (the mesh arrays may be NULL only
 * when nsub = 0, d_values only when nnz = 0), LOR_ECUDA. */
int lor_assemble_unstructured(lor_ctx* ctx, int64_t nsub, const double* d_corners, const int64_t* d_dofs,
                              const double* d_kappa_sub, const double* d_beta_sub, int64_t n, int64_t nnz,
                              const int64_t* d_rowptr, const int32_t* d_colidx, const uint8_t* d_ess, void* d_values,
                              int dtype, void* stream);

/* Discrete gradient of the LOR mesh (Section 3, Algorithm 1), for the
 * H(curl) auxiliary-space solver: the incidence matrix from the LOR vertices
 * (the N global GLL grid points) to the LOR edges, as CSR with two entries per
 * row: -1 at the edge's tail vertex, +1 at its head.  Edge order: all
 * x-directed edges, then y-, then z-directed, each set lexicographic by its
 * tail vertex (I fastest); an edge runs from its tail to the next vertex along
 * its axis (so columns ascend).  *nedge (host, may be NULL) receives the
 * number of edges; with all three arrays NULL only the count is returned.
 * d_rowptr int64[nedge+1], d_colidx int32[2 nedge] (8-byte aligned),
 * d_values f64[2 nedge] (16-byte aligned).  The matrix depends on the
 * topology and p only.  On a general mesh (lor_create_general) the edges are
 * the sub-hex edges through the element-to-DOF map, each oriented from its
 * lower to its higher global DOF and numbered by (tail, head) ascending; the
 * first call enumerates them (synchronises) and keeps them in the context.
 * Errors: LOR_EINVAL for a NULL ctx, when only some of the three arrays are
 * given, for misaligned arrays or 2^31 or more vertices; LOR_ENOMEM,
 * LOR_ECUDA. */
int lor_discrete_gradient(lor_ctx* ctx, int64_t* d_rowptr, int32_t* d_colidx, double* d_values, int64_t* nedge,
                          void* stream);

/* Coordinates of the LOR vertices without duplicates (the vector the
 * H(curl) solver of Section 3 takes besides the discrete gradient of
 * Algorithm 1): d_xyz f64[N][3], DOF d (structured: vertex I + nx(J + ny K))
 * at T_e(GLL node) of the lowest-index element holding it, i.e. the vertices
 * of the LOR mesh of Section 2.1.  Errors: LOR_EINVAL for a NULL ctx or
 * d_xyz, LOR_ECUDA. */
int lor_vertex_coordinates(lor_ctx* ctx, double* d_xyz, void* stream);

/* Step S2.1: y = A_p x, the high-order operator applied matrix-free by sum
 * factorisation (B = [B(x)B(x)d; B(x)d(x)B; d(x)B(x)B] with the 1D
 * interpolation/derivative matrices, D from lor_set_coefficient), in FP64.
 * Dirichlet rows: y_ess = x_ess; x_ess is ignored in the free rows.  With
 * lor_set_reaction the mass term is included.  d_x, d_y: f64[N], must not
 * alias.  Errors: LOR_EINVAL for a NULL ctx, NULL or aliased arrays,
 * LOR_ESTATE before lor_set_coefficient, LOR_ECUDA. */
int lor_apply(lor_ctx* ctx, const double* d_x, double* d_y, void* stream);

/* y = A_p x as lor_apply computes it, but with FP32 arithmetic inside the
 * kernel: the 1D tables, the stage buffers and D (and beta w detJ) are FP32
 * (rounded copies of the FP64 factors, made by the first FP32 call after
 * lor_set_coefficient / lor_set_reaction); x is read and y accumulated in
 * FP64.  Relative error about 1e-6 of |A_p| |x|.  It is the operator of the
 * inner solves of lor_pcg_solve_ir; the FP64 lor_apply stays the operator of
 * every residual that decides convergence.  d_x, d_y: f64[N], must not alias.
 * The operator is that of Step S2.1; the paper has no FP32 counterpart (it
 * runs the operator in FP64 only).  Errors: as lor_apply, and LOR_ENOMEM
 * for the FP32 factors. */
int lor_apply_f32(lor_ctx* ctx, const double* d_x, double* d_y, void* stream);

/* Backward of y = A_p(kappa) x for the cotangent d_gy (FP64):
 *   d_gx     = A_p gy (with the reaction term if set)     (f64[N], may be NULL)
 *   d_gkappa = d(gy^T A_p x)/d kappa = grad_ref(x)^T (D/kappa) grad_ref(gy)
 *              at every Gauss point, x and gy taken as 0 on essential DOFs
 *                                                          (f64[nel q^3], may be NULL).
 * This is the gradient used by the adjoint method for dJ/dkappa.  The
 * operator is that of Step S2.1 (Eq. (4) with D = kappa w detJ J^-1 J^-T);
 * the paper does not differentiate it.  Errors: LOR_EINVAL for a NULL ctx or
 * d_gy, d_gkappa without d_x, or d_gx aliasing d_gy; LOR_ESTATE before
 * lor_set_coefficient; LOR_ECUDA. */
int lor_apply_backward(lor_ctx* ctx, const double* d_x, const double* d_gy, double* d_gx, double* d_gkappa,
                       void* stream);

/* Load vector b_i = sum_e sum_g w_g detJ_g f_g phi_i(x_g) for f given at the
 * Gauss points (d_f [nel][q^3] f64) or f = 1 (d_f == NULL); b_ess = 0: the
 * right-hand side of the problem of Section 4.1, computed with the
 * quadrature of Step S2.1.  Needs only the mesh.  Errors: LOR_EINVAL for a
 * NULL ctx or d_b, LOR_ECUDA. */
int lor_load_vector(lor_ctx* ctx, const double* d_f, double* d_b, void* stream);

/* y = A_h x with the context's assembled LOR matrix of `dtype` (x, y f64;
 * in LOR_F32 mode x is rounded to f32 and the product accumulated in f32).
 * The kernel reads the CSR values only; the columns of the 27-point pattern
 * that lor_build_pattern writes are recomputed from the grid.  The SpMV is
 * the building block of Step S2.2 (the solve phase reduces to SpMVs and
 * vector updates).  Errors: LOR_EINVAL for a NULL ctx, NULL or aliased
 * arrays; LOR_ESTATE when no matrix of that dtype is assembled in the
 * context; LOR_ECUDA. */
int lor_spmv(lor_ctx* ctx, int dtype, const double* d_x, double* d_y, void* stream);

/* Preconditioner B_h on the context's assembled LOR matrix of `dtype`
 * (Section 2.2: any preconditioner of A_h preconditions A_p):
 *   LOR_PRECOND_JACOBI: z = D_h^-1 r, D_h = diag(A_h);
 *   LOR_PRECOND_CHEB:   `degree` steps of the Chebyshev semi-iteration for
 *                       A_h z = r with M = D_h from z_0 = 0 on the interval
 *                       [lo_ratio lmax, hi_ratio lmax] (Saad, Alg. 12.1).
 * lmax = lambda_max if > 0, else estimated by `power_iters` steps of the power
 * iteration w = D_h^-1 A_h v, lambda = |w|/|v|, v = w/|w| from d_v0 (f64[N],
 * device; NULL means all ones).  Returns lmax in *lambda_out (host, may be
 * NULL); synchronises the stream when it estimates lmax.  The smoother
 * computes in `dtype`.  Errors: LOR_EINVAL for a NULL ctx, a bad kind or
 * dtype, degree < 1, not 0 < lo_ratio < hi_ratio, or power_iters < 1 when
 * lmax is estimated; LOR_ESTATE before the context matrix of that dtype is
 * assembled; LOR_ENOMEM; LOR_ETIMEOUT; LOR_ECUDA. */
int lor_precond_setup(lor_ctx* ctx, int kind, int dtype, int degree, double lo_ratio, double hi_ratio,
                      double lambda_max, int power_iters, const double* d_v0, double* lambda_out, void* stream);

/* Step S2.2: z = B_h r with the preconditioner from lor_precond_setup
 * (r, z f64[N]; z = r when none is set).  Errors: LOR_EINVAL for a NULL ctx,
 * NULL or aliased arrays, LOR_ECUDA. */
int lor_precond_apply(lor_ctx* ctx, const double* d_r, double* d_z, void* stream);

/* Size in bytes of the device array used by lor_precond_apply_noalloc. */
#define LOR_NOALLOC_SCRATCH_BYTES (16u << 20)

/* z = B_h r exactly as lor_precond_apply computes it, for callers that must
 * not allocate device memory when they apply the preconditioner (for example
 * a solver loop whose device memory is reserved up front by another
 * allocator, or host code where CUDA allocation calls are not allowed).  The
 * call performs no cudaMalloc/cudaFree or other allocation: the smoother's
 * work vectors live in one static device array of LOR_NOALLOC_SCRATCH_BYTES
 * bytes that every GPU loading the library keeps until the process exits.
 * It needs 3 N values of the smoother's precision (N = DOFs): up to 699,050
 * DOFs for an FP64 smoother and 1,398,101 for FP32 (Jacobi and degree 1 need
 * none); larger sizes are rejected with LOR_EINVAL.  The first call on each
 * device looks up the array's device address (with that device current)
 * and keeps it for the life of the process, which assumes one primary CUDA
 * context per device (a cudaDeviceReset invalidates it); make that first
 * call before any stream capture.  All calls share the
 * array, which keeps the last call's contents (each call writes every element
 * it reads, so nothing needs clearing); calls that overlap on the GPU race
 * and must be ordered by the caller.  r, z: f64[N], distinct.
 * The paper has no counterpart (no passage): this is an interface for allocation-free
 * callers of this library. */
int lor_precond_apply_noalloc(lor_ctx* ctx, const double* d_r, double* d_z, void* stream);

/* Section 3, step S2: preconditioned CG for A_p x = b with x_0 = 0, the
 * operator of lor_apply (FP64) and the preconditioner of lor_precond_setup
 * (identity if none).  Dot products and recurrences are FP64.  Stops when
 * |r_k|/|b| <= rtol for the recurrence residual and the true residual
 * b - A_p x confirms it (otherwise continues from the true residual).
 * Returns the iteration count and final relative residual through host
 * pointers (may be NULL), LOR_ENOCONV after maxit iterations.  Synchronises
 * the stream (it reads the residual norm on the host).  Other errors:
 * LOR_EINVAL for a NULL ctx, NULL or aliased b and x, rtol <= 0 or
 * maxit < 0; LOR_ESTATE before lor_set_coefficient; LOR_ETIMEOUT;
 * LOR_ECUDA. */
int lor_pcg_solve(lor_ctx* ctx, const double* d_b, double* d_x, double rtol, int maxit, int* iters,
                  double* final_rel_residual, void* stream);

/* Mixed-precision iterative refinement (Wilkinson; Moler 1967) for the same
 * system, x_0 = 0, in one of two schemes:
 *   LOR_IR_RESTART:
 *     repeat: r = b - A_p x          (FP64 operator, FP64 vectors)
 *             stop if |r|/|b| <= rtol
 *             solve A_p d = r by PCG from d_0 = 0 until |r_k| <= inner_rtol |r|,
 *               with the FP32 operator of lor_apply_f32 and the preconditioner
 *               of lor_precond_setup (FP32 vectors, d and the dot products
 *               summed in FP64)
 *             x += d
 *   LOR_IR_REPLACE (residual replacement, van der Vorst and Ye 2000): one PCG
 *     on the FP32 operator whose vectors r, z, p, q are FP32 (x stays FP64;
 *     dot products are summed in FP64 across threads); whenever its
 *     recurrence residual has fallen by inner_rtol since the last outer step,
 *     the FP64 residual b - A_p x is formed, the solve stops if it meets rtol,
 *     and otherwise it replaces the recurrence residual (rounded to FP32; the
 *     search direction is kept).
 * Either way the stopping residual is always the FP64 one, while the inner
 * iterations run the FP32 operator (on this GPU the FP32 pipe is about 60x
 * the FP64 one).  maxit bounds the inner iterations over all outer steps;
 * LOR_IR_RESTART takes at most 64 outer steps.  *outer_iters (FP64
 * residuals formed), *inner_iters, *final_rel_residual (host, may be NULL)
 * receive the counts and the final FP64 relative residual.  LOR_ENOCONV when
 * maxit or the outer limit is reached first, or when an outer step does not
 * lower the FP64 residual.  Synchronises the stream.
 * The paper has no counterpart: it solves with PCG in FP64 (Section 3,
 * step S2).  Other errors: LOR_EINVAL for a NULL ctx, NULL or aliased b and
 * x, rtol <= 0, inner_rtol outside (0, 1), maxit < 0 or an unknown scheme;
 * LOR_ESTATE before lor_set_coefficient; LOR_ENOMEM; LOR_ETIMEOUT;
 * LOR_ECUDA. */
int lor_pcg_solve_ir(lor_ctx* ctx, const double* d_b, double* d_x, double rtol, double inner_rtol, int maxit,
                     int scheme, int* outer_iters, int* inner_iters, double* final_rel_residual, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LOR_H */
