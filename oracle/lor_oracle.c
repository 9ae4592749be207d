/*
 * lor_oracle.c -- plain, slow, FP64 CPU oracle for low-order-refined (LOR)
 * preconditioning of high-order H1 diffusion on hexahedral meshes
 * (Pazner, Kolev, Camier, "End-to-end GPU acceleration of low-order-refined
 * preconditioning for high-order finite element discretizations",
 * arXiv 2210.12253).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library in paper_2210_12253_gb300/.  Only tests/, the smoke check in
 * __graft_entry__.py and the cpu_baseline / reference legs of bench.py may
 * load it.  It shares no code, header, table or constant generator with the
 * CUDA path: every quantity (1D rules, geometry, operators, assembly, solver)
 * is computed here from its plain definition, in the order the paper states
 * it, with no blocking, fusion or reordering for speed.
 *
 * Problem (Section 2.2): -div(kappa grad u) = f on a hex mesh T_p of order-p
 * elements, homogeneous Dirichlet data on the whole boundary.
 *
 * Conventions (structured unit-cube meshes, nex x ney x nez elements):
 *   vertex (a,b,c)           -> a + (nex+1)*(b + (ney+1)*c), 3 doubles (x,y,z)
 *   element (ex,ey,ez)       -> ex + nex*(ey + ney*ez)
 *   global DOF (I,J,K)       -> I + nx*(J + ny*K), nx = nex*p+1 (etc.)
 *   element-local node (i,j,k) of element (ex,ey,ez) is DOF (ex*p+i, ey*p+j, ez*p+k)
 *   quadrature point (g0,g1,g2) of an element -> g0 + q*(g1 + q*g2)
 *   kappa                    -> [nel][q^3]
 *   symmetric 3x3 factors G  -> [nel][q^3][6], order (00,01,02,11,12,22)
 *   essential DOFs           -> I in {0,nx-1} or J in {0,ny-1} or K in {0,nz-1}
 *
 * Readings where the paper is silent (each one is listed with its reason in
 * the design notes of the repository):
 *   R1  kappa on an LOR sub-hex = Gauss-weight average of kappa over the
 *       high-order Gauss points whose reference coordinates fall in the
 *       sub-hex (per-axis binning; a point on a GLL node belongs to the
 *       lower interval).
 *   R2  each LOR sub-hex matrix is integrated with 2x2x2 Gauss points on the
 *       sub-hex's own trilinear map.
 *   R4  Dirichlet elimination keeps the sparsity pattern: rows and columns of
 *       essential DOFs are zeroed and the diagonal set to 1.
 *   R6  Chebyshev semi-iteration on D^-1 A (Saad, Iterative Methods for
 *       Sparse Linear Systems, 2nd ed., Algorithm 12.1) from z0 = 0.
 *   R7  PCG stops when ||r_k||/||b|| <= tol for the recurrence residual and
 *       the true residual b - A x confirms it.
 *
 * Parity pins: every function here is checked in tests/test_oracle_*.py
 * against closed forms, brute force or library routines (see each header).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EGEOM 2
#define ORC_ENOMEM 3
#define ORC_ENOCONV 5

#define ORC_MAXN 32 /* largest number of 1D points handled */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* 1D rules (Section 2.1: Gauss-Lobatto interpolation points; Gauss-Legendre  */
/* quadrature for the operator).                                              */
/* ------------------------------------------------------------------------- */

/* Legendre polynomial P_n(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}; also returns P_{n-1}(x).  Both
 * 1D rules of Section 2.1 are built on it. */
static void legendre_pair(int n, double x, double* Pn, double* Pnm1) {
  double pm1 = 1.0, p = x;
  if (n == 0) { *Pn = 1.0; *Pnm1 = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double pn = ((2.0 * k + 1.0) * x * p - k * pm1) / (k + 1.0);
    pm1 = p;
    p = pn;
  }
  *Pn = p;
  *Pnm1 = pm1;
}

static void sort_ascending(int n, double* x, double* w) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && x[j - 1] > x[j]; --j) {
      double t = x[j]; x[j] = x[j - 1]; x[j - 1] = t;
      if (w) { t = w[j]; w[j] = w[j - 1]; w[j - 1] = t; }
    }
}

/* Gauss-Legendre rule with q points on [-1,1]: roots of P_q by Newton's
 * method, weights w = 2 / ((1 - x^2) P_q'(x)^2), with
 * P_q'(x) = q (P_{q-1}(x) - x P_q(x)) / (1 - x^2). */
int orc_gauss_legendre(int q, double* x, double* w) {
  if (q < 1 || q > ORC_MAXN) return ORC_EINVAL;
  for (int i = 0; i < q; ++i) {
    double t = cos(ORC_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre_pair(q, t, &P, &Pm1);
      double dP = q * (Pm1 - t * P) / (1.0 - t * t);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double P, Pm1;
    legendre_pair(q, t, &P, &Pm1);
    double dP = q * (Pm1 - t * P) / (1.0 - t * t);
    x[i] = t;
    w[i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  sort_ascending(q, x, w);
  return ORC_OK;
}

/* Gauss-Lobatto points (p+1 of them) on [-1,1]: the endpoints and the roots
 * of P_p'.  Newton on f = P_p' with f' = P_p'' from the Legendre equation
 * (1 - x^2) P'' = 2 x P' - p (p+1) P. */
int orc_gauss_lobatto(int p, double* x) {
  if (p < 1 || p + 1 > ORC_MAXN) return ORC_EINVAL;
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double t = -cos(ORC_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre_pair(p, t, &P, &Pm1);
      double d1 = p * (Pm1 - t * P) / (1.0 - t * t);
      double d2 = (2.0 * t * d1 - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = d1 / d2;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    x[i] = t;
  }
  sort_ascending(p + 1, x, NULL);
  return ORC_OK;
}

/* Lagrange basis on the n nodes, evaluated at t by the product formula
 *   l_j(t)  = prod_{m != j} (t - x_m) / (x_j - x_m)
 *   l_j'(t) = sum_{l != j} 1/(x_j - x_l) prod_{m != j,l} (t - x_m)/(x_j - x_m).
 * On the Gauss-Lobatto nodes this is the nodal basis of the order-p space of
 * Section 2.1. */
void orc_lagrange(int n, const double* nodes, double t, double* phi, double* dphi) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
    phi[j] = v;
    double d = 0.0;
    for (int l = 0; l < n; ++l) {
      if (l == j) continue;
      double term = 1.0 / (nodes[j] - nodes[l]);
      for (int m = 0; m < n; ++m)
        if (m != j && m != l) term *= (t - nodes[m]) / (nodes[j] - nodes[m]);
      d += term;
    }
    if (dphi) dphi[j] = d;
  }
}

/* B_1D[g][i] = l_i(xg_g) and D_1D[g][i] = l_i'(xg_g): the one-dimensional
 * interpolation and differentiation matrices of Step S2.1 (q x (p+1)). */
int orc_basis_1d(int p, int q, double* B, double* D) {
  double gll[ORC_MAXN], xg[ORC_MAXN], wg[ORC_MAXN];
  int rc = orc_gauss_lobatto(p, gll);
  if (rc) return rc;
  rc = orc_gauss_legendre(q, xg, wg);
  if (rc) return rc;
  for (int g = 0; g < q; ++g) orc_lagrange(p + 1, gll, xg[g], B + g * (p + 1), D + g * (p + 1));
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Geometry: trilinear element maps T_e (p_g = 1) through the 8 element        */
/* vertices (Section 2.1), their Jacobians, and the symmetric factors          */
/* G = w detJ J^-1 J^-T of the diffusion D matrix (Step S1.1, Eq. (4)).        */
/* ------------------------------------------------------------------------- */

static int64_t vertex_index(int a, int b, int c, int nex, int ney) {
  return a + (int64_t)(nex + 1) * (b + (int64_t)(ney + 1) * c);
}

/* Corner c = c0 + 2 c1 + 4 c2 of element (ex,ey,ez). */
static void element_corners(const double* V, int nex, int ney, int ex, int ey, int ez, double X[8][3]) {
  for (int c = 0; c < 8; ++c) {
    int c0 = c & 1, c1 = (c >> 1) & 1, c2 = (c >> 2) & 1;
    const double* v = V + 3 * vertex_index(ex + c0, ey + c1, ez + c2, nex, ney);
    X[c][0] = v[0]; X[c][1] = v[1]; X[c][2] = v[2];
  }
}

/* Trilinear map through corners X at reference point xi in [-1,1]^3:
 * x(xi) = sum_c X_c prod_k l_{c_k}(xi_k), l_0 = (1-t)/2, l_1 = (1+t)/2,
 * J[i][j] = d x_i / d xi_j: the element map T_e of Section 2.1 with p_g = 1. */
static void trilinear_map(const double X[8][3], const double xi[3], double x[3], double J[3][3]) {
  for (int i = 0; i < 3; ++i) {
    if (x) x[i] = 0.0;
    for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
  }
  for (int c = 0; c < 8; ++c) {
    int ck[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    double l[3], dl[3];
    for (int k = 0; k < 3; ++k) {
      l[k] = ck[k] ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
      dl[k] = ck[k] ? 0.5 : -0.5;
    }
    double phi = l[0] * l[1] * l[2];
    double dphi[3] = {dl[0] * l[1] * l[2], l[0] * dl[1] * l[2], l[0] * l[1] * dl[2]};
    for (int i = 0; i < 3; ++i) {
      if (x) x[i] += X[c][i] * phi;
      for (int j = 0; j < 3; ++j) J[i][j] += X[c][i] * dphi[j];
    }
  }
}

/* Inverse of a 3x3 matrix by the cofactor formula; returns det (the J^-1
 * and detJ of Step S1.1). */
static double inverse3(const double A[3][3], double Ai[3][3]) {
  double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  Ai[0][0] = c00 / det;
  Ai[1][0] = c01 / det;
  Ai[2][0] = c02 / det;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
  return det;
}

/* G = w detJ J^-1 J^-T, stored as (00,01,02,11,12,22): the geometric part of
 * the quadrature-point factor D = kappa G of Step S1.1. */
static void diffusion_factor(const double J[3][3], double w, double* detJ, double G[6]) {
  double Ji[3][3];
  double det = inverse3(J, Ji);
  double M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Ji[a][k] * Ji[b][k];
      M[a][b] = w * det * s;
    }
  G[0] = M[0][0]; G[1] = M[0][1]; G[2] = M[0][2];
  G[3] = M[1][1]; G[4] = M[1][2]; G[5] = M[2][2];
  *detJ = det;
}

/* Geometric factors at the q^3 Gauss points of every element (Step S1.1):
 * detJ[e][g] and G[e][g][6] = w_g detJ J^-1 J^-T.  Returns ORC_EGEOM if any
 * detJ <= 0. */
int orc_geometry(int nex, int ney, int nez, const double* V, int q, double* detJ, double* G) {
  double xg[ORC_MAXN], wg[ORC_MAXN];
  int rc = orc_gauss_legendre(q, xg, wg);
  if (rc) return rc;
  int bad = 0;
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
        double X[8][3];
        element_corners(V, nex, ney, ex, ey, ez, X);
        for (int g2 = 0; g2 < q; ++g2)
          for (int g1 = 0; g1 < q; ++g1)
            for (int g0 = 0; g0 < q; ++g0) {
              int64_t g = g0 + q * (g1 + q * g2);
              double xi[3] = {xg[g0], xg[g1], xg[g2]};
              double J[3][3], d;
              trilinear_map(X, xi, NULL, J);
              diffusion_factor(J, wg[g0] * wg[g1] * wg[g2], &d, G + 6 * (e * q * q * q + g));
              if (detJ) detJ[e * q * q * q + g] = d;
              if (!(d > 0.0)) bad = 1;
            }
      }
  return bad ? ORC_EGEOM : ORC_OK;
}

/* Physical coordinates of every global GLL DOF: x = T_e(GLL tensor point),
 * i.e. the vertices of the LOR mesh of Section 2.1. */
int orc_dof_coordinates(int nex, int ney, int nez, const double* V, int p, double* xyz) {
  double gll[ORC_MAXN];
  int rc = orc_gauss_lobatto(p, gll);
  if (rc) return rc;
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1;
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        double X[8][3];
        element_corners(V, nex, ney, ex, ey, ez, X);
        for (int k = 0; k <= p; ++k)
          for (int j = 0; j <= p; ++j)
            for (int i = 0; i <= p; ++i) {
              double xi[3] = {gll[i], gll[j], gll[k]}, J[3][3];
              int64_t dof = (ex * (int64_t)p + i) + nx * ((ey * (int64_t)p + j) + ny * (ez * (int64_t)p + k));
              trilinear_map(X, xi, xyz + 3 * dof, J);
            }
      }
  return ORC_OK;
}

static int is_essential(int64_t I, int64_t J, int64_t K, int64_t nx, int64_t ny, int64_t nz) {
  return I == 0 || I == nx - 1 || J == 0 || J == ny - 1 || K == 0 || K == nz - 1;
}

/* ------------------------------------------------------------------------- */
/* High-order operator y = A_p x (Step S2.1, Eq. (4): A_p = G^T B^T D B G on a */
/* single rank), by sum factorisation with the 1D factors B_1D and D_1D.       */
/* B = [B (x) B (x) D ; B (x) D (x) B ; D (x) B (x) B] in 3D (Step S2.1), with */
/* D at each point = kappa * w detJ J^-1 J^-T (Step S1.1).                     */
/* beta != NULL adds the reaction (mass) term of the definite Helmholtz       */
/* problem of Section 4.1: B_m^T (beta w detJ) B_m with B_m = B (x) B (x) B.    */
/* If dirichlet != 0: x is taken as zero on essential DOFs on the input side,  */
/* no result is accumulated into essential rows, and y_ess = x_ess.            */
/* ------------------------------------------------------------------------- */

/* Reference gradient of the element field u[k][j][i] at every Gauss point,
 * gr[g][3] (d/dxi0, d/dxi1, d/dxi2), by the three tensor stages of B
 * (Step S2.1). */
static void element_reference_gradient(int n, int q, const double* B, const double* D, const double* u, double* gr) {
  /* stage along xi0 */
  double* Bu = (double*)malloc(sizeof(double) * n * n * q);
  double* Du = (double*)malloc(sizeof(double) * n * n * q);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int g0 = 0; g0 < q; ++g0) {
        double sb = 0.0, sd = 0.0;
        for (int i = 0; i < n; ++i) {
          sb += B[g0 * n + i] * u[(k * n + j) * n + i];
          sd += D[g0 * n + i] * u[(k * n + j) * n + i];
        }
        Bu[(k * n + j) * q + g0] = sb;
        Du[(k * n + j) * q + g0] = sd;
      }
  /* stage along xi1 */
  double* BBu = (double*)malloc(sizeof(double) * n * q * q);
  double* BDu = (double*)malloc(sizeof(double) * n * q * q); /* B in xi1, D in xi0 */
  double* DBu = (double*)malloc(sizeof(double) * n * q * q); /* D in xi1, B in xi0 */
  for (int k = 0; k < n; ++k)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int j = 0; j < n; ++j) {
          s0 += B[g1 * n + j] * Bu[(k * n + j) * q + g0];
          s1 += B[g1 * n + j] * Du[(k * n + j) * q + g0];
          s2 += D[g1 * n + j] * Bu[(k * n + j) * q + g0];
        }
        BBu[(k * q + g1) * q + g0] = s0;
        BDu[(k * q + g1) * q + g0] = s1;
        DBu[(k * q + g1) * q + g0] = s2;
      }
  /* stage along xi2 */
  for (int g2 = 0; g2 < q; ++g2)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < n; ++k) {
          s0 += B[g2 * n + k] * BDu[(k * q + g1) * q + g0];
          s1 += B[g2 * n + k] * DBu[(k * q + g1) * q + g0];
          s2 += D[g2 * n + k] * BBu[(k * q + g1) * q + g0];
        }
        int g = (g2 * q + g1) * q + g0;
        gr[3 * g + 0] = s0;
        gr[3 * g + 1] = s1;
        gr[3 * g + 2] = s2;
      }
  free(Bu); free(Du); free(BBu); free(BDu); free(DBu);
}

/* Transpose of element_reference_gradient: v[g][3] at Gauss points ->
 * element vector y[k][j][i] = sum_g (B^T v), the B^T of Eq. (4). */
static void element_reference_gradient_transpose(int n, int q, const double* B, const double* D, const double* v, double* y) {
  double* T0 = (double*)malloc(sizeof(double) * n * q * q);
  double* T1 = (double*)malloc(sizeof(double) * n * q * q);
  double* T2 = (double*)malloc(sizeof(double) * n * q * q);
  for (int k = 0; k < n; ++k)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int g2 = 0; g2 < q; ++g2) {
          int g = (g2 * q + g1) * q + g0;
          s0 += B[g2 * n + k] * v[3 * g + 0];
          s1 += B[g2 * n + k] * v[3 * g + 1];
          s2 += D[g2 * n + k] * v[3 * g + 2];
        }
        T0[(k * q + g1) * q + g0] = s0;
        T1[(k * q + g1) * q + g0] = s1;
        T2[(k * q + g1) * q + g0] = s2;
      }
  double* U0 = (double*)malloc(sizeof(double) * n * n * q); /* component 0: D still pending in xi0 */
  double* U1 = (double*)malloc(sizeof(double) * n * n * q); /* components 1,2: B pending in xi0 */
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int g0 = 0; g0 < q; ++g0) {
        double s0 = 0.0, s1 = 0.0;
        for (int g1 = 0; g1 < q; ++g1) {
          s0 += B[g1 * n + j] * T0[(k * q + g1) * q + g0];
          s1 += D[g1 * n + j] * T1[(k * q + g1) * q + g0] + B[g1 * n + j] * T2[(k * q + g1) * q + g0];
        }
        U0[(k * n + j) * q + g0] = s0;
        U1[(k * n + j) * q + g0] = s1;
      }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int g0 = 0; g0 < q; ++g0)
          s += D[g0 * n + i] * U0[(k * n + j) * q + g0] + B[g0 * n + i] * U1[(k * n + j) * q + g0];
        y[(k * n + j) * n + i] = s;
      }
  free(T0); free(T1); free(T2); free(U0); free(U1);
}

/* Values of the element field at every Gauss point, val[g] = ((B (x) B (x) B) u)_g:
 * the basis operator of the mass matrix (Section 3, Step S2.1: B is the
 * Kronecker product of the 1D evaluation matrix). */
static void element_values(int n, int q, const double* B, const double* u, double* val) {
  double* T1 = (double*)malloc(sizeof(double) * n * n * q);
  double* T2 = (double*)malloc(sizeof(double) * n * q * q);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int g0 = 0; g0 < q; ++g0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += B[g0 * n + i] * u[(k * n + j) * n + i];
        T1[(k * n + j) * q + g0] = s;
      }
  for (int k = 0; k < n; ++k)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += B[g1 * n + j] * T1[(k * n + j) * q + g0];
        T2[(k * q + g1) * q + g0] = s;
      }
  for (int g2 = 0; g2 < q; ++g2)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += B[g2 * n + k] * T2[(k * q + g1) * q + g0];
        val[(g2 * q + g1) * q + g0] = s;
      }
  free(T1); free(T2);
}

/* Transpose of element_values, accumulated: y[k][j][i] += ((B (x) B (x) B)^T v)_{ijk}
 * (the B_m^T of the reaction term of Section 4.1's problem). */
static void element_values_transpose_add(int n, int q, const double* B, const double* v, double* y) {
  double* T2 = (double*)malloc(sizeof(double) * n * q * q);
  double* T1 = (double*)malloc(sizeof(double) * n * n * q);
  for (int k = 0; k < n; ++k)
    for (int g1 = 0; g1 < q; ++g1)
      for (int g0 = 0; g0 < q; ++g0) {
        double s = 0.0;
        for (int g2 = 0; g2 < q; ++g2) s += B[g2 * n + k] * v[(g2 * q + g1) * q + g0];
        T2[(k * q + g1) * q + g0] = s;
      }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int g0 = 0; g0 < q; ++g0) {
        double s = 0.0;
        for (int g1 = 0; g1 < q; ++g1) s += B[g1 * n + j] * T2[(k * q + g1) * q + g0];
        T1[(k * n + j) * q + g0] = s;
      }
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int g0 = 0; g0 < q; ++g0) s += B[g0 * n + i] * T1[(k * n + j) * q + g0];
        y[(k * n + j) * n + i] += s;
      }
  free(T1); free(T2);
}

/* Element restriction G of Eq. (4): the element's (p+1)^3 values from the
 * global vector, zero on essential DOFs when dirichlet != 0. */
static void gather_element(int64_t nx, int64_t ny, int64_t nz, int p, int ex, int ey, int ez, const double* x, int dirichlet, double* xe) {
  int n = p + 1;
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int64_t I = (int64_t)ex * p + i, J = (int64_t)ey * p + j, K = (int64_t)ez * p + k;
        double v = x[I + nx * (J + ny * K)];
        if (dirichlet && is_essential(I, J, K, nx, ny, nz)) v = 0.0;
        xe[(k * n + j) * n + i] = v;
      }
}

/* y = A_p x (Step S2.1, Eq. (4)): restriction, reference gradient, the
 * factor D (Step S1.1), transposed stages, accumulation; see the banner
 * above for the reaction term and the Dirichlet treatment. */
int orc_ho_apply(int nex, int ney, int nez, const double* V, int p, int q, const double* kappa, const double* beta,
                 const double* x, double* y, int dirichlet) {
  if (p < 1 || q < 1 || p + 1 > ORC_MAXN || q > ORC_MAXN) return ORC_EINVAL;
  int n = p + 1, nq3 = q * q * q;
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  int64_t N = nx * ny * nz, nel = (int64_t)nex * ney * nez;
  double* B = (double*)malloc(sizeof(double) * q * n);
  double* D = (double*)malloc(sizeof(double) * q * n);
  orc_basis_1d(p, q, B, D);
  double* G = (double*)malloc(sizeof(double) * nel * nq3 * 6);
  double* detJ = beta ? (double*)malloc(sizeof(double) * nel * nq3) : NULL;
  int rc = orc_geometry(nex, ney, nez, V, q, detJ, G);
  if (rc) { free(B); free(D); free(G); free(detJ); return rc; }
  double xg[ORC_MAXN], wg[ORC_MAXN];
  orc_gauss_legendre(q, xg, wg);
  double* xe = (double*)malloc(sizeof(double) * n * n * n);
  double* ye = (double*)malloc(sizeof(double) * n * n * n);
  double* gr = (double*)malloc(sizeof(double) * 3 * nq3);
  double* val = (double*)malloc(sizeof(double) * nq3);
  for (int64_t i = 0; i < N; ++i) y[i] = 0.0;
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
        gather_element(nx, ny, nz, p, ex, ey, ez, x, dirichlet, xe); /* G (restriction) */
        element_reference_gradient(n, q, B, D, xe, gr);               /* B */
        for (int g = 0; g < nq3; ++g) {                                /* D */
          const double* Gq = G + 6 * (e * nq3 + g);
          double k = kappa[e * nq3 + g];
          double a = gr[3 * g], b = gr[3 * g + 1], c = gr[3 * g + 2];
          gr[3 * g + 0] = k * (Gq[0] * a + Gq[1] * b + Gq[2] * c);
          gr[3 * g + 1] = k * (Gq[1] * a + Gq[3] * b + Gq[4] * c);
          gr[3 * g + 2] = k * (Gq[2] * a + Gq[4] * b + Gq[5] * c);
        }
        element_reference_gradient_transpose(n, q, B, D, gr, ye);      /* B^T */
        if (beta) {                                                    /* reaction: B^T (beta w detJ) B */
          element_values(n, q, B, xe, val);
          for (int g2 = 0; g2 < q; ++g2)
            for (int g1 = 0; g1 < q; ++g1)
              for (int g0 = 0; g0 < q; ++g0) {
                int g = (g2 * q + g1) * q + g0;
                val[g] *= beta[e * nq3 + g] * wg[g0] * wg[g1] * wg[g2] * detJ[e * nq3 + g];
              }
          element_values_transpose_add(n, q, B, val, ye);
        }
        for (int k = 0; k < n; ++k)                                    /* G^T */
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int64_t I = (int64_t)ex * p + i, J = (int64_t)ey * p + j, K = (int64_t)ez * p + k;
              if (dirichlet && is_essential(I, J, K, nx, ny, nz)) continue;
              y[I + nx * (J + ny * K)] += ye[(k * n + j) * n + i];
            }
      }
  if (dirichlet)
    for (int64_t K = 0; K < nz; ++K)
      for (int64_t J = 0; J < ny; ++J)
        for (int64_t I = 0; I < nx; ++I)
          if (is_essential(I, J, K, nx, ny, nz)) y[I + nx * (J + ny * K)] = x[I + nx * (J + ny * K)];
  free(B); free(D); free(G); free(detJ); free(xe); free(ye); free(gr); free(val);
  return ORC_OK;
}

/* Backward of y = A_p(kappa) x for a cotangent gy (the Dirichlet-masked
 * operator is symmetric, so gx = A_p gy):
 *   gx = A_p gy,
 *   gkappa[e][g] = (grad_ref x)^T G_g (grad_ref gy) at Gauss point g, with
 *                  x and gy taken as zero on essential DOFs,
 * i.e. the derivative of gy^T A_p(kappa) x with respect to kappa[e][g].
 * Either output may be NULL; beta (may be NULL) is the reaction coefficient
 * of the operator, which enters gx only.  The operator is that of Step S2.1
 * (Eq. (4)); the paper does not differentiate it, so this is its plain
 * derivative written out. */
int orc_ho_apply_backward(int nex, int ney, int nez, const double* V, int p, int q, const double* kappa, const double* beta,
                          const double* x, const double* gy, double* gx, double* gkappa) {
  if (gx) {
    int rc = orc_ho_apply(nex, ney, nez, V, p, q, kappa, beta, gy, gx, 1);
    if (rc) return rc;
  }
  if (!gkappa) return ORC_OK;
  int n = p + 1, nq3 = q * q * q;
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  int64_t nel = (int64_t)nex * ney * nez;
  double* B = (double*)malloc(sizeof(double) * q * n);
  double* D = (double*)malloc(sizeof(double) * q * n);
  orc_basis_1d(p, q, B, D);
  double* G = (double*)malloc(sizeof(double) * nel * nq3 * 6);
  int rc = orc_geometry(nex, ney, nez, V, q, NULL, G);
  if (rc) { free(B); free(D); free(G); return rc; }
  double* xe = (double*)malloc(sizeof(double) * n * n * n);
  double* ge = (double*)malloc(sizeof(double) * n * n * n);
  double* grx = (double*)malloc(sizeof(double) * 3 * nq3);
  double* grg = (double*)malloc(sizeof(double) * 3 * nq3);
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
        gather_element(nx, ny, nz, p, ex, ey, ez, x, 1, xe);
        gather_element(nx, ny, nz, p, ex, ey, ez, gy, 1, ge);
        element_reference_gradient(n, q, B, D, xe, grx);
        element_reference_gradient(n, q, B, D, ge, grg);
        for (int g = 0; g < nq3; ++g) {
          const double* Gq = G + 6 * (e * nq3 + g);
          double a = grg[3 * g], b = grg[3 * g + 1], c = grg[3 * g + 2];
          double v0 = Gq[0] * a + Gq[1] * b + Gq[2] * c;
          double v1 = Gq[1] * a + Gq[3] * b + Gq[4] * c;
          double v2 = Gq[2] * a + Gq[4] * b + Gq[5] * c;
          gkappa[e * nq3 + g] = grx[3 * g] * v0 + grx[3 * g + 1] * v1 + grx[3 * g + 2] * v2;
        }
      }
  free(B); free(D); free(G); free(xe); free(ge); free(grx); free(grg);
  return ORC_OK;
}

/* Load vector b_i = sum_e sum_g w_g detJ_g f_g phi_i(x_g) for a right-hand
 * side given at Gauss points f[e][g] (f == NULL means f = 1); b_ess = 0: the
 * right-hand side of the problem of Section 2.2 (f = 1 in Section 4.1). */
int orc_load_vector(int nex, int ney, int nez, const double* V, int p, int q, const double* f, double* b) {
  int n = p + 1, nq3 = q * q * q;
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  int64_t N = nx * ny * nz, nel = (int64_t)nex * ney * nez;
  double gll[ORC_MAXN], xg[ORC_MAXN], wg[ORC_MAXN];
  orc_gauss_lobatto(p, gll);
  orc_gauss_legendre(q, xg, wg);
  double* detJ = (double*)malloc(sizeof(double) * nel * nq3);
  double* G = (double*)malloc(sizeof(double) * nel * nq3 * 6);
  int rc = orc_geometry(nex, ney, nez, V, q, detJ, G);
  if (rc) { free(detJ); free(G); return rc; }
  double L[ORC_MAXN][ORC_MAXN];
  for (int g = 0; g < q; ++g) orc_lagrange(n, gll, xg[g], L[g], NULL);
  for (int64_t i = 0; i < N; ++i) b[i] = 0.0;
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              double s = 0.0;
              for (int g2 = 0; g2 < q; ++g2)
                for (int g1 = 0; g1 < q; ++g1)
                  for (int g0 = 0; g0 < q; ++g0) {
                    int g = g0 + q * (g1 + q * g2);
                    double fv = f ? f[e * nq3 + g] : 1.0;
                    s += wg[g0] * wg[g1] * wg[g2] * detJ[e * nq3 + g] * fv * L[g0][i] * L[g1][j] * L[g2][k];
                  }
              int64_t I = (int64_t)ex * p + i, J = (int64_t)ey * p + j, K = (int64_t)ez * p + k;
              b[I + nx * (J + ny * K)] += s;
            }
      }
  for (int64_t K = 0; K < nz; ++K)
    for (int64_t J = 0; J < ny; ++J)
      for (int64_t I = 0; I < nx; ++I)
        if (is_essential(I, J, K, nx, ny, nz)) b[I + nx * (J + ny * K)] = 0.0;
  free(detJ); free(G);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Brute-force dense stiffness matrix on a general hex mesh: each element is   */
/* the trilinear image of [-1,1]^3 through its 8 corners, carries the degree-p */
/* Lagrange basis on the GLL tensor points, and is integrated with q^3 Gauss   */
/* points:  A_ij = sum_e sum_g kappa_g w_g detJ_g grad(phi_i) . grad(phi_j)    */
/* with grad(phi) = J^-T grad_ref(phi) evaluated from explicit 3D basis        */
/* functions (Section 2.2, the bilinear form (grad u, grad v)).                */
/* corners: [nel][8][3]; dofs: [nel][(p+1)^3] (local node i + n(j + n k));     */
/* kappa: [nel][q^3]; A: N x N row-major, accumulated (caller zeroes it).      */
/* beta (may be NULL): reaction coefficient, adds beta w detJ phi_i phi_j.     */
/* ------------------------------------------------------------------------- */
int orc_dense_general(int64_t nel, int p, int q, const double* corners, const int64_t* dofs, const double* kappa,
                      const double* beta, int64_t N, double* A) {
  if (p < 1 || q < 1 || p + 1 > ORC_MAXN || q > ORC_MAXN) return ORC_EINVAL;
  int n = p + 1, n3 = n * n * n, nq3 = q * q * q;
  double gll[ORC_MAXN], xg[ORC_MAXN], wg[ORC_MAXN];
  orc_gauss_lobatto(p, gll);
  orc_gauss_legendre(q, xg, wg);
  double L[ORC_MAXN][ORC_MAXN], dL[ORC_MAXN][ORC_MAXN];
  for (int g = 0; g < q; ++g) orc_lagrange(n, gll, xg[g], L[g], dL[g]);
  double* grad = (double*)malloc(sizeof(double) * 3 * n3);
  double* phi = (double*)malloc(sizeof(double) * n3);
  int bad = 0;
  for (int64_t e = 0; e < nel; ++e) {
    double X[8][3];
    for (int c = 0; c < 8; ++c)
      for (int d = 0; d < 3; ++d) X[c][d] = corners[(e * 8 + c) * 3 + d];
    for (int g2 = 0; g2 < q; ++g2)
      for (int g1 = 0; g1 < q; ++g1)
        for (int g0 = 0; g0 < q; ++g0) {
          double xi[3] = {xg[g0], xg[g1], xg[g2]}, J[3][3], Ji[3][3];
          trilinear_map(X, xi, NULL, J);
          double det = inverse3(J, Ji);
          if (!(det > 0.0)) bad = 1;
          double wk = wg[g0] * wg[g1] * wg[g2] * det * kappa[e * nq3 + g0 + q * (g1 + q * g2)];
          double wb = beta ? wg[g0] * wg[g1] * wg[g2] * det * beta[e * nq3 + g0 + q * (g1 + q * g2)] : 0.0;
          for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
              for (int i = 0; i < n; ++i) {
                double gr[3] = {dL[g0][i] * L[g1][j] * L[g2][k], L[g0][i] * dL[g1][j] * L[g2][k], L[g0][i] * L[g1][j] * dL[g2][k]};
                int a = i + n * (j + n * k);
                phi[a] = L[g0][i] * L[g1][j] * L[g2][k];
                for (int d = 0; d < 3; ++d) /* physical gradient: J^-T gr */
                  grad[3 * a + d] = Ji[0][d] * gr[0] + Ji[1][d] * gr[1] + Ji[2][d] * gr[2];
              }
          for (int a = 0; a < n3; ++a) {
            int64_t ra = dofs[e * n3 + a];
            for (int b = 0; b < n3; ++b) {
              int64_t cb = dofs[e * n3 + b];
              A[ra * N + cb] += wk * (grad[3 * a] * grad[3 * b] + grad[3 * a + 1] * grad[3 * b + 1] + grad[3 * a + 2] * grad[3 * b + 2]);
              if (beta) A[ra * N + cb] += wb * phi[a] * phi[b];
            }
          }
        }
  }
  free(grad);
  free(phi);
  return bad ? ORC_EGEOM : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* LOR matrix (Sections 2.1-2.2 and Step S1.2): the p = 1 H1 stiffness matrix */
/* on the LOR mesh T_h, whose elements are the p^3 sub-hexes of each macro     */
/* element, with vertices T_e(GLL tensor points).                              */
/* ------------------------------------------------------------------------- */

/* Reading R1: kappa_s = sum_{g in s} w_g kappa_g / sum_{g in s} w_g over the
 * high-order Gauss points g of the element whose reference coordinates lie
 * in sub-hex s = (a,b,c), binned per axis; interval(t) = #{interior GLL nodes
 * strictly below t}.  ksub: [nel][p^3], sub-hex a + p(b + p c). */
int orc_lor_kappa_sub(int p, int q, int64_t nel, const double* kappa, double* ksub) {
  double gll[ORC_MAXN], xg[ORC_MAXN], wg[ORC_MAXN];
  orc_gauss_lobatto(p, gll);
  orc_gauss_legendre(q, xg, wg);
  int bin[ORC_MAXN];
  for (int g = 0; g < q; ++g) {
    int c = 0;
    for (int m = 1; m < p; ++m)
      if (gll[m] < xg[g]) ++c;
    bin[g] = c;
  }
  int p3 = p * p * p, nq3 = q * q * q;
  double* num = (double*)malloc(sizeof(double) * p3);
  double* den = (double*)malloc(sizeof(double) * p3);
  int bad = 0;
  for (int64_t e = 0; e < nel; ++e) {
    for (int s = 0; s < p3; ++s) num[s] = den[s] = 0.0;
    for (int g2 = 0; g2 < q; ++g2)
      for (int g1 = 0; g1 < q; ++g1)
        for (int g0 = 0; g0 < q; ++g0) {
          int s = bin[g0] + p * (bin[g1] + p * bin[g2]);
          double w = wg[g0] * wg[g1] * wg[g2];
          num[s] += w * kappa[e * nq3 + g0 + q * (g1 + q * g2)];
          den[s] += w;
        }
    for (int s = 0; s < p3; ++s) {
      if (!(den[s] > 0.0)) bad = 1;
      ksub[e * p3 + s] = num[s] / den[s];
    }
  }
  free(num); free(den);
  return bad ? ORC_EINVAL : ORC_OK;
}

/* Reading R2: the 8 x 8 stiffness matrix of sub-hex (a,b,c) of an element
 * with corners X, kappa_s times 2x2x2 Gauss quadrature on the sub-hex's own
 * trilinear map through its 8 vertices T_e(GLL points); with a reaction
 * term, plus beta_s times the trilinear mass matrix by the same quadrature
 * (beta_s binned like kappa_s, reading R16).  Local vertex
 * r = r0 + 2 r1 + 4 r2 is the element node (a + r0, b + r1, c + r2). */
static int lor_subhex_matrix(const double X[8][3], const double* gll, int a, int b, int c, double kappa_s, double beta_s,
                             double K[8][8]) {
  double S[8][3];
  for (int r = 0; r < 8; ++r) {
    int r0 = r & 1, r1 = (r >> 1) & 1, r2 = (r >> 2) & 1;
    double xi[3] = {gll[a + r0], gll[b + r1], gll[c + r2]}, J[3][3];
    trilinear_map(X, xi, S[r], J);
  }
  const double g1 = 1.0 / sqrt(3.0);
  const double pts[2] = {-g1, g1};
  for (int r = 0; r < 8; ++r)
    for (int s = 0; s < 8; ++s) K[r][s] = 0.0;
  int bad = 0;
  for (int t2 = 0; t2 < 2; ++t2)
    for (int t1 = 0; t1 < 2; ++t1)
      for (int t0 = 0; t0 < 2; ++t0) {
        double xi[3] = {pts[t0], pts[t1], pts[t2]}, J[3][3], Ji[3][3];
        trilinear_map(S, xi, NULL, J);
        double det = inverse3(J, Ji);
        if (!(det > 0.0)) bad = 1;
        double grad[8][3], phi[8];
        for (int r = 0; r < 8; ++r) {
          int rk[3] = {r & 1, (r >> 1) & 1, (r >> 2) & 1};
          double l[3], dl[3];
          for (int k = 0; k < 3; ++k) {
            l[k] = rk[k] ? 0.5 * (1.0 + xi[k]) : 0.5 * (1.0 - xi[k]);
            dl[k] = rk[k] ? 0.5 : -0.5;
          }
          double gr[3] = {dl[0] * l[1] * l[2], l[0] * dl[1] * l[2], l[0] * l[1] * dl[2]};
          for (int d = 0; d < 3; ++d) grad[r][d] = Ji[0][d] * gr[0] + Ji[1][d] * gr[1] + Ji[2][d] * gr[2];
          phi[r] = l[0] * l[1] * l[2];
        }
        double wk = kappa_s * det, wb = beta_s * det; /* 2-point Gauss weights are 1 */
        for (int r = 0; r < 8; ++r)
          for (int s = 0; s < 8; ++s)
            K[r][s] += wk * (grad[r][0] * grad[s][0] + grad[r][1] * grad[s][1] + grad[r][2] * grad[s][2]) +
                       wb * phi[r] * phi[s];
      }
  return bad;
}

typedef struct {
  int64_t row, col;
  double val;
} orc_triplet;

static int triplet_cmp(const void* A, const void* B) {
  const orc_triplet* a = (const orc_triplet*)A;
  const orc_triplet* b = (const orc_triplet*)B;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  return 0;
}

typedef struct {
  int64_t n, nnz;
  int64_t* rowptr;
  int64_t* colidx;
  double* values;
} orc_csr;

/* Full LOR matrix as CSR: A_h = sum_s P_s^T K_s P_s over all sub-hexes s
 * (Step S1.2, A1-A2), formed as triplets, sorted by (row, col) and merged;
 * then (dirichlet != 0) essential rows/columns eliminated with the pattern
 * kept and the diagonal set to 1 (Step S1.2, A4; reading R4). */
void* orc_lor_assemble(int nex, int ney, int nez, const double* V, int p, int q, const double* kappa, const double* beta,
                       int dirichlet, int* status) {
  *status = ORC_OK;
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  int64_t N = nx * ny * nz, nel = (int64_t)nex * ney * nez;
  int p3 = p * p * p;
  double gll[ORC_MAXN];
  if (orc_gauss_lobatto(p, gll)) { *status = ORC_EINVAL; return NULL; }
  double* ksub = (double*)malloc(sizeof(double) * nel * p3);
  double* bsub = (double*)calloc((size_t)(nel * p3), sizeof(double));
  if (orc_lor_kappa_sub(p, q, nel, kappa, ksub) || (beta && orc_lor_kappa_sub(p, q, nel, beta, bsub))) {
    free(ksub); free(bsub); *status = ORC_EINVAL; return NULL;
  }
  int64_t ntrip = nel * p3 * 64;
  orc_triplet* T = (orc_triplet*)malloc(sizeof(orc_triplet) * ntrip);
  if (!T) { free(ksub); free(bsub); *status = ORC_ENOMEM; return NULL; }
  int64_t t = 0;
  int bad = 0;
  for (int ez = 0; ez < nez; ++ez)
    for (int ey = 0; ey < ney; ++ey)
      for (int ex = 0; ex < nex; ++ex) {
        int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
        double X[8][3];
        element_corners(V, nex, ney, ex, ey, ez, X);
        for (int c = 0; c < p; ++c)
          for (int b = 0; b < p; ++b)
            for (int a = 0; a < p; ++a) {
              double K[8][8];
              bad |= lor_subhex_matrix(X, gll, a, b, c, ksub[e * p3 + a + p * (b + p * c)], bsub[e * p3 + a + p * (b + p * c)], K);
              int64_t dof[8];
              for (int r = 0; r < 8; ++r) {
                int64_t I = (int64_t)ex * p + a + (r & 1), J = (int64_t)ey * p + b + ((r >> 1) & 1), Kk = (int64_t)ez * p + c + ((r >> 2) & 1);
                dof[r] = I + nx * (J + ny * Kk);
              }
              for (int r = 0; r < 8; ++r)
                for (int s = 0; s < 8; ++s) {
                  T[t].row = dof[r];
                  T[t].col = dof[s];
                  T[t].val = K[r][s];
                  ++t;
                }
            }
      }
  free(ksub);
  free(bsub);
  qsort(T, (size_t)ntrip, sizeof(orc_triplet), triplet_cmp);
  orc_csr* A = (orc_csr*)calloc(1, sizeof(orc_csr));
  A->n = N;
  A->rowptr = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
  int64_t nnz = 0;
  for (int64_t i = 0; i < ntrip; ++i)
    if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) ++nnz;
  A->nnz = nnz;
  A->colidx = (int64_t*)malloc(sizeof(int64_t) * nnz);
  A->values = (double*)malloc(sizeof(double) * nnz);
  int64_t k = -1;
  for (int64_t i = 0; i < ntrip; ++i) {
    if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) {
      ++k;
      A->colidx[k] = T[i].col;
      A->values[k] = 0.0;
      A->rowptr[T[i].row + 1]++;
    }
    A->values[k] += T[i].val;
  }
  free(T);
  for (int64_t i = 0; i < N; ++i) A->rowptr[i + 1] += A->rowptr[i];
  if (dirichlet) {
    for (int64_t r = 0; r < N; ++r) {
      int64_t I = r % nx, J = (r / nx) % ny, Kk = r / (nx * ny);
      int er = is_essential(I, J, Kk, nx, ny, nz);
      for (int64_t j = A->rowptr[r]; j < A->rowptr[r + 1]; ++j) {
        int64_t cc = A->colidx[j];
        int64_t cI = cc % nx, cJ = (cc / nx) % ny, cK = cc / (nx * ny);
        if (er || is_essential(cI, cJ, cK, nx, ny, nz)) A->values[j] = (cc == r) ? 1.0 : 0.0;
      }
    }
  }
  if (bad) *status = ORC_EGEOM;
  return A;
}

int64_t orc_csr_nnz(void* h) { return ((orc_csr*)h)->nnz; }
int64_t orc_csr_n(void* h) { return ((orc_csr*)h)->n; }
void orc_csr_copy(void* h, int64_t* rowptr, int64_t* colidx, double* values) {
  orc_csr* A = (orc_csr*)h;
  memcpy(rowptr, A->rowptr, sizeof(int64_t) * (A->n + 1));
  memcpy(colidx, A->colidx, sizeof(int64_t) * A->nnz);
  memcpy(values, A->values, sizeof(double) * A->nnz);
}
void orc_csr_free(void* h) {
  orc_csr* A = (orc_csr*)h;
  if (!A) return;
  free(A->rowptr); free(A->colidx); free(A->values); free(A);
}

/* ------------------------------------------------------------------------- */
/* LOR matrix of a general conforming hex mesh given in element-restriction    */
/* form (Step S1.1's maps G: corners [nel][8][3] and element-to-DOF map        */
/* [nel][(p+1)^3], local node i + n(j + n k)): the same sub-hex blocks as      */
/* orc_lor_assemble (readings R1, R2), their 8 DOFs looked up through the map, */
/* triplets sorted by (row, col) and merged; then (dirichlet != 0) the rows    */
/* and columns of the DOFs with ess[i] != 0 eliminated, pattern kept,          */
/* diagonal 1 (A4, reading R4).  ess may be NULL (no essential DOFs).          */
/* ------------------------------------------------------------------------- */
void* orc_lor_assemble_general(int64_t nel, int p, int q, const double* corners, const int64_t* dofs, int64_t N,
                               const uint8_t* ess, const double* kappa, const double* beta, int dirichlet, int* status) {
  *status = ORC_OK;
  int n = p + 1, n3 = n * n * n, p3 = p * p * p;
  double gll[ORC_MAXN];
  if (orc_gauss_lobatto(p, gll)) { *status = ORC_EINVAL; return NULL; }
  double* ksub = (double*)malloc(sizeof(double) * nel * p3);
  double* bsub = (double*)calloc((size_t)(nel * p3), sizeof(double));
  if (orc_lor_kappa_sub(p, q, nel, kappa, ksub) || (beta && orc_lor_kappa_sub(p, q, nel, beta, bsub))) {
    free(ksub); free(bsub); *status = ORC_EINVAL; return NULL;
  }
  int64_t ntrip = nel * p3 * 64;
  orc_triplet* T = (orc_triplet*)malloc(sizeof(orc_triplet) * ntrip);
  if (!T) { free(ksub); free(bsub); *status = ORC_ENOMEM; return NULL; }
  int64_t t = 0;
  int bad = 0;
  for (int64_t e = 0; e < nel; ++e) {
    double X[8][3];
    for (int cc = 0; cc < 8; ++cc)
      for (int d = 0; d < 3; ++d) X[cc][d] = corners[(e * 8 + cc) * 3 + d];
    for (int c = 0; c < p; ++c)
      for (int b = 0; b < p; ++b)
        for (int a = 0; a < p; ++a) {
          double K[8][8];
          int s = a + p * (b + p * c);
          bad |= lor_subhex_matrix(X, gll, a, b, c, ksub[e * p3 + s], bsub[e * p3 + s], K);
          int64_t dof[8];
          for (int r = 0; r < 8; ++r) {
            int i = a + (r & 1), j = b + ((r >> 1) & 1), k = c + ((r >> 2) & 1);
            dof[r] = dofs[e * n3 + i + n * (j + n * k)];
            if (dof[r] < 0 || dof[r] >= N) bad = 2;
          }
          for (int r = 0; r < 8; ++r)
            for (int s2 = 0; s2 < 8; ++s2) {
              T[t].row = dof[r];
              T[t].col = dof[s2];
              T[t].val = K[r][s2];
              ++t;
            }
        }
  }
  free(ksub);
  free(bsub);
  if (bad == 2) { free(T); *status = ORC_EINVAL; return NULL; }
  qsort(T, (size_t)ntrip, sizeof(orc_triplet), triplet_cmp);
  orc_csr* A = (orc_csr*)calloc(1, sizeof(orc_csr));
  A->n = N;
  A->rowptr = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
  int64_t nnz = 0;
  for (int64_t i = 0; i < ntrip; ++i)
    if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) ++nnz;
  A->nnz = nnz;
  A->colidx = (int64_t*)malloc(sizeof(int64_t) * (nnz > 0 ? nnz : 1));
  A->values = (double*)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
  int64_t k = -1;
  for (int64_t i = 0; i < ntrip; ++i) {
    if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) {
      ++k;
      A->colidx[k] = T[i].col;
      A->values[k] = 0.0;
      A->rowptr[T[i].row + 1]++;
    }
    A->values[k] += T[i].val;
  }
  free(T);
  for (int64_t i = 0; i < N; ++i) A->rowptr[i + 1] += A->rowptr[i];
  if (dirichlet && ess) {
    for (int64_t r = 0; r < N; ++r)
      for (int64_t j = A->rowptr[r]; j < A->rowptr[r + 1]; ++j) {
        int64_t cc = A->colidx[j];
        if (ess[r] || ess[cc]) A->values[j] = (cc == r) ? 1.0 : 0.0;
      }
  }
  if (bad) *status = ORC_EGEOM;
  return A;
}

/* Selected rows of the LOR matrix, each computed on its own from the
 * sub-hexes that contain the row's vertex (no global assembly): for every
 * sub-hex s touching DOF r, add row r of K_s.  Entries are returned sorted
 * by column, at most cap per row: cols/vals are [nrows][cap], counts[nrows].
 * Same Dirichlet treatment as orc_lor_assemble (Step S1.2, A4); the rows of
 * the LOR matrix at full size, computed one by one. */
int orc_lor_rows(int nex, int ney, int nez, const double* V, int p, int q, const double* kappa, const double* beta, int dirichlet,
                 int64_t nrows, const int64_t* rows, int cap, int32_t* counts, int64_t* cols, double* vals) {
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  int nq3 = q * q * q, p3 = p * p * p;
  double gll[ORC_MAXN];
  orc_gauss_lobatto(p, gll);
  double* ks = (double*)malloc(sizeof(double) * p3);
  double* bs = (double*)calloc((size_t)p3, sizeof(double));
  int bad = 0;
  for (int64_t t = 0; t < nrows; ++t) {
    int64_t r = rows[t];
    int64_t I = r % nx, J = (r / nx) % ny, Kk = r / (nx * ny);
    int cnt = 0;
    int64_t* rc = cols + t * cap;
    double* rv = vals + t * cap;
    for (int64_t sc = Kk - 1; sc <= Kk; ++sc)
      for (int64_t sb = J - 1; sb <= J; ++sb)
        for (int64_t sa = I - 1; sa <= I; ++sa) {
          if (sa < 0 || sb < 0 || sc < 0 || sa >= nx - 1 || sb >= ny - 1 || sc >= nz - 1) continue;
          int ex = (int)(sa / p), ey = (int)(sb / p), ez = (int)(sc / p);
          int a = (int)(sa % p), b = (int)(sb % p), c = (int)(sc % p);
          int64_t e = ex + (int64_t)nex * (ey + (int64_t)ney * ez);
          if (orc_lor_kappa_sub(p, q, 1, kappa + e * nq3, ks)) bad = 1;
          if (beta && orc_lor_kappa_sub(p, q, 1, beta + e * nq3, bs)) bad = 1;
          double X[8][3], K[8][8];
          element_corners(V, nex, ney, ex, ey, ez, X);
          bad |= lor_subhex_matrix(X, gll, a, b, c, ks[a + p * (b + p * c)], bs[a + p * (b + p * c)], K);
          int rloc = (int)(I - sa) + 2 * (int)(J - sb) + 4 * (int)(Kk - sc);
          for (int s = 0; s < 8; ++s) {
            int64_t cI = sa + (s & 1), cJ = sb + ((s >> 1) & 1), cK = sc + ((s >> 2) & 1);
            int64_t col = cI + nx * (cJ + ny * cK);
            int found = -1;
            for (int m = 0; m < cnt; ++m)
              if (rc[m] == col) found = m;
            if (found < 0) {
              if (cnt == cap) { free(ks); free(bs); return ORC_EINVAL; }
              rc[cnt] = col;
              rv[cnt] = 0.0;
              found = cnt++;
            }
            rv[found] += K[rloc][s];
          }
        }
    /* sort this row by column */
    for (int i = 1; i < cnt; ++i)
      for (int j = i; j > 0 && rc[j - 1] > rc[j]; --j) {
        int64_t tc = rc[j]; rc[j] = rc[j - 1]; rc[j - 1] = tc;
        double tv = rv[j]; rv[j] = rv[j - 1]; rv[j - 1] = tv;
      }
    if (dirichlet) {
      int er = is_essential(I, J, Kk, nx, ny, nz);
      for (int m = 0; m < cnt; ++m) {
        int64_t cc = rc[m];
        int64_t cI = cc % nx, cJ = (cc / nx) % ny, cK = cc / (nx * ny);
        if (er || is_essential(cI, cJ, cK, nx, ny, nz)) rv[m] = (cc == r) ? 1.0 : 0.0;
      }
    }
    counts[t] = cnt;
  }
  free(ks);
  free(bs);
  return bad ? ORC_EGEOM : ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Discrete gradient of the LOR mesh (Section 3, the matrix Algorithm 1 builds */
/* for the H(curl) solver): it maps the H1 LOR space (values at the LOR       */
/* vertices, i.e. the global GLL grid points) to the lowest-order H(curl)     */
/* space on the LOR edges.  Row i (an edge) holds -1 at the edge's tail vertex */
/* and +1 at its head vertex.  Reading R17 (the paper leaves the numbering to  */
/* the element restriction): the x-directed edges first, then the y- and      */
/* z-directed ones, each set lexicographic by its tail vertex (I fastest); an */
/* edge runs from its tail (I,J,K) to the next vertex along its axis, so the  */
/* tail has the lower global index and each row's columns are ascending.      */
/* ------------------------------------------------------------------------- */
int64_t orc_lor_edge_count(int nex, int ney, int nez, int p) {
  int64_t nx = (int64_t)nex * p + 1, ny = (int64_t)ney * p + 1, nz = (int64_t)nez * p + 1;
  return (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
}

/* The matrix of Algorithm 1 in the numbering above:
 * rowptr[nedge+1], colidx[2 nedge], values[2 nedge]. */
int orc_discrete_gradient(int nex, int ney, int nez, int p, int64_t* rowptr, int64_t* colidx, double* values) {
  int64_t n[3] = {(int64_t)nex * p + 1, (int64_t)ney * p + 1, (int64_t)nez * p + 1};
  int64_t stride[3] = {1, n[0], n[0] * n[1]};
  int64_t e = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t m[3] = {n[0], n[1], n[2]};
    m[d] -= 1; /* tails: all vertices but the last along the edge's axis */
    for (int64_t K = 0; K < m[2]; ++K)
      for (int64_t J = 0; J < m[1]; ++J)
        for (int64_t I = 0; I < m[0]; ++I) {
          int64_t tail = I + n[0] * (J + n[1] * K);
          rowptr[e] = 2 * e;
          colidx[2 * e] = tail;
          colidx[2 * e + 1] = tail + stride[d];
          values[2 * e] = -1.0;
          values[2 * e + 1] = 1.0;
          ++e;
        }
  }
  rowptr[e] = 2 * e;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Sparse kernels and preconditioners on a CSR matrix (Step S2.2: the solve    */
/* phase reduces to spmv and vector updates).                                  */
/* ------------------------------------------------------------------------- */

/* y = A x (Step S2.2's SpMV). */
void orc_csr_spmv(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* values, const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) s += values[j] * x[colidx[j]];
    y[i] = s;
  }
}

/* d = diag(A), the Jacobi scaling of the smoother (Step S2.2, reading R6). */
void orc_csr_diagonal(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* values, double* d) {
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j)
      if (colidx[j] == i) d[i] += values[j];
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Power iteration for the largest eigenvalue of D^-1 A (reading R6):
 * v = v0; repeat m times { w = D^-1 A v; lambda = ||w|| / ||v||; v = w / ||w|| }. */
double orc_power_lambda_max(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* values, const double* v0, int m) {
  double* d = (double*)malloc(sizeof(double) * n);
  double* v = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  orc_csr_diagonal(n, rowptr, colidx, values, d);
  for (int64_t i = 0; i < n; ++i) v[i] = v0[i];
  double lambda = 0.0;
  for (int it = 0; it < m; ++it) {
    orc_csr_spmv(n, rowptr, colidx, values, v, w);
    for (int64_t i = 0; i < n; ++i) w[i] /= d[i];
    double nw = sqrt(dot(n, w, w)), nv = sqrt(dot(n, v, v));
    lambda = nw / nv;
    for (int64_t i = 0; i < n; ++i) v[i] = w[i] / nw;
  }
  free(d); free(v); free(w);
  return lambda;
}

/* Chebyshev semi-iteration for A z = r preconditioned by M = diag(A)
 * (reading R6; Saad, Algorithm 12.1), k steps from z_0 = 0 on the interval
 * [lo, hi] of the spectrum of D^-1 A:
 *   theta = (hi+lo)/2, delta = (hi-lo)/2, sigma = theta/delta, rho_0 = 1/sigma,
 *   d_0 = M^-1 r / theta, z_1 = d_0,
 *   for j = 1..k-1: r_j = r - A z_j; rho_j = 1/(2 sigma - rho_{j-1});
 *                   d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) M^-1 r_j;
 *                   z_{j+1} = z_j + d_j.
 * k = 1 gives z = M^-1 r / theta.  diag may be NULL (taken from A). */
void orc_chebyshev(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* values, const double* diag, int k, double lo, double hi, const double* r, double* z) {
  double* dg = (double*)malloc(sizeof(double) * n);
  if (diag) memcpy(dg, diag, sizeof(double) * n);
  else orc_csr_diagonal(n, rowptr, colidx, values, dg);
  double* dvec = (double*)malloc(sizeof(double) * n);
  double* res = (double*)malloc(sizeof(double) * n);
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int64_t i = 0; i < n; ++i) {
    dvec[i] = r[i] / dg[i] / theta;
    z[i] = dvec[i];
  }
  for (int j = 1; j < k; ++j) {
    orc_csr_spmv(n, rowptr, colidx, values, z, res);
    for (int64_t i = 0; i < n; ++i) res[i] = r[i] - res[i];
    double rho_new = 1.0 / (2.0 * sigma - rho);
    for (int64_t i = 0; i < n; ++i) {
      dvec[i] = rho_new * rho * dvec[i] + (2.0 * rho_new / delta) * res[i] / dg[i];
      z[i] += dvec[i];
    }
    rho = rho_new;
  }
  free(dg); free(dvec); free(res);
}

/* Preconditioned conjugate gradient (Section 3, step S2) for A_p x = b with
 * x_0 = 0 and preconditioner B_h built on the LOR CSR matrix
 * (precond 0: identity, 1: Jacobi z = D^-1 r, 2: Chebyshev(k, lo, hi)).
 * Stopping rule R7: ||r||/||b|| <= rtol on the recurrence residual, then
 * confirmed on the true residual b - A_p x (otherwise iteration continues
 * from the true residual).  Returns ORC_ENOCONV after maxit iterations. */
int orc_pcg(int nex, int ney, int nez, const double* V, int p, int q, const double* kappa, const double* beta,
            const int64_t* rowptr, const int64_t* colidx, const double* values,
            int precond, int cheb_k, double lo, double hi,
            const double* b, double* x, double rtol, int maxit, int* iters, double* relres) {
  int64_t N = ((int64_t)nex * p + 1) * ((int64_t)ney * p + 1) * ((int64_t)nez * p + 1);
  double* r = (double*)malloc(sizeof(double) * N);
  double* z = (double*)malloc(sizeof(double) * N);
  double* pv = (double*)malloc(sizeof(double) * N);
  double* Ap = (double*)malloc(sizeof(double) * N);
  double* dg = (double*)malloc(sizeof(double) * N);
  orc_csr_diagonal(N, rowptr, colidx, values, dg);
#define ORC_PREC(rr, zz)                                                               \
  do {                                                                                  \
    if (precond == 0) memcpy(zz, rr, sizeof(double) * N);                               \
    else if (precond == 1) for (int64_t i_ = 0; i_ < N; ++i_) zz[i_] = rr[i_] / dg[i_]; \
    else orc_chebyshev(N, rowptr, colidx, values, dg, cheb_k, lo, hi, rr, zz);          \
  } while (0)
  for (int64_t i = 0; i < N; ++i) { x[i] = 0.0; r[i] = b[i]; }
  double nb = sqrt(dot(N, b, b));
  int status = ORC_ENOCONV, it = 0;
  double rel = 0.0;
  if (nb == 0.0) {
    status = ORC_OK;
  } else {
    ORC_PREC(r, z);
    memcpy(pv, z, sizeof(double) * N);
    double rz = dot(N, r, z);
    while (it < maxit) {
      orc_ho_apply(nex, ney, nez, V, p, q, kappa, beta, pv, Ap, 1);
      double alpha = rz / dot(N, pv, Ap);
      for (int64_t i = 0; i < N; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * Ap[i]; }
      ++it;
      rel = sqrt(dot(N, r, r)) / nb;
      if (rel <= rtol) {
        orc_ho_apply(nex, ney, nez, V, p, q, kappa, beta, x, Ap, 1);
        for (int64_t i = 0; i < N; ++i) r[i] = b[i] - Ap[i];
        rel = sqrt(dot(N, r, r)) / nb;
        if (rel <= rtol) { status = ORC_OK; break; }
      }
      ORC_PREC(r, z);
      double rz_new = dot(N, r, z);
      double beta = rz_new / rz;
      rz = rz_new;
      for (int64_t i = 0; i < N; ++i) pv[i] = z[i] + beta * pv[i];
    }
  }
#undef ORC_PREC
  *iters = it;
  *relres = rel;
  free(r); free(z); free(pv); free(Ap); free(dg);
  return status;
}
