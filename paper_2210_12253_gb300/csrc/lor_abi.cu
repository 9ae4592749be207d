// lor_abi.cu -- the extern "C" entry points of liblor (include/lor.h), the
// context, and the host-side 1D tables.
//
// 1D tables (Section 2.1 GLL nodes; Gauss-Legendre quadrature of the
// high-order operator; the LOR sub-hex quadrature) are computed here in long
// double:
//   Gauss-Legendre nodes: Newton on P_q with P_q' from the derivative
//     recurrence P'_{k+1} = P'_{k-1} + (2k+1) P_k; weights from the
//     Christoffel sum 1 / w_i = sum_{k<q} (k + 1/2) P_k(x_i)^2;
//   Gauss-Lobatto nodes: +-1 and the roots of P_{p+1} - P_{p-1} (which is
//     proportional to (1 - x^2) P_p'), by Newton;
//   Lagrange basis and derivative at the Gauss points: barycentric form
//     (Berrut & Trefethen, SIAM Review 2004) with l_j'/l_j = sum_{m!=j} 1/(t-x_m).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>

#include "fixed_point.cuh"
#include "lor_internal.cuh"

namespace {

thread_local std::string g_create_error;
std::atomic<long long> g_launches{0};

typedef long double ld;

// P_0..P_n and P'_0..P'_n at x.
void legendre_all(int n, ld x, ld* P, ld* dP) {
  P[0] = 1.0L;
  dP[0] = 0.0L;
  if (n == 0) return;
  P[1] = x;
  dP[1] = 1.0L;
  for (int k = 1; k < n; ++k) {
    P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
    dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
  }
}

void gauss_legendre_rule(int q, double* x, double* w) {
  const ld pi = 3.14159265358979323846264338327950288L;
  ld P[64], dP[64];
  for (int i = 0; i < q; ++i) {
    // initial guess (Tricomi), roots numbered from the right
    ld t = cosl(pi * (4 * (i + 1) - 1) / (4 * q + 2));
    for (int it = 0; it < 60; ++it) {
      legendre_all(q, t, P, dP);
      const ld dt = P[q] / dP[q];
      t -= dt;
      if (fabsl(dt) < 1e-30L) break;
    }
    legendre_all(q, t, P, dP);
    ld s = 0.0L;
    for (int k = 0; k < q; ++k) s += (k + 0.5L) * P[k] * P[k];
    x[q - 1 - i] = (double)t;  // ascending
    w[q - 1 - i] = (double)(1.0L / s);
  }
}

void gauss_lobatto_nodes(int p, double* x) {
  const ld pi = 3.14159265358979323846264338327950288L;
  ld P[64], dP[64];
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    ld t = -cosl(pi * i / p);
    for (int it = 0; it < 60; ++it) {
      legendre_all(p + 1, t, P, dP);
      const ld f = P[p + 1] - P[p - 1], df = dP[p + 1] - dP[p - 1];
      const ld dt = f / df;
      t -= dt;
      if (fabsl(dt) < 1e-30L) break;
    }
    x[i] = (double)t;
  }
}

void lagrange_barycentric(int n, const double* nodes, ld t, ld* phi, ld* dphi) {
  ld lam[64];
  for (int j = 0; j < n; ++j) {
    ld v = 1.0L;
    for (int m = 0; m < n; ++m)
      if (m != j) v *= ((ld)nodes[j] - (ld)nodes[m]);
    lam[j] = 1.0L / v;
  }
  ld den = 0.0L;
  for (int m = 0; m < n; ++m) den += lam[m] / (t - (ld)nodes[m]);
  for (int j = 0; j < n; ++j) {
    phi[j] = (lam[j] / (t - (ld)nodes[j])) / den;
    ld sl = 0.0L;
    for (int m = 0; m < n; ++m)
      if (m != j) sl += 1.0L / (t - (ld)nodes[m]);
    dphi[j] = phi[j] * sl;
  }
}

void build_tables(int p, LorTables* T) {
  memset(T, 0, sizeof(*T));
  const int q = p + 2, n = p + 1;
  T->p = p;
  T->q = q;
  T->n = n;
  gauss_legendre_rule(q, T->gx, T->gw);
  gauss_lobatto_nodes(p, T->gll);
  for (int g = 0; g < q; ++g) {
    T->gl0[g] = (double)(0.5L * (1.0L - (ld)T->gx[g]));
    T->gl1[g] = (double)(0.5L * (1.0L + (ld)T->gx[g]));
  }
  for (int g = 0; g < q; ++g) {
    ld phi[64], dphi[64];
    lagrange_barycentric(n, T->gll, (ld)T->gx[g], phi, dphi);
    for (int i = 0; i < n; ++i) {
      T->B[g * n + i] = (double)phi[i];
      T->Dm[g * n + i] = (double)dphi[i];
    }
  }
  const ld inv_sqrt3 = 0.577350269189625764509148780501957456L;
  for (int a = 0; a < p; ++a) {
    const ld lo = T->gll[a], hi = T->gll[a + 1];
    const ld r = 0.5L * (hi - lo), mid = 0.5L * (hi + lo);
    T->sub_r[a] = (double)r;
    T->sub_rinv[a] = (double)(1.0L / r);
    for (int s = 0; s < 2; ++s) {
      const ld t = mid + (s ? 1.0L : -1.0L) * r * inv_sqrt3;
      T->sub_t[2 * a + s] = (double)t;
      T->sub_l0[2 * a + s] = (double)(0.5L * (1.0L - t));
      T->sub_l1[2 * a + s] = (double)(0.5L * (1.0L + t));
    }
  }
  // Gauss points of each LOR interval: interval(t) = #{interior GLL nodes < t}
  int bin[LOR_MAX_Q];
  for (int g = 0; g < q; ++g) {
    int c = 0;
    for (int m = 1; m < p; ++m)
      if (T->gll[m] < T->gx[g]) ++c;
    bin[g] = c;
  }
  for (int a = 0; a < p; ++a) {
    T->bin_first[a] = -1;
    T->bin_count[a] = 0;
  }
  for (int g = 0; g < q; ++g) {
    if (T->bin_first[bin[g]] < 0) T->bin_first[bin[g]] = g;
    T->bin_count[bin[g]]++;
  }
  for (int g = 0; g < q; ++g) {
    ld s = 0.0L;
    for (int h = 0; h < q; ++h)
      if (bin[h] == bin[g]) s += T->gw[h];
    T->bin_w[g] = (double)((ld)T->gw[g] / s);
  }
}

int set_err(lor_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_err(lor_ctx* c, cudaError_t e, const char* what) {
  return set_err(c, LOR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Host-side fault injection: with LOR_DEVICE_ALLOC_LIMIT=<bytes> in the
// environment, an allocation that would take a context's own device buffers
// above that many bytes fails as a failed cudaMalloc does (LOR_ENOMEM), before
// any device call.  Unset, empty or not a number: no limit.
size_t device_alloc_limit() {
  const char* s = getenv("LOR_DEVICE_ALLOC_LIMIT");
  if (!s || !*s) return SIZE_MAX;
  char* end = nullptr;
  const unsigned long long v = strtoull(s, &end, 10);
  return *end == 0 ? (size_t)v : SIZE_MAX;
}

template <typename T>
int alloc(lor_ctx* c, T** p, size_t count, const char* what) {
  if (*p) return LOR_OK;
  const size_t bytes = sizeof(T) * (count ? count : 1), limit = device_alloc_limit();
  if (c->device_bytes > limit || bytes > limit - c->device_bytes) {
    *p = nullptr;
    return set_err(c, LOR_ENOMEM, std::string("device allocation failed: ") + what + " (over LOR_DEVICE_ALLOC_LIMIT)");
  }
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(c, LOR_ENOMEM, std::string("device allocation failed: ") + what);
  }
  c->device_bytes += bytes;
  return LOR_OK;
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

// The same budget for blocks allocated by the general-mesh builders.
cudaError_t ctx_device_alloc(void* cv, void** p, size_t bytes) {
  lor_ctx* c = (lor_ctx*)cv;
  const size_t limit = device_alloc_limit();
  if (c->device_bytes > limit || bytes > limit - c->device_bytes) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e;
  }
  c->device_bytes += bytes;
  return cudaSuccess;
}

void ctx_device_release(void* cv, void* p, size_t bytes) {
  lor_ctx* c = (lor_ctx*)cv;
  cudaFree(p);
  c->device_bytes -= bytes;
}

LorDeviceAlloc device_allocator(lor_ctx* c) { return LorDeviceAlloc{c, ctx_device_alloc, ctx_device_release}; }

// A failed allocation through the budget is LOR_ENOMEM, anything else LOR_ECUDA.
int builder_err(lor_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return set_err(c, LOR_ENOMEM, std::string("device allocation failed: ") + what);
  return cuda_err(c, e, what);
}

void free_all(lor_ctx* c) {
  cudaFree(c->verts);
  cudaFree(c->Dq);
  cudaFree(c->kappa);
  cudaFree(c->beta);
  cudaFree(c->Mq);
  cudaFree(c->rowptr);
  cudaFree(c->colidx);
  cudaFree(c->vals64);
  cudaFree(c->vals32);
  cudaFree(c->d_status);
  cudaFree(c->dinv64);
  cudaFree(c->dinv32);
  cudaFree(c->pc_work);
  cudaFree(c->pcg_work);
  cudaFree(c->red);
  cudaFree(c->red_count);
  cudaFree(c->ecorners);
  cudaFree(c->edofs);
  cudaFree(c->ess);
  cudaFree(c->etail);
  cudaFree(c->ehead);
  cudaFree(c->Dq32);
  cudaFree(c->Mq32);
  cudaFree(c->ir_work);
  if (c->h_scalar) cudaFreeHost(c->h_scalar);
}

int read_status(lor_ctx* c, cudaStream_t s, int* flags) {
  cudaError_t e = cudaMemcpyAsync(c->h_scalar, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(c, e, "status read");
  memcpy(flags, c->h_scalar, sizeof(int));
  return LOR_OK;
}

}  // namespace

void lor_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int lor_ensure_f32_factors(lor_ctx* c, cudaStream_t s) {
  if (c->have_d32) return LOR_OK;
  const int64_t nq = c->m.nel * (int64_t)c->T.q * c->T.q * c->T.q;
  int rc = alloc(c, &c->Dq32, 6 * nq, "FP32 D");
  if (!rc && c->have_beta) rc = alloc(c, &c->Mq32, nq, "FP32 beta w detJ");
  if (rc) return rc;
  cudaError_t e = lor_launch_d_to_f32(c->m, c->Dq, c->Dq32, s);
  if (e == cudaSuccess && c->have_beta) e = lor_launch_to_f32(c->Mq, c->Mq32, nq, s);
  if (e != cudaSuccess) return cuda_err(c, e, "FP32 operator factors");
  c->have_d32 = true;
  return LOR_OK;
}

int lor_alloc_ir_work(lor_ctx* c) { return alloc(c, &c->ir_work, 2 * c->m.ndof, "refinement work"); }

extern "C" {

const char* lor_last_error(const lor_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int lor_create(lor_ctx** out, const lor_config* cfg, const double* d_vertices, void* stream) {
  if (!out) return set_err(nullptr, LOR_EINVAL, "lor_create: out is NULL");
  *out = nullptr;
  if (!cfg || !d_vertices) return set_err(nullptr, LOR_EINVAL, "lor_create: cfg or vertices is NULL");
  if (cfg->p < 1 || cfg->p > LOR_MAX_P)
    return set_err(nullptr, LOR_EINVAL, "lor_create: p must be in [1, " + std::to_string(LOR_MAX_P) + "]");
  if (cfg->nex < 1 || cfg->ney < 1 || cfg->nez < 1) return set_err(nullptr, LOR_EINVAL, "lor_create: empty mesh");
  const int64_t p = cfg->p;
  const int64_t nx = cfg->nex * p + 1, ny = cfg->ney * p + 1, nz = cfg->nez * p + 1;
  const int64_t lim = int64_t(1) << 31;  // each factor bounded before the next product: no int64 overflow
  if (nx >= lim || ny >= lim || nz >= lim || nx * ny >= lim || nx * ny * nz >= lim)
    return set_err(nullptr, LOR_EINVAL, "lor_create: more than 2^31-1 DOFs (int32 column indices)");
  lor_ctx* c = new (std::nothrow) lor_ctx();
  if (!c) return set_err(nullptr, LOR_ENOMEM, "lor_create: host allocation failed");
  c->cfg = *cfg;
  cudaGetDevice(&c->device);
  build_tables(cfg->p, &c->T);
  LorMesh& m = c->m;
  m.nex = cfg->nex;
  m.ney = cfg->ney;
  m.nez = cfg->nez;
  m.p = cfg->p;
  m.nx = nx;
  m.ny = ny;
  m.nz = nz;
  m.ndof = nx * ny * nz;
  m.nel = (int64_t)cfg->nex * cfg->ney * cfg->nez;
  m.nnz = (3 * nx - 2) * (3 * ny - 2) * (3 * nz - 2);
  const int64_t nv = (int64_t)(cfg->nex + 1) * (cfg->ney + 1) * (cfg->nez + 1);
  int rc = LOR_OK;
  if (!rc) rc = alloc(c, &c->verts, 3 * nv, "vertices");
  if (!rc) rc = alloc(c, &c->d_status, 4, "status");
  if (!rc) rc = alloc(c, &c->red, LOR_RED_BLOCKS + 16 + 2 * LOR_PCG_MAX_BLOCKS, "reduction");
  if (!rc) rc = alloc(c, &c->red_count, 8, "reduction counters");
  if (!rc) rc = alloc(c, &c->pcg_work, 4 * m.ndof, "pcg work");
  if (!rc && cudaMallocHost((void**)&c->h_scalar, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->h_scalar = nullptr;
    rc = set_err(c, LOR_ENOMEM, "pinned host allocation failed");
  }
  if (rc) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return rc;
  }
  m.verts = c->verts;
  cudaError_t e = cudaMemcpyAsync(c->verts, d_vertices, sizeof(double) * 3 * nv, cudaMemcpyDeviceToDevice, S(stream));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), S(stream));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->red_count, 0, 8 * sizeof(unsigned), S(stream));
  if (e == cudaSuccess) e = lor_launch_geometry_check(m, c->T, c->d_status, S(stream));
  int flags = 0;
  if (e == cudaSuccess) {
    rc = read_status(c, S(stream), &flags);
  } else {
    rc = cuda_err(c, e, "lor_create");
  }
  if (!rc && (flags & LOR_FLAG_BAD_GEOM)) rc = set_err(c, LOR_EGEOM, "lor_create: a Jacobian determinant is <= 0");
  if (rc) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return rc;
  }
  *out = c;
  return LOR_OK;
}

int lor_create_general(lor_ctx** out, int p, int64_t nel, int64_t ndof, const double* d_corners,
                       const int64_t* d_elem_dofs, const uint8_t* d_ess, void* stream) {
  if (!out) return set_err(nullptr, LOR_EINVAL, "lor_create_general: out is NULL");
  *out = nullptr;
  if (!d_corners || !d_elem_dofs) return set_err(nullptr, LOR_EINVAL, "lor_create_general: corners or map is NULL");
  if (p < 1 || p > LOR_MAX_P)
    return set_err(nullptr, LOR_EINVAL, "lor_create_general: p must be in [1, " + std::to_string(LOR_MAX_P) + "]");
  if (nel < 1 || ndof < 1) return set_err(nullptr, LOR_EINVAL, "lor_create_general: empty mesh");
  if (ndof >= (int64_t(1) << 31))
    return set_err(nullptr, LOR_EINVAL, "lor_create_general: more than 2^31-1 DOFs (int32 column indices)");
  if (nel > (INT64_MAX / 8) / ((int64_t)(LOR_MAX_P + 1) * (LOR_MAX_P + 1) * (LOR_MAX_P + 1)))
    return set_err(nullptr, LOR_EINVAL, "lor_create_general: element count overflows the byte size of its arrays");
  lor_ctx* c = new (std::nothrow) lor_ctx();
  if (!c) return set_err(nullptr, LOR_ENOMEM, "lor_create_general: host allocation failed");
  c->cfg.p = p;
  c->cfg.nex = c->cfg.ney = c->cfg.nez = 0;
  c->general = true;
  cudaGetDevice(&c->device);
  build_tables(p, &c->T);
  LorMesh& m = c->m;
  // the structured extents are unused on a general mesh; 1 keeps any index
  // arithmetic that is evaluated but not used free of divisions by zero
  m.nex = m.ney = m.nez = 1;
  m.p = p;
  m.nx = m.ny = m.nz = 1;
  m.ndof = ndof;
  m.nel = nel;
  m.verts = nullptr;
  const int64_t n3 = (int64_t)(p + 1) * (p + 1) * (p + 1);
  int rc = LOR_OK;
  if (!rc) rc = alloc(c, &c->ecorners, 24 * nel, "element corners");
  if (!rc) rc = alloc(c, &c->edofs, n3 * nel, "element-to-DOF map");
  if (!rc) rc = alloc(c, &c->ess, ndof, "essential mask");
  if (!rc) rc = alloc(c, &c->d_status, 4, "status");
  if (!rc) rc = alloc(c, &c->red, LOR_RED_BLOCKS + 16 + 2 * LOR_PCG_MAX_BLOCKS, "reduction");
  if (!rc) rc = alloc(c, &c->red_count, 8, "reduction counters");
  if (!rc) rc = alloc(c, &c->pcg_work, 4 * ndof, "pcg work");
  if (!rc && cudaMallocHost((void**)&c->h_scalar, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->h_scalar = nullptr;
    rc = set_err(c, LOR_ENOMEM, "pinned host allocation failed");
  }
  cudaError_t e = cudaSuccess;
  if (!rc) {
    m.ecorners = c->ecorners;
    m.edofs = c->edofs;
    m.ess = c->ess;
    e = cudaMemcpyAsync(c->ecorners, d_corners, sizeof(double) * 24 * nel, cudaMemcpyDeviceToDevice, S(stream));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->edofs, d_elem_dofs, sizeof(int64_t) * n3 * nel, cudaMemcpyDeviceToDevice, S(stream));
    if (e == cudaSuccess)
      e = d_ess ? cudaMemcpyAsync(c->ess, d_ess, ndof, cudaMemcpyDeviceToDevice, S(stream))
                : cudaMemsetAsync(c->ess, 0, ndof, S(stream));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), S(stream));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->red_count, 0, 8 * sizeof(unsigned), S(stream));
    if (e == cudaSuccess) e = lor_launch_geometry_check(m, c->T, c->d_status, S(stream));
    if (e != cudaSuccess) rc = cuda_err(c, e, "lor_create_general");
  }
  if (!rc) {
    e = lor_general_pattern(m, device_allocator(c), &c->rowptr, &c->colidx, &m.nnz, c->d_status, S(stream));
    if (e != cudaSuccess) rc = builder_err(c, e, "lor_create_general: LOR pattern");
  }
  int flags = 0;
  if (!rc) rc = read_status(c, S(stream), &flags);
  if (!rc && (flags & LOR_FLAG_BAD_MAP))
    rc = set_err(c, LOR_EINVAL, "lor_create_general: element-to-DOF map entry out of [0, ndof) or vertex valence > 64");
  if (!rc && (flags & LOR_FLAG_BAD_GEOM))
    rc = set_err(c, LOR_EGEOM, "lor_create_general: a Jacobian determinant is <= 0");
  if (rc) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return rc;
  }
  m.rowptr = c->rowptr;
  m.colidx = c->colidx;
  c->have_pattern = true;
  *out = c;
  return LOR_OK;
}

int lor_launch_count(int64_t* count) {
  if (!count) return LOR_EINVAL;
  *count = g_launches.load(std::memory_order_relaxed);
  return LOR_OK;
}

int lor_destroy(lor_ctx* ctx) {
  if (!ctx) return LOR_OK;
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return LOR_OK;
}

int lor_sizes(const lor_ctx* ctx, int64_t* ndof, int64_t* nnz, int64_t* nel, int64_t* nqpt) {
  if (!ctx) return LOR_EINVAL;
  if (ndof) *ndof = ctx->m.ndof;
  if (nnz) *nnz = ctx->m.nnz;
  if (nel) *nel = ctx->m.nel;
  if (nqpt) *nqpt = ctx->m.nel * (int64_t)ctx->T.q * ctx->T.q * ctx->T.q;
  return LOR_OK;
}

int lor_set_coefficient(lor_ctx* c, const double* d_kappa, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_kappa) return set_err(c, LOR_EINVAL, "lor_set_coefficient: kappa is NULL");
  const int64_t nq = c->m.nel * (int64_t)c->T.q * c->T.q * c->T.q;
  int rc = alloc(c, &c->Dq, (size_t)lor_d_doubles(nq), "D");
  if (!rc) rc = alloc(c, &c->kappa, nq, "kappa");
  if (rc) return rc;
  cudaError_t e = lor_launch_setup(c->m, c->T, d_kappa, c->kappa, c->Dq, c->d_status, S(stream));
  if (e != cudaSuccess) return cuda_err(c, e, "lor_set_coefficient");
  c->have_coeff = true;
  c->have_d32 = false;
  return LOR_OK;
}

int lor_set_reaction(lor_ctx* c, const double* d_beta, void* stream) {
  if (!c) return LOR_EINVAL;
  c->have_d32 = false;
  if (!d_beta) {
    c->have_beta = false;
    return LOR_OK;
  }
  const int64_t nq = c->m.nel * (int64_t)c->T.q * c->T.q * c->T.q;
  int rc = alloc(c, &c->beta, nq, "beta");
  if (!rc) rc = alloc(c, &c->Mq, nq, "beta w detJ");
  if (rc) return rc;
  cudaError_t e = lor_launch_reaction_setup(c->m, c->T, d_beta, c->beta, c->Mq, c->d_status, S(stream));
  if (e != cudaSuccess) return cuda_err(c, e, "lor_set_reaction");
  c->have_beta = true;
  return LOR_OK;
}

int lor_lor_mesh(lor_ctx* c, double* d_corners, int64_t* d_dofs, double* d_kappa_sub, double* d_beta_sub,
                 uint8_t* d_ess, void* stream) {
  if (!c) return LOR_EINVAL;
  if (c->general) return set_err(c, LOR_ESTATE, "lor_lor_mesh: structured (lor_create) meshes only");
  if (!d_corners || !d_dofs || !d_kappa_sub) return set_err(c, LOR_EINVAL, "lor_lor_mesh: NULL output array");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_lor_mesh: call lor_set_coefficient first");
  if (d_beta_sub && !c->have_beta) return set_err(c, LOR_ESTATE, "lor_lor_mesh: beta_sub asked without lor_set_reaction");
  cudaError_t e = lor_launch_lor_mesh(c->m, c->T, c->kappa, d_beta_sub ? c->beta : nullptr, d_corners, d_dofs,
                                      d_kappa_sub, d_beta_sub, d_ess, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_lor_mesh");
}

int lor_assemble_unstructured(lor_ctx* c, int64_t nsub, const double* d_corners, const int64_t* d_dofs,
                              const double* d_kappa_sub, const double* d_beta_sub, int64_t n, int64_t nnz,
                              const int64_t* d_rowptr, const int32_t* d_colidx, const uint8_t* d_ess, void* d_values,
                              int dtype, void* stream) {
  if (!c) return LOR_EINVAL;
  if (dtype != LOR_F64 && dtype != LOR_F32) return set_err(c, LOR_EINVAL, "lor_assemble_unstructured: bad dtype");
  if (nsub < 0 || n < 0 || nnz < 0 || (nsub > 0 && (!d_corners || !d_dofs || !d_kappa_sub)) || !d_rowptr ||
      !d_colidx || (nnz > 0 && !d_values))
    return set_err(c, LOR_EINVAL, "lor_assemble_unstructured: bad arguments");
  cudaError_t e = lor_launch_assemble_unstructured(nsub, d_corners, d_dofs, d_kappa_sub, d_beta_sub, n, nnz, d_rowptr,
                                                   d_colidx, d_ess, d_values, dtype, c->d_status, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_assemble_unstructured");
}

int lor_discrete_gradient(lor_ctx* c, int64_t* d_rowptr, int32_t* d_colidx, double* d_values, int64_t* nedge,
                          void* stream) {
  if (!c) return LOR_EINVAL;
  if (c->general && c->nedge < 0) {  // enumerate the LOR edges once
    cudaError_t e = lor_general_edges(c->m, device_allocator(c), &c->etail, &c->ehead, &c->nedge, c->d_status,
                                      S(stream));
    if (e != cudaSuccess) return builder_err(c, e, "lor_discrete_gradient: LOR edges");
  }
  const int64_t ne = c->general ? c->nedge : lor_edge_count(c->m);
  if (nedge) *nedge = ne;
  if (!d_rowptr && !d_colidx && !d_values) return LOR_OK;
  if (!d_rowptr || !d_colidx || !d_values)
    return set_err(c, LOR_EINVAL, "lor_discrete_gradient: give all three output arrays or none");
  if (((uintptr_t)d_colidx & 7) || ((uintptr_t)d_values & 15))
    return set_err(c, LOR_EINVAL, "lor_discrete_gradient: colidx must be 8-byte and values 16-byte aligned");
  if (c->m.ndof > INT32_MAX) return set_err(c, LOR_EINVAL, "lor_discrete_gradient: more vertices than int32 columns");
  cudaError_t e = c->general
                      ? lor_launch_general_gradient(ne, c->etail, c->ehead, d_rowptr, d_colidx, d_values, S(stream))
                      : lor_launch_discrete_gradient(c->m, d_rowptr, d_colidx, d_values, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_discrete_gradient");
}

int lor_vertex_coordinates(lor_ctx* c, double* d_xyz, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_xyz) return set_err(c, LOR_EINVAL, "lor_vertex_coordinates: xyz is NULL");
  cudaError_t e = c->general ? lor_launch_general_vertices(c->m, c->T, d_xyz, S(stream))
                             : lor_launch_vertex_coordinates(c->m, c->T, d_xyz, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_vertex_coordinates");
}

int lor_check(lor_ctx* c, void* stream) {
  if (!c) return LOR_EINVAL;
  int flags = 0;
  int rc = read_status(c, S(stream), &flags);
  if (rc) return rc;
  if (flags) {
    cudaMemsetAsync(c->d_status, 0, sizeof(int), S(stream));
    cudaStreamSynchronize(S(stream));
    if (flags & LOR_FLAG_TIMEOUT)
      return set_err(c, LOR_ETIMEOUT, "a bounded device wait expired (a bulk copy into shared memory never completed)");
    if (flags & LOR_FLAG_BAD_GEOM) return set_err(c, LOR_EGEOM, "a Jacobian determinant is <= 0");
    if (flags & LOR_FLAG_BAD_PATTERN)
      return set_err(c, LOR_EINVAL, "lor_assemble_unstructured: a coupling is missing from the given CSR pattern");
    return set_err(c, LOR_EINVAL, "kappa (and beta) must be finite and > 0 at every Gauss point");
  }
  return LOR_OK;
}

int lor_set_test_hooks(lor_ctx* c, unsigned flags) {
  if (!c) return LOR_EINVAL;
  if (flags & ~(LOR_TEST_EXPIRE_WAITS | LOR_TEST_UNSTAGED_CSR))
    return set_err(c, LOR_EINVAL, "lor_set_test_hooks: unknown flag");
  c->m.test_flags = flags;
  return LOR_OK;
}

int lor_build_pattern(lor_ctx* c, int64_t* d_rowptr, int32_t* d_colidx, void* stream) {
  if (!c) return LOR_EINVAL;
  if ((d_rowptr == nullptr) != (d_colidx == nullptr))
    return set_err(c, LOR_EINVAL, "lor_build_pattern: give both output arrays or neither");
  int rc = alloc(c, &c->rowptr, c->m.ndof + 1, "rowptr");
  if (!rc) rc = alloc(c, &c->colidx, c->m.nnz, "colidx");
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!c->have_pattern) {
    e = lor_launch_pattern(c->m, c->rowptr, c->colidx, S(stream));
    if (e != cudaSuccess) return cuda_err(c, e, "lor_build_pattern");
    c->have_pattern = true;
  }
  if (d_rowptr) {
    e = cudaMemcpyAsync(d_rowptr, c->rowptr, sizeof(int64_t) * (c->m.ndof + 1), cudaMemcpyDeviceToDevice, S(stream));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_colidx, c->colidx, sizeof(int32_t) * c->m.nnz, cudaMemcpyDeviceToDevice, S(stream));
    if (e != cudaSuccess) return cuda_err(c, e, "lor_build_pattern copy");
  }
  return LOR_OK;
}

int lor_assemble(lor_ctx* c, void* d_values, int dtype, void* stream) {
  if (!c) return LOR_EINVAL;
  if (dtype != LOR_F64 && dtype != LOR_F32) return set_err(c, LOR_EINVAL, "lor_assemble: bad dtype");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_assemble: call lor_set_coefficient first");
  void* out = d_values;
  if (!out) {
    if (!c->have_pattern) return set_err(c, LOR_ESTATE, "lor_assemble: call lor_build_pattern first");
    int rc = dtype == LOR_F64 ? alloc(c, &c->vals64, c->m.nnz + LOR_VALS_PAD, "values f64")
                                : alloc(c, &c->vals32, c->m.nnz + LOR_VALS_PAD, "values f32");
    if (rc) return rc;
    out = dtype == LOR_F64 ? (void*)c->vals64 : (void*)c->vals32;
  }
  cudaError_t e = lor_launch_assemble(c->m, c->T, c->kappa, c->have_beta ? c->beta : nullptr, out, dtype, S(stream));
  if (e != cudaSuccess) return cuda_err(c, e, "lor_assemble");
  if (!d_values) {
    if (dtype == LOR_F64) c->have_vals64 = true;
    else c->have_vals32 = true;
  }
  return LOR_OK;
}

int lor_apply(lor_ctx* c, const double* d_x, double* d_y, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_x || !d_y || d_x == d_y) return set_err(c, LOR_EINVAL, "lor_apply: x, y must be distinct device arrays");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_apply: call lor_set_coefficient first");
  cudaError_t e = lor_launch_apply(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, d_x, d_y, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_apply");
}

int lor_apply_f32(lor_ctx* c, const double* d_x, double* d_y, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_x || !d_y || d_x == d_y) return set_err(c, LOR_EINVAL, "lor_apply_f32: x, y must be distinct device arrays");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_apply_f32: call lor_set_coefficient first");
  int rc = lor_ensure_f32_factors(c, S(stream));
  if (rc) return rc;
  cudaError_t e = lor_launch_apply_f32(c->m, c->T, c->Dq32, c->have_beta ? c->Mq32 : nullptr, d_x, d_y, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_apply_f32");
}

int lor_apply_backward(lor_ctx* c, const double* d_x, const double* d_gy, double* d_gx, double* d_gkappa,
                       void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_gy || (d_gkappa && !d_x) || (d_gx && d_gx == d_gy))
    return set_err(c, LOR_EINVAL, "lor_apply_backward: bad arguments");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_apply_backward: call lor_set_coefficient first");
  cudaError_t e = lor_launch_apply_backward(c->m, c->T, c->Dq, c->have_beta ? c->Mq : nullptr, c->kappa, d_x, d_gy, d_gx,
                                            d_gkappa, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_apply_backward");
}

int lor_load_vector(lor_ctx* c, const double* d_f, double* d_b, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_b) return set_err(c, LOR_EINVAL, "lor_load_vector: b is NULL");
  cudaError_t e = lor_launch_load_vector(c->m, c->T, d_f, d_b, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_load_vector");
}

int lor_spmv(lor_ctx* c, int dtype, const double* d_x, double* d_y, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_x || !d_y || d_x == d_y) return set_err(c, LOR_EINVAL, "lor_spmv: x, y must be distinct device arrays");
  const bool have = dtype == LOR_F64 ? c->have_vals64 : dtype == LOR_F32 ? c->have_vals32 : false;
  if (!have) return set_err(c, LOR_ESTATE, "lor_spmv: no assembled matrix of that dtype in the context");
  cudaError_t e = lor_launch_spmv(c->m, dtype == LOR_F64 ? (const void*)c->vals64 : (const void*)c->vals32, dtype, d_x,
                                  d_y, c->d_status, S(stream));
  return e == cudaSuccess ? LOR_OK : cuda_err(c, e, "lor_spmv");
}

int lor_precond_setup(lor_ctx* c, int kind, int dtype, int degree, double lo_ratio, double hi_ratio,
                      double lambda_max, int power_iters, const double* d_v0, double* lambda_out, void* stream) {
  if (!c) return LOR_EINVAL;
  if (kind == LOR_PRECOND_NONE) {
    c->pc_kind = kind;
    return LOR_OK;
  }
  if (kind != LOR_PRECOND_JACOBI && kind != LOR_PRECOND_CHEB) return set_err(c, LOR_EINVAL, "lor_precond_setup: bad kind");
  if (dtype != LOR_F64 && dtype != LOR_F32) return set_err(c, LOR_EINVAL, "lor_precond_setup: bad dtype");
  const bool have = dtype == LOR_F64 ? c->have_vals64 : c->have_vals32;
  if (!have) return set_err(c, LOR_ESTATE, "lor_precond_setup: assemble the context matrix of that dtype first");
  if (kind == LOR_PRECOND_CHEB && (degree < 1 || !(lo_ratio > 0) || !(hi_ratio > lo_ratio)))
    return set_err(c, LOR_EINVAL, "lor_precond_setup: need degree >= 1 and 0 < lo_ratio < hi_ratio");
  const int64_t n = c->m.ndof;
  int rc = dtype == LOR_F64 ? alloc(c, &c->dinv64, n, "dinv") : alloc(c, &c->dinv32, n, "dinv");
  if (!rc && kind == LOR_PRECOND_CHEB) {
    if (c->pc_work && c->pc_dtype != dtype) {
      cudaFree(c->pc_work);
      c->pc_work = nullptr;
      c->device_bytes -= (size_t)(3 * n * (c->pc_dtype == LOR_F64 ? 8 : 4));
    }
    rc = alloc(c, (char**)&c->pc_work, 3 * n * (dtype == LOR_F64 ? 8 : 4), "smoother work");
  }
  if (rc) return rc;
  cudaError_t e = lor_launch_diag_inv(c->m, dtype == LOR_F64 ? (const void*)c->vals64 : (const void*)c->vals32, dtype,
                                      dtype == LOR_F64 ? (void*)c->dinv64 : (void*)c->dinv32, S(stream));
  if (e != cudaSuccess) return cuda_err(c, e, "lor_precond_setup");
  c->pc_kind = kind;
  c->pc_dtype = dtype;
  c->pc_degree = degree;
  double lmax = lambda_max;
  if (kind == LOR_PRECOND_CHEB && !(lmax > 0)) {
    if (power_iters < 1) return set_err(c, LOR_EINVAL, "lor_precond_setup: power_iters must be >= 1");
    rc = lor_power_iteration(c, dtype, power_iters, d_v0, &lmax, S(stream));
    if (rc) {
      c->pc_kind = LOR_PRECOND_NONE;
      return rc;
    }
  }
  c->pc_lmax = lmax;
  c->pc_lo = lo_ratio * lmax;
  c->pc_hi = hi_ratio * lmax;
  if (lambda_out) *lambda_out = lmax;
  return LOR_OK;
}

int lor_precond_apply(lor_ctx* c, const double* d_r, double* d_z, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_r || !d_z || d_r == d_z) return set_err(c, LOR_EINVAL, "lor_precond_apply: r, z must be distinct device arrays");
  return lor_precond_apply_impl(c, d_r, d_z, S(stream));
}

int lor_pcg_solve(lor_ctx* c, const double* d_b, double* d_x, double rtol, int maxit, int* iters,
                  double* final_rel_residual, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_b || !d_x || d_b == d_x) return set_err(c, LOR_EINVAL, "lor_pcg_solve: b, x must be distinct device arrays");
  if (!(rtol > 0) || maxit < 0) return set_err(c, LOR_EINVAL, "lor_pcg_solve: need rtol > 0 and maxit >= 0");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_pcg_solve: call lor_set_coefficient first");
  return lor_pcg_impl(c, d_b, d_x, rtol, maxit, iters, final_rel_residual, S(stream));
}

int lor_pcg_solve_ir(lor_ctx* c, const double* d_b, double* d_x, double rtol, double inner_rtol, int maxit,
                     int scheme, int* outer_iters, int* inner_iters, double* final_rel_residual, void* stream) {
  if (!c) return LOR_EINVAL;
  if (!d_b || !d_x || d_b == d_x) return set_err(c, LOR_EINVAL, "lor_pcg_solve_ir: b, x must be distinct device arrays");
  if (!(rtol > 0) || !(inner_rtol > 0) || !(inner_rtol < 1) || maxit < 0)
    return set_err(c, LOR_EINVAL, "lor_pcg_solve_ir: need rtol > 0, 0 < inner_rtol < 1 and maxit >= 0");
  if (scheme != LOR_IR_RESTART && scheme != LOR_IR_REPLACE)
    return set_err(c, LOR_EINVAL, "lor_pcg_solve_ir: unknown scheme");
  if (!c->have_coeff) return set_err(c, LOR_ESTATE, "lor_pcg_solve_ir: call lor_set_coefficient first");
  return lor_pcg_ir_impl(c, d_b, d_x, rtol, inner_rtol, maxit, scheme, outer_iters, inner_iters, final_rel_residual,
                         S(stream));
}

}  // extern "C"
