"""Pins of the oracle's solve phase: CSR spmv, the Chebyshev-Jacobi
preconditioner (reading R6), the power iteration, PCG (Section 3, step S2;
reading R7), the Poisson solution for f = 1, and the adjoint gradient."""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb

import oracle
from meshutil import element_corners, element_dofs, eliminate, essential_mask
from paper_2210_12253_gb300.inputs import make_problem, unit_cube_vertices


def random_spd_csr(n, seed, density=0.2):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=density, random_state=np.random.RandomState(seed)).toarray()
    A = A + A.T + n * np.eye(n) * (0.5 + rng.random(n))[:, None]
    S = sp.csr_matrix(A)
    S.sort_indices()
    return A, S.indptr.astype(np.int64), S.indices.astype(np.int64), S.data.copy()


def test_spmv_and_diagonal_match_scipy():
    A, rp, ci, v = random_spd_csr(40, 1)
    x = np.random.default_rng(2).standard_normal(40)
    np.testing.assert_allclose(oracle.csr_spmv(rp, ci, v, x), A @ x, rtol=1e-14)
    np.testing.assert_allclose(oracle.csr_diagonal(rp, ci, v), np.diag(A), rtol=0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_chebyshev_residual_polynomial_closed_form(k):
    """z = p_k(M^-1 A) M^-1 r with residual polynomial
    1 - t p_k(t) = T_k((theta - t)/delta) / T_k(theta/delta)."""
    A, rp, ci, v = random_spd_csr(30, 3)
    d = np.diag(A)
    S = A / np.sqrt(d)[:, None] / np.sqrt(d)[None, :]
    lam, Q = np.linalg.eigh(S)
    lo, hi = lam.max() / 30, 1.1 * lam.max()
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    Tk = npcheb.Chebyshev.basis(k)
    R = Tk((theta - lam) / delta) / Tk(theta / delta)
    pk = (1 - R) / lam
    r = np.random.default_rng(4).standard_normal(30)
    ref = (Q @ (pk * (Q.T @ (r / np.sqrt(d))))) / np.sqrt(d)
    z = oracle.chebyshev(rp, ci, v, r, k, lo, hi)
    np.testing.assert_allclose(z, ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_chebyshev_is_symmetric_positive():
    A, rp, ci, v = random_spd_csr(25, 5)
    lmax = scipy.linalg.eigh(A, np.diag(np.diag(A)), eigvals_only=True).max()
    P = np.stack([oracle.chebyshev(rp, ci, v, e, 3, lmax / 30, 1.1 * lmax) for e in np.eye(25)], axis=1)
    np.testing.assert_allclose(P, P.T, atol=1e-14 * np.abs(P).max())
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0


def test_power_iteration_converges_to_lambda_max():
    A, rp, ci, v = random_spd_csr(50, 6)
    lmax = scipy.linalg.eigh(A, np.diag(np.diag(A)), eigvals_only=True).max()
    v0 = np.random.default_rng(7).standard_normal(50)
    l20 = oracle.power_lambda_max(rp, ci, v, v0, 20)
    l500 = oracle.power_lambda_max(rp, ci, v, v0, 500)
    assert l20 <= lmax * (1 + 1e-12)
    assert abs(l500 - lmax) < 1e-9 * lmax


def test_power_iteration_on_diagonal_scaled_matrix():
    """For A = D T with T symmetric and D diagonal the estimate tracks the
    top eigenvalue of D^-1 A exactly after convergence (closed form)."""
    lam = np.array([1.0, 2.0, 5.0, 9.0])
    A = np.diag(lam)
    S = sp.csr_matrix(A)
    rp, ci, v = S.indptr.astype(np.int64), S.indices.astype(np.int64), S.data
    # D^-1 A = I for a diagonal A: every estimate is exactly 1
    assert abs(oracle.power_lambda_max(rp, ci, v, np.ones(4), 5) - 1.0) < 1e-15


def small_problem(p=2, dims=(2, 2, 2), seed=3):
    prob = make_problem("t", *dims, p, seed=seed, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    return prob, mesh


@pytest.mark.parametrize("precond", [oracle.PRECOND_NONE, oracle.PRECOND_JACOBI, oracle.PRECOND_CHEB])
def test_pcg_matches_dense_solve(precond):
    prob, mesh = small_problem()
    p, q = prob.p, prob.q
    A = eliminate(oracle.dense_general(element_corners(mesh.V, *(prob.nex, prob.ney, prob.nez)),
                                       element_dofs(prob.nex, prob.ney, prob.nez, p), prob.kappa, p, q, prob.ndof),
                  essential_mask(prob.nex, prob.ney, prob.nez, p))
    ref = scipy.linalg.solve(A, prob.rhs, assume_a="pos")
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True)
    lmax = oracle.power_lambda_max(*csr, np.random.default_rng(1).standard_normal(prob.ndof), 20)
    x, it, rel, rc = oracle.pcg(mesh, p, q, prob.kappa, csr, prob.rhs, 1e-12, 500, precond, 3, lmax / 30, 1.1 * lmax)
    assert rc == oracle.OK and rel <= 1e-12
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    r = prob.rhs - A @ x
    assert np.linalg.norm(r) <= 1.0000001e-12 * np.linalg.norm(prob.rhs)


def test_pcg_reports_no_convergence():
    prob, mesh = small_problem()
    csr = oracle.lor_assemble(mesh, prob.p, prob.q, prob.kappa, True)
    x, it, rel, rc = oracle.pcg(mesh, prob.p, prob.q, prob.kappa, csr, prob.rhs, 1e-14, 3,
                                oracle.PRECOND_JACOBI, raise_on_noconv=False)
    assert rc == oracle.ENOCONV and it == 3 and rel > 1e-14


def poisson_series(terms=301):
    """Exact solution of -Lap u = 1 on the unit cube with u = 0 on the
    boundary, by its sine series: int u and u(1/2,1/2,1/2)."""
    k = np.arange(1, terms + 1, 2, dtype=np.float64)
    I, J, K = np.meshgrid(k, k, k, indexing="ij")
    s2 = I ** 2 + J ** 2 + K ** 2
    coef = 64.0 / (np.pi ** 3 * I * J * K) / (np.pi ** 2 * s2)
    integral = (coef * 8.0 / (np.pi ** 3 * I * J * K)).sum()
    sgn = ((-1.0) ** ((I - 1) / 2)) * ((-1.0) ** ((J - 1) / 2)) * ((-1.0) ** ((K - 1) / 2))
    centre = (coef * sgn).sum()
    return integral, centre


def test_unit_source_poisson_solution():
    """4^3 undistorted elements, kappa = 1, f = 1, Jacobi-on-LOR PCG to 1e-10.
    The spaces Q_p are nested, so the Galerkin energy b^T u_h = a(u_h,u_h)
    increases monotonically with p and stays below int u (series value);
    the energy error and u_h(1/2,1/2,1/2) converge to the series solution."""
    integral, centre = poisson_series()
    assert abs(integral - 0.0201685) < 5e-7
    ne = 4
    mesh = oracle.Mesh(ne, ne, ne, unit_cube_vertices(ne, ne, ne))
    energies, centres = [], []
    for p in (2, 3, 4):
        q = p + 2
        k1 = np.ones((mesh.nel, q ** 3))
        b = oracle.load_vector(mesh, p, q)
        csr = oracle.lor_assemble(mesh, p, q, k1, True)
        u, it, rel, rc = oracle.pcg(mesh, p, q, k1, csr, b, 1e-10, 1000, oracle.PRECOND_JACOBI)
        assert rc == oracle.OK
        energies.append(b @ u)
        n = ne * p + 1
        c = n // 2
        centres.append(u[c + n * (c + n * c)])
    assert energies[0] < energies[1] < energies[2] <= integral + 1e-12
    err = [integral - e for e in energies]
    assert err[2] < 0.5 * err[0] and err[1] < 2e-4 * integral
    assert abs(centres[2] - centre) < abs(centres[0] - centre) and abs(centres[2] - centre) < 2e-4 * centre


def test_adjoint_gradient_matches_finite_differences():
    """J(theta) = 1/2 |u(theta) - u*|^2 with A(e^theta) u = b.  Adjoint:
    A lambda = u - u*, dJ/dkappa = -grad_kappa(u, lambda), dJ/dtheta = kappa dJ/dkappa."""
    dims, p = (2, 1, 2), 2
    prob = make_problem("t", *dims, p, seed=5, kappa="theta", rhs="normal")
    mesh = oracle.Mesh(*dims, prob.vertices)
    q = prob.q
    C, Dm = element_corners(mesh.V, *dims), element_dofs(*dims, p)
    ess = essential_mask(*dims, p)

    def solve(theta, rhs):
        A = eliminate(oracle.dense_general(C, Dm, np.exp(theta), p, q, prob.ndof), ess)
        return scipy.linalg.solve(A, rhs, assume_a="pos")

    ustar = solve(prob.theta_star, prob.rhs)

    def J(theta):
        d = solve(theta, prob.rhs) - ustar
        return 0.5 * d @ d

    u = solve(prob.theta, prob.rhs)
    lam = solve(prob.theta, u - ustar)
    _, gk = oracle.ho_apply_backward(mesh, p, q, np.exp(prob.theta), u, lam, want_gx=False)
    grad = -np.exp(prob.theta) * gk
    rng = np.random.default_rng(11)
    for _ in range(4):
        v = rng.standard_normal(prob.theta.shape)
        eps = 1e-6 * np.linalg.norm(prob.theta) / np.linalg.norm(v)
        fd = (J(prob.theta + eps * v) - J(prob.theta - eps * v)) / (2 * eps)
        assert abs(fd - (grad * v).sum()) <= 1e-6 * abs(fd) + 1e-14
