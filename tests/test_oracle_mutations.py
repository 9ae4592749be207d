"""Mutation tests of the oracle's pins: each case plants one plausible
mistake in a copy of oracle/lor_oracle.c (a dropped term, a wrong weight,
sign or index, a swapped operand), builds it, and runs the CPU pin suite
against that build; at least one pin must fail.  The planted copies live in
a temporary directory and are loaded through LOR_ORACLE_LIB; the oracle
itself is untouched."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "lor_oracle.c")
PINS = ["tests/test_oracle_basis.py", "tests/test_oracle_ho.py", "tests/test_oracle_lor.py",
        "tests/test_oracle_solver.py", "tests/test_oracle_helmholtz.py", "tests/test_oracle_hcurl.py"]

# (name, original text, planted text)
MUTATIONS = [
    ("x-derivative uses the interpolation matrix",
     "sd += D[g0 * n + i] * u[(k * n + j) * n + i];", "sd += B[g0 * n + i] * u[(k * n + j) * n + i];"),
    ("z-stage derivative uses the interpolation matrix",
     "s2 += D[g2 * n + k] * BBu[(k * q + g1) * q + g0];", "s2 += B[g2 * n + k] * BBu[(k * q + g1) * q + g0];"),
    ("quadrature weight dropped from the metric factor",
     "M[a][b] = w * det * s;", "M[a][b] = det * s;"),
    ("transposed inverse Jacobian",
     "Ai[1][0] = c01 / det;", "Ai[1][0] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;"),
    ("Dirichlet rows of the apply set to zero",
     "y[I + nx * (J + ny * K)] = x[I + nx * (J + ny * K)];", "y[I + nx * (J + ny * K)] = 0.0;"),
    ("kappa_s as an unweighted average",
     "den[s] += w;", "den[s] += 1.0;"),
    ("sub-hex Gauss points at +-1/3",
     "const double g1 = 1.0 / sqrt(3.0);", "const double g1 = 1.0 / 3.0;"),
    ("reaction term without detJ",
     "* wg[g0] * wg[g1] * wg[g2] * detJ[e * nq3 + g];", "* wg[g0] * wg[g1] * wg[g2];"),
    ("LOR mass block uses phi_r twice",
     "wb * phi[r] * phi[s];", "wb * phi[r] * phi[r];"),
    ("Chebyshev step coefficient halved",
     "(2.0 * rho_new / delta) * res[i] / dg[i];", "(rho_new / delta) * res[i] / dg[i];"),
    ("PCG beta inverted",
     "double beta = rz_new / rz;", "double beta = rz / rz_new;"),
    ("Gauss-Lobatto Newton stopped after one step",
     "for (int it = 0; it < 100; ++it) {\n      double P, Pm1;\n      legendre_pair(p, t, &P, &Pm1);\n      double d1",
     "for (int it = 0; it < 1; ++it) {\n      double P, Pm1;\n      legendre_pair(p, t, &P, &Pm1);\n      double d1"),
    ("discrete gradient orientation lost",
     "values[2 * e] = -1.0;", "values[2 * e] = 1.0;"),
    ("power iteration without the diagonal scaling",
     "for (int64_t i = 0; i < n; ++i) w[i] /= d[i];", ""),
    ("load vector without detJ",
     "s += wg[g0] * wg[g1] * wg[g2] * detJ[e * nq3 + g] * fv * L[g0][i] * L[g1][j] * L[g2][k];",
     "s += wg[g0] * wg[g1] * wg[g2] * fv * L[g0][i] * L[g1][j] * L[g2][k];"),
    ("kappa_s bins shifted by half an interval",
     "      if (gll[m] < xg[g]) ++c;",
     "      if (0.5 * (gll[m] + gll[m - 1]) < xg[g]) ++c;"),
    ("kappa gradient with a wrong metric entry",
     "          double v1 = Gq[1] * a + Gq[3] * b + Gq[4] * c;",
     "          double v1 = Gq[2] * a + Gq[3] * b + Gq[4] * c;"),
    ("discrete gradient head on the wrong axis",
     "          colidx[2 * e + 1] = tail + stride[d];",
     "          colidx[2 * e + 1] = tail + stride[(d + 1) % 3];"),
    ("load vector reads f at the neighbouring Gauss point",
     "double fv = f ? f[e * nq3 + g] : 1.0;", "double fv = f ? f[e * nq3 + (g + 1) % nq3] : 1.0;"),
    ("apply with a wrong metric entry",
     "gr[3 * g + 1] = k * (Gq[1] * a + Gq[3] * b + Gq[4] * c);", "gr[3 * g + 1] = k * (Gq[2] * a + Gq[3] * b + Gq[4] * c);"),
    ("sub-hex coefficient of the transposed sub-hex",
     "bad |= lor_subhex_matrix(X, gll, a, b, c, ksub[e * p3 + a + p * (b + p * c)],",
     "bad |= lor_subhex_matrix(X, gll, a, b, c, ksub[e * p3 + b + p * (a + p * c)],"),
    ("CSR diagonal taken from the row's first entry",
     "      if (colidx[j] == i) d[i] += values[j];", "      if (j == rowptr[i]) d[i] += values[j];"),
    ("PCG step length against p.p",
     "double alpha = rz / dot(N, pv, Ap);", "double alpha = rz / dot(N, pv, pv);"),
    ("Chebyshev interval centre taken as its half-width",
     "double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;",
     "double theta = 0.5 * (hi - lo), delta = 0.5 * (hi - lo), sigma = theta / delta;"),
    ("transposed y stage pairs the derivative with the wrong component",
     "          s1 += D[g1 * n + j] * T1[(k * q + g1) * q + g0] + B[g1 * n + j] * T2[(k * q + g1) * q + g0];",
     "          s1 += B[g1 * n + j] * T1[(k * q + g1) * q + g0] + D[g1 * n + j] * T2[(k * q + g1) * q + g0];"),
    ("Gauss-Legendre weight without the 1 - x^2 factor",
     "    w[i] = 2.0 / ((1.0 - t * t) * dP * dP);",
     "    w[i] = 2.0 / (dP * dP);"),
    ("Lagrange derivative without the 1/(x_j - x_l) factor",
     "      double term = 1.0 / (nodes[j] - nodes[l]);",
     "      double term = 1.0;"),
    ("dense brute force maps reference gradients by J^-1 instead of J^-T",
     "grad[3 * a + d] = Ji[0][d] * gr[0] + Ji[1][d] * gr[1] + Ji[2][d] * gr[2];",
     "grad[3 * a + d] = Ji[d][0] * gr[0] + Ji[d][1] * gr[1] + Ji[d][2] * gr[2];"),
    ("selected LOR rows take the sub-hex row with y and z swapped",
     "          int rloc = (int)(I - sa) + 2 * (int)(J - sb) + 4 * (int)(Kk - sc);",
     "          int rloc = (int)(I - sa) + 2 * (int)(Kk - sc) + 4 * (int)(J - sb);"),
    ("DOF coordinates with the y and z reference coordinates swapped",
     "              double xi[3] = {gll[i], gll[j], gll[k]}, J[3][3];",
     "              double xi[3] = {gll[i], gll[k], gll[j]}, J[3][3];"),
    ("SpMV reads x at the row instead of the column",
     "    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) s += values[j] * x[colidx[j]];",
     "    for (int64_t j = rowptr[i]; j < rowptr[i + 1]; ++j) s += values[j] * x[i];"),
    ("general-mesh LOR looks up the element map with j and k swapped",
     "            dof[r] = dofs[e * n3 + i + n * (j + n * k)];",
     "            dof[r] = dofs[e * n3 + i + n * (k + n * j)];"),
    ("LOR Dirichlet diagonal left at zero",
     "        if (er || is_essential(cI, cJ, cK, nx, ny, nz)) A->values[j] = (cc == r) ? 1.0 : 0.0;",
     "        if (er || is_essential(cI, cJ, cK, nx, ny, nz)) A->values[j] = 0.0;"),
]


@pytest.mark.parametrize("name,orig,planted", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, orig, planted, tmp_path):
    src = open(SRC).read()
    assert src.count(orig) == 1, "mutation site not found (oracle source changed?): " + name
    bad = tmp_path / "lor_oracle_mutant.c"
    bad.write_text(src.replace(orig, planted))
    lib = tmp_path / "liblor_oracle_mutant.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib), str(bad),
                    "-lm"], check=True)
    env = dict(os.environ, LOR_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "no pin caught: " + name + "\n" + r.stdout[-2000:]
