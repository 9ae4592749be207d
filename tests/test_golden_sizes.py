"""Section 4.1 prints the DOF and LOR-nonzero counts of its p = 6 problems
(tests/golden/paper_problem_sizes.txt).  On a Cartesian grid with n = n_e p + 1
points per axis the LOR pattern has 3n-2 couplings per axis (2 at each end,
3 inside), so nnz = (3n-2)^d; the oracle's assembled pattern obeys the same
per-axis count (test_oracle_lor.test_sparsity_pattern)."""
import os

import numpy as np

import oracle
from paper_2210_12253_gb300.inputs import unit_cube_vertices

HERE = os.path.dirname(os.path.abspath(__file__))


def rows():
    with open(os.path.join(HERE, "golden", "paper_problem_sizes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                yield tuple(int(t) for t in line.split())


def test_paper_sizes_follow_from_the_lor_pattern():
    for dim, nel, dofs, nnz in rows():
        ne = round(nel ** (1.0 / dim))
        assert ne ** dim == nel
        n = ne * 6 + 1
        assert n ** dim == dofs
        assert (3 * n - 2) ** dim == nnz


def test_oracle_pattern_count_matches_formula_on_small_grid():
    ne, p = 3, 6
    mesh = oracle.Mesh(ne, ne, ne, unit_cube_vertices(ne, ne, ne))
    rp, _, _ = oracle.lor_assemble(mesh, p, p + 2, np.ones((mesh.nel, (p + 2) ** 3)), True)
    n = ne * p + 1
    assert rp[-1] == (3 * n - 2) ** 3
