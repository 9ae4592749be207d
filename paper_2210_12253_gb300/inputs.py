"""Seeded synthetic inputs for LOR-preconditioned H1 diffusion.

This module only draws inputs; it holds none of the method's arithmetic.
Both the CUDA library and the CPU oracle consume exactly these arrays.

Recipe (one ``numpy.random.default_rng(seed)`` per workload, draws in this
order):

1. mesh jitter: unit-cube lattice of nex x ney x nez hexes; every interior
   vertex gets an independent U(-j*h_d, +j*h_d) offset per coordinate d
   (h_d = 1/ne_d, j = 0.10), drawn vertex by vertex in lexicographic order
   (x fastest), x then y then z.  Boundary vertices stay on the lattice, so
   the domain stays the unit cube;
2. the coefficient: kappa = exp(N(0,1)) i.i.d. per (element, Gauss point)
   ("lognormal(0,1)"), or theta ~ N(0, 0.5^2) with kappa = exp(theta);
3. theta* for the adjoint workload (same generator, right after theta);
4. the right-hand side: N(0,1) per DOF, then zero on the boundary DOFs
   (homogeneous Dirichlet data).

Layouts: vertices [(nex+1)(ney+1)(nez+1), 3] f64, lexicographic x fastest;
coefficients [nel, q^3] f64, elements lexicographic, Gauss points
g0 + q (g1 + q g2); DOF vectors [N] f64, DOF (I,J,K) at I + nx (J + ny K),
nx = nex p + 1.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


def unit_cube_vertices(nex, ney, nez, jitter=0.0, rng=None):
    """Lattice vertices of the unit cube, interior ones jittered by
    U(-jitter*h, jitter*h) per coordinate."""
    ax = [np.linspace(0.0, 1.0, n + 1) for n in (nex, ney, nez)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if jitter:
        a = np.arange(nex + 1)
        b = np.arange(ney + 1)
        c = np.arange(nez + 1)
        C3, B3, A3 = np.meshgrid(c, b, a, indexing="ij")
        interior = ((A3 > 0) & (A3 < nex) & (B3 > 0) & (B3 < ney) & (C3 > 0) & (C3 < nez)).ravel()
        h = np.array([1.0 / nex, 1.0 / ney, 1.0 / nez])
        r = rng.uniform(-1.0, 1.0, size=(int(interior.sum()), 3))
        V[interior] += jitter * h * r
    return V


def boundary_mask(nex, ney, nez, p):
    """Boolean mask of the DOFs on the boundary of the unit cube."""
    nx, ny, nz = nex * p + 1, ney * p + 1, nez * p + 1
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = (I == 0) | (I == nx - 1) | (J == 0) | (J == ny - 1) | (K == 0) | (K == nz - 1)
    return m.ravel()


@dataclass
class Problem:
    name: str
    nex: int
    ney: int
    nez: int
    p: int
    vertices: np.ndarray
    kappa: np.ndarray
    rhs: Optional[np.ndarray] = None
    theta: Optional[np.ndarray] = None
    theta_star: Optional[np.ndarray] = None
    extra: dict = field(default_factory=dict)

    @property
    def q(self):
        return self.p + 2

    @property
    def nel(self):
        return self.nex * self.ney * self.nez

    @property
    def ndof(self):
        return (self.nex * self.p + 1) * (self.ney * self.p + 1) * (self.nez * self.p + 1)


def make_problem(name, nex, ney, nez, p, seed=None, jitter=0.10, kappa="lognormal", rhs="normal",
                 theta_sigma=0.5):
    """Draw one synthetic workload (see the module docstring for the order)."""
    rng = np.random.default_rng(seed)
    V = unit_cube_vertices(nex, ney, nez, jitter, rng if jitter else None)
    q = p + 2
    nel = nex * ney * nez
    theta = theta_star = None
    if kappa == "one":
        K = np.ones((nel, q ** 3))
    elif kappa == "lognormal":
        K = np.exp(rng.standard_normal((nel, q ** 3)))
    elif kappa == "theta":
        theta = theta_sigma * rng.standard_normal((nel, q ** 3))
        theta_star = theta_sigma * rng.standard_normal((nel, q ** 3))
        K = np.exp(theta)
    else:
        raise ValueError(kappa)
    b = None
    if rhs == "normal":
        b = rng.standard_normal((nex * p + 1) * (ney * p + 1) * (nez * p + 1))
        b[boundary_mask(nex, ney, nez, p)] = 0.0
    elif rhs is not None and rhs != "unit_source":
        raise ValueError(rhs)
    return Problem(name, nex, ney, nez, p, V, K, b, theta, theta_star)


# The five workloads (sizes from the paper's 3D experiment and the build's
# configuration list).  "unit_source" means f = 1, whose load vector is an
# output of the method, not a drawn input.
WORKLOADS = {
    "c1_4x4x4_p3": dict(nex=4, ney=4, nez=4, p=3, seed=None, jitter=0.0, kappa="one", rhs="unit_source"),
    "c2_16x16x16_p4": dict(nex=16, ney=16, nez=16, p=4, seed=1, kappa="lognormal", rhs="normal"),
    "c3_32x32x32_p6": dict(nex=32, ney=32, nez=32, p=6, seed=2, kappa="lognormal", rhs="normal"),
    "c4_24x24x24_p5": dict(nex=24, ney=24, nez=24, p=5, seed=3, kappa="theta", rhs="normal"),
}

# p-sweep at about 20M DOFs: n_e = round(20e6^(1/3) / p).
PSWEEP_NE = {2: 136, 3: 90, 4: 68, 5: 54, 6: 45, 7: 39, 8: 34, 9: 30, 10: 27}


def workload(name):
    if name in WORKLOADS:
        return make_problem(name, **WORKLOADS[name])
    if name.startswith("c5_p"):
        p = int(name[4:])
        ne = PSWEEP_NE[p]
        return make_problem(name, ne, ne, ne, p, seed=4, kappa="lognormal", rhs="normal")
    raise KeyError(name)


def power_start_vector(n, seed=12345):
    """Seeded start vector for the power iteration that estimates the largest
    eigenvalue of D^-1 A (a random input of the method, passed to both sides)."""
    return np.random.default_rng(seed).standard_normal(n)


def reaction_coefficient(nel, q, seed=777):
    """Seeded reaction coefficient beta = exp(N(0,1)) per (element, Gauss
    point) for the definite Helmholtz (diffusion-reaction) workloads; drawn
    from its own generator so the diffusion workloads' draws are unchanged."""
    return np.exp(np.random.default_rng(seed).standard_normal((nel, q ** 3)))
