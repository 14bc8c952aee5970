"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws parameters (Gaussian weights, exponents and centres)
with numpy's PCG64 generator; it holds none of the method's arithmetic and is
the one module both the CUDA path's harness and the oracle-side tests use to
obtain identical inputs.  Seeds follow ``1000 * config + instance``.

The paper's own workloads are analytic Gaussian densities (Sec. 6.1: three
Gaussians of exponent 300 and their negative Laplacian); no public dataset is
involved.  Each density is a sum of terms (c + b |x - x0|^2) exp(-a |x - x0|^2).
"""
import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Density:
    coef: np.ndarray          # c_g
    expo: np.ndarray          # a_g
    centers: np.ndarray       # (n, 3)
    r2coef: np.ndarray        # b_g (coefficient of |x - x0|^2)

    @property
    def n(self):
        return len(self.coef)


@dataclass
class Config:
    name: str
    mu: float
    alpha: float
    eps: float
    k: int
    max_level: int
    uniform_level: int = -1
    init_level: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)


def unit_mass(expo, centers):
    expo = np.asarray(expo, dtype=np.float64)
    coef = (expo / math.pi) ** 1.5
    return Density(coef, expo, np.asarray(centers, dtype=np.float64).reshape(-1, 3),
                   np.zeros_like(coef))


def poisson_small(instance=0):
    """3-D Poisson, k=4, eps=1e-4, uniform level-3 tree (512 leaves); 4 unit-mass
    Gaussians, exponents U[100, 1000], centres U[0.3, 0.7]^3."""
    rng = np.random.default_rng(1000 * 1 + instance)
    expo = rng.uniform(100.0, 1000.0, 4)
    cen = rng.uniform(0.3, 0.7, (4, 3))
    cfg = Config("poisson_k4_eps1e-4_uniform3", 0.0, 1.0, 1e-4, 4, 3, uniform_level=3)
    return cfg, unit_mass(expo, cen)


def poisson_k8(instance=0, n_gauss=64):
    """3-D Poisson, k=8, eps=1e-6, adaptive tree to depth 7; 64 unit-mass
    Gaussians, log10 exponent U[2, 5], centres U[0.1, 0.9]^3."""
    rng = np.random.default_rng(1000 * 2 + instance)
    expo = 10.0 ** rng.uniform(2.0, 5.0, n_gauss)
    cen = rng.uniform(0.1, 0.9, (n_gauss, 3))
    cfg = Config("poisson_k8_eps1e-6_adaptive7", 0.0, 1.0, 1e-6, 8, 7, init_level=2)
    return cfg, unit_mass(expo, cen)


def poisson_resolved(instance=0, n_gauss=16):
    """3-D Poisson, k=8, eps=1e-6, adaptive to depth 7 with every density
    resolved (no depth cap reached): 16 unit-mass Gaussians, log10 exponent
    U[2, 3.5], centres U[0.2, 0.8]^3.  Used to compare the output on the input's
    skeleton with the output on a refined one."""
    rng = np.random.default_rng(1000 * 6 + instance)
    expo = 10.0 ** rng.uniform(2.0, 3.5, n_gauss)
    cen = rng.uniform(0.2, 0.8, (n_gauss, 3))
    cfg = Config("poisson_resolved_k8_eps1e-6_adaptive7", 0.0, 1.0, 1e-6, 8, 7, init_level=2)
    return cfg, unit_mass(expo, cen)


def slater_fit(n_terms=5, zeta=2.0):
    """Least-squares fit of exp(-zeta r) by n_terms Gaussians (weights and
    exponents), on 400 log-spaced radii in [1e-3, 4]; exponents are kept as
    logs so they stay positive.  Deterministic (fixed start, scipy LM)."""
    from scipy.optimize import least_squares
    r = np.exp(np.linspace(math.log(1e-3), math.log(4.0), 400))
    target = np.exp(-zeta * r)

    def resid(p):
        c, la = p[:n_terms], p[n_terms:]
        return np.exp(-np.outer(r * r, np.exp(la))) @ c - target

    la0 = np.linspace(math.log(0.3), math.log(300.0), n_terms)
    c0 = np.full(n_terms, 1.0 / n_terms)
    sol = least_squares(resid, np.concatenate([c0, la0]), method="lm", xtol=1e-14, ftol=1e-14)
    return sol.x[:n_terms], np.exp(sol.x[n_terms:])


def helmholtz_slater(instance=0):
    """Bound-state Helmholtz (mu = 1.5, alpha = 1), k=8, eps=1e-6, adaptive to
    depth 8; density is a 5-Gaussian fit of exp(-2r) centred at (0.5, 0.5, 0.5)."""
    c, a = slater_fit()
    cen = np.tile([0.5, 0.5, 0.5], (len(c), 1))
    cfg = Config("helmholtz_mu1.5_k8_eps1e-6_adaptive8", 1.5, 1.0, 1e-6, 8, 8, init_level=2)
    return cfg, Density(c, a, cen, np.zeros_like(c))


def batched_rhs(n_rhs=256, instance=0):
    """n_rhs independent Poisson right-hand sides at eps=1e-5, k=6: each has
    U{1..32} unit-mass Gaussians, log10 exponent U[1, 4], centres U[0.1,0.9]^3."""
    rng = np.random.default_rng(1000 * 4 + instance)
    out = []
    for _ in range(n_rhs):
        n = int(rng.integers(1, 33))
        expo = 10.0 ** rng.uniform(1.0, 4.0, n)
        cen = rng.uniform(0.1, 0.9, (n, 3))
        out.append(unit_mass(expo, cen))
    cfg = Config("batched_poisson_k6_eps1e-5", 0.0, 1.0, 1e-5, 6, 7, init_level=2)
    return cfg, out


def schedule_set(n, instance0, k=8):
    """Training / held-out densities for the learned schedule: Poisson or
    Helmholtz, 16-128 unit-mass Gaussians, log10 exponent U[2, 5]."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(1000 * 5 + instance0 + i)
        ng = int(rng.integers(16, 129))
        expo = 10.0 ** rng.uniform(2.0, 5.0, ng)
        cen = rng.uniform(0.1, 0.9, (ng, 3))
        mu = 0.0 if rng.random() < 0.5 else 1.5
        out.append((mu, unit_mass(expo, cen)))
    return out


def paper_poisson(a=300.0, k=8, eps=1e-6, max_level=6):
    """The paper's Poisson test (Sec. 6.1): rho = -Laplacian sum_i exp(-a|r-r_i|^2)
    with a = 300 and the three centres given there; (4 pi) T rho = phi exactly.
    rho = sum_i (6a - 4a^2 |r - r_i|^2) exp(-a |r - r_i|^2)."""
    cen = np.array([[0.5, 0.5, 0.5], [0.6, 0.6, 0.5], [0.35, 0.6, 0.5]])
    coef = np.full(3, 6.0 * a)
    r2 = np.full(3, -4.0 * a * a)
    cfg = Config(f"paper_poisson_a{a:g}_k{k}", 0.0, 1.0, eps, k, max_level, init_level=1)
    return cfg, Density(coef, np.full(3, a), cen, r2)


def slater_expansion(zeta, h=0.4, r_min=1e-4):
    """Gaussian expansion (c, a) of exp(-zeta r): the trapezoid rule with step
    h in s on exp(-zeta r) = zeta / (2 sqrt(pi)) int exp(-s/2 - zeta^2 e^{-s}/4
    - r^2 e^s) ds (the Laplace-transform identity of exp(-zeta sqrt(y)) with
    y = r^2), over s in [ln(zeta^2 / 150), 2 ln(1 / r_min) + 2].  Absolute
    error about 1e-10 for r >= r_min at h = 0.4 (66 terms at zeta = 1)."""
    s = np.arange(math.log(zeta * zeta / 150.0), 2.0 * math.log(1.0 / r_min) + 2.0 + h, h)
    c = zeta / (2.0 * math.sqrt(math.pi)) * h * np.exp(-s / 2.0 - zeta * zeta * np.exp(-s) / 4.0)
    return c, np.exp(s)


@dataclass
class Hydrogen:
    """The hydrogen ground-state iteration (Sec. 6.2): a cube of side L
    (atomic units) with the nucleus at the cube point u0, the starting
    function exp(-zeta0 r), the starting mu0, and the apply's k / eps /
    max_level.  The starting tree is Algorithm 1 on the Gaussian expansion
    of exp(-zeta0 r) in cube coordinates (exponents a L^2)."""
    name: str
    L: float
    u0: tuple
    zeta0: float
    mu0: float
    k: int
    eps: float
    max_level: int
    init_level: int

    def start_density(self):
        c, a = slater_expansion(self.zeta0)
        return Density(c, a * self.L * self.L, np.tile(np.asarray(self.u0, dtype=np.float64), (len(c), 1)),
                       np.zeros_like(c))


def hydrogen(k=8, eps=1e-6, max_level=12):
    """Hydrogen ground state: L = 32, nucleus at the cube centre (a corner of
    boxes at every level, so no GL node meets it), exp(-0.7 r) and mu0 = 0.8
    to start."""
    return Hydrogen(f"hydrogen_k{k}_eps{eps:g}_level{max_level}", 32.0, (0.5, 0.5, 0.5), 0.7, 0.8, k, eps,
                    max_level, 3)


def hydrogen_small():
    """A small hydrogen case the oracle finishes in seconds: k = 5,
    eps = 1e-3, depth 5."""
    return Hydrogen("hydrogen_k5_eps1e-3_level5", 32.0, (0.5, 0.5, 0.5), 0.7, 0.8, 5, 1e-3, 5, 2)


def unit_mass2(expo, centers):
    """Unit-mass Gaussians in R^2: (a/pi) exp(-a |x - x0|^2)."""
    expo = np.asarray(expo, dtype=np.float64)
    return Density(expo / math.pi, expo, np.asarray(centers, dtype=np.float64).reshape(-1, 2), np.zeros_like(expo))


def poisson2d(instance=0, n_gauss=64):
    """The d = 2 variant at full size: the kernel 1/(2 pi r) of
    (-Laplacian)^{-1/2} in R^2 (alpha = 1/2, mu = 0), k = 8, eps = 1e-6,
    adaptive to depth 12; 64 unit-mass Gaussians, log10 exponent U[2.5, 5],
    centres U[0.2, 0.8]^2, so that each Gaussian's mass outside the square is
    below 3e-7 of it and the output can be checked against the free-space
    closed form."""
    rng = np.random.default_rng(1000 * 8 + instance)
    expo = 10.0 ** rng.uniform(2.5, 5.0, n_gauss)
    cen = rng.uniform(0.2, 0.8, (n_gauss, 2))
    cfg = Config("poisson2d_half_k8_eps1e-6_adaptive12", 0.0, 0.5, 1e-6, 8, 12, init_level=2)
    return cfg, unit_mass2(expo, cen)


def poisson2d_small(instance=0):
    """A d = 2 case the oracle finishes in seconds: k = 5, eps = 1e-4, depth 6;
    4 unit-mass Gaussians, log10 exponent U[1.5, 3], centres U[0.25, 0.75]^2."""
    rng = np.random.default_rng(1000 * 9 + instance)
    expo = 10.0 ** rng.uniform(1.5, 3.0, 4)
    cen = rng.uniform(0.25, 0.75, (4, 2))
    cfg = Config("poisson2d_half_k5_eps1e-4_adaptive6", 0.0, 0.5, 1e-4, 5, 6, init_level=1)
    return cfg, unit_mass2(expo, cen)


@dataclass
class OneElectron:
    """A one-electron system for the ground-state iteration of Sec. 6.2 with
    several nuclei: charges Z_n at cube points (the potential is
    sum_n -Z_n / |x - R_n|), the starting function sum_n exp(-zeta0 |x - R_n|),
    mu0, the apply's k / eps / max_level, and the exact electronic energy the
    iteration must reach."""
    name: str
    L: float
    nuclei: tuple
    charges: tuple
    zeta0: float
    mu0: float
    k: int
    eps: float
    max_level: int
    init_level: int
    exact_energy: float

    def start_density(self):
        c, a = slater_expansion(self.zeta0)
        cen = np.concatenate([np.tile(np.asarray(u, dtype=np.float64), (len(c), 1)) for u in self.nuclei])
        coef = np.concatenate([c for _ in self.nuclei])
        return Density(coef, np.concatenate([a * self.L * self.L for _ in self.nuclei]), cen, np.zeros_like(coef))

    def potential_charges(self):
        """(charges, positions) in cube coordinates: -Z_n / L at u_n."""
        return [-z / self.L for z in self.charges], [list(u) for u in self.nuclei]


def h2plus(k=8, eps=1e-6, max_level=12):
    """The hydrogen molecular ion at the bond length R = 2 bohr: two protons
    at the cube points (1/2 -+ 1/32, 1/2, 1/2) of a 32-bohr cube (corners of
    boxes from level 5 on, so no GL node meets them); exact electronic energy
    -1.10263421 hartree (the total, with the protons' repulsion 1/R = 1/2, is
    -0.60263421)."""
    return OneElectron(f"h2plus_R2_k{k}_eps{eps:g}_level{max_level}", 32.0,
                       ((0.5 - 1.0 / 32.0, 0.5, 0.5), (0.5 + 1.0 / 32.0, 0.5, 0.5)), (1.0, 1.0), 0.7, 1.2,
                       k, eps, max_level, 3, -1.10263421)
