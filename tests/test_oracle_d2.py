"""Pins of the d = 2 oracle (oracle/d2.py and the d = 2 Gaussian sum):
the integral representation by direct quadrature and the closed form
1/(2 pi r), dense Galerkin matrices on uniform and adaptive trees, the
potential of a Gaussian under 1/(2 pi r) (closed form checked by radial
quadrature), the two-factor estimate against the true block difference, the
transforms' round trip and Parseval, Algorithm 1's bound and projections of
polynomials."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg
from scipy import integrate, special

from oracle import d2 as D
from oracle import gauss_sum as GS
from tests.test_oracle_apply import dense_level

DENS = D.Density2([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52], [0.62, 0.41]])


def integral_repr(mu, alpha, r, d):
    """C int exp(-r^2 e^{2s} - mu^2 e^{-2s}/4 + (d - 2 alpha) s) ds by quad."""
    c = 2.0 * 2.0 ** (-2 * alpha) * math.pi ** (-d / 2) / math.gamma(alpha)
    f = lambda s: math.exp(-r * r * math.exp(2 * s) - 0.25 * mu * mu * math.exp(-2 * s) + (d - 2 * alpha) * s)
    return c * integrate.quad(f, -60, 30, limit=400, epsabs=0, epsrel=1e-12)[0]


@pytest.mark.parametrize("mu,alpha", [(0.0, 0.5), (0.0, 0.25), (2.0, 0.5), (6.0, 0.75)])
def test_gauss_sum_d2(mu, alpha):
    """The d = 2 kernel: the closed form agrees with the integral
    representation; the sum meets eq. KernelApproxByGaussians's bound."""
    for r in (1e-3, 0.05, 0.4, 1.3):
        ref = integral_repr(mu, alpha, r, 2)
        assert abs(GS.kernel(mu, alpha, r, d=2) - ref) <= 1e-9 * ref
    eps = 1e-6
    w, tau = GS.gaussian_sum(mu, alpha, eps, d=2)
    r = np.exp(np.random.default_rng(3).uniform(math.log(eps / 10), math.log(math.sqrt(2)), 20000))
    err = np.abs(GS.kernel(mu, alpha, r, d=2) - np.exp(-np.outer(r * r, tau)) @ w) / GS.envelope(alpha, r, d=2)
    assert err.max() <= eps


def test_half_power_kernel_closed_form():
    """(-Laplacian)^{-1/2} in R^2 has the kernel 1/(2 pi r)."""
    r = np.array([1e-4, 0.01, 0.3, 1.4])
    assert np.allclose(GS.kernel(0.0, 0.5, r, d=2), 1.0 / (2 * math.pi * r), rtol=1e-14, atol=0)


def dense_apply2(op, Am, X):
    return np.einsum("m,mai,mbj,ij->ab", op.w, Am, Am, X, optimize=True)


def leaves_function(tr, k):
    """The piecewise polynomial of the leaves, evaluated test-side with
    numpy's Legendre series."""
    leaves = [(key, n.s) for key, n in tr.items() if n.leaf]

    def f(p):
        out = np.zeros(len(p))
        for key, s in leaves:
            jj, a = key[0], np.array(key[1:])
            u = p * 2 ** jj - a
            inside = np.all((u >= 0) & (u < 1), axis=1)
            if not inside.any():
                continue
            ui = u[inside]
            scale = np.sqrt(2 * np.arange(k) + 1)
            P = [npleg.legvander(2 * ui[:, d] - 1, k - 1) * scale for d in range(2)]   # (n, k)
            out[inside] = np.einsum("ij,ni,nj->n", s, P[0], P[1]) * 2.0 ** jj
        return out
    return f


def project_box(fn, k, j, a, sub=1, q=None):
    """Projection of fn on box (j, a) by a composite q-point GL rule with sub x sub
    panels (numpy leggauss, test-side)."""
    q = q or k + 2
    x, w = npleg.leggauss(q)
    x, w = (x + 1) / 2, w / 2
    h = 2.0 ** -j
    out = np.zeros((k, k))
    scale = np.sqrt(2 * np.arange(k) + 1)
    for p1 in range(sub):
        for p2 in range(sub):
            u1, u2 = (p1 + x) / sub, (p2 + x) / sub
            X1, X2 = np.meshgrid((a[0] + u1) * h, (a[1] + u2) * h, indexing="ij")
            vals = fn(np.stack([X1.ravel(), X2.ravel()], axis=1)).reshape(q, q)
            B1 = npleg.legvander(2 * u1 - 1, k - 1) * scale
            B2 = npleg.legvander(2 * u2 - 1, k - 1) * scale
            out += np.einsum("a,b,ab,ai,bj->ij", w, w, vals, B1, B2) / sub ** 2
    return out * 2.0 ** (-j)


def level_grid(tr, k, j):
    N = 2 ** j
    depth = max(key[0] for key in tr)
    f = leaves_function(tr, k)
    X = np.zeros((N * k, N * k))
    for a in np.ndindex(N, N):
        X[a[0] * k:(a[0] + 1) * k, a[1] * k:(a[1] + 1) * k] = project_box(f, k, j, a, sub=2 ** max(0, depth - j), q=k)
    return X


def block_of(X, k, a):
    return X[a[0] * k:(a[0] + 1) * k, a[1] * k:(a[1] + 1) * k]


@pytest.fixture(scope="module")
def op2():
    return D.operator(0.0, 0.5, 1e-4, 3, 3)


def test_dense_uniform_level2_exact(op2):
    tr, _ = D.build_tree(DENS, 3, 1e-4, 3, uniform_level=2)
    g = D.apply_full(op2, tr, screen=False)
    G = dense_apply2(op2, dense_level(op2, 2), level_grid(tr, 3, 2))
    err = math.sqrt(sum(((n.s - block_of(G, 3, key[1:])) ** 2).sum() for key, n in g.items() if n.leaf))
    assert err <= 1e-13 * np.linalg.norm(G)


def test_dense_adaptive_depth2_with_refined_inputs(op2):
    """Leaves at levels 1 and 2: Step 2 refines level-2 inputs from level-1
    leaves; an output leaf at level j receives [T_j f_j] on its box."""
    k = 3
    tr, _ = D.build_tree(DENS, k, 1e-4, 3, uniform_level=1)
    for key in [(1, 0, 1), (1, 1, 0)]:
        tr[key].leaf = False
        tr[key].s = None
        for ck in D.children(key):
            tr[ck] = D.Node(True, D.project_values(k, 2, DENS(D.grid(D.box_nodes(k, 2, ck[1:])))))
    st = {}
    g = D.apply_full(op2, tr, screen=False, stats=st)
    assert st["n_refined"] > 0
    for j in (1, 2):
        G = dense_apply2(op2, dense_level(op2, j), level_grid(tr, k, j))
        ref = math.sqrt(sum((block_of(G, k, key[1:]) ** 2).sum() for key, n in g.items() if n.leaf and key[0] == j))
        err = math.sqrt(sum(((n.s - block_of(G, k, key[1:])) ** 2).sum()
                            for key, n in g.items() if n.leaf and key[0] == j))
        assert err <= 1e-13 * ref


def test_screened_close_to_unscreened(op2):
    tr, _ = D.build_tree(DENS, 3, 1e-4, 3, uniform_level=3)
    st = {}
    g1 = D.apply_full(op2, tr, screen=True, stats=st)
    g0 = D.apply_full(op2, tr, screen=False)
    assert 0 < st["n_items"]
    num = sum(((g1[key].s - n.s) ** 2).sum() for key, n in g0.items() if n.leaf)
    den = sum((n.s ** 2).sum() for key, n in g0.items() if n.leaf)
    assert math.sqrt(num / den) <= 10 * op2.eps


def gaussian_potential_2d(a, r):
    """(1/(2 pi)) int (a/pi) exp(-a|y|^2) / |x - y| d^2y = sqrt(a/pi)/2 e^{-x} I_0(x),
    x = a r^2 / 2."""
    return 0.5 * math.sqrt(a / math.pi) * special.i0e(0.5 * a * np.asarray(r) ** 2)


def test_gaussian_potential_closed_form_by_radial_quadrature():
    """The closed form against the radial integral: the angular integral of
    1/|x - y| over a circle of radius s is 4 K(m) / (r + s), m = 4 r s / (r + s)^2
    (K with 1 - m = ((r - s)/(r + s))^2 passed directly, the log singularity at
    s = r at an end of each of the two pieces)."""
    a = 150.0
    for r in (0.0, 0.02, 0.1, 0.3):
        if r == 0.0:
            val = (a / math.pi) * integrate.quad(lambda s: math.exp(-a * s * s), 0, 2)[0]
        else:
            f = lambda s: ((a / math.pi) * math.exp(-a * s * s) * s * 4
                           * special.ellipkm1(((r - s) / (r + s)) ** 2) / (r + s))
            val = sum(integrate.quad(f, lo, hi, limit=400, epsabs=0, epsrel=1e-12)[0]
                      for lo, hi in ((0.0, r), (r, 2.0))) / (2 * math.pi)
        assert abs(val - float(gaussian_potential_2d(a, r))) <= 1e-9 * val


def test_apply_matches_gaussian_potential():
    """End to end: T (kernel 1/(2 pi r)) of a unit-mass Gaussian well inside the
    square equals the closed form, projected on the output leaves, to 10 eps."""
    k, eps, a, c = 6, 1e-5, 200.0, np.array([0.47, 0.53])
    dens = D.Density2([a / math.pi], [a], [c])
    tr, _ = D.build_tree(dens, k, eps, 6, init_level=2)
    op = D.operator(0.0, 0.5, eps, k, 6)
    g = D.apply_full(op, tr)
    fn = lambda p: gaussian_potential_2d(a, np.linalg.norm(p - c, axis=1))
    num = den = 0.0
    for key, n in g.items():
        if n.leaf:
            ref = project_box(fn, k, key[0], key[1:], sub=2, q=k + 4)
            num += float(((n.s - ref) ** 2).sum())
            den += float((ref ** 2).sum())
    assert math.sqrt(num / den) <= 10 * eps


def test_two_factor_estimate_bounds_true_difference(op2):
    """The d = 2 estimate bounds ||FF1 x FF2 - UP1 x UP2|| (Kronecker products)."""
    j = 2
    for m in range(0, op2.M, 5):
        FF, UP = {}, {}
        for L in (-1, 0, 1):
            F = op2.F[j, m]
            FF[L] = np.block([[F[2 * L + 3], F[2 * L + 2]], [F[2 * L + 4], F[2 * L + 3]]])
            UP[L] = op2.U @ op2.F[j - 1, m, L + 3] @ op2.U.T
        for Ls in [(0, 0), (1, -1), (1, 1), (-1, 0)]:
            diff = np.linalg.norm(np.kron(FF[Ls[0]], FF[Ls[1]]) - np.kron(UP[Ls[0]], UP[Ls[1]]))
            assert diff <= op2.estimate(j, m, tuple(L + 1 for L in Ls)) * (1 + 1e-12) + 1e-300


def test_compress_round_trip_and_parseval():
    k = 4
    tr, _ = D.build_tree(DENS, k, 1e-5, 5, init_level=1)
    before = {key: n.s.copy() for key, n in tr.items() if n.leaf}
    t = D.copy_tree(tr)
    D.compress(t, k)
    # Parseval: the leaves' energy = the root block's + every wavelet block's
    e_leaves = sum((s ** 2).sum() for s in before.values())
    e_tree = (t[(0, 0, 0)].s ** 2).sum() + sum(n.dnorm ** 2 for n in t.values() if not n.leaf)
    assert abs(e_leaves - e_tree) <= 1e-13 * e_leaves
    D.reconstruct(t, k)
    for key, s in before.items():
        assert np.abs(t[key].s - s).max() <= 1e-13 * max(1.0, np.abs(s).max())


def test_projection_of_polynomials_is_exact():
    k = 5
    c = np.random.default_rng(4).standard_normal((k, k))       # degree < k per direction
    fn = lambda p: npleg.legval2d(2 * p[:, 0] - 1, 2 * p[:, 1] - 1, c)
    for j, a in [(0, (0, 0)), (2, (1, 3)), (3, (5, 2))]:
        s = D.project_values(k, j, fn(D.grid(D.box_nodes(k, j, a))))
        pts = np.random.default_rng(5).uniform(0, 1, (50, 2))
        x = (np.array(a) + pts) * 2.0 ** -j
        assert np.allclose(D.eval_block(k, j, a, s, x), fn(x), rtol=0, atol=1e-12 * np.abs(c).sum())


def test_algorithm1_bound():
    k, eps = 5, 1e-6
    tr, hit = D.build_tree(DENS, k, eps, 8, init_level=1)
    assert not hit
    f = leaves_function(tr, k)
    pts = np.random.default_rng(6).uniform(0, 1, (3000, 2))
    assert np.abs(f(pts) - DENS(pts)).max() <= 10 * eps * DENS.scale()


def test_truncation_removes_little():
    op = D.operator(0.0, 0.5, 1e-4, 4, 5)
    tr, _ = D.build_tree(DENS, 4, 1e-4, 5, init_level=1)
    st = {}
    g = D.apply_full(op, tr, truncate_out=True, stats=st)
    g0 = D.apply_full(op, tr)
    assert len(g) <= len(g0)
    assert st["truncation_l2"] <= op.eps * D.norm2(g0)
