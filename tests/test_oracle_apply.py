"""Pins for oracle/apply.py (Algorithm 3, eqs. apply_algo, g_assemble, Step 2).

(c1) brute force: dense Galerkin matrices T_j = sum_m w_m A_m x A_m x A_m built
     from the F blocks, on trees of depth <= 2 where the band of width 3 covers
     the whole domain, so the unscreened ns-form must agree to rounding; at
     depth 3 only band truncation separates them.
(b1) Poisson of a centred unit-mass Gaussian = erf(sqrt(a) r)/(4 pi r).
(b2) Gaussian-sum kernel applied exactly to a box-truncated off-centre Gaussian.
(b3) the paper's Table 2 workload: (4 pi) T rho = phi.
(b4) Helmholtz (Yukawa) of a Gaussian, closed form verified by radial quadrature.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import apply as A, gauss_sum, operator as O, tree as T
from tests import closed_forms as CF


def dense_level(op, j):
    N = 2 ** j
    k = op.k
    pe = O._PhiEval(k)
    Am = np.zeros((op.M, N * k, N * k))
    for m in range(op.M):
        for a in range(N):
            for b in range(N):
                l = a - b
                blk = op.F[j, m, l + 3] if abs(l) <= 3 else O.f_block(pe, j, op.tau[m], l)
                Am[m, a * k:(a + 1) * k, b * k:(b + 1) * k] = blk
    return Am


def leaves_function(tr, k):
    """f~ as a callable (piecewise polynomial from the leaves), test-side code."""
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
            P = [CF.legendre_scaled(k, ui[:, d]) for d in range(3)]
            out[inside] = np.einsum("ijk,in,jn,kn->n", s, *P) * 2 ** (1.5 * jj)
        return out
    return f


def level_grid(tr, k, j):
    """f~ projected on every box of level j (test-side composite GL)."""
    N = 2 ** j
    depth = max(key[0] for key in tr)
    f = leaves_function(tr, k)
    sub = 2 ** max(0, depth - j)
    X = np.zeros((N * k,) * 3)
    for a in np.ndindex(N, N, N):
        X[a[0] * k:(a[0] + 1) * k, a[1] * k:(a[1] + 1) * k, a[2] * k:(a[2] + 1) * k] = \
            CF.project_leaf(f, k, j, a, sub=sub, q=k)
    return X


def dense_apply(op, Am, X):
    return np.einsum("m,mai,mbj,mck,ijk->abc", op.w, Am, Am, Am, X, optimize=True)


def block_of(X, k, a):
    return X[a[0] * k:(a[0] + 1) * k, a[1] * k:(a[1] + 1) * k, a[2] * k:(a[2] + 1) * k]


DENS = T.Density([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47]])


@pytest.fixture(scope="module")
def op_k3():
    return O.Operator(0.0, 1.0, 1e-4, 3, 3)


def test_dense_uniform_level2_exact(op_k3):
    op = op_k3
    tr, _ = T.build_tree(DENS, 3, 1e-4, 3, uniform_level=2)
    g = A.apply_full(op, tr, screen=False)
    X = level_grid(tr, 3, 2)
    G = dense_apply(op, dense_level(op, 2), X)
    err = math.sqrt(sum(((n.s - block_of(G, 3, key[1:])) ** 2).sum() for key, n in g.items() if n.leaf))
    assert err <= 1e-13 * np.linalg.norm(G)


def test_dense_adaptive_depth2_with_refined_inputs(op_k3):
    """Leaves at levels 1 and 2: Step 2 must refine level-2 inputs from level-1
    leaves.  Unscreened, an output leaf at level j receives [T_j f_j] on its
    box (eq. apply_algo with whole bands covering the domain)."""
    op = op_k3
    k = 3
    tr, _ = T.build_tree(DENS, k, 1e-4, 3, uniform_level=1)
    # refine two of the level-1 boxes by hand -> adaptive depth-2 tree
    for key in [(1, 0, 1, 0), (1, 1, 0, 0)]:
        node = tr[key]
        node.leaf = False
        for ck in T.children(key):
            xs = T.box_nodes(k, 2, ck[1:])
            tr[ck] = T.Node(True, T.project_values(k, 2, DENS(T.grid(xs))))
        node.s = None
    st = {}
    g = A.apply_full(op, tr, screen=False, stats=st)
    assert st["n_refined"] > 0
    for j in (1, 2):
        G = dense_apply(op, dense_level(op, j), level_grid(tr, k, j))
        ref = math.sqrt(sum((block_of(G, k, key[1:]) ** 2).sum() for key, n in g.items() if n.leaf and key[0] == j))
        err = math.sqrt(sum(((n.s - block_of(G, k, key[1:])) ** 2).sum()
                            for key, n in g.items() if n.leaf and key[0] == j))
        assert err <= 1e-13 * ref


def test_screened_close_to_unscreened(op_k3):
    op = op_k3
    tr, _ = T.build_tree(DENS, 3, 1e-4, 3, uniform_level=2)
    st = {}
    g1 = A.apply_full(op, tr, screen=True, stats=st)
    g0 = A.apply_full(op, tr, screen=False)
    assert st["n_items"] > 0
    num = sum(((g1[key].s - n.s) ** 2).sum() for key, n in g0.items() if n.leaf)
    den = sum((n.s ** 2).sum() for key, n in g0.items() if n.leaf)
    assert math.sqrt(num / den) <= 10 * op.eps


def test_band_truncation_level3():
    op = O.Operator(0.0, 1.0, 1e-3, 3, 3)
    tr, _ = T.build_tree(DENS, 3, 1e-3, 3, uniform_level=3)
    g = A.apply_full(op, tr, screen=False)
    X = level_grid(tr, 3, 3)
    G = dense_apply(op, dense_level(op, 3), X)
    err = math.sqrt(sum(((n.s - block_of(G, 3, key[1:])) ** 2).sum() for key, n in g.items() if n.leaf))
    assert err <= op.eps * np.linalg.norm(G)


def rel_err_vs(fun, g, k):
    num = den = 0.0
    for key, n in g.items():
        if n.leaf:
            e = CF.project_leaf(fun, k, key[0], key[1:], sub=2)
            num += ((n.s - e) ** 2).sum()
            den += (e ** 2).sum()
    return math.sqrt(num / den)


def test_poisson_centered_gaussian_closed_form():
    k, eps, a = 5, 1e-4, 300.0
    c = [0.5, 0.5, 0.5]
    dens = T.Density([(a / math.pi) ** 1.5], [a], [c])
    tr, hit = T.build_tree(dens, k, eps, 5, init_level=1)
    op = O.Operator(0.0, 1.0, eps, k, 5)
    g = A.apply_full(op, tr)
    assert rel_err_vs(CF.poisson_gaussian(a, c), g, k) <= 10 * eps


def test_truncated_offcentre_gaussian_closed_form():
    """(b2): the Gaussian-sum kernel applied exactly to a Gaussian whose tail
    crosses the box face (the method computes T(f 1_B) on B)."""
    k, eps, a = 5, 1e-4, 120.0
    c = [0.22, 0.5, 0.6]
    dens = T.Density([1.0], [a], [c])
    tr, _ = T.build_tree(dens, k, eps, 5, init_level=1)
    op = O.Operator(0.0, 1.0, eps, k, 5)
    g = A.apply_full(op, tr)
    ref = CF.truncated_gauss_sum_potential(op.w, op.tau, a, c)
    assert rel_err_vs(ref, g, k) <= 10 * eps


def test_paper_poisson_workload():
    """(b3) Sec. 6.1: rho = -Laplacian sum_i exp(-a|r-r_i|^2), a = 300, the three
    centres of the paper; (4 pi) T rho = sum_i exp(-a |r - r_i|^2)."""
    k, eps, a = 5, 1e-4, 300.0
    cen = np.array([[0.5, 0.5, 0.5], [0.6, 0.6, 0.5], [0.35, 0.6, 0.5]])
    dens = T.Density(np.full(3, 6 * a), np.full(3, a), cen, np.full(3, -4 * a * a))
    tr, _ = T.build_tree(dens, k, eps, 5, init_level=1)
    op = O.Operator(0.0, 1.0, eps, k, 5)
    g = A.apply_full(op, tr)

    def phi(p):
        return sum(np.exp(-a * ((p - c0) ** 2).sum(axis=1)) for c0 in cen)
    assert rel_err_vs(phi, g, k) <= 10 * eps


def test_yukawa_closed_form_by_radial_quadrature():
    a, mu = 200.0, 1.5
    V = CF.yukawa_gaussian(a, mu, [0, 0, 0]).radial
    rho = lambda s: (a / math.pi) ** 1.5 * math.exp(-a * s * s)
    for r in [0.01, 0.05, 0.2, 0.7]:
        # V(r) = (2 pi / r) int rho(s) s int_{|r-s|}^{r+s} e^{-mu u}/(4 pi u) u du ds... (shell theorem)
        inner = lambda s: rho(s) * s * (math.exp(-mu * abs(r - s)) - math.exp(-mu * (r + s))) / mu
        val = integrate.quad(inner, 0, 2.0, limit=200, epsabs=0, epsrel=1e-13)[0] * 2 * math.pi / r / (4 * math.pi)
        assert abs(val - V(np.array([r]))[0]) <= 1e-11 * abs(val)


def test_helmholtz_centered_gaussian_closed_form():
    k, eps, a, mu = 5, 1e-4, 300.0, 1.5
    c = [0.5, 0.5, 0.5]
    dens = T.Density([(a / math.pi) ** 1.5], [a], [c])
    tr, _ = T.build_tree(dens, k, eps, 5, init_level=1)
    op = O.Operator(mu, 1.0, eps, k, 5)
    g = A.apply_full(op, tr)
    assert rel_err_vs(CF.yukawa_gaussian(a, mu, c), g, k) <= 10 * eps


def test_truncation_bounded():
    k, eps = 4, 1e-3
    tr, _ = T.build_tree(DENS, k, 1e-5, 4, init_level=1)
    op = O.Operator(0.0, 1.0, eps, k, 4)
    st = {}
    g_full = A.apply_full(op, tr)
    g_tr = A.apply_full(op, tr, truncate_out=True, stats=st)
    assert len(g_tr) < len(g_full)
    nrm = T.norm2(g_full)
    assert st["truncation_l2"] <= eps * nrm
    # merged leaves hold the projection of the untruncated output (the removed
    # part is the wavelet detail), and the removed l2 mass obeys Pythagoras
    f_full = leaves_function(g_full, k)
    diff = 0.0
    for key, n in g_tr.items():
        if n.leaf and key not in g_full or (n.leaf and not g_full[key].leaf):
            e = CF.project_leaf(f_full, k, key[0], key[1:], sub=2 ** (T.levels(g_full) - 1 - key[0]), q=k)
            diff += ((n.s - e) ** 2).sum()
    assert math.sqrt(diff) <= 1e-12 * nrm
    assert abs(math.sqrt(max(nrm ** 2 - T.norm2(g_tr) ** 2, 0.0)) - st["truncation_l2"]) <= 1e-6 * nrm
