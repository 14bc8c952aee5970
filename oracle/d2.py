"""Oracle: the d = 2 variant of the method (Sec. 6 remark that the apply was
implemented for d = 2 and d = 3; Algorithm 3 as the paper illustrates it for
d = 2; Sec. 4: three subsets Core / Boundary-1 / Boundary-2 in d = 2).

Test infrastructure only (see ``oracle/__init__``).

Everything follows the d = 3 modules with one direction fewer:
* a tree is a dict keyed by (j, a1, a2) with blocks s[i1, i2] (k x k) in the
  basis phi^j_{i1,a1}(x1) phi^j_{i2,a2}(x2); every internal node has its 4
  children (Algorithm 1 in d = 2, the l-infinity test at the children's GL
  nodes with threshold eps * max_g |f(x_g)|);
* the redundant tree: the 2k x 2k filter applied in both directions to the
  (2k)^2 square of the 4 children (eqs. decomp_scaling / decomp_wavelet);
* the operator: the d = 2 Gaussian sum (gauss_sum with d = 2) and the same
  1-D blocks F^{j;m,l}; the estimate of the product of two factors
  (operator.Operator with d = 2);
* Algorithm 3: band t_d in [-3, 2] (even a_d) or [-2, 3] (odd a_d) per
  direction, J_m, ranges [m1, m2] per scale and subset S = number of
  directions with |t_d| <= 1 (S = 0, 1, 2), trimmed while the cumulative
  w_m prod_d max N_F stays <= eta / (2 * 36) (36 = 6^2 translations);
  ghat^j_a += sum_m w_m F^{j;m,t1} f_{a-t} (F^{j;m,t2})^T (the nested sums of
  Algorithm 3, Step 3); Step 2 by the d = 0 refinement from the ancestor
  leaf; eq. g_assemble; truncation as in d = 3.

Parity pins (tests/test_oracle_d2.py): dense Galerkin matrices on uniform
and adaptive trees (unscreened apply to rounding), the closed form of the
alpha = 1/2 kernel 1/(2 pi r) applied to a Gaussian (verified by radial
quadrature), compress / reconstruct round trip and Parseval, exact
projection of polynomials, Algorithm 1's bound, the d = 2 Gaussian sum
against the integral representation, and the two-factor estimate against the
true block difference.
"""
import itertools

import numpy as np

from . import basis
from . import operator as O
from .tree import Node

QUADS = list(itertools.product((0, 1), repeat=2))     # child quadrant (p1, p2)
BAND_EVEN = (-3, -2, -1, 0, 1, 2)
BAND_ODD = (-2, -1, 0, 1, 2, 3)


class Density2:
    """f(x) = sum_g (c_g + b_g |x - x_g|^2) exp(-a_g |x - x_g|^2), x in R^2."""

    def __init__(self, coef, expo, centers, r2coef=None):
        self.coef = np.asarray(coef, dtype=np.float64)
        self.expo = np.asarray(expo, dtype=np.float64)
        self.centers = np.asarray(centers, dtype=np.float64).reshape(-1, 2)
        self.r2coef = (np.zeros_like(self.coef) if r2coef is None
                       else np.asarray(r2coef, dtype=np.float64))

    def __call__(self, pts):
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
        out = np.zeros(len(pts))
        for c, b, a, x0 in zip(self.coef, self.r2coef, self.expo, self.centers):
            r2 = ((pts - x0) ** 2).sum(axis=1)
            out += (c + b * r2) * np.exp(-a * r2)
        return out

    def scale(self):
        return float(np.abs(self(self.centers)).max())


def box_nodes(k, j, a):
    g, _ = basis.gl01(k)
    return np.array([(g + a[d]) / 2.0 ** j for d in range(2)])


def grid(xs):
    X = np.meshgrid(xs[0], xs[1], indexing="ij")
    return np.stack([x.ravel() for x in X], axis=1)


def project_values(k, j, vals):
    """s = 2^{-j} sum_q f(x_q) prod_d phi_{i_d}(g_{q_d}) w_{q_d} (eq. fvals2coefs, d = 2)."""
    g, w = basis.gl01(k)
    P = basis.phi(k, g) * w
    return np.einsum("ia,jb,ab->ij", P, P, vals.reshape(k, k), optimize=True) / 2.0 ** j


def eval_block(k, j, a, s, pts):
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
    u = pts * 2.0 ** j - np.asarray(a, dtype=np.float64)
    P = [basis.phi(k, u[:, d]) for d in range(2)]
    return np.einsum("ij,in,jn->n", s, P[0], P[1], optimize=True) * 2.0 ** j


def children(key):
    j, a = key[0], key[1:]
    return [(j + 1, 2 * a[0] + p[0], 2 * a[1] + p[1]) for p in QUADS]


def levels(tree):
    return max(key[0] for key in tree) + 1


def build_tree(dens, k, eps, max_level, uniform_level=-1, init_level=0):
    """Algorithm 1 in d = 2; returns (tree, depth_hit)."""
    tol = eps * dens.scale()
    g, _ = basis.gl01(k)
    Q = [basis.phi(k, 0.5 * (g + p)).T for p in (0, 1)]       # (q, i): child-node values
    tree = {}
    depth_hit = False
    boxes = [(0, 0)]
    j = 0
    while boxes:
        nxt = []
        for b in boxes:
            s = project_values(k, j, dens(grid(box_nodes(k, j, b))))
            if uniform_level >= 0:
                refine = j < uniform_level
            elif j < init_level:
                refine = True
            else:
                err = 0.0
                for p in QUADS:
                    cb = (2 * b[0] + p[0], 2 * b[1] + p[1])
                    direct = dens(grid(box_nodes(k, j + 1, cb)))
                    interp = np.einsum("ij,ai,bj->ab", s, Q[p[0]], Q[p[1]]).ravel() * 2.0 ** j
                    err = max(err, float(np.abs(direct - interp).max()))
                refine = err > tol
                if refine and j >= max_level:
                    depth_hit = True
            if j >= max_level:
                refine = False
            key = (j,) + tuple(b)
            if refine:
                tree[key] = Node(False)
                nxt += [(2 * b[0] + p[0], 2 * b[1] + p[1]) for p in QUADS]
            else:
                tree[key] = Node(True, s)
        boxes = nxt
        j += 1
    return tree, depth_hit


def _square_of_children(tree, key, k):
    sq = np.zeros((2 * k, 2 * k))
    for p, ck in zip(QUADS, children(key)):
        sq[p[0] * k:(p[0] + 1) * k, p[1] * k:(p[1] + 1) * k] = tree[ck].s
    return sq


def compress(tree, k):
    """Redundant tree in d = 2: s^j and the 3 wavelet blocks of every internal
    node from the (2k)^2 square of its children, W sq W^T."""
    Wm = basis.filter_matrix(k)
    for j in range(levels(tree) - 2, -1, -1):
        for key, node in tree.items():
            if key[0] != j or node.leaf:
                continue
            out = Wm @ _square_of_children(tree, key, k) @ Wm.T
            node.s = out[:k, :k].copy()
            out[:k, :k] = 0.0
            node.d = out
            node.dnorm = float(np.linalg.norm(out))
    return tree


def reconstruct(tree, k):
    """Inverse of compress: children from s and d with W^T . W."""
    Wm = basis.filter_matrix(k)
    for j in range(levels(tree) - 1):
        for key, node in tree.items():
            if key[0] != j or node.leaf:
                continue
            sq = node.d.copy()
            sq[:k, :k] = node.s
            full = Wm.T @ sq @ Wm
            for p, ck in zip(QUADS, children(key)):
                tree[ck].s = full[p[0] * k:(p[0] + 1) * k, p[1] * k:(p[1] + 1) * k].copy()
    return tree


def upsample(k, s, p):
    """s^{j+1}_{2a+p} = H^(p1)T s^j_a H^(p2) (the d = 0 half of eqs.
    recon_even / recon_odd in d = 2)."""
    H = basis.two_scale_H(k)
    return H[p[0]].T @ s @ H[p[1]]


def norm2(tree):
    return float(np.sqrt(sum((n.s ** 2).sum() for n in tree.values() if n.leaf)))


def copy_tree(tree):
    out = {}
    for key, n in tree.items():
        m = Node(n.leaf, None if n.s is None else n.s.copy())
        m.d = None if n.d is None else n.d.copy()
        m.dnorm = n.dnorm
        out[key] = m
    return out


def operator(mu, alpha, eps, k, max_level):
    """The d = 2 operator tables (gauss_sum and the two-factor estimate)."""
    return O.Operator(mu, alpha, eps, k, max_level, d=2)


def band(a):
    return itertools.product(*[(BAND_EVEN if a[d] % 2 == 0 else BAND_ODD) for d in range(2)])


class Schedule:
    """J_m and [m1, m2] per scale and subset S = 0, 1, 2 (Sec. 4 for d = 2)."""

    def __init__(self, op, sigma, fnorm, nlev, screen=True):
        M = op.M
        self.eta = op.eps * sigma / fnorm if fnorm > 0 else 0.0
        if not screen:
            self.Jm = np.full(M, nlev - 1, dtype=np.int64)
            self.m1 = np.zeros((nlev, 3), dtype=np.int64)
            self.m2 = np.full((nlev, 3), M - 1, dtype=np.int64)
            return
        self.Jm = np.zeros(M, dtype=np.int64)
        for m in range(M):
            for j in range(1, nlev):
                if op.w[m] * op.est_core[j, m] > self.eta / M:
                    self.Jm[m] = j
        nFc = op.nF[:, :, 2:5].max(axis=2)
        nFb = op.nF[:, :, [0, 1, 5, 6]].max(axis=2)
        self.m1 = np.zeros((nlev, 3), dtype=np.int64)
        self.m2 = np.full((nlev, 3), -1, dtype=np.int64)
        budget = self.eta / (2.0 * 36.0)
        for j in range(nlev):
            cand = [m for m in range(M) if self.Jm[m] >= j]
            for S in range(3):
                if not cand:
                    continue
                e = [op.w[m] * nFc[j, m] ** S * nFb[j, m] ** (2 - S) for m in cand]
                lo, acc = 0, 0.0
                while lo < len(cand) and acc + e[lo] <= budget:
                    acc += e[lo]
                    lo += 1
                hi, acc = len(cand) - 1, 0.0
                while hi >= lo and acc + e[hi] <= budget:
                    acc += e[hi]
                    hi -= 1
                if hi >= lo:
                    self.m1[j, S] = cand[lo]
                    self.m2[j, S] = cand[hi]

    def terms(self, j, t, leaf):
        S = sum(1 for v in t if abs(v) <= 1)
        core = S == 2
        out = []
        for m in range(self.m1[j, S], self.m2[j, S] + 1):
            if self.Jm[m] < j:
                continue
            if core and not leaf and self.Jm[m] > j:
                continue
            out.append(m)
        return out


def separated_apply(w, F1, F2, x):
    """sum_m w_m F1_m x F2_m^T; shapes w (M,), F* (M, k, k), x (k, k)."""
    return np.einsum("m,mai,ij,mbj->ab", w, F1, x, F2, optimize=True)


def pilot_sigma(op, tree):
    F0 = op.F[0, :, 3]
    return float(np.linalg.norm(separated_apply(op.w, F0, F0, tree[(0, 0, 0)].s)))


class _Inputs:
    """Step 2 of Algorithm 3 in d = 2."""

    def __init__(self, tree, k):
        self.tree, self.k, self.cache = tree, k, {}
        self.n_refined = 0

    def get(self, j, b):
        key = (j,) + tuple(b)
        if key in self.tree:
            return self.tree[key].s
        if key in self.cache:
            return self.cache[key]
        for jj in range(j - 1, -1, -1):
            anc = (jj,) + tuple(v >> (j - jj) for v in b)
            if anc in self.tree:
                break
        s = self.tree[anc].s
        for lev in range(jj, j):
            sh = j - lev - 1
            s = upsample(self.k, s, tuple((v >> sh) & 1 for v in b))
        self.cache[key] = s
        self.n_refined += 1
        return s


def apply_ns(op, tree, stats=None, screen=True, nodes=None):
    """Algorithm 3 in d = 2, Steps 1-3, on a compressed tree: ghat per node."""
    k = op.k
    nlev = levels(tree)
    if nlev - 1 > op.max_level:
        raise ValueError("tree deeper than the operator tables")
    fnorm = norm2(tree)
    sigma = pilot_sigma(op, tree)
    sch = Schedule(op, sigma, fnorm, nlev, screen=screen)
    inp = _Inputs(tree, k)
    ghat, n_items, n_pairs = {}, 0, 0
    for key in (sorted(tree.keys()) if nodes is None else list(nodes)):
        j, a = key[0], key[1:]
        leaf = tree[key].leaf
        y = np.zeros((k, k))
        for t in band(a):
            b = (a[0] - t[0], a[1] - t[1])
            if min(b) < 0 or max(b) >= 2 ** j:
                continue
            ms = sch.terms(j, t, leaf)
            if not ms:
                continue
            ms = np.array(ms)
            y += separated_apply(op.w[ms], op.F[j, ms, t[0] + 3], op.F[j, ms, t[1] + 3], inp.get(j, b))
            n_items += len(ms)
            n_pairs += 1
        ghat[key] = y
    if stats is not None:
        stats.update(dict(n_items=n_items, n_pairs=n_pairs, n_refined=inp.n_refined, eta=sch.eta,
                          sigma=sigma, fnorm=fnorm, Jm=sch.Jm.copy(), m1=sch.m1.copy(), m2=sch.m2.copy()))
    return ghat


def assemble(op, tree, ghat):
    """Eq. g_assemble in d = 2."""
    k = op.k
    out = {key: Node(n.leaf, ghat[key].copy()) for key, n in tree.items()}
    for j in range(levels(tree) - 1):
        for key, node in out.items():
            if key[0] != j or node.leaf:
                continue
            for p, ck in zip(QUADS, children(key)):
                out[ck].s += upsample(k, node.s, p)
    return out


def truncate(g, k, eps):
    """Algorithm 3, Step 4 in d = 2: compress, then merge leaf siblings whose
    parent's wavelet norm is below eps ||g|| / sqrt(N), bottom-up."""
    compress(g, k)
    thr = eps * norm2(g) / np.sqrt(len(g))
    removed2 = 0.0
    for j in range(levels(g) - 2, -1, -1):
        for key in [kk for kk in g if kk[0] == j]:
            node = g[key]
            if node.leaf:
                continue
            ch = children(key)
            if all(g[c].leaf for c in ch) and node.dnorm < thr:
                removed2 += node.dnorm ** 2
                for c in ch:
                    del g[c]
                node.leaf = True
                node.d = None
    return g, float(np.sqrt(removed2))


def apply_full(op, tree, truncate_out=False, stats=None, screen=True):
    t = copy_tree(tree)
    compress(t, op.k)
    g = assemble(op, t, apply_ns(op, t, stats=stats, screen=screen))
    if truncate_out:
        g, rem = truncate(g, op.k, op.eps)
        if stats is not None:
            stats["truncation_l2"] = rem
    return g
