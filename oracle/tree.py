"""Oracle: adaptive / redundant trees in d = 3 (Sec. 2.2, Algorithm 1, Appendix).

Test infrastructure only (see ``oracle/__init__``).

A tree is a dict keyed by (j, a1, a2, a3) -- level j (root j = 0) and box
index a in [0, 2^j)^3 -- whose values are Node objects.  Every internal node
has all 8 children (Algorithm 1 refines the 8 children together).  Blocks are
(k, k, k) arrays s[i1, i2, i3] of scaling coefficients in the tensor basis
phi^j_{i1,a1}(x1) phi^j_{i2,a2}(x2) phi^j_{i3,a3}(x3).

Densities are sums of Gaussians with an optional r^2 factor per term,
f(x) = sum_g (c_g + b_g |x - x_g|^2) exp(-a_g |x - x_g|^2), which covers the
paper's Poisson test density rho = -Laplacian(sum exp(-a r^2)) (Sec. 6.1).

Readings (the paper is silent): the l-infinity test of Algorithm 1 uses the
threshold eps * fscale with fscale = max_g |f(x_g)| over the Gaussian
centres; refinement stops at max_level (a leaf that still fails the test sets
``depth_hit``); ``init_level`` refines uniformly before the adaptive test
starts (the paper's "appropriate choice of the initial sampling scale");
``uniform_level >= 0`` builds the uniform tree of that depth.

Parity pins (tests/test_oracle_tree.py): projection of polynomials of degree
< k is exact; compress/reconstruct round trip and Parseval; Algorithm 1 meets
its l-infinity bound at sample points of the leaves.
"""
import itertools

import numpy as np

from . import basis

OCTS = list(itertools.product((0, 1), repeat=3))     # child octant (p1, p2, p3)


class Node:
    __slots__ = ("leaf", "s", "d", "dnorm")

    def __init__(self, leaf, s=None):
        self.leaf = leaf
        self.s = s
        self.d = None
        self.dnorm = 0.0


class Density:
    def __init__(self, coef, expo, centers, r2coef=None):
        self.coef = np.asarray(coef, dtype=np.float64)
        self.expo = np.asarray(expo, dtype=np.float64)
        self.centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        self.r2coef = (np.zeros_like(self.coef) if r2coef is None
                       else np.asarray(r2coef, dtype=np.float64))

    def __call__(self, pts):
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
        out = np.zeros(len(pts))
        for c, b, a, x0 in zip(self.coef, self.r2coef, self.expo, self.centers):
            r2 = ((pts - x0) ** 2).sum(axis=1)
            out += (c + b * r2) * np.exp(-a * r2)
        return out

    def scale(self):
        return float(np.abs(self(self.centers)).max())


def box_nodes(k, j, a):
    """GL nodes of box (j, a) per direction: array (3, k)."""
    g, _ = basis.gl01(k)
    return np.array([(g + a[d]) / 2.0 ** j for d in range(3)])


def grid(xs):
    """Tensor grid of three 1-D node sets -> (n1*n2*n3, 3) points, C order."""
    X = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
    return np.stack([x.ravel() for x in X], axis=1)


def project_values(k, j, vals):
    """Coefficients from values at the box's k^3 GL nodes (eq. fvals2coefs,
    tensor form): s = 2^{-3j/2} sum_q f(x_q) prod_d phi_{i_d}(g_{q_d}) w_{q_d}."""
    g, w = basis.gl01(k)
    P = basis.phi(k, g) * w                      # (i, q)
    v = vals.reshape(k, k, k)
    s = np.einsum("ia,jb,kc,abc->ijk", P, P, P, v)
    return s / 2.0 ** (1.5 * j)


def eval_block(k, j, a, s, pts):
    """f(x) = sum_i s_i prod_d phi^j_{i_d, a_d}(x_d) (eq. func_interp_2d in 3-D)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    u = pts * 2.0 ** j - np.asarray(a, dtype=np.float64)
    P = [basis.phi(k, u[:, d]) for d in range(3)]  # (i, n)
    return np.einsum("ijk,in,jn,kn->n", s, P[0], P[1], P[2]) * 2.0 ** (1.5 * j)


def build_tree(dens, k, eps, max_level, uniform_level=-1, init_level=0):
    """Algorithm 1 (adaptive function decomposition) in d = 3.

    Returns (tree, depth_hit)."""
    tol = eps * dens.scale()
    tree = {}
    depth_hit = False
    todo = [(0, 0, 0, 0)]
    while todo:
        nxt = []
        for key in todo:
            j, a = key[0], key[1:]
            vals = dens(grid(box_nodes(k, j, a)))
            s = project_values(k, j, vals)
            if uniform_level >= 0:
                refine = j < uniform_level
            elif j < init_level:
                refine = True
            else:
                err = 0.0
                for p in OCTS:
                    c = tuple(2 * a[d] + p[d] for d in range(3))
                    pts = grid(box_nodes(k, j + 1, c))
                    err = max(err, float(np.abs(dens(pts) - eval_block(k, j, a, s, pts)).max()))
                refine = err > tol
                if refine and j >= max_level:
                    depth_hit = True
                    refine = False
            if refine:
                tree[key] = Node(False)
                for p in OCTS:
                    nxt.append((j + 1,) + tuple(2 * a[d] + p[d] for d in range(3)))
            else:
                tree[key] = Node(True, s)
        todo = nxt
    return tree, depth_hit


def levels(tree):
    return max(key[0] for key in tree) + 1


def children(key):
    j, a = key[0], key[1:]
    return [(j + 1,) + tuple(2 * a[d] + p[d] for d in range(3)) for p in OCTS]


def _cube_of_children(tree, key, k):
    cube = np.zeros((2 * k, 2 * k, 2 * k))
    for p, ck in zip(OCTS, children(key)):
        cube[p[0] * k:(p[0] + 1) * k, p[1] * k:(p[1] + 1) * k, p[2] * k:(p[2] + 1) * k] = tree[ck].s
    return cube


def _apply3(Wm, cube):
    return np.einsum("ai,bj,ck,ijk->abc", Wm, Wm, Wm, cube)


def compress(tree, k):
    """Redundant tree (Sec. 2.2.1): bottom-up, every internal node gets
    s^j = sum_p (H^(p1) x H^(p2) x H^(p3)) s^{j+1}_{child p} (eq. decomp_scaling)
    and the seven wavelet blocks (eq. decomp_wavelet), i.e. the 2k x 2k
    filter matrix W applied in each direction to the (2k)^3 cube of the
    children.  d holds that cube with its scaling corner zeroed."""
    Wm = basis.filter_matrix(k)
    for j in range(levels(tree) - 2, -1, -1):
        for key, node in tree.items():
            if key[0] != j or node.leaf:
                continue
            out = _apply3(Wm, _cube_of_children(tree, key, k))
            node.s = out[:k, :k, :k].copy()
            out[:k, :k, :k] = 0.0
            node.d = out
            node.dnorm = float(np.linalg.norm(out))
    return tree


def reconstruct(tree, k):
    """Inverse of ``compress`` (eqs. recon_even / recon_odd; the filter matrix
    is orthogonal, so the inverse is its transpose): top-down, the children's
    s blocks are rebuilt from each internal node's s and d."""
    Wm = basis.filter_matrix(k)
    for j in range(levels(tree) - 1):
        for key, node in tree.items():
            if key[0] != j or node.leaf:
                continue
            cube = node.d.copy()
            cube[:k, :k, :k] = node.s
            full = _apply3(Wm.T, cube)
            for p, ck in zip(OCTS, children(key)):
                tree[ck].s = full[p[0] * k:(p[0] + 1) * k, p[1] * k:(p[1] + 1) * k,
                                  p[2] * k:(p[2] + 1) * k].copy()
    return tree


def upsample(k, s, p):
    """s^{j+1}_{2a+p} = (H^(p1)T x H^(p2)T x H^(p3)T) s^j_a (the d = 0 half of
    eqs. recon_even / recon_odd)."""
    H = basis.two_scale_H(k)
    return np.einsum("ia,jb,kc,ijk->abc", H[p[0]], H[p[1]], H[p[2]], s)


def norm2(tree):
    """L2 norm by Parseval from the leaves."""
    return float(np.sqrt(sum((n.s ** 2).sum() for n in tree.values() if n.leaf)))


def copy_tree(tree):
    out = {}
    for key, n in tree.items():
        m = Node(n.leaf, None if n.s is None else n.s.copy())
        m.d = None if n.d is None else n.d.copy()
        m.dnorm = n.dnorm
        out[key] = m
    return out


def to_arrays(tree, k):
    """Flat export: keys (n, 4) int64 rows (j, a1, a2, a3) sorted by level then
    box, leaf flags (n,), and blocks (n, k, k, k) (zeros where undefined)."""
    keys = sorted(tree.keys())
    K = np.array(keys, dtype=np.int64).reshape(-1, 4)
    leaf = np.array([tree[key].leaf for key in keys], dtype=np.int32)
    S = np.zeros((len(keys), k, k, k))
    for i, key in enumerate(keys):
        if tree[key].s is not None:
            S[i] = tree[key].s
    return K, leaf, S


def from_arrays(K, leaf, S):
    tree = {}
    for row, lf, s in zip(np.asarray(K), np.asarray(leaf), np.asarray(S)):
        tree[tuple(int(v) for v in row)] = Node(bool(lf), np.array(s, dtype=np.float64))
    return tree
