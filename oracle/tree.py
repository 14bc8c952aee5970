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

    def on_grids(self, X):
        """Values on tensor grids: X is a list of three (n, q) arrays of
        per-direction coordinates; returns (n, q, q, q).  Each term factors as
        exp(-a|x-c|^2) = prod_d exp(-a (x_d - c_d)^2), and the r^2 factor as a
        sum over directions."""
        n, q = X[0].shape
        out = np.zeros((n, q, q, q))
        for c, b, a, x0 in zip(self.coef, self.r2coef, self.expo, self.centers):
            R = [(X[d] - x0[d]) ** 2 for d in range(3)]
            E = [np.exp(-a * R[d]) for d in range(3)]
            prod = E[0][:, :, None, None] * E[1][:, None, :, None] * E[2][:, None, None, :]
            out += c * prod
            if b != 0.0:
                out += b * ((R[0] * E[0])[:, :, None, None] * E[1][:, None, :, None] * E[2][:, None, None, :]
                            + E[0][:, :, None, None] * (R[1] * E[1])[:, None, :, None] * E[2][:, None, None, :]
                            + E[0][:, :, None, None] * E[1][:, None, :, None] * (R[2] * E[2])[:, None, None, :])
        return out


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
    s = np.einsum("ia,jb,kc,abc->ijk", P, P, P, v, optimize=True)
    return s / 2.0 ** (1.5 * j)


def eval_block(k, j, a, s, pts):
    """f(x) = sum_i s_i prod_d phi^j_{i_d, a_d}(x_d) (eq. func_interp_2d in 3-D)."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    u = pts * 2.0 ** j - np.asarray(a, dtype=np.float64)
    P = [basis.phi(k, u[:, d]) for d in range(3)]  # (i, n)
    return np.einsum("ijk,in,jn,kn->n", s, P[0], P[1], P[2], optimize=True) * 2.0 ** (1.5 * j)


def _level_projection(dens, k, j, boxes, P, g):
    """Values at each box's k^3 GL nodes and their projections, for a batch
    of boxes (n, 3) at level j: eq. fvals2coefs in tensor form."""
    h = 2.0 ** -j
    X = [(g[None, :] + boxes[:, d:d + 1]) * h for d in range(3)]          # (n, k) per direction
    vals = dens.on_grids(X)
    return np.einsum("ia,jb,kc,nabc->nijk", P, P, P, vals, optimize=True) * 2.0 ** (-1.5 * j)


def _children_error(dens, k, j, boxes, s, g, Q):
    """max over the 8 children of |f - f~| at the children's GL nodes, where
    f~ interpolates the parent's coefficients (Algorithm 1's test)."""
    hc = 2.0 ** -(j + 1)
    n = len(boxes)
    err = np.zeros(n)
    for p in OCTS:
        X = [(g[None, :] + 2 * boxes[:, d:d + 1] + p[d]) * hc for d in range(3)]
        direct = dens.on_grids(X)
        interp = np.einsum("nijk,ai,bj,ck->nabc", s, Q[p[0]], Q[p[1]], Q[p[2]], optimize=True) * 2.0 ** (1.5 * j)
        err = np.maximum(err, np.abs(direct - interp).reshape(n, -1).max(axis=1))
    return err


def build_tree(dens, k, eps, max_level, uniform_level=-1, init_level=0, chunk=64):
    """Algorithm 1 (adaptive function decomposition) in d = 3, processed one
    level at a time (the boxes of a level are independent).

    Returns (tree, depth_hit)."""
    tol = eps * dens.scale()
    g, w = basis.gl01(k)
    P = basis.phi(k, g) * w                                   # (i, q): projection
    Q = [basis.phi(k, 0.5 * (g + p)).T for p in (0, 1)]       # (q, i): child-node values
    tree = {}
    depth_hit = False
    boxes = np.zeros((1, 3), dtype=np.int64)
    j = 0
    while len(boxes):
        refine = np.zeros(len(boxes), dtype=bool)
        S = np.zeros((len(boxes), k, k, k))
        for c0 in range(0, len(boxes), chunk):
            bx = boxes[c0:c0 + chunk]
            s = _level_projection(dens, k, j, bx, P, g)
            S[c0:c0 + chunk] = s
            if uniform_level >= 0:
                refine[c0:c0 + chunk] = j < uniform_level
            elif j < init_level:
                refine[c0:c0 + chunk] = True
            else:
                fail = _children_error(dens, k, j, bx, s, g, Q) > tol
                if j >= max_level:
                    depth_hit = depth_hit or bool(fail.any())
                    fail[:] = False
                refine[c0:c0 + chunk] = fail
        if j >= max_level:
            refine[:] = False
        nxt = []
        for b, r, s in zip(boxes, refine, S):
            key = (j,) + tuple(int(v) for v in b)
            if r:
                tree[key] = Node(False)
                for p in OCTS:
                    nxt.append([2 * b[0] + p[0], 2 * b[1] + p[1], 2 * b[2] + p[2]])
            else:
                tree[key] = Node(True, s)
        boxes = np.array(nxt, dtype=np.int64).reshape(-1, 3)
        j += 1
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
    return np.einsum("ai,bj,ck,ijk->abc", Wm, Wm, Wm, cube, optimize=True)


def compress(tree, k):
    """Redundant tree (Sec. 2.2.1): bottom-up, every internal node gets
    s^j = sum_p (H^(p1) x H^(p2) x H^(p3)) s^{j+1}_{child p} (eq. decomp_scaling)
    and the seven wavelet blocks (eq. decomp_wavelet), i.e. the 2k x 2k
    filter matrix W applied in each direction to the (2k)^3 cube of the
    children.  d holds that cube with its scaling corner zeroed.  The
    internal nodes of one level are transformed together."""
    Wm = basis.filter_matrix(k)
    for j in range(levels(tree) - 2, -1, -1):
        keys = [key for key, node in tree.items() if key[0] == j and not node.leaf]
        if not keys:
            continue
        cubes = np.stack([_cube_of_children(tree, key, k) for key in keys])
        out = np.einsum("ai,bj,ck,nijk->nabc", Wm, Wm, Wm, cubes, optimize=True)
        for key, o in zip(keys, out):
            node = tree[key]
            node.s = o[:k, :k, :k].copy()
            o[:k, :k, :k] = 0.0
            node.d = o
            node.dnorm = float(np.linalg.norm(o))
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
    return np.einsum("ia,jb,kc,ijk->abc", H[p[0]], H[p[1]], H[p[2]], s, optimize=True)


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


def refine_graded(tree, k, passes=1, max_level=12):
    """Output skeleton refinement (the paper copies the input skeleton for the
    output and leaves the removal of that assumption for later, Algorithm 2/3,
    Initialization).  Reading: one pass splits every leaf at level j <
    max_level that has an internal node among the 26 boxes around it at level
    j, each child receiving the exact refinement of the leaf's block
    (``upsample``, the d = 0 half of eqs. recon_even / recon_odd); the split
    leaf keeps its own block and a zero wavelet norm.  The function is
    unchanged.  Returns (new tree, leaves split)."""
    cur = copy_tree(tree)
    total = 0
    for _ in range(passes):
        internal = {key for key, n in cur.items() if not n.leaf}
        split = []
        for key, n in cur.items():
            j, a = key[0], key[1:]
            if not n.leaf or j >= max_level:
                continue
            for dt in itertools.product((-1, 0, 1), repeat=3):
                if dt == (0, 0, 0):
                    continue
                if (j,) + tuple(a[d] + dt[d] for d in range(3)) in internal:
                    split.append(key)
                    break
        for key in split:
            node = cur[key]
            node.leaf = False
            node.dnorm = 0.0
            for p, ck in zip(OCTS, children(key)):
                cur[ck] = Node(True, upsample(k, node.s, p))
        total += len(split)
        if not split:
            break
    return cur, total
