"""Oracle: pointwise products and inner products of trees, for the hydrogen
ground-state iteration of Sec. 6.2 (Steps 2 and 4).

Test infrastructure only (see ``oracle/__init__``).

The paper computes products and inner products by the method of its
reference [A-B-G-V:2002] and does not describe it.  Reading used here (and by
the library): the product V f is projected leaf by leaf on f's skeleton with
the box's k-point Gauss-Legendre rule per direction -- f's values at the
box's k^3 GL nodes (the block evaluated, eq. func_interp_2d in tensor form),
times V there, projected back (eq. fvals2coefs in tensor form).  This is the
exact L2 projection of V f whenever V f restricted to the box is a
polynomial of degree <= k per direction (the rule integrates degree 2k - 1).

The inner product of two functions on one skeleton is the sum over the
leaves of the coefficient products (Parseval: the leaf blocks are
coefficients in an orthonormal basis of the piecewise polynomials).

Potentials: V(x) = sum_g (c_g + b_g |x - x_g|^2) exp(-a_g |x - x_g|^2)
+ sum_n q_n / |x - R_n|, a_g >= 0.  A point at distance 0 from some R_n takes
0 from that term.

Parity pins (tests/test_oracle_product.py): a polynomial potential times a
polynomial block against the exact product projected by a 24-point rule
(1-D polynomial arithmetic); a charge outside the cube against a 32-point
projection of the smooth product; multiplication by the constant 1 is the
identity; the inner product of two projected Gaussians against their
closed-form overlap.
"""
import numpy as np

from . import tree as T


class Potential:
    def __init__(self, coef=(), expo=(), centers=(), r2coef=None, charges=(), positions=()):
        self.coef = np.asarray(coef, dtype=np.float64).reshape(-1)
        self.expo = np.asarray(expo, dtype=np.float64).reshape(-1)
        self.centers = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        self.r2coef = (np.zeros_like(self.coef) if r2coef is None
                       else np.asarray(r2coef, dtype=np.float64).reshape(-1))
        self.charges = np.asarray(charges, dtype=np.float64).reshape(-1)
        self.positions = np.asarray(positions, dtype=np.float64).reshape(-1, 3)

    def __call__(self, pts):
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
        v = np.zeros(len(pts))
        for c, b, a, x0 in zip(self.coef, self.r2coef, self.expo, self.centers):
            r2 = ((pts - x0) ** 2).sum(axis=1)
            v += (c + b * r2) * np.exp(-a * r2)
        for q, R in zip(self.charges, self.positions):
            r = np.sqrt(((pts - R) ** 2).sum(axis=1))
            with np.errstate(divide="ignore"):
                v += np.where(r > 0.0, q / np.where(r > 0.0, r, 1.0), 0.0)
        return v


def multiply(tree, k, pot, scale=1.0):
    """scale * P(V f) on f's skeleton: leaves get the projected product,
    internal nodes zero blocks."""
    out = {}
    for key, node in tree.items():
        if not node.leaf:
            out[key] = T.Node(False, np.zeros((k, k, k)))
            continue
        j, a = key[0], key[1:]
        pts = T.grid(T.box_nodes(k, j, a))                 # (k^3, 3), C order
        fvals = T.eval_block(k, j, a, node.s, pts)
        out[key] = T.Node(True, scale * T.project_values(k, j, fvals * pot(pts)))
    return out


def dot(ta, tb):
    """sum over the leaves of <s_a, s_b>; the two trees share a skeleton."""
    assert ta.keys() == tb.keys()
    total = 0.0
    for key, node in ta.items():
        assert node.leaf == tb[key].leaf
        if node.leaf:
            total += float((node.s * tb[key].s).sum())
    return total


def scale(tree, alpha):
    return {key: T.Node(n.leaf, None if n.s is None else alpha * n.s) for key, n in tree.items()}


def project_onto(tree, k, fn):
    """The projection of a function (callable on (n, 3) points) onto the
    leaves of ``tree`` by the same GL rule."""
    out = {}
    for key, node in tree.items():
        if not node.leaf:
            out[key] = T.Node(False, np.zeros((k, k, k)))
            continue
        j, a = key[0], key[1:]
        pts = T.grid(T.box_nodes(k, j, a))
        out[key] = T.Node(True, T.project_values(k, j, fn(pts)))
    return out

