"""Closed forms and projections used to pin the oracle.

Written independently of ``oracle/`` (own quadrature and Legendre evaluation),
so that an error in the oracle's basis code cannot cancel out of a pin.
"""
import math

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy import special


def gl(n):
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1), 0.5 * w


def legendre_scaled(k, u):
    """sqrt(2i+1) P_i(2u-1), i < k, for u in [0,1] -> (k, n)."""
    v = 2.0 * np.asarray(u) - 1.0
    out = np.empty((k, v.size))
    p0, p1 = np.ones_like(v), v
    for i in range(k):
        if i == 0:
            p = p0
        elif i == 1:
            p = p1
        else:
            p = ((2 * i - 1) * v * p1 - (i - 1) * p0) / i
            p0, p1 = p1, p
        out[i] = math.sqrt(2 * i + 1) * p
    return out


def project_leaf(fun, k, j, b, sub=4, q=None):
    """Coefficients of fun on box (j, b) by composite GL (sub^3 sub-boxes,
    q points per direction each): s_i = int_box fun phi^j_i."""
    q = q or k + 3
    g, w = gl(q)
    x1 = np.concatenate([(u + g) / sub for u in range(sub)])
    w1 = np.concatenate([w / sub for _ in range(sub)])
    P = legendre_scaled(k, x1) * w1
    ax = [(x1 + b[d]) / 2.0 ** j for d in range(3)]
    X = np.meshgrid(*ax, indexing="ij")
    pts = np.stack([x.ravel() for x in X], axis=1)
    v = fun(pts).reshape(len(x1), len(x1), len(x1))
    return np.einsum("ia,jb,kc,abc->ijk", P, P, P, v) / 2.0 ** (1.5 * j)


def poisson_gaussian(a, c):
    """Potential of a unit-mass Gaussian (a/pi)^{3/2} exp(-a|x-c|^2) under
    K = 1/(4 pi r): erf(sqrt(a) r) / (4 pi r)."""
    c = np.asarray(c, dtype=np.float64)

    def f(p):
        r = np.linalg.norm(p - c, axis=1)
        small = r < 1e-8
        rs = np.where(small, 1.0, r)
        return np.where(small, 2.0 * math.sqrt(a / math.pi), special.erf(math.sqrt(a) * rs) / rs) / (4 * math.pi)
    return f


def yukawa_gaussian(a, mu, c):
    """Potential of a unit-mass Gaussian under K = exp(-mu r)/(4 pi r):
    V(r) = e^{mu^2/(4a)} / (2r) [e^{-mu r} erfc(mu/(2 sqrt a) - sqrt(a) r)
                                 - e^{mu r} erfc(mu/(2 sqrt a) + sqrt(a) r)] / (4 pi),
    evaluated with erfcx to avoid overflow."""
    c = np.asarray(c, dtype=np.float64)
    sa = math.sqrt(a)
    z0 = mu / (2 * sa)

    def V(r):
        r = np.maximum(r, 1e-12)
        z1 = z0 - sa * r
        z2 = z0 + sa * r
        # e^{mu^2/4a - mu r} erfc(z1) = e^{-a r^2} e^{-z1^2}... use erfcx(z) = e^{z^2} erfc(z)
        # mu^2/(4a) - mu r - z1^2 = -a r^2 ; mu^2/(4a) + mu r - z2^2 = -a r^2
        t1 = np.where(z1 >= 0, np.exp(-a * r * r) * special.erfcx(z1),
                      np.exp(mu * mu / (4 * a) - mu * r) * special.erfc(z1))
        t2 = np.exp(-a * r * r) * special.erfcx(z2)
        return (t1 - t2) / (2 * r) / (4 * math.pi)

    def f(p):
        return V(np.linalg.norm(p - c, axis=1))
    f.radial = V
    return f


def truncated_gauss_sum_potential(w, tau, a, c, coef=1.0):
    """sum_m w_m prod_d int_0^1 exp(-tau_m (x_d - y)^2) coef^(1/3) exp(-a (y - c_d)^2) dy:
    the Gaussian-sum kernel applied exactly to a Gaussian truncated to [0,1]^3.
    Completing the square: exp(-tau(x-y)^2 - a(y-c)^2) =
    exp(-tau a/(tau+a) (x-c)^2) exp(-(tau+a)(y - y0)^2), y0 = (tau x + a c)/(tau+a)."""
    c = np.asarray(c, dtype=np.float64)

    def one_dim(x, cd):
        s = tau[None, :] + a
        y0 = (tau[None, :] * x[:, None] + a * cd) / s
        rs = np.sqrt(s)
        lo, hi = -y0 * rs, (1.0 - y0) * rs
        # int_lo^hi e^{-u^2} du * sqrt(pi)/2 ... via erf differences, erfc for same-sign tails
        val = np.where(lo >= 0, special.erfc(lo) - special.erfc(hi),
                       np.where(hi <= 0, special.erfc(-hi) - special.erfc(-lo),
                                special.erf(hi) - special.erf(lo)))
        return np.exp(-(tau[None, :] * a / s) * (x[:, None] - cd) ** 2) * val * math.sqrt(math.pi) / (2 * rs)

    def f(p):
        prod = one_dim(p[:, 0], c[0]) * one_dim(p[:, 1], c[1]) * one_dim(p[:, 2], c[2])
        return coef * (prod @ w)
    return f
