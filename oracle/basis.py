"""Oracle: 1-D Legendre multiwavelet basis (paper Appendix, Secs. A.1-A.4).

Test infrastructure only (see ``oracle/__init__``).

Parity pins (tests/test_oracle_basis.py):
* ``gl01``           -- against numpy's Gauss-Legendre rule on monomials.
* ``phi``            -- orthonormality on [0,1] (Appendix, scaling functions).
* ``filters``        -- the 2k x 2k matrix [[H0 H1],[G0 G1]] is orthogonal;
                        the wavelets have k vanishing moments (Appendix,
                        multiwavelets); the two-scale relation holds pointwise.
* ``cross_corr``     -- Proposition 1 items 1-5 and 7; Phi_00(x) = 1-|x|.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gl01(n):
    """Gauss-Legendre nodes and weights on [0,1] (roots of P_n(2x-1)).

    Appendix, eq. fvals2coefs: x_i are the roots of P_p(2x-1) and w_i the
    matching weights.  numpy's rule on [-1,1] is mapped affinely.
    """
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def phi(k, x):
    """phi_i(x) = sqrt(2i+1) P_i(2x-1) on [0,1], zero outside (eq. scalingFNC).

    Returns an array of shape (k, len(x)).
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((k,) + x.shape)
    inside = (x >= 0.0) & (x <= 1.0)
    u = 2.0 * x - 1.0
    for i in range(k):
        c = np.zeros(i + 1)
        c[i] = 1.0
        out[i] = np.where(inside, np.sqrt(2 * i + 1) * npleg.legval(u, c), 0.0)
    return out


def two_scale_H(k):
    """Scaling filters H^(0), H^(1) of the two-scale relation (Appendix A.3).

    phi_i(x) = sqrt(2) sum_i' (h0_ii' phi_i'(2x) + h1_ii' phi_i'(2x-1)), so by
    orthonormality h^(p)_ii' = (1/sqrt 2) int_0^1 phi_i((u+p)/2) phi_i'(u) du.
    The integrand is a polynomial of degree <= 2k-2, so k-point GL is exact.
    """
    u, w = gl01(k)
    pu = phi(k, u)
    H = []
    for p in (0, 1):
        ph = phi(k, 0.5 * (u + p))
        H.append((ph * w) @ pu.T / np.sqrt(2.0))
    return H[0], H[1]


def two_scale_G(k):
    """Wavelet filters G^(0), G^(1) (Appendix A.3).

    The paper defers the construction of G to Alpert et al.  Reading used
    here: G is the orthonormal completion of the rows [H0 H1] to an
    orthogonal 2k x 2k matrix, obtained by modified Gram-Schmidt (two passes)
    of the start vectors (e_i, -e_i)/sqrt(2), i = 0..k-1, against the rows of
    [H0 H1] and then against each other.  Every orthonormal completion spans
    the same space W_0, so wavelet-coefficient norms (the only way wavelet
    coefficients enter the apply and the truncation) do not depend on it.
    """
    H0, H1 = two_scale_H(k)
    rows = [np.concatenate([H0[i], H1[i]]) for i in range(k)]
    G = []
    for i in range(k):
        v = np.zeros(2 * k)
        v[i] = 1.0 / np.sqrt(2.0)
        v[k + i] = -1.0 / np.sqrt(2.0)
        for _ in range(2):
            for r in rows + G:
                v = v - np.dot(r, v) * r
        v = v / np.linalg.norm(v)
        G.append(v)
    G = np.array(G)
    return G[:, :k].copy(), G[:, k:].copy()


def filter_matrix(k):
    """The 2k x 2k matrix W = [[H0, H1], [G0, G1]] (rows: s then d)."""
    H0, H1 = two_scale_H(k)
    G0, G1 = two_scale_G(k)
    return np.block([[H0, H1], [G0, G1]])


def cross_corr(k, x):
    """Cross-correlations Phi_ii'(x) (eqs. CrossCor, crosscor.00, crosscor.01).

    Phi+_ii'(x) = int_0^{1-x} phi_i(x+y) phi_i'(y) dy   for 0 <= x <= 1,
    Phi-_ii'(x) = int_{-x}^{1} phi_i(x+y) phi_i'(y) dy  for -1 <= x < 0,
    zero for |x| > 1.  Each integrand is a polynomial of degree <= 2k-2 on an
    interval of length 1-|x|, so k-point GL on that interval is exact.
    Returns an array of shape (k, k, len(x)).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    g, gw = gl01(k)
    out = np.zeros((k, k, x.size))
    for n, xv in enumerate(x):
        if abs(xv) > 1.0:
            continue
        if xv >= 0.0:
            lo, hi = 0.0, 1.0 - xv
        else:
            lo, hi = -xv, 1.0
        y = lo + (hi - lo) * g
        wy = (hi - lo) * gw
        a = phi(k, xv + y)          # phi_i(x+y)
        b = phi(k, y)               # phi_i'(y)
        out[:, :, n] = (a * wy) @ b.T
    return out
