"""Oracle: 1-D operator blocks, block norms and the norm estimate (Secs. 3-4).

Test infrastructure only (see ``oracle/__init__``).

F^{j;m,l}_ii' = 2^{-j} int_{-1}^{1} exp(-tau_m (x+l)^2 / 4^j) Phi_ii'(x) dx
(eq. KernelFactor), l = (output box) - (input box) in one direction.

Oracle route (independent of the CUDA route): Phi+ and Phi- are polynomials
of degree <= 2k-1 on [0,1] and [-1,0]; each is recovered exactly from its
values at 2k Gauss-Legendre points (``basis.cross_corr``), and the integral is
taken piecewise on [-1,0] and [0,1] by composite 16-point GL restricted to the
window |x + l| <= sqrt(45 / c), c = tau/4^j (outside it the Gaussian is below
e^-45), with panels no wider than min(1/4, 1/(2 sqrt c)).

Norms (eq. BlockNorms), per direction, Frobenius norm (reading: the paper
does not name the norm; Frobenius bounds the operator norm and is
multiplicative under Kronecker products):
* nF[j,m,l]       = ||F^{j;m,l}||                       (k x k, l = -3..3)
* for j >= 1 and a coarse shift L, the fine 2 x 2 block matrix
  FF = [[F^{j;2L}, F^{j;2L-1}], [F^{j;2L+1}, F^{j;2L}]]  (rows: output child,
  columns: input child), its upsampled coarse counterpart
  UP = U F^{j-1;L} U^T with U = [H0^T; H1^T], and
  N_F = ||FF||, N_upF = ||F^{j-1;L}|| (= ||UP||, U has orthonormal columns),
  N_dif = ||FF - UP||.
* the symmetrised 18-term estimate of eq. NormEstimateUsing1DBlocks for a
  3-D coarse shift (L1, L2, L3): the mean over the 6 orderings sigma of
  Nd(s1) NF(s2) NF(s3) + NU(s1) Nd(s2) NF(s3) + NU(s1) NU(s2) Nd(s3).
* d = 2 (the paper's d = 2 variant): the same telescoping of a product of two
  factors, F1 F2 - G1 G2 = (F1 - G1) F2 + G1 (F2 - G2), symmetrised over the 2
  orderings: the mean of Nd(s1) NF(s2) + NU(s1) Nd(s2) over sigma (4 terms).

Parity pins (tests/test_oracle_operator.py): the erf closed form of F_00
(Phi_00 = 1 - |x|), the transposition/reflection symmetries implied by
Proposition 1, the vanishing moments in the wide-Gaussian limit, a direct
2-D quadrature of the Galerkin integral, and the telescoping identity
FF = UP for an exactly quadratic-free case (tau -> 0).
"""
import itertools
import math

import numpy as np
from numpy.polynomial import legendre as npleg

from . import basis
from . import gauss_sum

NT = 7          # translations l = -3..3 stored per level and term
TOFF = 3        # index of l = 0


def _phi_pm_coeffs(k):
    """Legendre-series coefficients of Phi+ on [0,1] and Phi- on [-1,0].

    Returns (cp, cm) with shape (k, k, 2k); Phi+(x) = legval(2x-1, cp),
    Phi-(x) = legval(2x+1, cm).
    """
    n = 2 * k
    g, _ = basis.gl01(n)
    vp = basis.cross_corr(k, g)            # x in (0,1)
    vm = basis.cross_corr(k, g - 1.0)      # x in (-1,0)
    V = npleg.legvander(2.0 * g - 1.0, n - 1)   # same abscissae u = 2x-1 (+)
    Vinv = np.linalg.inv(V)
    cp = np.einsum("qn,abn->abq", Vinv, vp)
    cm = np.einsum("qn,abn->abq", Vinv, vm)
    return cp, cm


class _PhiEval:
    def __init__(self, k):
        self.k = k
        self.cp, self.cm = _phi_pm_coeffs(k)

    def plus(self, x):
        V = npleg.legvander(2.0 * x - 1.0, 2 * self.k - 1)
        return np.einsum("abq,nq->abn", self.cp, V)

    def minus(self, x):
        V = npleg.legvander(2.0 * x + 1.0, 2 * self.k - 1)
        return np.einsum("abq,nq->abn", self.cm, V)


_G16 = basis.gl01(16)


def _panels(lo, hi, width):
    n = max(1, int(math.ceil((hi - lo) / width)))
    edges = np.linspace(lo, hi, n + 1)
    x = (edges[:-1, None] + (edges[1:] - edges[:-1])[:, None] * _G16[0][None, :]).ravel()
    w = ((edges[1:] - edges[:-1])[:, None] * _G16[1][None, :]).ravel()
    return x, w


def f_block(pe, j, tau, l):
    """F^{j;m,l} for one term (tau) and one integer shift l (eq. KernelFactor)."""
    k = pe.k
    c = tau / 4.0 ** j
    x0 = -float(l)
    half = math.sqrt(45.0 / c)
    width = min(0.25, 0.5 / math.sqrt(c))
    out = np.zeros((k, k))
    for lo, hi, ev in ((-1.0, 0.0, pe.minus), (0.0, 1.0, pe.plus)):
        a = max(lo, x0 - half)
        b = min(hi, x0 + half)
        if b <= a:
            continue
        x, w = _panels(a, b, width)
        g = w * np.exp(-c * (x - x0) ** 2)
        out += ev(x) @ g
    return out / 2.0 ** j


class Operator:
    """Operator tables for K_{mu,alpha} at order k on levels 0..max_level."""

    def __init__(self, mu, alpha, eps, k, max_level, delta=None, d=3):
        if not (1 <= k <= 16):
            raise ValueError("k must be in [1, 16]")
        if max_level < 0:
            raise ValueError("max_level must be >= 0")
        if d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        self.mu, self.alpha, self.eps, self.k = float(mu), float(alpha), float(eps), int(k)
        self.max_level, self.d = int(max_level), int(d)
        self.w, self.tau = gauss_sum.gaussian_sum(mu, alpha, eps, delta=delta, d=d)
        self.M = len(self.w)
        self.H0, self.H1 = basis.two_scale_H(k)
        self.U = np.vstack([self.H0.T, self.H1.T])          # 2k x k
        pe = _PhiEval(k)
        J = self.max_level
        F = np.zeros((J + 1, self.M, NT, k, k))
        for j in range(J + 1):
            for m in range(self.M):
                for l in range(-3, 4):
                    F[j, m, l + TOFF] = f_block(pe, j, self.tau[m], l)
        self.F = F
        self.nF = np.sqrt((F ** 2).sum(axis=(3, 4)))        # (J+1, M, 7)
        # 2x2 fine block matrices vs upsampled coarse blocks, coarse L = -1..1
        self.NdF = np.zeros((J + 1, self.M, 3))
        self.NFF = np.zeros((J + 1, self.M, 3))
        self.NUF = np.zeros((J + 1, self.M, 3))
        for j in range(1, J + 1):
            for m in range(self.M):
                for L in (-1, 0, 1):
                    FF = np.block([[F[j, m, 2 * L + TOFF], F[j, m, 2 * L - 1 + TOFF]],
                                   [F[j, m, 2 * L + 1 + TOFF], F[j, m, 2 * L + TOFF]]])
                    Fc = F[j - 1, m, L + TOFF]
                    UP = self.U @ Fc @ self.U.T
                    self.NFF[j, m, L + 1] = np.linalg.norm(FF)
                    self.NUF[j, m, L + 1] = np.linalg.norm(Fc)
                    self.NdF[j, m, L + 1] = np.linalg.norm(FF - UP)
        # max over the coarse core L in {-1,0,1}^d of the estimate
        self.est_core = np.zeros((J + 1, self.M))
        for j in range(1, J + 1):
            for m in range(self.M):
                best = 0.0
                for Ls in itertools.product(range(3), repeat=self.d):
                    best = max(best, self.estimate(j, m, Ls))
                self.est_core[j, m] = best

    def estimate(self, j, m, Lidx):
        """Eq. NormEstimateUsing1DBlocks (without w_m) for coarse shifts given
        as indices 0..2 (L = -1..1), symmetrised over the 6 orderings."""
        Nd = self.NdF[j, m]
        NF = self.NFF[j, m]
        NU = self.NUF[j, m]
        tot = 0.0
        if len(Lidx) == 2:   # d = 2: two factors, two orderings
            for a, b in itertools.permutations(Lidx):
                tot += Nd[a] * NF[b] + NU[a] * Nd[b]
            return tot / 2.0
        for s in itertools.permutations(Lidx):
            a, b, c = s
            tot += (Nd[a] * NF[b] * NF[c] + NU[a] * Nd[b] * NF[c] + NU[a] * NU[b] * Nd[c])
        return tot / 6.0
