"""Oracle: Gaussian-sum approximation of K_{mu,alpha} (Sec. 3).

Test infrastructure only (see ``oracle/__init__``).

K_{mu,alpha}(r) = C_alpha int_R exp(-r^2 e^{2s} - mu^2 e^{-2s}/4 + (3-2alpha)s) ds
(eq. IntegralRepr), C_alpha = 2 * 2^{-2 alpha} pi^{-3/2} / Gamma(alpha), is
discretised by the trapezoidal rule s_m = A + m h, m = 1..M, giving
tau_m = e^{2 s_m}, w_m = h C_alpha exp(-mu^2 e^{-2 s_m}/4 + (3-2alpha) s_m)
(eq. KernelApproxByGaussians).

The paper takes A, B and h from an external reference that is not part of the
paper.  Reading used here (both halves of the library use the same rule):

* h0 = pi^2 / (2 ln(1/eps))  (trapezoid error ~ exp(-pi^2/(2h)) for an
  integrand analytic in the strip |Im s| < pi/4);
* A: lower tail below 0.1 eps K_{0,alpha}(R):
  A0 = ln(0.1 eps (3-2a) Gamma(3/2-a) / (2 R^{3-2a})) / (3-2a); for mu > 0 also
  A_mu = -1/2 ln(4 (ln(1/eps) + 10) / mu^2); A = max(A0, A_mu);
* B = 1/2 ln((ln(1/eps) + 5) / delta^2);
* M = ceil((B - A)/h); while max_{r in [delta, R]} |K - sum| / K_{0,alpha}(r)
  exceeds eps on 4000 log-spaced r, shrink h by 3 % and recount.
* defaults delta = eps/10, R = sqrt(3) (the diameter of the unit cube): an
  over-provisioned range, as the paper intends; the per-scale screen discards
  the excess terms.

Dimension d.  The same integral gives the kernel of (-Laplacian + mu^2)^{-alpha}
in R^d (the paper's d = 2 variant, Sec. 6 and Algorithm 3 as illustrated for
d = 2): the heat-kernel route t^{alpha-1} (4 pi t)^{-d/2} exp(-r^2/(4t) - mu^2 t)
with 1/(4t) = e^{2s} gives C^{(d)}_alpha int exp(-r^2 e^{2s} - mu^2 e^{-2s}/4
+ (d - 2alpha) s) ds, C^{(d)}_alpha = 2 * 2^{-2 alpha} pi^{-d/2} / Gamma(alpha)
(d = 3: the paper's C_alpha).  In closed form K^{(d)}_{mu,alpha}(r) =
C^{(d)}_alpha (mu/(2r))^{d/2 - alpha} K_{d/2 - alpha}(mu r), and at mu = 0
C^{(d)}_alpha Gamma(d/2 - alpha) / (2 r^{d - 2 alpha}), the envelope of the
sup-norm test (0 < alpha < d/2).  Every rule above carries over with 3 replaced
by d (R = sqrt(d), the diameter of the unit cube of R^d).

Parity pin (tests/test_oracle_gauss_sum.py): the sup relative error bound of
eq. KernelApproxByGaussians against scipy's Bessel K, and the term count of
Fig. 3 (about 300 terms for eps = 1e-10 over 15 decades); for d = 2
(tests/test_oracle_d2.py) the closed form against a direct quadrature of the
integral representation, the bound, and 1/(2 pi r) at alpha = 1/2.
"""
import math

import numpy as np
from scipy import special


def c_alpha(alpha, d=3):
    """C_alpha = 2 * 2^{-2 alpha} pi^{-d/2} / Gamma(alpha) (Sec. 3 for d = 3)."""
    return 2.0 * 2.0 ** (-2.0 * alpha) * math.pi ** (-0.5 * d) / math.gamma(alpha)


def kernel(mu, alpha, r, d=3):
    """K_{mu,alpha}(r) (Sec. 3): modified-Bessel form; mu = 0 limit closed form."""
    r = np.asarray(r, dtype=np.float64)
    ca = c_alpha(alpha, d)
    nu = 0.5 * d - alpha
    if mu == 0.0:
        return math.gamma(nu) * ca / (2.0 * r ** (2.0 * nu))
    return ca * (mu / (2.0 * r)) ** nu * special.kv(nu, mu * r)


def envelope(alpha, r, d=3):
    """K_{0,alpha}(r), the right-hand side scale of eq. KernelApproxByGaussians."""
    return kernel(0.0, alpha, r, d)


def _terms(mu, alpha, A, h, M, d=3):
    ca = c_alpha(alpha, d)
    s = A + h * np.arange(1, M + 1, dtype=np.float64)
    tau = np.exp(2.0 * s)
    w = h * ca * np.exp(-0.25 * mu * mu * np.exp(-2.0 * s) + (d - 2.0 * alpha) * s)
    return w, tau


def eval_sum(w, tau, r):
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-np.outer(r * r, tau)) @ w


def max_rel_error(mu, alpha, w, tau, delta, R, n=4000, d=3):
    r = np.exp(np.linspace(math.log(delta), math.log(R), n))
    err = np.abs(kernel(mu, alpha, r, d) - eval_sum(w, tau, r)) / envelope(alpha, r, d)
    return float(err.max())


def gaussian_sum(mu, alpha, eps, delta=None, R=None, d=3):
    """Return (w, tau) with |K_{mu,alpha}(r) - sum_m w_m e^{-tau_m r^2}| <=
    eps K_{0,alpha}(r) on [delta, R] (eq. KernelApproxByGaussians) in R^d
    (R = sqrt(d) by default).

    tau is increasing in m (s_m increases with m).
    """
    if not (0.0 < alpha < 0.5 * d):
        raise ValueError("alpha must lie in (0, d/2)")
    if not (eps > 0.0) or mu < 0.0:
        raise ValueError("eps must be > 0 and mu >= 0")
    if delta is None:
        delta = eps / 10.0
    if R is None:
        R = math.sqrt(d)
    L = math.log(1.0 / eps)
    q = d - 2.0 * alpha
    A = math.log(0.1 * eps * q * math.gamma(0.5 * q) / (2.0 * R ** q)) / q
    if mu > 0.0:
        A = max(A, -0.5 * math.log(4.0 * (L + 10.0) / (mu * mu)))
    B = 0.5 * math.log((L + 5.0) / (delta * delta))
    h = math.pi ** 2 / (2.0 * L)
    for _ in range(200):
        M = int(math.ceil((B - A) / h))
        w, tau = _terms(mu, alpha, A, h, M, d)
        if max_rel_error(mu, alpha, w, tau, delta, R, d=d) <= eps:
            return w, tau
        h *= 0.97
    raise RuntimeError("Gaussian-sum construction did not reach eps")
