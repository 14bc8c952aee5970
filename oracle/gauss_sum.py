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

Parity pin (tests/test_oracle_gauss_sum.py): the sup relative error bound of
eq. KernelApproxByGaussians against scipy's Bessel K, and the term count of
Fig. 3 (about 300 terms for eps = 1e-10 over 15 decades).
"""
import math

import numpy as np
from scipy import special


def c_alpha(alpha):
    """C_alpha = 2 * 2^{-2 alpha} pi^{-3/2} / Gamma(alpha) (Sec. 3)."""
    return 2.0 * 2.0 ** (-2.0 * alpha) * math.pi ** (-1.5) / math.gamma(alpha)


def kernel(mu, alpha, r):
    """K_{mu,alpha}(r) (Sec. 3): modified-Bessel form; mu = 0 limit closed form."""
    r = np.asarray(r, dtype=np.float64)
    ca = c_alpha(alpha)
    if mu == 0.0:
        return math.gamma(1.5 - alpha) * ca / (2.0 * r ** (3.0 - 2.0 * alpha))
    nu = 1.5 - alpha
    return 2.0 ** (-1.5 + alpha) * ca * (mu / r) ** nu * special.kv(nu, mu * r)


def envelope(alpha, r):
    """K_{0,alpha}(r), the right-hand side scale of eq. KernelApproxByGaussians."""
    return kernel(0.0, alpha, r)


def _terms(mu, alpha, A, h, M):
    ca = c_alpha(alpha)
    s = A + h * np.arange(1, M + 1, dtype=np.float64)
    tau = np.exp(2.0 * s)
    w = h * ca * np.exp(-0.25 * mu * mu * np.exp(-2.0 * s) + (3.0 - 2.0 * alpha) * s)
    return w, tau


def eval_sum(w, tau, r):
    r = np.asarray(r, dtype=np.float64)
    return np.exp(-np.outer(r * r, tau)) @ w


def max_rel_error(mu, alpha, w, tau, delta, R, n=4000):
    r = np.exp(np.linspace(math.log(delta), math.log(R), n))
    err = np.abs(kernel(mu, alpha, r) - eval_sum(w, tau, r)) / envelope(alpha, r)
    return float(err.max())


def gaussian_sum(mu, alpha, eps, delta=None, R=math.sqrt(3.0)):
    """Return (w, tau) with |K_{mu,alpha}(r) - sum_m w_m e^{-tau_m r^2}| <=
    eps K_{0,alpha}(r) on [delta, R] (eq. KernelApproxByGaussians).

    tau is increasing in m (s_m increases with m).
    """
    if not (0.0 < alpha < 1.5):
        raise ValueError("alpha must lie in (0, 3/2)")
    if not (eps > 0.0) or mu < 0.0:
        raise ValueError("eps must be > 0 and mu >= 0")
    if delta is None:
        delta = eps / 10.0
    L = math.log(1.0 / eps)
    q = 3.0 - 2.0 * alpha
    A = math.log(0.1 * eps * q * math.gamma(1.5 - alpha) / (2.0 * R ** q)) / q
    if mu > 0.0:
        A = max(A, -0.5 * math.log(4.0 * (L + 10.0) / (mu * mu)))
    B = 0.5 * math.log((L + 5.0) / (delta * delta))
    h = math.pi ** 2 / (2.0 * L)
    for _ in range(200):
        M = int(math.ceil((B - A) / h))
        w, tau = _terms(mu, alpha, A, h, M)
        if max_rel_error(mu, alpha, w, tau, delta, R) <= eps:
            return w, tau
        h *= 0.97
    raise RuntimeError("Gaussian-sum construction did not reach eps")
