"""Pins for oracle/gauss_sum.py (Sec. 3, eqs. IntegralRepr and
KernelApproxByGaussians; Proposition trapez; Fig. 3)."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import gauss_sum


def kernel_ref(mu, alpha, r):
    """K_{mu,alpha} written out independently: alpha = 1 closed forms
    e^{-mu r}/(4 pi r); otherwise the Bessel form with scipy's kv."""
    if alpha == 1.0:
        return np.exp(-mu * r) / (4 * math.pi * r)
    ca = 2 * 2 ** (-2 * alpha) * math.pi ** -1.5 / math.gamma(alpha)
    if mu == 0.0:
        return math.gamma(1.5 - alpha) * ca / (2 * r ** (3 - 2 * alpha))
    nu = 1.5 - alpha
    return 2 ** (-1.5 + alpha) * ca * (mu / r) ** nu * special.kv(nu, mu * r)


def test_c_alpha_normalisation():
    # K_{0,1} = 1/(4 pi r): the Poisson Green's function of Sec. 6.1
    assert abs(gauss_sum.c_alpha(1.0) - 1 / (2 * math.pi ** 1.5)) < 1e-16
    assert abs(gauss_sum.kernel(0.0, 1.0, 0.7) - 1 / (4 * math.pi * 0.7)) < 1e-15


@pytest.mark.parametrize("mu,alpha,eps", [(0.0, 1.0, 1e-4), (0.0, 1.0, 1e-6), (1.5, 1.0, 1e-6),
                                          (0.0, 0.5, 1e-6), (0.7, 0.75, 1e-5)])
def test_sup_relative_error(mu, alpha, eps):
    w, tau = gauss_sum.gaussian_sum(mu, alpha, eps)
    assert np.all(w > 0) and np.all(np.diff(tau) > 0)
    rng = np.random.default_rng(5)
    delta, R = eps / 10, math.sqrt(3)
    r = np.exp(rng.uniform(math.log(delta), math.log(R), 20000))
    approx = np.exp(-np.outer(r * r, tau)) @ w
    env = kernel_ref(0.0, alpha, r)
    assert np.max(np.abs(kernel_ref(mu, alpha, r) - approx) / env) <= eps


def test_fig3_term_count():
    # Fig. 3: about 300 terms (299) for eps = 1e-10 over roughly 15 decades of r
    w, tau = gauss_sum.gaussian_sum(0.0, 1.0, 1e-10, delta=math.sqrt(3) * 1e-15)
    assert 250 <= len(w) <= 350


def test_term_count_grows_like_log():
    # Proposition trapez: M = O(log 1/delta) at fixed eps
    m1 = len(gauss_sum.gaussian_sum(0.0, 1.0, 1e-6, delta=1e-4)[0])
    m2 = len(gauss_sum.gaussian_sum(0.0, 1.0, 1e-6, delta=1e-8)[0])
    m3 = len(gauss_sum.gaussian_sum(0.0, 1.0, 1e-6, delta=1e-12)[0])
    assert m1 < m2 < m3 and abs((m3 - m2) - (m2 - m1)) <= 4


def test_rejects_bad_arguments():
    for args in [(0.0, 0.0, 1e-6), (0.0, 1.5, 1e-6), (0.0, 1.0, 0.0), (-1.0, 1.0, 1e-6)]:
        with pytest.raises(ValueError):
            gauss_sum.gaussian_sum(*args)


@pytest.mark.parametrize("mu,alpha", [(0.7, 0.75), (1.5, 1.25), (0.0, 0.75), (1.5, 1.0)])
def test_kernel_matches_fourier_definition(mu, alpha):
    """K_{mu,alpha} is the Green's function of (-Lap + mu^2)^alpha in R^3 (Sec. 3):
    its radial Fourier inversion (1 / (2 pi^2 r)) int_0^inf xi sin(xi r) (xi^2 +
    mu^2)^(-alpha) d xi, evaluated by quadrature, pins the oracle's Bessel form and
    the normalisation C_alpha without using either."""
    from scipy import integrate
    f = lambda x: x * (x * x + mu * mu) ** (-alpha)
    for r in (0.05, 0.3, 1.2):
        head, _ = integrate.quad(lambda x: f(x) * math.sin(x * r), 0.0, 1.0, limit=200)
        tail, _ = integrate.quad(f, 1.0, np.inf, weight="sin", wvar=r, limlst=200)
        ref = (head + tail) / (2.0 * math.pi ** 2 * r)
        assert abs(float(gauss_sum.kernel(mu, alpha, r)) - ref) <= 1e-9 * abs(ref)
