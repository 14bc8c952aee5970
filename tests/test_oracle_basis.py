"""Pins for oracle/basis.py (paper Appendix: scaling functions, multiwavelets,
two-scale relations, Proposition 1)."""
import numpy as np
import pytest
from scipy import special

from oracle import basis
from tests.closed_forms import legendre_scaled


@pytest.mark.parametrize("n", [1, 3, 8, 12])
def test_gl_exact_for_monomials(n):
    x, w = basis.gl01(n)
    for p in range(2 * n):
        assert abs((w * x ** p).sum() - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("k", [2, 4, 6, 8, 10])
def test_phi_orthonormal_and_matches_recurrence(k):
    x, w = basis.gl01(k + 2)
    P = basis.phi(k, x)
    assert np.allclose((P * w) @ P.T, np.eye(k), atol=1e-13)
    assert np.allclose(P, legendre_scaled(k, x), atol=1e-12)


@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_filter_matrix_orthogonal(k):
    W = basis.filter_matrix(k)
    assert np.allclose(W @ W.T, np.eye(2 * k), atol=1e-13)


@pytest.mark.parametrize("k", [3, 6, 8])
def test_two_scale_relation_pointwise(k):
    H0, H1 = basis.two_scale_H(k)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, 50)
    lhs = basis.phi(k, x)
    rhs = np.sqrt(2) * (H0 @ basis.phi(k, 2 * x) + H1 @ basis.phi(k, 2 * x - 1))
    assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("k", [2, 5, 8])
def test_wavelets_vanishing_moments_and_orthonormal(k):
    G0, G1 = basis.two_scale_G(k)
    g, w = basis.gl01(2 * k + 2)
    # psi_i(x) = sqrt 2 sum (g0 phi(2x) + g1 phi(2x-1)); integrate each half
    xl, xr = g / 2, (g + 1) / 2
    psil = np.sqrt(2) * G0 @ basis.phi(k, 2 * xl)
    psir = np.sqrt(2) * G1 @ basis.phi(k, 2 * xr - 1)
    for q in range(k):
        mom = (psil * xl ** q * w / 2).sum(axis=1) + (psir * xr ** q * w / 2).sum(axis=1)
        assert np.abs(mom).max() < 1e-13
    gram = (psil * w / 2) @ psil.T + (psir * w / 2) @ psir.T
    assert np.allclose(gram, np.eye(k), atol=1e-13)


def gegenbauer_mhalf(n, x):
    """C_n^{(-1/2)}(x): C_0 = 1, C_1 = -x, C_n = (P_{n-2} - P_n)/(2n-1), n >= 2."""
    if n == 0:
        return np.ones_like(x)
    if n == 1:
        return -x
    return (special.eval_legendre(n - 2, x) - special.eval_legendre(n, x)) / (2 * n - 1)


@pytest.mark.parametrize("k", [3, 6, 8])
def test_cross_correlation_proposition1(k):
    x = np.linspace(0.0, 1.0, 41)
    Pp = basis.cross_corr(k, x)
    Pm = basis.cross_corr(k, -x)
    sgn = (-1.0) ** np.add.outer(np.arange(k), np.arange(k))
    # item 1: transposition
    assert np.allclose(Pp, sgn[:, :, None] * Pp.transpose(1, 0, 2), atol=1e-13)
    # item 2: Phi-(-x) = (-1)^{i+i'} Phi+(x)
    assert np.allclose(Pm[:, :, 1:], (sgn[:, :, None] * Pp)[:, :, 1:], atol=1e-13)
    # item 3: values at zero
    assert np.allclose(basis.cross_corr(k, [0.0])[:, :, 0], np.eye(k), atol=1e-13)
    # item 4: bounded by one
    assert np.abs(Pp).max() <= 1.0 + 1e-13
    # item 5: Gegenbauer connection
    u = 2 * x - 1
    assert np.allclose(Pp[0, 0], 0.5 * gegenbauer_mhalf(1, u) + 0.5, atol=1e-13)
    for l in range(1, k):
        assert np.allclose(Pp[l, 0], 0.5 * np.sqrt(2 * l + 1) * gegenbauer_mhalf(l + 1, u), atol=1e-12)
    # Phi_00 = 1 - |x|
    assert np.allclose(Pp[0, 0], 1 - x, atol=1e-14) and np.allclose(Pm[0, 0], 1 - x, atol=1e-14)


@pytest.mark.parametrize("k", [3, 6])
def test_cross_correlation_vanishing_moments(k):
    g, w = basis.gl01(2 * k + 2)
    for i in range(k):
        for ip in range(k):
            vp = basis.cross_corr(k, g)[i, ip]
            vm = basis.cross_corr(k, g - 1)[i, ip]
            for q in range(max(1, i + ip)):
                mom = (w * g ** q * vp).sum() + (w * (g - 1) ** q * vm).sum()
                expect = 1.0 if (i == 0 and ip == 0 and q == 0) else 0.0
                assert abs(mom - expect) < 1e-13
