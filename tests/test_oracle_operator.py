"""Pins for oracle/operator.py (eq. KernelFactor, eq. BlockNorms,
eq. NormEstimateUsing1DBlocks, Proposition 1)."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import operator as O
from tests.closed_forms import gl, legendre_scaled


@pytest.fixture(scope="module")
def op():
    return O.Operator(0.0, 1.0, 1e-6, 6, 4)


def f00_closed(j, tau, l):
    """2^{-j} int_{-1}^{1} exp(-c (x+l)^2) (1-|x|) dx, c = tau/4^j, via erf."""
    c = tau / 4.0 ** j
    sc = math.sqrt(c)

    def I0(lo, hi):  # int exp(-c(x+l)^2)
        a, b = sc * (lo + l), sc * (hi + l)
        if a >= 0:
            d = special.erfc(a) - special.erfc(b)
        elif b <= 0:
            d = special.erfc(-b) - special.erfc(-a)
        else:
            d = special.erf(b) - special.erf(a)
        return math.sqrt(math.pi) / (2 * sc) * d

    def I1(lo, hi):  # int x exp(-c(x+l)^2) = int (u - l) e^{-c u^2}
        ua, ub = lo + l, hi + l
        return (math.exp(-c * ua * ua) - math.exp(-c * ub * ub)) / (2 * c) - l * I0(lo, hi)

    val = I0(-1, 0) + I1(-1, 0) + I0(0, 1) - I1(0, 1)
    return val / 2.0 ** j


def test_f00_closed_form(op):
    for j in range(op.max_level + 1):
        for m in range(0, op.M, 7):
            for l in range(-3, 4):
                ref = f00_closed(j, op.tau[m], l)
                # the erf form loses ~1e-16/c to cancellation when c = tau/4^j is tiny
                c = op.tau[m] / 4.0 ** j
                tol = (1e-13 + 1e-15 / c) / 2 ** j
                assert abs(op.F[j, m, l + 3, 0, 0] - ref) <= tol


def test_symmetries_from_proposition1(op):
    k = op.k
    sgn = (-1.0) ** np.add.outer(np.arange(k), np.arange(k))
    F = op.F
    # Phi_ii' = (-1)^{i+i'} Phi_i'i  =>  F^l_ii' = (-1)^{i+i'} F^l_i'i
    assert np.allclose(F, sgn * F.transpose(0, 1, 2, 4, 3), atol=1e-15, rtol=1e-12)
    # Phi(-x) = (-1)^{i+i'} Phi(x)    =>  F^{-l} = (-1)^{i+i'} F^{l}
    assert np.allclose(F[:, :, ::-1], sgn * F, atol=1e-15, rtol=1e-12)


def test_wide_gaussian_limit(op):
    # tau -> 0: F -> 2^{-j} int Phi_ii' = 2^{-j} delta_i0 delta_i'0 (vanishing moments)
    pe = O._PhiEval(op.k)
    for j in range(3):
        Fb = O.f_block(pe, j, 1e-12, 1)
        ref = np.zeros((op.k, op.k))
        ref[0, 0] = 2.0 ** -j
        assert np.allclose(Fb, ref, atol=1e-11)


def test_narrow_gaussian_limit(op):
    # c -> inf: F^{j;m,0} -> 2^{-j} sqrt(pi/c) Phi(0) = sqrt(pi/tau) I; next term O(1/c)
    pe = O._PhiEval(op.k)
    tau = 1e14
    for j in range(3):
        Fb = O.f_block(pe, j, tau, 0)
        c = tau / 4.0 ** j
        assert np.allclose(Fb, math.sqrt(math.pi / tau) * np.eye(op.k), atol=200.0 / c / 2 ** j)


def galerkin_direct(k, j, tau, l, panels=48, q=12):
    """<phi^j_{i,a}, exp(-tau (x-y)^2) phi^j_{i',b}>, l = a - b, by a tensor GL
    rule over [0,1]^2 in the box variables (no cross-correlations involved)."""
    g, w = gl(q)
    u = np.concatenate([(p + g) / panels for p in range(panels)])
    wu = np.concatenate([w / panels for _ in range(panels)])
    P = legendre_scaled(k, u) * wu
    c = tau / 4.0 ** j
    Kmat = np.exp(-c * (u[:, None] - u[None, :] + l) ** 2)
    return P @ Kmat @ P.T / 2.0 ** j


def test_direct_galerkin_quadrature(op):
    for (j, m, l) in [(0, 20, 0), (1, 30, 1), (2, 40, -2), (3, 45, 3), (4, 50, -1), (2, 35, 0)]:
        if op.tau[m] / 4.0 ** j > 2e3:
            continue
        ref = galerkin_direct(op.k, j, op.tau[m], l)
        assert np.allclose(op.F[j, m, l + 3], ref, atol=1e-13 * max(1.0, np.abs(ref).max()))


def test_norm_tables(op):
    # N_upF(j, L) = ||F^{j-1;L}||; N_dif vanishes for a constant kernel (tau -> 0)
    assert np.allclose(op.NUF[1:, :, :], op.nF[:-1, :, 2:5])
    pe = O._PhiEval(op.k)
    j = 2
    Ff = {l: O.f_block(pe, j, 1e-12, l) for l in range(-3, 4)}
    Fc = {l: O.f_block(pe, j - 1, 1e-12, l) for l in range(-1, 2)}
    for L in (-1, 0, 1):
        FF = np.block([[Ff[2 * L], Ff[2 * L - 1]], [Ff[2 * L + 1], Ff[2 * L]]])
        UP = op.U @ Fc[L] @ op.U.T
        assert np.abs(FF - UP).max() < 1e-10


def test_estimate_bounds_true_difference(op):
    """Eq. NormEstimateUsing1DBlocks bounds the Frobenius norm of the 3-D block
    difference F1F2F3 - UP1 UP2 UP3 (assembled by Kronecker products)."""
    j = 2
    for m in range(0, op.M, 9):
        FF, UP = {}, {}
        for L in (-1, 0, 1):
            F = op.F[j, m]
            FF[L] = np.block([[F[2 * L + 3], F[2 * L + 2]], [F[2 * L + 4], F[2 * L + 3]]])
            UP[L] = op.U @ op.F[j - 1, m, L + 3] @ op.U.T
        for Ls in [(0, 0, 0), (1, 0, -1), (1, 1, 1)]:
            A = np.kron(np.kron(FF[Ls[0]], FF[Ls[1]]), FF[Ls[2]])
            B = np.kron(np.kron(UP[Ls[0]], UP[Ls[1]]), UP[Ls[2]])
            est = op.estimate(j, m, tuple(L + 1 for L in Ls))
            assert np.linalg.norm(A - B) <= est * (1 + 1e-12) + 1e-300


def test_coarse_blocks_are_two_scale_projections(op):
    """The level-(j-1) block of translation L equals the 2x2 fine block matrix
    [[F^{2L}, F^{2L-1}], [F^{2L+1}, F^{2L}]] at level j (rows: output child, columns:
    input child) projected by the two-scale filters, D FF D^T with D = [H0 | H1] --
    an identity of the scaling spaces (V_{j-1} inside V_j) that holds for any
    kernel.  The two levels' tables come from separate quadratures, so this pins
    the fine-block layout the norm estimate uses; the transposed layout fails."""
    D = op.U.T
    worst_wrong = 0.0
    for j in range(1, op.max_level + 1):
        for m in range(0, op.M, 5):
            F = op.F[j, m]
            for L in (-1, 0, 1):
                C = op.F[j - 1, m, L + 3]
                FF = np.block([[F[2 * L + 3], F[2 * L + 2]], [F[2 * L + 4], F[2 * L + 3]]])
                # quadrature and rounding errors are relative to the term's blocks (for a
                # narrow Gaussian the off-diagonal blocks are tiny tails of them)
                scale = max(np.abs(op.F[j - 1, m]).max(), np.abs(F).max(), 1e-300)
                assert np.abs(D @ FF @ D.T - C).max() <= 1e-10 * scale
                FT = np.block([[F[2 * L + 3], F[2 * L + 4]], [F[2 * L + 2], F[2 * L + 3]]])
                worst_wrong = max(worst_wrong, np.abs(D @ FT @ D.T - C).max() / scale)
    assert worst_wrong > 1e-4
