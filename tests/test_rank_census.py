"""The rank census behind leaving a rank-structured apply out (tests/census_ranks.py):
its per-item bound is valid, and on the 3-D Poisson k = 4 workload only a few per cent
of the static screen's items could use rank-one blocks even at tolerances far looser
than the screen's."""
import numpy as np

from oracle import operator as O
from tests.census_ranks import census


def test_rank_one_bound_holds():
    """||F1 x F2 x F3 - R1 x R2 x R3||_2 <= (sum_d s2/s1) s1(F1) s1(F2) s1(F3) with R_d
    the best rank-one approximations (spectral norms; the bound the census uses)."""
    op = O.Operator(0.0, 1.0, 1e-4, 4, 3)
    rng = np.random.default_rng(3)
    for _ in range(20):
        j, m = int(rng.integers(1, 4)), int(rng.integers(0, op.M))
        t = rng.integers(-3, 4, 3)
        Fs = [op.F[j, m, int(td) + 3] for td in t]
        Rs, s1, ratio = [], 1.0, 0.0
        for F in Fs:
            U, S, Vt = np.linalg.svd(F)
            Rs.append(S[0] * np.outer(U[:, 0], Vt[0]))
            s1 *= S[0]
            ratio += S[1] / S[0] if S[0] > 0 else 0.0  # a zero block (a far, narrow term)
        A = np.kron(np.kron(Fs[0], Fs[1]), Fs[2])
        B = np.kron(np.kron(Rs[0], Rs[1]), Rs[2])
        assert np.linalg.norm(A - B, 2) <= ratio * s1 * (1 + 1e-12) + 1e-300


def test_few_items_have_rank_one_blocks():
    cfg, op, total, below = census("poisson_small")
    assert total == 589430
    assert below[1e-4] / total < 0.05 and below[1e-6] / total < 0.01 and below[1e-8] / total < 1e-4
