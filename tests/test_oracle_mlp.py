"""Pins of the learned schedule's oracle (oracle/mlp.py) and of the exact
per-pair screen that judges it (oracle/apply.py, pair_screen / screen_data).

Each pin is fixed by something other than the code under test: central
finite differences, a closed form, a hand-derived case, or an inequality
that any correct norm bound must satisfy."""
import math

import numpy as np
import pytest

from oracle import apply as OA, mlp as OM, operator as OO, tree as OT

DENS = OT.Density([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47]])


def rand_problem(n_in=5, hidden=6, n=7, seed=3):
    rng = np.random.default_rng(seed)
    shapes = OM.param_shapes(n_in, OM.N_OUT, hidden)
    theta = np.concatenate([rng.normal(0, 0.7, int(np.prod(s))) for s in shapes])
    x = rng.normal(0, 1, (n, n_in))
    tgt = np.zeros((n, 12))
    for S in range(4):
        E = (rng.random(n) < 0.4).astype(float)
        tgt[:, 3 * S] = E
        tgt[:, 3 * S + 1] = (1 - E) * rng.random(n) * 0.5
        tgt[:, 3 * S + 2] = (1 - E) * (0.5 + rng.random(n) * 0.5)
    return theta, x, tgt


def test_gradient_matches_central_differences():
    n_in, hidden = 5, 6
    theta, x, tgt = rand_problem(n_in, hidden)
    L, g = OM.loss_grad(theta, x, tgt, n_in, fp16_storage=False, hidden=hidden)
    h = 1e-6
    fd = np.zeros_like(theta)
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd[i] = (OM.loss_grad(tp, x, tgt, n_in, False, hidden)[0] -
                 OM.loss_grad(tm, x, tgt, n_in, False, hidden)[0]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_zero_network_closed_form():
    n_in = 4
    theta = np.zeros(sum(int(np.prod(s)) for s in OM.param_shapes(n_in)))
    _, x, tgt = rand_problem(n_in=n_in)
    L, g = OM.loss_grad(theta, x, tgt, n_in)
    E, LO, HI = tgt[:, 0::3], tgt[:, 1::3], tgt[:, 2::3]
    L_ref = np.mean(np.sum(math.log(2.0) + (1 - E) * (LO ** 2 + HI ** 2), axis=1))
    assert abs(L - L_ref) <= 1e-14
    gb4 = g[-12:]
    assert np.allclose(gb4[0::3], np.mean(0.5 - E, axis=0), atol=1e-15)
    assert np.allclose(gb4[1::3], np.mean(-2 * (1 - E) * LO, axis=0), atol=1e-15)
    assert np.allclose(gb4[2::3], np.mean(-2 * (1 - E) * HI, axis=0), atol=1e-15)
    # a zero hidden layer blocks every other gradient
    assert np.all(g[:-12] == 0.0)


def test_single_unit_by_hand():
    # hidden = 1, n_in = 1: y = w4 relu(w3 relu(w2 relu(w1 x + b1) + b2) + b3) + b4
    w1, b1, w2, b2, w3, b3 = 2.0, -1.0, 3.0, 0.5, -1.0, 4.0
    w4 = np.arange(1, 13, dtype=float).reshape(12, 1) / 8.0
    b4 = np.zeros(12)
    params = [np.array([[w1]]), np.array([b1]), np.array([[w2]]), np.array([b2]), np.array([[w3]]),
              np.array([b3]), w4, b4]
    y, _ = OM.forward(params, np.array([[1.5]]), fp16_storage=False)
    h1 = max(w1 * 1.5 + b1, 0)          # 2
    h2 = max(w2 * h1 + b2, 0)           # 6.5
    h3 = max(w3 * h2 + b3, 0)           # 0 (negative pre-activation)
    assert h1 == 2.0 and h2 == 6.5 and h3 == 0.0
    assert np.all(y == b4)


def test_fp16_storage_exact_on_representable_values():
    # weights and activations that FP16 holds exactly: the FP16 network is the FP64 one
    n_in, hidden = 3, 4
    rng = np.random.default_rng(5)
    shapes = OM.param_shapes(n_in, OM.N_OUT, hidden)
    theta = np.concatenate([rng.integers(-4, 5, int(np.prod(s))) / 8.0 for s in shapes])
    x = rng.integers(-4, 5, (6, n_in)) / 4.0
    p = OM.unflatten(theta, n_in, OM.N_OUT, hidden)
    y16, _ = OM.forward(p, x, True)
    y64, _ = OM.forward(p, x, False)
    assert np.array_equal(y16, y64)


def test_adam_first_step_is_signed_lr():
    g = np.array([3.0, -0.25, 1e-3, 0.0])
    th, m, v = OM.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    # m_hat = g, v_hat = g^2: the step is -lr g / (|g| + eps)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)


@pytest.fixture(scope="module")
def screened():
    k, eps = 4, 1e-4
    tree, _ = OT.build_tree(DENS, k, eps, 3, init_level=1)
    OT.compress(tree, k)
    op = OO.Operator(0.0, 1.0, eps, k, 3)
    return k, eps, tree, op


def test_pair_screen_error_within_dropped_bounds(screened):
    """Every box's change from the static apply is at most the sum of the
    norm bounds w_m prod N_F ||x_b|| of the items the pair screen dropped (a
    property of the bound itself: ||F1 x F2 x F3 x|| <= prod ||F_d||_F ||x||)."""
    k, eps, tree, op = screened
    st0, st1, st2 = {}, {}, {}
    g0 = OA.apply_ns(op, tree, stats=st0)
    g1 = OA.apply_ns(op, tree, stats=st1, pair_screen=True)
    OA.apply_ns(op, tree, stats=st2, block_screen=True)
    assert st2["n_items"] <= st1["n_items"] <= st0["n_items"]
    assert st1["n_items"] < st0["n_items"]
    # rebuild the dropped items' bounds box by box
    sch = OA.Schedule(op, st0["sigma"], st0["fnorm"], OT.levels(tree))
    eta_blk = op.eps * st0["sigma"] / np.sqrt(len(tree) * 216.0 * op.M)
    inp = OA._Inputs(tree, k)
    for key in tree:
        j, a = key[0], key[1:]
        bound = 0.0
        for t in OA.band(a):
            b = tuple(a[d] - t[d] for d in range(3))
            if min(b) < 0 or max(b) >= 2 ** j:
                continue
            ms = sch.terms(j, t, tree[key].leaf)
            if not ms:
                continue
            xn = float(np.linalg.norm(inp.get(j, b)))
            est = {m: op.w[m] * op.nF[j, m, t[0] + 3] * op.nF[j, m, t[1] + 3] * op.nF[j, m, t[2] + 3] * xn
                   for m in ms}
            keep = [m for m in ms if est[m] > eta_blk]
            kept = [m for m in ms if keep and keep[0] <= m <= keep[-1]]
            bound += sum(est[m] for m in ms if m not in kept)
        assert np.linalg.norm(g1[key] - g0[key]) <= bound * (1 + 1e-12) + 1e-300


def test_screen_data_consistent_with_pair_screen(screened):
    k, eps, tree, op = screened
    keys, X, Y = OA.screen_data(op, tree)
    st = {}
    OA.apply_ns(op, tree, stats=st)
    # pair counts per class add up to the static screen's pairs
    assert int(round(64 * X[:, 11:15].sum())) == st["n_pairs"]
    assert X.shape == (len(tree), 16) and Y.shape == (len(tree), 12)
    E = Y[:, 0::3]
    assert set(np.unique(E)) <= {0.0, 1.0}
    lo, hi = Y[:, 1::3], Y[:, 2::3]
    assert np.all(lo[E == 0] <= hi[E == 0]) and np.all((lo[E == 1] == 0) & (hi[E == 1] == 0))
    # a box with no pair in a class has that class empty
    assert np.all(E[X[:, 11:15] == 0] == 1)
    # the per-class ranges hold every item the pair screen applies
    st1 = {}
    OA.apply_ns(op, tree, stats=st1, pair_screen=True)
    assert st1["n_items"] > 0 and np.any(E == 0)
