"""GPU parity of the learned schedule (mra_mlp_*, mra_screen_data and the
pair / learned screens of mra_apply_ns) against the oracle.

* the network's forward pass, loss, gradients and Adam step against
  oracle/mlp.py on seeded parameters and inputs (FP16 weights and
  activations on both sides; the GPU accumulates in FP32);
* the per-box inputs and exact-screen targets against oracle screen_data;
* the exact per-pair screen against the oracle's pair_screen apply;
* the learned screen: with a network that predicts "empty" everywhere the
  judge restores exactly the exact screen's ranges; with one that predicts
  "everything" the static schedule comes back; a trained network keeps the
  result within the 10 eps gate and applies fewer items than the static
  screen (the gain), every miss counted.
"""
import numpy as np
import pytest

from oracle import apply as OA, mlp as OM, operator as OO, tree as OT
from paper_0706_0747_gb300 import workloads as W
from tests.helpers import arrays_to_dict, oracle_density, oracle_to_arrays, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

N_IN = 16


def seeded_params(seed=7, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for shp in OM.param_shapes(N_IN):
        if len(shp) == 2:
            out.append(rng.normal(0.0, scale * np.sqrt(2.0 / shp[1]), shp))
        else:
            out.append(rng.normal(0.0, 0.1, shp))
    return OM.flatten(out).astype(np.float32)


def seeded_batch(n=301, seed=9):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, (n, N_IN)).astype(np.float32)
    t = np.zeros((n, 12), dtype=np.float32)
    for S in range(4):
        E = (rng.random(n) < 0.3).astype(np.float32)
        lo = rng.random(n).astype(np.float32) * 0.5
        t[:, 3 * S] = E
        t[:, 3 * S + 1] = (1 - E) * lo
        t[:, 3 * S + 2] = (1 - E) * (lo + 0.3)
    return x, t


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_forward_matches_oracle():
    theta = seeded_params()
    x, _ = seeded_batch()
    net = mra.mlp_create(params=theta)
    y = torch.empty((x.shape[0], 12), dtype=torch.float32, device="cuda")
    net.forward(dev(x), y)
    torch.cuda.synchronize()
    ref, _ = OM.forward(OM.unflatten(theta.astype(np.float64), N_IN), x.astype(np.float64))
    got = y.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max()
    assert np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()) <= 1e-4


def test_loss_and_gradient_match_oracle():
    theta = seeded_params()
    x, t = seeded_batch()
    net = mra.mlp_create(params=theta)
    L, g = net.loss_grad(dev(x), dev(t))
    L_o, g_o = OM.loss_grad(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64), N_IN)
    assert abs(L - L_o) <= 1e-5 * abs(L_o)
    o = 0
    for shp in OM.param_shapes(N_IN):
        size = int(np.prod(shp))
        a, b = g[o:o + size], g_o[o:o + size]
        assert np.abs(a - b).max() <= 2e-3 * np.abs(b).max() + 1e-7, shp
        o += size


def test_adam_step_matches_oracle():
    theta = seeded_params()
    x, t = seeded_batch()
    net = mra.mlp_create(params=theta)
    lr = 1e-3
    net.train_step(dev(x), dev(t), lr)
    got = net.get_params()
    _, g_o = OM.loss_grad(theta.astype(np.float64), x.astype(np.float64), t.astype(np.float64), N_IN)
    ref, _, _ = OM.adam_step(theta.astype(np.float64), np.zeros_like(g_o), np.zeros_like(g_o), g_o, 1, lr)
    # the first step moves each weight by about lr sign(g); tiny gradients are
    # sensitive to the accumulation order, so compare with a fraction of lr
    assert np.abs(got - ref).max() <= 0.05 * lr
    assert np.mean(np.abs(got - ref) <= 1e-3 * lr) > 0.99


DENS = OT.Density([30.0, 12.0, 8.0], [70.0, 150.0, 900.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47],
                                                          [0.3, 0.66, 0.58]])


@pytest.fixture(scope="module")
def small():
    k, eps, J = 6, 1e-5, 4
    tree, _ = OT.build_tree(DENS, k, eps, J, init_level=1)
    OT.compress(tree, k)
    op_o = OO.Operator(0.0, 1.0, eps, k, J)
    op_g = mra.make_operator(0.0, 1.0, eps, k, J)
    c, l, b = oracle_to_arrays(tree, k)
    return k, eps, tree, op_o, op_g, (c, l, b)


def gpu_tree(arrs, k):
    c, l, b = arrs
    t = mra.tree_import(k, c, l, b)
    mra.compress(t)
    return t


def test_screen_data_matches_oracle(small):
    k, eps, tree, op_o, op_g, arrs = small
    tg = gpu_tree(arrs, k)
    X, Y = mra.screen_data(op_g, tg)
    keys, Xo, Yo = OA.screen_data(op_o, tree)
    c = tg.export()[0]
    order = {tuple(int(v) for v in cc): i for i, cc in enumerate(c)}
    idx = np.array([order[key] for key in keys])
    Xg, Yg = X.cpu().numpy()[idx], Y.cpu().numpy()[idx]
    assert np.abs(Xg - Xo).max() <= 2e-6
    same = np.all(np.abs(Yg - Yo) <= 1e-6, axis=1)
    # decisions are FP64 on both sides; allow a handful of boxes within
    # rounding of the threshold, each off by at most one term
    assert same.mean() >= 0.995
    assert np.abs(Yg - Yo).max() <= 1.0 / (op_o.M - 1) + 1e-6


def test_pair_screen_matches_oracle(small):
    k, eps, tree, op_o, op_g, arrs = small
    tg = gpu_tree(arrs, k)
    g, st = mra.apply_ns(op_g, tg, precision="fp64", screen="pair")
    st_o = {}
    ref = OA.apply_ns(op_o, tree, stats=st_o, pair_screen=True)
    st_s = {}
    OA.apply_ns(op_o, tree, stats=st_s)
    assert abs(st["n_items"] - st_o["n_items"]) <= max(2, st_o["n_items"] // 100000)
    assert st["n_items"] < st_s["n_items"]
    c, _, bl, _ = g.export()
    assert rel_l2(arrays_to_dict(c, bl), ref) <= 1e-10


def constant_net(empty_logit, lo=0.0, hi=1.0):
    """A network whose output ignores its input: every weight 0, and the
    output bias per class [empty_logit, lo, hi]."""
    theta = np.zeros(sum(int(np.prod(s)) for s in OM.param_shapes(N_IN)), dtype=np.float32)
    theta[-12:] = np.tile([empty_logit, lo, hi], 4)
    return mra.mlp_create(params=theta)


def test_learned_screen_judge_restores_exact_ranges(small):
    k, eps, tree, op_o, op_g, arrs = small
    tg = gpu_tree(arrs, k)
    gp, sp = mra.apply_ns(op_g, tg, precision="fp64", screen="pair")
    # "every class empty": every passing item is a miss and is restored
    ge, se = mra.apply_ns(op_g, tg, precision="fp64", screen="learned", schedule=constant_net(10.0), margin=0)
    assert se["n_items"] == sp["n_items"]
    assert se["n_misses"] > 0
    assert np.array_equal(ge.export()[2], gp.export()[2])
    # "every term": the static schedule comes back, with no miss
    gs, ss = mra.apply_ns(op_g, tg, precision="fp64")
    ga, sa = mra.apply_ns(op_g, tg, precision="fp64", screen="learned", schedule=constant_net(-10.0), margin=0)
    assert sa["n_items"] == ss["n_items"] and sa["n_misses"] == 0
    assert np.array_equal(ga.export()[2], gs.export()[2])


def train_small(op_g, dens_list, k, eps, J, steps=300, seed=1):
    xs, ys = [], []
    for d in dens_list:
        t, _ = mra.build_tree(d, k, eps, J, init_level=1)
        mra.compress(t)
        X, Y = mra.screen_data(op_g, t)
        xs.append(X)
        ys.append(Y)
    X = torch.cat(xs)
    Y = torch.cat(ys)
    net = mra.mlp_create(seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    for s in range(steps):
        idx = torch.randint(0, X.shape[0], (1024,), device="cuda", generator=gen)
        net.train_step(X[idx].contiguous(), Y[idx].contiguous(), 2e-3)
    loss0 = net.loss_grad(X, Y)[0]
    return net, loss0


def test_trained_network_gain_and_gate(small):
    """Trained on seeded densities of the learned-schedule family, the learned
    screen applies fewer items than the static screen on a held-out density,
    stays within the 10 eps gate against the oracle, and counts its misses."""
    k, eps, _, op_o, op_g, _ = small
    dens = [d for mu, d in W.schedule_set(12, 0, k=k)]
    net, loss = train_small(op_g, dens, k, eps, 4)
    assert np.isfinite(loss)
    held = W.schedule_set(1, 100, k=k)[0][1]
    t_o, _ = OT.build_tree(oracle_density(held), k, eps, 3, init_level=1)
    OT.compress(t_o, k)
    tg = gpu_tree(oracle_to_arrays(t_o, k), k)
    gs, ss = mra.apply_ns(op_g, tg, precision="fp64")
    gl, sl = mra.apply_ns(op_g, tg, precision="fp64", screen="learned", schedule=net)
    gp, sp = mra.apply_ns(op_g, tg, precision="fp64", screen="pair")
    assert sp["n_items"] <= sl["n_items"] < ss["n_items"]
    assert sl["n_misses"] >= 0
    ref = OA.apply_ns(op_o, t_o)
    c, _, bl, _ = gl.export()
    assert rel_l2(arrays_to_dict(c, bl), ref) <= 10 * eps
    # the tensor-core path takes the same schedule
    gt, st = mra.apply_ns(op_g, tg, precision="tc", screen="learned", schedule=net)
    assert st["n_items"] == sl["n_items"]
    c, _, bl, _ = gt.export()
    assert rel_l2(arrays_to_dict(c, bl), ref) <= 10 * eps
