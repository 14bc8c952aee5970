"""GPU parity of the batched apply (mra_plan_*): one operator, many trees,
one screen over the forest and one Step-3 launch over all nodes.

* per tree, the batch applies exactly the items of the oracle's Algorithm 3
  on that tree (same eta, same item count) and agrees with it to rounding
  (FP64) or within the 10 eps gate (tensor cores);
* the batch and the single-tree apply give the same blocks (the tensor-core
  kernel treats every node alike, whatever else is in the launch);
* graph replays, rewritten coefficients (the screen is scale-invariant:
  doubling f doubles g exactly), autotuned variants and trees of different
  depths in one batch;
* the sizes of the 256-input batch: per-tree item counts equal the
  single-tree apply's, and two of its trees against the oracle on sampled
  output nodes.
"""
import numpy as np
import pytest

from oracle import apply as OA, operator as OO, tree as OT
from paper_0706_0747_gb300 import workloads as W
from tests.helpers import arrays_to_dict, oracle_density, oracle_to_arrays, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

K, EPS, JMAX = 6, 1e-5, 4


def small_batch(n_rhs=5, seed=4900):
    """Seeded inputs shaped like the multi-RHS workload, shallow enough for
    the oracle: 1-6 Gaussians each, log10 exponent U[1, 3]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_rhs):
        n = int(rng.integers(1, 7))
        out.append(W.unit_mass(10.0 ** rng.uniform(1.0, 3.0, n), rng.uniform(0.15, 0.85, (n, 3))))
    return out


@pytest.fixture(scope="module")
def batch():
    dens = small_batch()
    trees_o = []
    for d in dens:
        t, _ = OT.build_tree(oracle_density(d), K, EPS, JMAX, init_level=1)
        OT.compress(t, K)
        trees_o.append(t)
    # a root-only tree and a uniform level-1 tree make the depths differ
    t, _ = OT.build_tree(oracle_density(dens[0]), K, EPS, 0, uniform_level=0)
    OT.compress(t, K)
    trees_o.append(t)
    t, _ = OT.build_tree(oracle_density(dens[1]), K, EPS, 1, uniform_level=1)
    OT.compress(t, K)
    trees_o.append(t)
    op_o = OO.Operator(0.0, 1.0, EPS, K, JMAX)
    op_g = mra.make_operator(0.0, 1.0, EPS, K, JMAX)
    ref = []
    for t in trees_o:
        st = {}
        g = OA.apply_ns(op_o, t, stats=st)
        ref.append((g, st))
    return trees_o, op_o, op_g, ref


def gpu_trees(trees_o):
    out = []
    for t in trees_o:
        # the oracle's tree after compress carries s on every node; import
        # its leaves and compress on the GPU
        c, l, b = oracle_to_arrays(t, K)
        tg = mra.tree_import(K, c, l, b)
        mra.compress(tg)
        out.append(tg)
    return out


def outputs(plan, n):
    res = []
    for b in range(n):
        c, _, bl, _ = plan.output(b).export()
        res.append(arrays_to_dict(c, bl))
    return res


@pytest.mark.parametrize("precision,use_graph", [("fp64", False), ("fp64", True), ("tc", True), ("fp32", False),
                                                 ("tc_ladder", True)])
def test_batch_matches_oracle_per_tree(batch, precision, use_graph):
    trees_o, op_o, op_g, ref = batch
    tg = gpu_trees(trees_o)
    plan = mra.plan_create(op_g, tg, precision=precision, use_graph=use_graph)
    plan.execute()
    info = plan.info()
    outs = outputs(plan, len(tg))
    tol = 1e-12 if precision == "fp64" else 10 * EPS
    total = 0
    for b, (g_o, st_o) in enumerate(ref):
        ts = plan.tree_stats(b)
        assert abs(ts["eta"] - st_o["eta"]) <= 1e-13 * st_o["eta"]
        assert ts["n_items"] == st_o["n_items"]
        assert ts["n_pairs"] == st_o["n_pairs"]
        total += st_o["n_items"]
        assert rel_l2(outs[b], g_o) <= tol, (b, rel_l2(outs[b], g_o))
    assert info["n_items"] == total
    assert info["n_ghosts"] == sum(st["n_refined"] for _, st in ref)
    assert info["graph"] == int(use_graph)
    if precision == "tc_ladder":
        assert 0 < info["n_items_lowp"] <= info["n_items"]


def test_batch_equals_single_tree_tc(batch):
    trees_o, _, op_g, _ = batch
    tg = gpu_trees(trees_o)
    plan = mra.plan_create(op_g, tg, precision="tc")
    plan.execute()
    outs = outputs(plan, len(tg))
    for b, t in enumerate(tg):
        g, st = mra.apply_ns(op_g, t, precision="tc")
        c, _, bl, _ = g.export()
        single = arrays_to_dict(c, bl)
        assert plan.tree_stats(b)["n_items"] == st["n_items"]
        assert rel_l2(outs[b], single) <= 1e-14


def test_graph_replay_and_rewritten_blocks(batch):
    trees_o, _, op_g, _ = batch
    tg = gpu_trees(trees_o)
    plan = mra.plan_create(op_g, tg, precision="tc", use_graph=True)
    plan.execute()
    first = outputs(plan, len(tg))
    launches = mra.kernel_launches()
    plan.execute()
    info = plan.info()
    assert info["graph"] == 1 and info["graph_kernels"] >= 4
    assert mra.kernel_launches() - launches == info["graph_kernels"]
    again = outputs(plan, len(tg))
    for a, b in zip(first, again):
        assert all(np.array_equal(a[key], b[key]) for key in a)
    # scale every tree's coefficients by 16: eta = eps sigma / ||f|| is
    # unchanged, so the plan's screen still holds; block scales are powers of
    # 16, so the FP16 operands are the same bits and every output is exactly
    # 16 times the first (blocks below the scale clamp aside)
    for t in tg:
        s_ptr, _ = t.device_arrays()
        n, k3 = t.n, K ** 3
        buf = torch.empty(n * k3, dtype=torch.float64, device="cuda")
        c, l, bl, _ = t.export()
        buf.copy_(torch.from_numpy(16.0 * bl.reshape(-1)))
        mra.tree_set_blocks(t, buf.data_ptr())
        torch.cuda.synchronize()
    plan.execute()
    scaled = outputs(plan, len(tg))
    for a, b in zip(first, scaled):
        assert rel_l2(b, {key: 16.0 * v for key, v in a.items()}) <= 1e-13


def test_autotune_variants_agree(batch):
    trees_o, _, op_g, ref = batch
    tg = gpu_trees(trees_o)
    plan = mra.plan_create(op_g, tg, precision="tc")
    info = plan.autotune(reps=2)
    assert info["tuned"] == 1
    assert all(ms > 0.0 for ms in info["ms_variant"])
    assert info["terms_per_chunk"] in (4, 8) and info["ctas_per_sm"] in (1, 2, 3, 4)
    by_variant = {}
    for v in range(10):
        mc, ctas = [(8, 3), (8, 2), (4, 3), (4, 2), (4, 4)][v % 5]
        plan.set_variant(terms_per_chunk=mc, ctas_per_sm=ctas, heavy_first=v >= 5)
        plan.execute()
        outs = outputs(plan, len(tg))
        by_variant[(mc, ctas, v >= 5)] = outs
        assert plan.info()["n_items"] == sum(st["n_items"] for _, st in ref)
        for b, (g_o, _) in enumerate(ref):
            assert rel_l2(outs[b], g_o) <= 10 * EPS
    # the wide-MMA kernel (8 terms, two CTAs per SM) sums the same split products in
    # another order (and adds the lo*lo products of stages II and III): the same blocks
    # to FP32 rounding
    for a, b in zip(by_variant[(8, 2, False)], by_variant[(8, 3, False)]):
        assert rel_l2(a, b) <= 1e-6


def test_plan_rejects_bad_inputs(batch):
    trees_o, _, op_g, _ = batch
    tg = gpu_trees(trees_o[:2])
    with pytest.raises(mra.MraError) as e:
        mra.plan_create(op_g, [], precision="fp64")
    assert e.value.code == mra.EINVAL
    c, l, b = oracle_to_arrays(trees_o[0], K)
    raw = mra.tree_import(K, c, l, b)           # not compressed
    with pytest.raises(mra.MraError) as e:
        mra.plan_create(op_g, [tg[0], raw], precision="fp64")
    assert e.value.code == mra.ESTATE
    op4 = mra.make_operator(0.0, 1.0, EPS, 4, JMAX)
    with pytest.raises(mra.MraError) as e:
        mra.plan_create(op4, tg, precision="fp64")
    assert e.value.code == mra.EINVAL
    plan = mra.plan_create(op_g, tg, precision="fp64")
    with pytest.raises(mra.MraError) as e:
        plan.output(5)
    assert e.value.code == mra.EINVAL


# ------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def rhs256():
    cfg, dens = W.batched_rhs()
    trees = [mra.build_tree(d, cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)[0] for d in dens]
    for t in trees:
        mra.compress(t)
    op_g = mra.make_operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    return cfg, dens, trees, op_g


def test_rhs256_items_equal_single_tree(rhs256):
    cfg, dens, trees, op_g = rhs256
    plan = mra.plan_create(op_g, trees, precision="tc")
    plan.execute()
    info = plan.info()
    total = 0
    for b, t in enumerate(trees):
        _, st = mra.apply_ns(op_g, t, precision="fp64")
        ts = plan.tree_stats(b)
        assert ts["n_items"] == st["n_items"], b
        assert abs(ts["eta"] - st["eta"]) <= 1e-12 * st["eta"]
        total += st["n_items"]
    assert info["n_items"] == total
    assert info["n_nodes"] == sum(t.n for t in trees)


def sample_nodes(keys, per_level=4, seed=41):
    rng = np.random.default_rng(seed)
    out = []
    for j in sorted({key[0] for key in keys}):
        lv = sorted(key for key in keys if key[0] == j)
        pick = rng.choice(len(lv), size=min(per_level, len(lv)), replace=False)
        out += [lv[i] for i in sorted(pick)]
    return out


def test_rhs256_sampled_against_oracle(rhs256):
    cfg, dens, trees, op_g = rhs256
    plan = mra.plan_create(op_g, trees, precision="tc")
    plan.execute()
    op_o = OO.Operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    # the two inputs with the fewest Gaussians keep the oracle's tree small
    pick = sorted(range(len(dens)), key=lambda b: (dens[b].n, b))[:2]
    for b in pick:
        t_o, _ = OT.build_tree(oracle_density(dens[b]), cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
        c, _, bl, _ = plan.output(b).export()
        got = arrays_to_dict(c, bl)
        assert set(got) == set(t_o)
        OT.compress(t_o, cfg.k)
        nodes = sample_nodes(list(t_o))
        st_o = {}
        ref = OA.apply_ns(op_o, t_o, stats=st_o, nodes=nodes)
        assert abs(plan.tree_stats(b)["eta"] - st_o["eta"]) <= 1e-12 * st_o["eta"]
        assert rel_l2({key: got[key] for key in nodes}, ref) <= 10 * cfg.eps


@pytest.mark.parametrize("precision", ["fp64", "tc"])
def test_batch_pair_screen_matches_oracle(batch, precision):
    """The exact per-pair screen in a batch: per tree the items of the oracle's
    pair_screen apply and its result (rounding for FP64, the gate for tc)."""
    trees_o, op_o, op_g, _ = batch
    tg = gpu_trees(trees_o)
    plan = mra.plan_create(op_g, tg, precision=precision, screen="pair")
    plan.execute()
    outs = outputs(plan, len(tg))
    for b, t in enumerate(trees_o):
        st_o = {}
        ref = OA.apply_ns(op_o, t, stats=st_o, pair_screen=True)
        got = plan.tree_stats(b)["n_items"]
        assert abs(got - st_o["n_items"]) <= max(2, st_o["n_items"] // 100000)
        assert rel_l2(outs[b], ref) <= (1e-10 if precision == "fp64" else 10 * EPS)


def _net(theta_tail=None, seed=None):
    """A schedule network: constant outputs (zero weights, the given output
    biases) or seeded random weights."""
    from oracle import mlp as OM
    n = sum(int(np.prod(s)) for s in OM.param_shapes(16))
    if seed is not None:
        rng = np.random.default_rng(seed)
        theta = rng.normal(0.0, 0.05, n).astype(np.float32)
        return mra.mlp_create(params=theta)
    theta = np.zeros(n, dtype=np.float32)
    theta[-12:] = np.tile(theta_tail, 4)
    return mra.mlp_create(params=theta)


def test_batch_learned_screen(batch):
    """The learned screen inside the batched plan (learned + tensor cores +
    one persistent graph-captured launch): per tree the same items, misses
    and blocks as the single-tree learned apply with the same network; a
    network predicting "empty" everywhere gives back the exact per-pair
    screen (every passing item a miss, restored), one predicting every term
    the static schedule."""
    trees_o, op_o, op_g, ref = batch
    tg = gpu_trees(trees_o)
    for net, margin in ((_net(seed=11), 2), (_net(seed=12), 0)):
        plan = mra.plan_create(op_g, tg, precision="tc", screen="learned", schedule=net, margin=margin)
        plan.execute()
        info = plan.info()
        assert info["screen_mode"] == mra.SCREEN["learned"]
        outs = outputs(plan, len(tg))
        misses = 0
        for b, t in enumerate(tg):
            g, st = mra.apply_ns(op_g, t, precision="tc", screen="learned", schedule=net, margin=margin)
            c, _, bl, _ = g.export()
            assert plan.tree_stats(b)["n_items"] == st["n_items"]
            misses += st["n_misses"]
            assert rel_l2(outs[b], arrays_to_dict(c, bl)) <= 1e-14
            assert rel_l2(outs[b], ref[b][0]) <= 10 * EPS
        assert info["n_misses"] == misses
    empty = mra.plan_create(op_g, tg, precision="tc", screen="learned", schedule=_net([10.0, 0.0, 0.0]), margin=0)
    pair = mra.plan_create(op_g, tg, precision="tc", screen="pair")
    empty.execute()
    pair.execute()
    assert empty.info()["n_items"] == pair.info()["n_items"] and empty.info()["n_misses"] > 0
    for a, b in zip(outputs(empty, len(tg)), outputs(pair, len(tg))):
        assert rel_l2(a, b) == 0.0
    full = mra.plan_create(op_g, tg, precision="tc", screen="learned", schedule=_net([-10.0, 0.0, 1.0]), margin=0)
    full.execute()
    assert full.info()["n_items"] == sum(st["n_items"] for _, st in ref) and full.info()["n_misses"] == 0
    with pytest.raises(mra.MraError):
        mra.plan_create(op_g, tg, precision="tc", screen="learned")
