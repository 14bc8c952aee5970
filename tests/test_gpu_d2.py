"""GPU parity of the d = 2 variant through the C ABI against oracle/d2.py:
operator tables, Algorithm 1, the redundant tree, Algorithm 3 (with Step 2)
and the assembly / truncation on the oracle-sized case, and sampled output
nodes of every level on the full-size case.

Tolerances: FP64 on both sides, the same decisions (item and pair counts
equal), so blocks agree to rounding (relative L2 <= 1e-12, per block 1e-12 of
its largest entry)."""
import numpy as np
import pytest

from oracle import d2 as D
from paper_0706_0747_gb300 import workloads as W
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

DENS = D.Density2([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52], [0.62, 0.41]])


def spread2(v):
    out = 0
    for b in range(21):
        out |= ((v >> b) & 1) << (2 * b)
    return out


def to_arrays(tree, k):
    keys = sorted(tree.keys(), key=lambda key: (key[0], (spread2(key[1]) << 1) | spread2(key[2])))
    coords = np.array(keys, dtype=np.int32).reshape(-1, 3)
    leaf = np.array([tree[key].leaf for key in keys], dtype=np.int32)
    blocks = np.zeros((len(keys), k, k))
    for i, key in enumerate(keys):
        if tree[key].s is not None:
            blocks[i] = tree[key].s
    return coords, leaf, blocks


def import2(tree, k):
    return mra.tree2_import(k, *to_arrays(tree, k))


def as_dicts(t):
    c, l, b, dn = t.export()
    keys = [tuple(int(v) for v in cc) for cc in c]
    return dict(zip(keys, b)), dict(zip(keys, l.astype(bool))), dict(zip(keys, dn))


def oracle_density(d):
    return D.Density2(d.coef, d.expo, d.centers)


@pytest.mark.parametrize("mu,alpha,eps,k,J", [(0.0, 0.5, 1e-4, 4, 4), (2.0, 0.75, 1e-6, 6, 5),
                                              (0.0, 0.25, 1e-5, 5, 3)])
def test_operator2_tables(mu, alpha, eps, k, J):
    op = mra.make_operator2(mu, alpha, eps, k, J)
    g = op.export()
    o = D.operator(mu, alpha, eps, k, J)
    assert len(g["w"]) == o.M
    assert np.allclose(g["w"], o.w, rtol=1e-13, atol=0)
    assert np.allclose(g["tau"], o.tau, rtol=1e-13, atol=0)
    assert np.abs(g["F"] - o.F).max() <= 2e-14
    assert np.allclose(g["nF"], o.nF, rtol=1e-12, atol=k * 2e-14)
    scale = o.nF.max(axis=2) ** 2
    assert np.all(np.abs(g["est"] - o.est_core) <= 1e-7 * np.abs(o.est_core) + 1e-12 * scale)


def test_build_tree2_matches_algorithm1():
    k, eps = 4, 1e-5
    tg, hit = mra.build_tree2(DENS, k, eps, 6, init_level=1)
    to, hito = D.build_tree(DENS, k, eps, 6, init_level=1)
    assert hit == hito
    blocks, leaf, _ = as_dicts(tg)
    assert set(blocks) == set(to)
    for key, n in to.items():
        assert leaf[key] == n.leaf
        if n.leaf:
            assert np.abs(blocks[key] - n.s).max() <= 1e-12 * max(1.0, np.abs(n.s).max())


def test_build_tree2_depth_cap():
    narrow = D.Density2([1.0], [3e4], [[0.52, 0.47]])
    tg, hit = mra.build_tree2(narrow, 4, 1e-6, 3, init_level=1)
    to, hito = D.build_tree(narrow, 4, 1e-6, 3, init_level=1)
    assert hit and hito and tg.n == len(to)


def test_compress2_matches_oracle():
    k = 5
    to, _ = D.build_tree(DENS, k, 1e-5, 5, init_level=1)
    tg = import2(to, k)
    mra.compress2(tg)
    t = D.copy_tree(to)
    D.compress(t, k)
    blocks, _, dn = as_dicts(tg)
    for key, n in t.items():
        assert np.abs(blocks[key] - n.s).max() <= 1e-13 * max(1.0, np.abs(n.s).max())
        if not n.leaf:
            assert abs(dn[key] - n.dnorm) <= 1e-12 * max(1.0, n.dnorm)


def apply_both(tree_o, k, op_args):
    op_g = mra.make_operator2(*op_args)
    op_o = D.operator(*op_args)
    tg = import2(tree_o, k)
    mra.compress2(tg)
    g, st = mra.apply_ns2(op_g, tg)
    t = D.copy_tree(tree_o)
    D.compress(t, k)
    sto = {}
    ghat = D.apply_ns(op_o, t, stats=sto)
    return g, st, ghat, sto, op_g, op_o, tg


def test_apply2_parity_small_case():
    """Algorithm 3 in d = 2 on the oracle-sized workload: every block of ghat,
    the item and pair counts and eta."""
    cfg, dens = W.poisson2d_small()
    to, _ = D.build_tree(oracle_density(dens), cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    g, st, ghat, sto, *_ = apply_both(to, cfg.k, (cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level))
    blocks, _, _ = as_dicts(g)
    assert st["n_items"] == sto["n_items"] and st["n_pairs"] == sto["n_pairs"]
    assert abs(st["eta"] - sto["eta"]) <= 1e-12 * sto["eta"]
    assert rel_l2(blocks, ghat) <= 1e-12
    assert st["n_ghosts"] > 0


def test_apply2_parity_adaptive_with_refined_inputs():
    """A hand-made adaptive tree whose level-2 inputs must be refined from
    level-1 leaves (Step 2), unscreened terms included by a loose operator."""
    k = 4
    to, _ = D.build_tree(DENS, k, 1e-4, 3, uniform_level=1)
    for key in [(1, 0, 1), (1, 1, 0)]:
        to[key].leaf = False
        to[key].s = None
        for ck in D.children(key):
            to[ck] = D.Node(True, D.project_values(k, 2, DENS(D.grid(D.box_nodes(k, 2, ck[1:])))))
    g, st, ghat, sto, *_ = apply_both(to, k, (0.0, 0.5, 1e-4, k, 3))
    blocks, _, _ = as_dicts(g)
    assert st["n_items"] == sto["n_items"]
    assert rel_l2(blocks, ghat) <= 1e-12


@pytest.mark.parametrize("mu,alpha", [(4.0, 0.75), (0.0, 0.25)])
def test_apply2_parity_other_kernels(mu, alpha):
    """Other members of the d = 2 family: a screened kernel (mu > 0) and a
    weaker singularity (alpha = 1/4), on the oracle-sized tree."""
    cfg, dens = W.poisson2d_small()
    to, _ = D.build_tree(oracle_density(dens), cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    g, st, ghat, sto, *_ = apply_both(to, cfg.k, (mu, alpha, cfg.eps, cfg.k, cfg.max_level))
    blocks, _, _ = as_dicts(g)
    assert st["n_items"] == sto["n_items"] and st["n_pairs"] == sto["n_pairs"]
    assert rel_l2(blocks, ghat) <= 1e-12


def test_reconstruct2_and_truncation_parity():
    cfg, dens = W.poisson2d_small()
    od = oracle_density(dens)
    to, _ = D.build_tree(od, cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    op_args = (cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    tg = import2(to, cfg.k)
    mra.compress2(tg)
    g, _ = mra.apply_ns2(mra.make_operator2(*op_args), tg)
    removed = mra.reconstruct2(g, truncate=True, eps=cfg.eps)
    sto = {}
    go = D.apply_full(D.operator(*op_args), to, truncate_out=True, stats=sto)
    blocks, leaf, _ = as_dicts(g)
    assert set(blocks) == set(go)
    assert all(leaf[key] == n.leaf for key, n in go.items())
    assert rel_l2({k_: b for k_, b in blocks.items() if leaf[k_]}, {k_: n.s for k_, n in go.items() if n.leaf}) <= 1e-12
    assert abs(removed - sto["truncation_l2"]) <= 1e-9 * max(sto["truncation_l2"], 1e-300)


def test_full_size_sampled_parity():
    """The full-size d = 2 workload (64 Gaussians, k = 8, eps = 1e-6, depth 12,
    2,717 nodes): the GPU tree is handed to the oracle, and the ns-form
    output of sampled nodes of every level (Step 2 blocks included) agrees with
    the oracle's Algorithm 3 to rounding; eta agrees."""
    cfg, dens = W.poisson2d()
    op_args = (cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    t, hit = mra.build_tree2(dens, cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    assert not hit
    c, l, b, _ = t.export()
    to = {tuple(int(v) for v in cc): D.Node(bool(ll), bb.copy() if ll else None) for cc, ll, bb in zip(c, l, b)}
    mra.compress2(t)
    g, st = mra.apply_ns2(mra.make_operator2(*op_args), t)
    D.compress(to, cfg.k)
    rng = np.random.default_rng(12)
    keys = sorted(to)
    levels = sorted({key[0] for key in keys})
    sample = []
    for j in levels:
        lv = [key for key in keys if key[0] == j]
        sample += [lv[i] for i in rng.choice(len(lv), size=min(6, len(lv)), replace=False)]
    sto = {}
    ghat = D.apply_ns(D.operator(*op_args), to, stats=sto, nodes=sample)
    blocks, _, _ = as_dicts(g)
    assert abs(st["eta"] - sto["eta"]) <= 1e-12 * sto["eta"]
    for key in sample:
        ref = ghat[key]
        assert np.abs(blocks[key] - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300) + 1e-300, key


def test_dimension_mismatch_is_rejected():
    op3 = mra.make_operator(0.0, 1.0, 1e-4, 4, 3)
    op2 = mra.make_operator2(0.0, 0.5, 1e-4, 4, 3)
    t2, _ = mra.build_tree2(DENS, 4, 1e-4, 3)
    mra.compress2(t2)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns2(op3, t2)
    assert e.value.code == mra.EINVAL
    t3, _ = mra.build_tree(W.Density(np.array([1.0]), np.array([50.0]), np.array([[0.5, 0.5, 0.5]]), np.zeros(1)),
                           4, 1e-4, 3)
    mra.compress(t3)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op2, t3)
    assert e.value.code == mra.EINVAL
    with pytest.raises(mra.MraError) as e:
        mra.make_operator2(0.0, 1.0, 1e-4, 4, 3)      # alpha must be below 1 in d = 2
    assert e.value.code == mra.EINVAL
