"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Trees given to both sides are built by the oracle
and imported, so apply parity does not depend on Algorithm 1's decisions;
Algorithm 1 itself is compared separately.

Tolerances: FP64 paths agree with the oracle to rounding (relative L2
<= 1e-12; term/translation decisions are FP64 on both sides, so item counts
match exactly); the FP32 path is gated at 10 eps (the per-config bound)."""
import math

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

DENS2 = OT.Density([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47]])


def gpu_tree_from_oracle(tree, k):
    c, l, b = oracle_to_arrays(tree, k)
    return mra.tree_import(k, c, l, b)


def export_dict(t):
    c, l, b, dn = t.export()
    return arrays_to_dict(c, b), {tuple(int(v) for v in cc): bool(x) for cc, x in zip(c, l)}, \
        {tuple(int(v) for v in cc): d for cc, d in zip(c, dn)}


@pytest.mark.parametrize("mu,alpha,eps,k,J", [(0.0, 1.0, 1e-4, 4, 3), (1.5, 1.0, 1e-6, 6, 4),
                                              (0.0, 0.5, 1e-5, 5, 3)])
def test_operator_tables(mu, alpha, eps, k, J):
    op = mra.make_operator(mu, alpha, eps, k, J)
    g = op.export()
    o = OO.Operator(mu, alpha, eps, k, J)
    assert len(g["w"]) == o.M
    assert np.allclose(g["w"], o.w, rtol=1e-13, atol=0)
    assert np.allclose(g["tau"], o.tau, rtol=1e-13, atol=0)
    # F entries are O(1) at most; both quadratures are accurate to ~1e-15
    assert np.abs(g["F"] - o.F).max() <= 2e-14
    # norms inherit the entries' absolute rounding (k entries per row)
    assert np.allclose(g["nF"], o.nF, rtol=1e-12, atol=k * 2e-14)
    # the estimate contains N_dif = ||FF - U F U^T||, a difference of nearly
    # equal blocks: its rounding is relative to the blocks' own scale (nF^3)
    scale = o.nF.max(axis=2) ** 3
    assert np.all(np.abs(g["est"] - o.est_core) <= 1e-7 * np.abs(o.est_core) + 1e-12 * scale)
    op.free()


def test_build_tree_matches_algorithm1():
    k, eps = 4, 1e-4
    tg, hit = mra.build_tree(DENS2, k, eps, 4, init_level=1)
    to, hito = OT.build_tree(DENS2, k, eps, 4, init_level=1)
    assert hit == hito
    blocks, leaf, _ = export_dict(tg)
    assert set(blocks) == set(to)
    for key, n in to.items():
        assert leaf[key] == n.leaf
        if n.leaf:
            assert np.abs(blocks[key] - n.s).max() <= 1e-12 * max(1.0, np.abs(n.s).max())


def test_build_uniform_and_depth_cap():
    tg, _ = mra.build_tree(DENS2, 3, 1e-3, 5, uniform_level=2)
    assert tg.n == 1 + 8 + 64
    # a Gaussian that level-2 boxes cannot resolve reports the cap
    narrow = OT.Density([1.0], [2e3], [[0.52, 0.47, 0.5]])
    tg2, hit = mra.build_tree(narrow, 4, 1e-6, 2, init_level=1)
    to2, hito = OT.build_tree(narrow, 4, 1e-6, 2, init_level=1)
    assert hit and hito and tg2.n == len(to2)


def test_compress_and_inverse_round_trip():
    k = 5
    to, _ = OT.build_tree(DENS2, k, 1e-5, 4, init_level=1)
    tg = gpu_tree_from_oracle(to, k)
    mra.compress(tg, store_d=True)
    OT.compress(to, k)
    blocks, leaf, dn = export_dict(tg)
    for key, n in to.items():
        assert np.abs(blocks[key] - n.s).max() <= 1e-13 * max(1.0, np.abs(n.s).max())
        if not n.leaf:
            assert abs(dn[key] - n.dnorm) <= 1e-12 * max(n.dnorm, 1e-300) + 1e-14
    ref = {key: b.copy() for key, b in blocks.items() if leaf[key]}
    # zero the leaves on the device, then rebuild them from s^0 and d
    c, l, b, _ = tg.export()
    b[l.astype(bool)] = 0.0
    dev = torch.from_numpy(b).cuda()
    mra.tree_set_blocks(tg, dev.data_ptr())
    mra.reconstruct(tg, mode="inverse")
    blocks2, leaf2, _ = export_dict(tg)
    err = math.sqrt(sum(((blocks2[key] - ref[key]) ** 2).sum() for key in ref))
    nrm = math.sqrt(sum((b ** 2).sum() for b in ref.values()))
    assert err <= 1e-13 * nrm * OT.levels(to)


@pytest.mark.parametrize("k", [3, 8])
def test_compress_without_stored_cubes(k):
    """The default compress (scaling blocks by the H half of the filter, wavelet
    norms as ||children - up(parent)||) against the oracle's full transform."""
    to, _ = OT.build_tree(DENS2, k, 1e-5, 4, init_level=1)
    tg = gpu_tree_from_oracle(to, k)
    mra.compress(tg)
    OT.compress(to, k)
    blocks, leaf, dn = export_dict(tg)
    scale = max(n.dnorm for n in to.values())
    for key, n in to.items():
        assert np.abs(blocks[key] - n.s).max() <= 1e-13 * max(1.0, np.abs(n.s).max())
        if not n.leaf:
            assert abs(dn[key] - n.dnorm) <= 1e-12 * n.dnorm + 1e-14 * scale


@pytest.mark.parametrize("k", [3, 8])
def test_compress_scaling_only(k):
    """MRA_COMPRESS_SCALING: the same scaling blocks as the full compress (bit
    for bit: the same H stages run), wavelet norms left at zero, the same
    apply output; an unknown mode is refused, and a recompress without cubes
    drops the stored ones (the inverse transform then refuses)."""
    to, _ = OT.build_tree(DENS2, k, 1e-5, 4, init_level=1)
    ta = gpu_tree_from_oracle(to, k)
    tb = gpu_tree_from_oracle(to, k)
    mra.compress(ta)
    mra.compress(tb, norms=False)
    _, _, ba, dna = ta.export()
    _, _, bb, dnb = tb.export()
    assert np.array_equal(ba, bb)
    assert not dnb.any() and dna.any()
    op = mra.make_operator(0.0, 1.0, 1e-5, k, 4)
    ga, _ = mra.apply_ns(op, ta)
    gb, _ = mra.apply_ns(op, tb)
    assert np.array_equal(ga.export()[2], gb.export()[2])
    with pytest.raises(mra.MraError) as e:
        mra._check(mra.lib().mra_compress(ta.h, 3, None))
    assert e.value.code == mra.EINVAL
    mra.compress(ta, store_d=True)
    mra.compress(ta, norms=False)
    with pytest.raises(mra.MraError) as e:
        mra.reconstruct(ta, mode="inverse")
    assert e.value.code == mra.ESTATE


def run_both(tree_o, op_o, op_g, k, precision="fp64", **kw):
    tg = gpu_tree_from_oracle(tree_o, k)
    mra.compress(tg)
    tc = OT.copy_tree(tree_o)
    OT.compress(tc, k)
    st_o = {}
    kw_o = dict(kw)
    kw_o.pop("itemwise", None)
    if kw_o.pop("unscreened", False):
        kw_o["screen"] = False
    ghat_o = OA.apply_ns(op_o, tc, stats=st_o, **kw_o)
    g, st_g = mra.apply_ns(op_g, tg, precision=precision, **kw)
    ghat_g, _, _ = export_dict(g)
    return tc, tg, g, ghat_o, ghat_g, st_o, st_g


@pytest.fixture(scope="module")
def small_cfg():
    cfg, d = W.poisson_small()
    dens = oracle_density(d)
    tree, _ = OT.build_tree(dens, cfg.k, cfg.eps, cfg.max_level, uniform_level=cfg.uniform_level)
    op_o = OO.Operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    op_g = mra.make_operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    return cfg, tree, op_o, op_g


def test_apply_parity_poisson_k4_uniform3(small_cfg):
    cfg, tree, op_o, op_g = small_cfg
    tc, tg, g, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, cfg.k)
    assert st_g["n_items"] == st_o["n_items"]
    assert st_g["n_pairs"] == st_o["n_pairs"]
    assert abs(st_g["eta"] - st_o["eta"]) <= 1e-13 * st_o["eta"]
    assert rel_l2(ghat_g, ghat_o) <= 1e-12
    # eq. g_assemble and the redundant output tree
    gg = OA.assemble(op_o, tc, ghat_o)
    OT.compress(gg, cfg.k)
    mra.reconstruct(g, mode="assemble")
    out_g, leaf_g, _ = export_dict(g)
    assert rel_l2(out_g, {key: n.s for key, n in gg.items()}) <= 1e-12


def test_apply_fp32_within_gate(small_cfg):
    cfg, tree, op_o, op_g = small_cfg
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, cfg.k, precision="fp32")
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= 10 * cfg.eps


@pytest.fixture(scope="module")
def adaptive_cfg():
    k, eps = 5, 1e-4
    tree, _ = OT.build_tree(DENS2, k, eps, 4, init_level=1)
    op_o = OO.Operator(0.0, 1.0, eps, k, 4)
    op_g = mra.make_operator(0.0, 1.0, eps, k, 4)
    return k, eps, tree, op_o, op_g


def test_apply_parity_adaptive_with_ghosts(adaptive_cfg):
    k, eps, tree, op_o, op_g = adaptive_cfg
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k)
    assert st_g["n_ghosts"] == st_o["n_refined"] > 0
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_apply_parity_itemwise_kernel(adaptive_cfg, precision):
    """The per-item formulation (three mode products per item) and the default
    nested-sum formulation apply the same items."""
    k, eps, tree, op_o, op_g = adaptive_cfg
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, precision=precision, itemwise=True)
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= (1e-12 if precision == "fp64" else 10 * eps)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_apply_tensor_core_split_k8(eps):
    """tcgen05 FP16 hi/lo split products with FP32 accumulation: same items as
    the oracle, every output block within the 10 eps gate."""
    k = 8
    tree, _ = OT.build_tree(DENS2, k, eps, 3, init_level=1)
    op_o = OO.Operator(0.0, 1.0, eps, k, 3)
    op_g = mra.make_operator(0.0, 1.0, eps, k, 3)
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, precision="tc")
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= 10 * eps


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_apply_tensor_core_ladder_k8(eps):
    """Precision ladder: single FP16 products for the terms whose bounded
    rounding error fits the node's budget, FP16 hi+lo for the rest; same items,
    within the 10 eps gate, and some items do take the single-FP16 rung."""
    k = 8
    tree, _ = OT.build_tree(DENS2, k, eps, 3, init_level=1)
    op_o = OO.Operator(0.0, 1.0, eps, k, 3)
    op_g = mra.make_operator(0.0, 1.0, eps, k, 3)
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, precision="tc_ladder")
    assert st_g["n_items"] == st_o["n_items"]
    assert 0 < st_g["n_items_lowp"] <= st_g["n_items"]
    # the budget is eps ||T_0 f_0|| / 4 in L2 on top of the hi+lo error
    assert rel_l2(ghat_g, ghat_o) <= 10 * eps


@pytest.mark.parametrize("k,eps", [(4, 1e-4), (6, 1e-5)])
def test_apply_tensor_core_padded_orders(k, eps):
    """Orders below 8 run on the same 8 x 8 MMA tiles with zero padding: the
    padded rows and columns contribute nothing and the output keeps k^3."""
    tree, _ = OT.build_tree(DENS2, k, eps, 3, init_level=1)
    op_o = OO.Operator(0.0, 1.0, eps, k, 3)
    op_g = mra.make_operator(0.0, 1.0, eps, k, 3)
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, precision="tc")
    assert st_g["n_items"] == st_o["n_items"]
    assert st_g["n_ghosts"] == st_o["n_refined"]
    assert rel_l2(ghat_g, ghat_o) <= 10 * eps


def test_tensor_core_rejects_orders_above_8():
    tree, _ = OT.build_tree(DENS2, 10, 1e-4, 1, uniform_level=1)
    op_g = mra.make_operator(0.0, 1.0, 1e-4, 10, 1)
    tg = gpu_tree_from_oracle(tree, 10)
    mra.compress(tg)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op_g, tg, precision="tc")
    assert e.value.code == mra.EINVAL


def test_apply_parity_unscreened(adaptive_cfg):
    k, eps, tree, op_o, op_g = adaptive_cfg
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, unscreened=True)
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= 1e-12


def test_apply_parity_block_screen(adaptive_cfg):
    k, eps, tree, op_o, op_g = adaptive_cfg
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k, block_screen=True)
    # per-block decisions compare FP64 norms computed in different orders:
    # allow a handful of items within rounding of the threshold
    assert abs(st_g["n_items"] - st_o["n_items"]) <= max(2, st_o["n_items"] // 100000)
    assert rel_l2(ghat_g, ghat_o) <= 1e-10


@pytest.mark.parametrize("mu,alpha", [(1.5, 1.0), (0.0, 0.5)])
def test_apply_parity_other_kernels(mu, alpha):
    k, eps = 4, 1e-4
    tree, _ = OT.build_tree(DENS2, k, eps, 3, init_level=1)
    op_o = OO.Operator(mu, alpha, eps, k, 3)
    op_g = mra.make_operator(mu, alpha, eps, k, 3)
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k)
    assert st_g["n_items"] == st_o["n_items"]
    assert rel_l2(ghat_g, ghat_o) <= 1e-12


def test_truncation_parity(adaptive_cfg):
    k, eps, tree, op_o, op_g = adaptive_cfg
    tc, tg, g, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k)
    gg = OA.assemble(op_o, tc, ghat_o)
    gg, rem_o = OA.truncate(gg, k, 10 * eps)
    rem_g = mra.reconstruct(g, mode="assemble", truncate=True, eps=10 * eps)
    out_g, leaf_g, _ = export_dict(g)
    assert set(out_g) == set(gg)
    assert abs(rem_g - rem_o) <= 1e-9 * max(rem_o, 1e-300) + 1e-15
    assert rel_l2(out_g, {key: n.s for key, n in gg.items()}) <= 1e-12


def test_root_only_tree():
    k = 4
    tree, _ = OT.build_tree(DENS2, k, 1e-4, 0, uniform_level=0)
    op_o = OO.Operator(0.0, 1.0, 1e-4, k, 0)
    op_g = mra.make_operator(0.0, 1.0, 1e-4, k, 0)
    _, _, _, ghat_o, ghat_g, st_o, st_g = run_both(tree, op_o, op_g, k)
    assert st_g["n_pairs"] == st_o["n_pairs"] == 1
    assert rel_l2(ghat_g, ghat_o) <= 1e-13


def test_rejects_deeper_tree_than_operator():
    tree, _ = OT.build_tree(DENS2, 3, 1e-3, 3, uniform_level=3)
    op_g = mra.make_operator(0.0, 1.0, 1e-3, 3, 2)
    tg = gpu_tree_from_oracle(tree, 3)
    mra.compress(tg)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op_g, tg)
    assert e.value.code == mra.EINVAL


def test_import_rejects_malformed_node_lists():
    """mra_tree_import checks the node list and names the first bad node:
    out-of-range levels and boxes, an unsorted list, a list without the root
    first, an internal node without its children, a node without a parent."""
    to, _ = OT.build_tree(DENS2, 3, 1e-3, 3, init_level=1)
    c, l, b = oracle_to_arrays(to, 3)
    tg = mra.tree_import(3, c, l, b)          # the valid list imports
    assert tg.info().n_nodes == len(to)
    cases = []
    bad = c.copy(); bad[5, 0] = 99; cases.append((bad, l, "out of range"))
    bad = c.copy(); bad[5, 1] = 1 << int(bad[5, 0]); cases.append((bad, l, "box index out of range"))
    bad = c.copy(); bad[[3, 4]] = bad[[4, 3]]; cases.append((bad, l, "not sorted"))
    bad = c[1:].copy(); cases.append((bad, l[1:].copy(), "root"))
    li = l.copy(); li[int(np.nonzero(l)[0][-1])] = 0; cases.append((c, li, "lacks child"))
    keep = np.ones(len(c), bool); keep[int(np.nonzero(c[:, 0] == 1)[0][0])] = False   # drop one level-1 box
    cases.append((c[keep].copy(), l[keep].copy(), ""))
    for cc, ll, msg in cases:
        with pytest.raises(mra.MraError) as e:
            mra.tree_import(3, np.ascontiguousarray(cc), np.ascontiguousarray(ll), b[:len(cc)].copy())
        assert e.value.code == mra.EINVAL
        assert msg in str(e.value)
