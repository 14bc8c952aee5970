"""GPU parity of the output skeleton refinement (mra_tree_refine) against the
oracle's refine_graded: the same node set, leaf flags and blocks; the apply
on the refined tree against the oracle's apply on it; and the output nearer
the closed-form potential than on the input's own skeleton."""
import numpy as np
import pytest

from oracle import apply as OA, operator as OO, tree as OT
from tests.closed_forms import poisson_gaussian, project_leaf
from tests.helpers import arrays_to_dict, oracle_to_arrays, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

K, EPS, J, A, C = 4, 1e-4, 5, 3e3, [0.43, 0.51, 0.57]


@pytest.fixture(scope="module")
def case():
    dens = OT.Density([(A / np.pi) ** 1.5], [A], [C])
    tree, _ = OT.build_tree(dens, K, EPS, J, init_level=1)
    c, l, b = oracle_to_arrays(tree, K)
    tg = mra.tree_import(K, c, l, b)
    return tree, tg


@pytest.mark.parametrize("passes", [0, 1, 2])
def test_refine_matches_oracle(case, passes):
    tree, tg = case
    ref, ns = OT.refine_graded(tree, K, passes=passes, max_level=J)
    got, ns_g = mra.tree_refine(tg, passes=passes, max_level=J)
    assert ns_g == ns
    c, l, b, dn = got.export()
    keys = [tuple(int(v) for v in r) for r in c]
    assert sorted(keys) == sorted(ref.keys()) and len(keys) == len(ref)
    scale = max(np.abs(n.s).max() for n in ref.values() if n.s is not None)
    for key, lf, blk in zip(keys, l, b):
        assert bool(lf) == ref[key].leaf
        if ref[key].leaf:
            assert np.abs(blk - ref[key].s).max() <= 1e-13 * scale
    assert got.info().state == mra.TREE_LEAVES


def test_refine_rejects_bad_arguments(case):
    _, tg = case
    with pytest.raises(mra.MraError) as e:
        mra.tree_refine(tg, passes=-1)
    assert e.value.code == mra.EINVAL
    with pytest.raises(mra.MraError) as e:
        mra.tree_refine(tg, passes=1, max_level=99)
    assert e.value.code == mra.EINVAL


@pytest.mark.parametrize("precision", ["fp64", "tc"])
def test_apply_on_refined_skeleton(case, precision):
    """Algorithm 3 on the refined tree: the oracle's items and result (rounding for
    FP64, the 10 eps gate on the tensor cores), and after assembly the output is an
    order of magnitude nearer erf(sqrt(a) r) / (4 pi r) than on the input's skeleton."""
    tree, tg = case
    op_g = mra.make_operator(0.0, 1.0, EPS, K, J)
    op_o = OO.Operator(0.0, 1.0, EPS, K, J)
    pot = poisson_gaussian(A, C)

    def err_closed(g):
        c, l, b, _ = g.export()
        num = den = 0.0
        for row, lf, blk in zip(c, l, b):
            if lf:
                r = project_leaf(pot, K, int(row[0]), tuple(int(v) for v in row[1:]), sub=2)
                num += float(((blk - r) ** 2).sum())
                den += float((r ** 2).sum())
        return (num / den) ** 0.5

    errs = []
    for passes in (0, 1):
        t_o, _ = OT.refine_graded(tree, K, passes=passes, max_level=J)
        t_g, _ = mra.tree_refine(tg, passes=passes, max_level=J)
        mra.compress(t_g)
        g, st = mra.apply_ns(op_g, t_g, precision=precision)
        T = OT.copy_tree(t_o)
        OT.compress(T, K)
        st_o = {}
        ref = OA.apply_ns(op_o, T, stats=st_o)
        c, _, b, _ = g.export()
        assert st["n_items"] == st_o["n_items"]
        assert rel_l2(arrays_to_dict(c, b), ref) <= (1e-12 if precision == "fp64" else 10 * EPS)
        mra.reconstruct(g, mode="assemble")
        errs.append(err_closed(g))
    assert errs[1] < errs[0] / 4, errs
