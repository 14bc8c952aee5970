"""mra_apply_ns_noalloc (the apply for callers that cannot allocate) against
mra_apply_ns.

Some callers cannot call cudaMalloc/cudaFree while the apply runs: code where
another component owns the device allocator, or work that must not change the
device's memory map.  The no-alloc entry point serves them from one fixed
scratch array inside the library.  This test calls it through the C ABI twice
in a row on the same input and compares each result with the allocating entry
point's output, at the parity tests' tolerances (relative L2 1e-12 in FP64,
10 eps in FP32).  The file is named so that pytest collects it last."""
import numpy as np
import pytest

from oracle import tree as OT
from tests.helpers import oracle_to_arrays

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

DENS = OT.Density([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47]])


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    k, eps = 5, 1e-4
    tree, _ = OT.build_tree(DENS, k, eps, 4, init_level=1)   # adaptive: Step 2 refines inputs
    c, l, b = oracle_to_arrays(tree, k)
    tg = mra.tree_import(k, c, l, b)
    mra.compress(tg)
    op = mra.make_operator(0.0, 1.0, eps, k, 4)
    return k, eps, tg, op


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_apply_ns_on_two_calls(case, precision):
    k, eps, tg, op = case
    n = tg.n
    assert n <= 1024
    g, st = mra.apply_ns(op, tg, precision=precision)
    _, _, ref, _ = g.export()
    g.free()
    tol = 1e-12 if precision == "fp64" else 10 * eps
    out = torch.empty(n * k ** 3, dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        items = mra.apply_ns_noalloc(op, tg, out.data_ptr(), precision=precision)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(n, k, k, k)
        assert np.isfinite(got).all(), f"call {call}: unwritten output"
        assert items == st["n_items"], f"call {call}"
        assert rel_l2(got, ref) <= tol, f"call {call}"


def test_noalloc_rejects_oversize_tree():
    k = 3
    tree, _ = OT.build_tree(DENS, k, 1e-3, 4, uniform_level=4)      # 4681 nodes > 1024
    c, l, b = oracle_to_arrays(tree, k)
    tg = mra.tree_import(k, c, l, b)
    mra.compress(tg)
    op = mra.make_operator(0.0, 1.0, 1e-3, k, 4)
    out = torch.empty(tg.n * k ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns_noalloc(op, tg, out.data_ptr())
    assert e.value.code == mra.EINVAL and "1024" in str(e.value)


def test_noalloc_without_item_count(case):
    """n_items_host is optional: with NULL the call still checks the device's
    error words and writes the same output."""
    import ctypes
    k, eps, tg, op = case
    n = tg.n
    g, _ = mra.apply_ns(op, tg, precision="fp64")
    ref = g.export()[2]
    g.free()
    out = torch.empty(n * k ** 3, dtype=torch.float64, device="cuda")
    out.fill_(float("nan"))
    rc = mra.lib().mra_apply_ns_noalloc(op.h, tg.h, mra.PREC["fp64"], out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream, None)
    assert rc == mra.OK, mra.last_error()
    got = out.cpu().numpy().reshape(n, k, k, k)
    assert rel_l2(got, ref) <= 1e-12


def test_noalloc_rejects_too_many_refined_blocks(case):
    """A tree within the node limit (825 nodes) whose Step 2 needs more than
    4096 refined input blocks (5,725: four narrow Gaussians refined to level 7)
    is refused after the screen with MRA_EINVAL; a valid call right after it
    still matches mra_apply_ns."""
    kk, e2 = 5, 1e-3
    cens = [[0.37, 0.52, 0.61], [0.18, 0.81, 0.47], [0.62, 0.37, 0.21], [0.83, 0.66, 0.77]]
    tree, _ = OT.build_tree(OT.Density([1.0] * 4, [1e4] * 4, cens), kk, e2, 8, init_level=1)
    c, l, b = oracle_to_arrays(tree, kk)
    tb = mra.tree_import(kk, c, l, b)
    mra.compress(tb)
    assert tb.n <= 1024
    opb = mra.make_operator(0.0, 1.0, e2, kk, 8)
    _, st = mra.apply_ns(opb, tb, precision="fp64")
    assert st["n_ghosts"] > 4096
    out = torch.empty(tb.n * kk ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns_noalloc(opb, tb, out.data_ptr())
    assert e.value.code == mra.EINVAL and "4096" in str(e.value)
    k, eps, tg, op = case
    g, st2 = mra.apply_ns(op, tg, precision="fp64")
    ref = g.export()[2]
    g.free()
    out2 = torch.empty(tg.n * k ** 3, dtype=torch.float64, device="cuda")
    items = mra.apply_ns_noalloc(op, tg, out2.data_ptr())
    assert items == st2["n_items"]
    assert rel_l2(out2.cpu().numpy().reshape(tg.n, k, k, k), ref) <= 1e-12
