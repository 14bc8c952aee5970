"""The boundary's error contract on the GPU, produced without faulting it.

* MRA_ENOMEM: an allocator hook that returns NULL on its n-th call, for every
  n across one make_operator -> build_tree -> compress -> apply_ns (tensor
  cores) -> reconstruct -> plan sequence.  The failing call must return
  MRA_ENOMEM with a NULL output handle, and once the handles that were made
  are freed the hook must hold no live block (nothing leaked on any error
  path), with torch's allocated byte count back where it started.
* MRA_ETIMEOUT: the tensor-core apply's bounded completion wait.  With the
  test hook MRA_TEST_WITHHOLD_MMA the issuing threads send no MMA and no
  commit for the first group, so the first wait of every CTA can only end by
  its limit (4096 polls here): nothing is in flight when it gives up, the
  kernel frees its tensor memory and returns, and the call reports
  MRA_ETIMEOUT.  The context stays usable: the next apply is checked against
  the FP64 path.
* mra_free on every handle kind.
"""
import ctypes
import gc

import numpy as np
import pytest

from oracle import tree as OT
from paper_0706_0747_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0706_0747_gb300 import mra  # noqa: E402

DENS = OT.Density([30.0, 12.0], [70.0, 150.0], [[0.45, 0.52, 0.5], [0.62, 0.41, 0.47]])


class FailingAlloc:
    """torch caching-allocator hook that returns NULL on call number fail_at
    (never when fail_at is 0) and records the blocks it has handed out."""

    def __init__(self, fail_at):
        self.calls, self.fail_at, self.live = 0, fail_at, {}

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, stream, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self._fa, self._ff = mra.ALLOC_FN(_alloc), mra.FREE_FN(_free)
        self.hook = mra.Alloc(self._fa, self._ff, None)


def _sequence(A, made):
    """The calls under test, through the C ABI; returns the first status that
    is not OK (with the output handle it left), or OK."""
    L = mra.lib()
    st = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p()
    rc = L.mra_make_operator(0.0, 1.0, 1e-4, 4, 3, ctypes.byref(A.hook), st, ctypes.byref(h))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    op = h.value
    coef = np.array(DENS.coef, dtype=np.float64)
    expo = np.array(DENS.expo, dtype=np.float64)
    cen = np.ascontiguousarray(np.array(DENS.centers, dtype=np.float64).reshape(-1))
    r2 = np.zeros_like(coef)
    d = mra.Density(len(coef), mra._dp(coef), mra._dp(r2), mra._dp(expo), mra._dp(cen))
    h = ctypes.c_void_p()
    rc = L.mra_build_tree(ctypes.byref(d), 4, 1e-4, 3, -1, 1, ctypes.byref(A.hook), st, ctypes.byref(h))
    if rc not in (mra.OK, mra.EDEPTH):
        return rc, h.value
    made.append(h.value)
    tree = h.value
    rc = L.mra_compress(tree, 0, st)
    if rc != mra.OK:
        return rc, None
    o = mra.ApplyOpts(mra.PREC["tc"], 0, 0, 0, 0, 0, 0, 0)
    s = mra.ApplyStats()
    h = ctypes.c_void_p()
    rc = L.mra_apply_ns(op, tree, ctypes.byref(o), st, ctypes.byref(h), ctypes.byref(s))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    g = h.value
    rem = ctypes.c_double(0.0)
    rc = L.mra_reconstruct(g, 0, 1, 1e-4, st, ctypes.byref(rem))
    if rc != mra.OK:
        return rc, None
    arr = (ctypes.c_void_p * 1)(tree)
    po = mra.PlanOpts(mra.PREC["tc"], 0, 0)
    h = ctypes.c_void_p()
    rc = L.mra_plan_create(op, arr, 1, ctypes.byref(po), st, ctypes.byref(h))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    rc = L.mra_plan_execute(h.value, st)
    if rc != mra.OK:
        return rc, None
    h2 = ctypes.c_void_p()
    rc = L.mra_plan_output(made[-1], 0, st, ctypes.byref(h2))
    if rc != mra.OK:
        return rc, h2.value
    made.append(h2.value)
    return mra.OK, None


def _free_all(made):
    for hd in reversed(made):  # the plan before the trees it borrows
        assert mra.lib().mra_free(hd) == mra.OK


def test_enomem_on_every_allocation_leaks_nothing():
    # handles left over from earlier tests are released first, so that the
    # byte count below measures this test's calls only
    gc.collect()
    mra.release_cached()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    probe = FailingAlloc(0)
    made = []
    rc, _ = _sequence(probe, made)
    assert rc == mra.OK, mra.last_error()
    _free_all(made)
    mra.release_cached()
    torch.cuda.synchronize()
    total = probe.calls
    assert not probe.live and total > 20
    for n in range(1, total + 1):
        A = FailingAlloc(n)
        made = []
        rc, out = _sequence(A, made)
        assert rc == mra.ENOMEM, f"allocation {n} of {total}: status {rc} ({mra.last_error()})"
        assert out is None, f"allocation {n}: output handle set on failure"
        _free_all(made)
        mra.release_cached()  # the reuse cache hands this hook's blocks back
        torch.cuda.synchronize()
        assert not A.live, f"allocation {n} of {total}: {len(A.live)} blocks leaked"
    gc.collect()
    mra.release_cached()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def _sequence_products_d2(A, made):
    """The hydrogen step's calls (product, inner product, two Kalos steps with
    an operator cache: a build, then a re-weighting) and the d = 2 variant
    (build_tree2, compress2, make_operator2, apply_ns2, reconstruct2 with
    truncation), with the allocator hook on every handle."""
    L = mra.lib()
    st = torch.cuda.current_stream().cuda_stream
    hc = W.hydrogen_small()
    dens = hc.start_density()
    coef, expo = np.ascontiguousarray(dens.coef), np.ascontiguousarray(dens.expo)
    cen, r2 = np.ascontiguousarray(dens.centers.reshape(-1)), np.zeros_like(coef)
    d = mra.Density(len(coef), mra._dp(coef), mra._dp(r2), mra._dp(expo), mra._dp(cen))
    h = ctypes.c_void_p()
    rc = L.mra_build_tree(ctypes.byref(d), hc.k, hc.eps, hc.max_level, -1, hc.init_level, ctypes.byref(A.hook), st,
                          ctypes.byref(h))
    if rc not in (mra.OK, mra.EDEPTH):
        return rc, h.value
    made.append(h.value)
    phi = h.value
    pot = mra.Potential(charges=[-1.0 / hc.L], positions=[hc.u0])
    pc = pot.c_struct()
    h = ctypes.c_void_p()
    rc = L.mra_tree_multiply(phi, ctypes.byref(pc), 1.0, st, ctypes.byref(h))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    dot = ctypes.c_double(0.0)
    rc = L.mra_tree_dot(h.value, phi, st, ctypes.byref(dot))
    if rc != mra.OK:
        return rc, None
    cache = ctypes.c_void_p()
    info = mra.KalosInfo()
    for mu in (0.8, 0.9):
        h = ctypes.c_void_p()
        rc = L.mra_kalos_step(phi, ctypes.byref(pc), hc.L, mu, hc.eps, hc.max_level, None, ctypes.byref(cache), st,
                              ctypes.byref(h), ctypes.byref(info))
        if cache.value and cache.value not in made:
            made.append(cache.value)
        if rc != mra.OK:
            return rc, h.value
        made.append(h.value)
    d2c = np.array([30.0, 12.0]), np.array([70.0, 150.0]), np.array([0.45, 0.52, 0.62, 0.41])
    r22 = np.zeros(2)
    dd = mra.Density(2, mra._dp(d2c[0]), mra._dp(r22), mra._dp(d2c[1]), mra._dp(d2c[2]))
    h = ctypes.c_void_p()
    rc = L.mra_build_tree2(ctypes.byref(dd), 4, 1e-4, 5, -1, 1, ctypes.byref(A.hook), st, ctypes.byref(h))
    if rc not in (mra.OK, mra.EDEPTH):
        return rc, h.value
    made.append(h.value)
    t2 = h.value
    rc = L.mra_compress2(t2, st)
    if rc != mra.OK:
        return rc, None
    h = ctypes.c_void_p()
    rc = L.mra_make_operator2(0.0, 0.5, 1e-4, 4, 5, ctypes.byref(A.hook), st, ctypes.byref(h))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    op2 = h.value
    h = ctypes.c_void_p()
    s = mra.ApplyStats()
    rc = L.mra_apply_ns2(op2, t2, st, ctypes.byref(h), ctypes.byref(s))
    if rc != mra.OK:
        return rc, h.value
    made.append(h.value)
    rem = ctypes.c_double(0.0)
    rc = L.mra_reconstruct2(h.value, 1, 1e-4, st, ctypes.byref(rem))
    if rc != mra.OK:
        return rc, None
    return mra.OK, None


def test_enomem_in_products_kalos_and_d2_leaks_nothing():
    """The same contract for the hydrogen step's entries and the d = 2
    variant: every failed allocation gives MRA_ENOMEM, no output handle, and
    no block left allocated once the handles made are freed."""
    gc.collect()
    mra.release_cached()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    probe = FailingAlloc(0)
    made = []
    rc, _ = _sequence_products_d2(probe, made)
    assert rc == mra.OK, mra.last_error()
    _free_all(made)
    mra.release_cached()
    torch.cuda.synchronize()
    total = probe.calls
    assert not probe.live and total > 20
    for n in range(1, total + 1):
        A = FailingAlloc(n)
        made = []
        rc, out = _sequence_products_d2(A, made)
        assert rc == mra.ENOMEM, f"allocation {n} of {total}: status {rc} ({mra.last_error()})"
        assert out is None, f"allocation {n}: output handle set on failure"
        _free_all(made)
        mra.release_cached()  # the reuse cache hands this hook's blocks back
        torch.cuda.synchronize()
        assert not A.live, f"allocation {n} of {total}: {len(A.live)} blocks leaked"
    gc.collect()
    mra.release_cached()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_bounded_wait_times_out_and_context_survives():
    k, eps = 4, 1e-4
    tree, _ = mra.build_tree(DENS, k, eps, 3, init_level=1)
    mra.compress(tree)
    op = mra.make_operator(0.0, 1.0, eps, k, 3)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op, tree, precision="tc", wait_limit=4096, test_flags=mra.TEST_WITHHOLD_MMA)
    assert e.value.code == mra.ETIMEOUT and "limit" in str(e.value)
    torch.cuda.synchronize()  # no sticky error: the kernel returned on its own
    g64, st64 = mra.apply_ns(op, tree, precision="fp64")
    gtc, sttc = mra.apply_ns(op, tree, precision="tc", wait_limit=4096)
    a, b = g64.export()[2], gtc.export()[2]
    assert sttc["n_items"] == st64["n_items"]
    assert np.linalg.norm(a - b) <= 10 * eps * np.linalg.norm(a)


def test_bounded_wait_rejects_bad_arguments():
    k, eps = 4, 1e-4
    tree, _ = mra.build_tree(DENS, k, eps, 2, uniform_level=2)
    mra.compress(tree)
    op = mra.make_operator(0.0, 1.0, eps, k, 2)
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op, tree, precision="tc", wait_limit=-1)
    assert e.value.code == mra.EINVAL
    with pytest.raises(mra.MraError) as e:
        mra.apply_ns(op, tree, precision="tc", test_flags=8)
    assert e.value.code == mra.EINVAL


def test_mra_free_every_handle_kind():
    k, eps = 4, 1e-4
    tree, _ = mra.build_tree(DENS, k, eps, 2, uniform_level=2)
    mra.compress(tree)
    op = mra.make_operator(0.0, 1.0, eps, k, 2)
    g, _ = mra.apply_ns(op, tree, precision="fp64")
    plan = mra.plan_create(op, [tree], precision="fp64", use_graph=False)
    net = mra.mlp_create(seed=3)
    for obj in (plan, net, g, tree, op):
        mra.free(obj)
        assert obj.h is None
    torch.cuda.synchronize()


def test_block_cache_reuses_and_releases():
    """The library's reuse cache: a repeated apply takes its blocks from the cache
    (no call reaches the hook) and gives the same output bit for bit; a tree made
    on another stream gets fresh blocks; mra_release_cached hands every cached
    block back (the hook then holds only the live handles' blocks)."""
    A = FailingAlloc(0)
    k, eps = 4, 1e-4
    tree, _ = mra.build_tree(DENS, k, eps, 3, uniform_level=2, allocator=A.hook)
    mra.compress(tree, norms=False)
    op = mra.make_operator(0.0, 1.0, eps, k, 3, allocator=A.hook)
    g1, _ = mra.apply_ns(op, tree, precision="tc")
    out1 = g1.export()[2]
    g1.free()
    calls = A.calls
    g2, _ = mra.apply_ns(op, tree, precision="tc")
    assert A.calls == calls  # every block of the second apply came from the cache
    assert np.array_equal(g2.export()[2], out1)
    g2.free()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        t2, _ = mra.build_tree(DENS, k, eps, 3, uniform_level=2, allocator=A.hook, stream=side.cuda_stream)
        mra.compress(t2, norms=False, stream=side.cuda_stream)
        g3, _ = mra.apply_ns(op, t2, precision="tc", stream=side.cuda_stream)
        side.synchronize()
    assert A.calls > calls  # blocks keyed by another stream: fresh ones from the hook
    assert np.array_equal(g3.export(stream=side.cuda_stream)[2], out1)
    g3.free()
    mra.free(t2)
    side.synchronize()
    live_handles = dict(A.live)
    released = mra.release_cached()
    torch.cuda.synchronize()
    assert released > 0 and len(A.live) < len(live_handles)
    mra.free(tree)
    mra.free(op)
    mra.release_cached()
    torch.cuda.synchronize()
    assert not A.live
