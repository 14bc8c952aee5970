"""Thin Python binding of the C ABI in include/mra_gb300.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library ``libmra_gb300.so`` (built in-tree by ``build.py``).  Importing this
module fails loudly when the library is missing; there is no CPU fallback.
PyTorch, when present, supplies the CUDA stream and (through the allocator
hook) the caching allocator's device memory.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmra_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDEPTH, ESTATE = 0, 1, 2, 3, 4, 5, 6
PREC = {"fp64": 0, "fp32": 1, "tc": 2, "tc_ladder": 3, "tc_fast": 4}
TEST_WITHHOLD_MMA = 1
TREE_LEAVES, TREE_REDUNDANT, TREE_NSFORM = 0, 1, 2
MAX_LEVEL = 12


class MraError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mra error {code}: {msg}")
        self.code = code


class Density(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("coef_host", ctypes.POINTER(ctypes.c_double)),
                ("r2coef_host", ctypes.POINTER(ctypes.c_double)),
                ("expo_host", ctypes.POINTER(ctypes.c_double)),
                ("center_host", ctypes.POINTER(ctypes.c_double))]


class PotentialC(ctypes.Structure):
    _fields_ = [("n_gauss", ctypes.c_int), ("coef_host", ctypes.POINTER(ctypes.c_double)),
                ("r2coef_host", ctypes.POINTER(ctypes.c_double)),
                ("expo_host", ctypes.POINTER(ctypes.c_double)),
                ("center_host", ctypes.POINTER(ctypes.c_double)),
                ("n_charge", ctypes.c_int), ("charge_host", ctypes.POINTER(ctypes.c_double)),
                ("position_host", ctypes.POINTER(ctypes.c_double))]


class KalosInfo(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("mu_next", ctypes.c_double), ("norm_new", ctypes.c_double),
                ("n_terms", ctypes.c_int), ("op_rebuilt", ctypes.c_int), ("n_items", ctypes.c_int64),
                ("ms_apply", ctypes.c_float)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Alloc(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_nodes", ctypes.c_int), ("n_levels", ctypes.c_int),
                ("state", ctypes.c_int), ("depth_hit", ctypes.c_int),
                ("level_offset", ctypes.c_int * (MAX_LEVEL + 2))]


class OpInfo(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("k", ctypes.c_int), ("max_level", ctypes.c_int),
                ("mu", ctypes.c_double), ("alpha", ctypes.c_double), ("eps", ctypes.c_double)]


SCREEN = {"static": 0, "pair": 1, "learned": 2}


class ApplyOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("block_screen", ctypes.c_int),
                ("unscreened", ctypes.c_int), ("itemwise", ctypes.c_int), ("screen_mode", ctypes.c_int),
                ("margin", ctypes.c_int), ("wait_limit", ctypes.c_int), ("test_flags", ctypes.c_int),
                ("schedule", ctypes.c_void_p)]


class ApplyStats(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("n_items", ctypes.c_int64), ("n_ghosts", ctypes.c_int64),
                ("n_out_nodes", ctypes.c_int64), ("eta", ctypes.c_double), ("sigma", ctypes.c_double),
                ("fnorm", ctypes.c_double), ("ms_screen", ctypes.c_float), ("ms_ghost", ctypes.c_float),
                ("ms_apply", ctypes.c_float), ("n_items_lowp", ctypes.c_int64), ("n_misses", ctypes.c_int64),
                ("n_pairs_empty", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("use_graph", ctypes.c_int), ("screen_mode", ctypes.c_int),
                ("margin", ctypes.c_int), ("reserved", ctypes.c_int * 4), ("schedule", ctypes.c_void_p)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_trees", ctypes.c_int), ("n_nodes", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("n_ghosts", ctypes.c_int64), ("n_items", ctypes.c_int64), ("precision", ctypes.c_int),
                ("terms_per_chunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("heavy_first", ctypes.c_int),
                ("tuned", ctypes.c_int), ("ms_variant", ctypes.c_float * 10), ("graph", ctypes.c_int),
                ("graph_kernels", ctypes.c_int), ("ms_screen", ctypes.c_float),
                ("n_items_lowp", ctypes.c_int64), ("screen_mode", ctypes.c_int), ("n_misses", ctypes.c_int64),
                ("n_pairs_empty", ctypes.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["ms_variant"] = list(self.ms_variant)
        return d


_lib = None
_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)

SIGNATURES = {
    "mra_build_tree": [ctypes.POINTER(Density), ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                       ctypes.c_int, ctypes.POINTER(Alloc), _P, ctypes.POINTER(_P)],
    "mra_tree_import": [ctypes.c_int, ctypes.c_int, _I32P, _I32P, _DP, ctypes.POINTER(Alloc), _P,
                        ctypes.POINTER(_P)],
    "mra_tree_export": [_P, _I32P, _I32P, _DP, _DP, _P],
    "mra_tree_get_info": [_P, ctypes.POINTER(TreeInfo)],
    "mra_tree_device_arrays": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)],
    "mra_tree_set_blocks": [_P, _P, _P],
    "mra_compress": [_P, ctypes.c_int, _P],
    "mra_tree_refine": [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int)],
    "mra_tree_multiply": [_P, ctypes.POINTER(PotentialC), ctypes.c_double, _P, ctypes.POINTER(_P)],
    "mra_tree_dot": [_P, _P, _P, _DP],
    "mra_tree_scale": [_P, ctypes.c_double, _P],
    "mra_kalos_step": [_P, ctypes.POINTER(PotentialC), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                       ctypes.c_int, ctypes.POINTER(ApplyOpts), ctypes.POINTER(_P), _P, ctypes.POINTER(_P),
                       ctypes.POINTER(KalosInfo)],
    "mra_op_retune": [_P, ctypes.c_double, _P],
    "mra_build_tree2": [ctypes.POINTER(Density), ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                        ctypes.c_int, ctypes.POINTER(Alloc), _P, ctypes.POINTER(_P)],
    "mra_tree2_import": [ctypes.c_int, ctypes.c_int, _I32P, _I32P, _DP, ctypes.POINTER(Alloc), _P,
                         ctypes.POINTER(_P)],
    "mra_tree2_export": [_P, _I32P, _I32P, _DP, _DP, _P],
    "mra_tree2_get_info": [_P, ctypes.POINTER(TreeInfo)],
    "mra_compress2": [_P, _P],
    "mra_make_operator2": [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(Alloc), _P, ctypes.POINTER(_P)],
    "mra_apply_ns2": [_P, _P, _P, ctypes.POINTER(_P), ctypes.POINTER(ApplyStats)],
    "mra_reconstruct2": [_P, ctypes.c_int, ctypes.c_double, _P, _DP],
    "mra_free_tree2": [_P],
    "mra_make_operator": [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                          ctypes.POINTER(Alloc), _P, ctypes.POINTER(_P)],
    "mra_op_get_info": [_P, ctypes.POINTER(OpInfo)],
    "mra_op_export": [_P, _DP, _DP, _DP, _DP, _DP, _P],
    "mra_apply_ns": [_P, _P, ctypes.POINTER(ApplyOpts), _P, ctypes.POINTER(_P), ctypes.POINTER(ApplyStats)],
    "mra_apply_ns_noalloc": [_P, _P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_int64)],
    "mra_reconstruct": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _DP],
    "mra_plan_create": [_P, ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(PlanOpts), _P, ctypes.POINTER(_P)],
    "mra_plan_execute": [_P, _P],
    "mra_plan_autotune": [_P, ctypes.c_int, _P],
    "mra_plan_set_variant": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "mra_plan_output": [_P, ctypes.c_int, _P, ctypes.POINTER(_P)],
    "mra_plan_get_info": [_P, ctypes.POINTER(PlanInfo), _P],
    "mra_plan_tree_stats": [_P, ctypes.c_int, _P, ctypes.POINTER(ApplyStats)],
    "mra_free_plan": [_P],
    "mra_mlp_create": [ctypes.c_int, ctypes.c_int, _FP, ctypes.c_ulonglong, ctypes.POINTER(Alloc), _P,
                       ctypes.POINTER(_P)],
    "mra_mlp_num_params": [_P, ctypes.POINTER(ctypes.c_int64)],
    "mra_mlp_get_params": [_P, _FP, _P],
    "mra_mlp_set_params": [_P, _FP, _P],
    "mra_mlp_forward": [_P, _P, ctypes.c_int64, _P, _P],
    "mra_mlp_loss_grad": [_P, _P, _P, ctypes.c_int64, _FP, _DP, _P],
    "mra_mlp_train_step": [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P, _DP],
    "mra_mlp_free": [_P],
    "mra_screen_data": [_P, _P, _P, _P, _P],
    "mra_free": [_P],
    "mra_free_tree": [_P],
    "mra_free_op": [_P],
    "mra_last_error": [],
    "mra_version": [],
    "mra_kernel_launches": [],
    "mra_release_cached": [],
}


def lib():
    """Load libmra_gb300.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_0706_0747_gb300/build.py "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            if name in ("mra_last_error", "mra_version"):
                fn.restype = ctypes.c_char_p
            elif name == "mra_kernel_launches":
                fn.restype = ctypes.c_ulonglong
            elif name == "mra_release_cached":
                fn.restype = ctypes.c_size_t
            else:
                fn.restype = ctypes.c_int
        _lib = L
    return _lib


def symbols_declared():
    return sorted(SIGNATURES)


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise MraError(rc, lib().mra_last_error().decode())
    return rc


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------- allocator hook
_torch_hook = None


def torch_allocator():
    """An mra_alloc hook backed by torch's CUDA caching allocator (or None)."""
    global _torch_hook
    if _torch_hook is not None:
        return _torch_hook
    try:
        import torch
        if not torch.cuda.is_available():
            return None
    except ImportError:
        return None

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    hook = Alloc(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _torch_hook = hook
    return hook


def _alloc_ptr(allocator):
    if allocator == "torch":
        h = torch_allocator()
        return ctypes.byref(h) if h is not None else None
    if allocator is None:
        return None
    return ctypes.byref(allocator)


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_I32P)


# ----------------------------------------------------------- handles
class Tree:
    def __init__(self, handle, keepalive=None):
        self.h = handle
        self._keep = keepalive

    def info(self):
        inf = TreeInfo()
        _check(lib().mra_tree_get_info(self.h, ctypes.byref(inf)))
        return inf

    @property
    def n(self):
        return self.info().n_nodes

    def export(self, stream=None, out=None):
        """(coords, leaf, blocks, dnorm) as host arrays; ``out`` may give
        arrays (e.g. in pinned memory) with room for them, filled in place."""
        inf = self.info()
        n, k = inf.n_nodes, inf.k
        if out is None:
            coords = np.zeros((n, 4), dtype=np.int32)
            leaf = np.zeros(n, dtype=np.int32)
            blocks = np.zeros((n, k, k, k))
            dnorm = np.zeros(n)
        else:
            coords, leaf, blocks, dnorm = (a.reshape(-1)[:m].reshape(shp) for a, m, shp in
                                           zip(out, (4 * n, n, n * k ** 3, n), ((n, 4), (n,), (n, k, k, k), (n,))))
        _check(lib().mra_tree_export(self.h, _ip(coords), _ip(leaf), _dp(blocks), _dp(dnorm), _stream(stream)))
        return coords, leaf, blocks, dnorm

    def device_arrays(self):
        b, l = _P(), _P()
        _check(lib().mra_tree_device_arrays(self.h, ctypes.byref(b), ctypes.byref(l)))
        return b.value, l.value

    def free(self):
        if self.h:
            lib().mra_free_tree(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Operator:
    def __init__(self, handle):
        self.h = handle

    def info(self):
        inf = OpInfo()
        _check(lib().mra_op_get_info(self.h, ctypes.byref(inf)))
        return inf

    def export(self, stream=None):
        inf = self.info()
        M, k, J = inf.M, inf.k, inf.max_level
        w, tau = np.zeros(M), np.zeros(M)
        F = np.zeros((J + 1, M, 7, k, k))
        nF = np.zeros((J + 1, M, 7))
        est = np.zeros((J + 1, M))
        _check(lib().mra_op_export(self.h, _dp(w), _dp(tau), _dp(F), _dp(nF), _dp(est), _stream(stream)))
        return dict(w=w, tau=tau, F=F, nF=nF, est=est)

    def free(self):
        if self.h:
            lib().mra_free_op(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ----------------------------------------------------------- entry points
def build_tree(density, k, eps, max_level, uniform_level=-1, init_level=0, stream=None, allocator="torch"):
    """mra_build_tree; density has coef, expo, centers (n,3), r2coef.  Returns
    (Tree, depth_hit)."""
    coef = np.ascontiguousarray(density.coef, dtype=np.float64)
    expo = np.ascontiguousarray(density.expo, dtype=np.float64)
    cen = np.ascontiguousarray(np.asarray(density.centers, dtype=np.float64).reshape(-1))
    r2 = np.ascontiguousarray(getattr(density, "r2coef", np.zeros_like(coef)), dtype=np.float64)
    d = Density(len(coef), _dp(coef), _dp(r2), _dp(expo), _dp(cen))
    h = _P()
    rc = lib().mra_build_tree(ctypes.byref(d), k, eps, max_level, uniform_level, init_level,
                              _alloc_ptr(allocator), _stream(stream), ctypes.byref(h))
    _check(rc, allow=(EDEPTH,))
    return Tree(h.value), rc == EDEPTH


def tree_import(k, coords, leaf, blocks, stream=None, allocator="torch"):
    coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 4)
    leaf = np.ascontiguousarray(leaf, dtype=np.int32)
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    h = _P()
    _check(lib().mra_tree_import(k, len(coords), _ip(coords), _ip(leaf), _dp(blocks), _alloc_ptr(allocator),
                                 _stream(stream), ctypes.byref(h)))
    return Tree(h.value)


def tree_set_blocks(tree, device_ptr, stream=None):
    """Overwrite the tree's blocks from device memory (n k^3 doubles)."""
    _check(lib().mra_tree_set_blocks(tree.h, device_ptr, _stream(stream)))


def tree_refine(tree, passes=1, max_level=MAX_LEVEL, stream=None):
    """mra_tree_refine: a new tree with the graded output skeleton (the same
    function); returns (Tree, leaves split)."""
    h = _P()
    ns = ctypes.c_int(0)
    _check(lib().mra_tree_refine(tree.h, int(passes), int(max_level), _stream(stream), ctypes.byref(h),
                                 ctypes.byref(ns)))
    return Tree(h.value), ns.value


class Potential:
    """V(x) = sum_g (coef_g + r2coef_g |x - c_g|^2) exp(-expo_g |x - c_g|^2)
    + sum_n charges_n / |x - positions_n| (unit-cube coordinates)."""

    def __init__(self, coef=(), expo=(), centers=(), r2coef=None, charges=(), positions=()):
        self.coef = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1))
        self.expo = np.ascontiguousarray(np.asarray(expo, dtype=np.float64).reshape(-1))
        self.centers = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1))
        self.r2coef = (np.zeros_like(self.coef) if r2coef is None
                       else np.ascontiguousarray(np.asarray(r2coef, dtype=np.float64).reshape(-1)))
        self.charges = np.ascontiguousarray(np.asarray(charges, dtype=np.float64).reshape(-1))
        self.positions = np.ascontiguousarray(np.asarray(positions, dtype=np.float64).reshape(-1))

    def c_struct(self):
        """The mra_potential view of the arrays (valid while self lives)."""
        def p(a):
            return _dp(a) if len(a) else None
        return PotentialC(len(self.coef), p(self.coef), p(self.r2coef), p(self.expo), p(self.centers),
                          len(self.charges), p(self.charges), p(self.positions))


def tree_multiply(tree, potential, scale=1.0, stream=None):
    """mra_tree_multiply: scale * (V f) projected leaf by leaf on f's skeleton."""
    v = potential.c_struct()
    h = _P()
    _check(lib().mra_tree_multiply(tree.h, ctypes.byref(v), float(scale), _stream(stream), ctypes.byref(h)))
    return Tree(h.value)


def tree_dot(a, b, stream=None):
    """mra_tree_dot: <a, b> over the unit cube (same skeleton)."""
    out = ctypes.c_double(0.0)
    _check(lib().mra_tree_dot(a.h, b.h, _stream(stream), ctypes.byref(out)))
    return out.value


def tree_scale(tree, alpha, stream=None):
    _check(lib().mra_tree_scale(tree.h, float(alpha), _stream(stream)))


class Tree2:
    """A tree of the d = 2 variant (mra_tree2): k x k blocks on the unit square."""

    def __init__(self, handle):
        self.h = handle

    def info(self):
        inf = TreeInfo()
        _check(lib().mra_tree2_get_info(self.h, ctypes.byref(inf)))
        return inf

    @property
    def n(self):
        return self.info().n_nodes

    def export(self, stream=None):
        """(coords (n, 3), leaf (n,), blocks (n, k, k), dnorm (n,)) on the host."""
        inf = self.info()
        n, k = inf.n_nodes, inf.k
        coords = np.zeros((n, 3), dtype=np.int32)
        leaf = np.zeros(n, dtype=np.int32)
        blocks = np.zeros((n, k, k))
        dnorm = np.zeros(n)
        _check(lib().mra_tree2_export(self.h, _ip(coords), _ip(leaf), _dp(blocks), _dp(dnorm), _stream(stream)))
        return coords, leaf, blocks, dnorm

    def free(self):
        if self.h:
            lib().mra_free_tree2(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_tree2(density, k, eps, max_level, uniform_level=-1, init_level=0, stream=None, allocator="torch"):
    """mra_build_tree2 (Algorithm 1 in d = 2); density.centers is (n, 2).
    Returns (Tree2, depth_hit)."""
    coef = np.ascontiguousarray(density.coef, dtype=np.float64)
    expo = np.ascontiguousarray(density.expo, dtype=np.float64)
    cen = np.ascontiguousarray(np.asarray(density.centers, dtype=np.float64).reshape(-1))
    r2 = np.ascontiguousarray(getattr(density, "r2coef", np.zeros_like(coef)), dtype=np.float64)
    d = Density(len(coef), _dp(coef), _dp(r2), _dp(expo), _dp(cen))
    h = _P()
    rc = lib().mra_build_tree2(ctypes.byref(d), k, eps, max_level, uniform_level, init_level,
                               _alloc_ptr(allocator), _stream(stream), ctypes.byref(h))
    _check(rc, allow=(EDEPTH,))
    return Tree2(h.value), rc == EDEPTH


def tree2_import(k, coords, leaf, blocks, stream=None, allocator="torch"):
    coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 3)
    leaf = np.ascontiguousarray(leaf, dtype=np.int32)
    blocks = np.ascontiguousarray(blocks, dtype=np.float64)
    h = _P()
    _check(lib().mra_tree2_import(k, len(coords), _ip(coords), _ip(leaf), _dp(blocks), _alloc_ptr(allocator),
                                  _stream(stream), ctypes.byref(h)))
    return Tree2(h.value)


def compress2(tree, stream=None):
    _check(lib().mra_compress2(tree.h, _stream(stream)))


def make_operator2(mu, alpha, eps, k, max_level, stream=None, allocator="torch"):
    """mra_make_operator2: K_{mu,alpha} in R^2 (0 < alpha < 1)."""
    h = _P()
    _check(lib().mra_make_operator2(mu, alpha, eps, k, max_level, _alloc_ptr(allocator), _stream(stream),
                                    ctypes.byref(h)))
    return Operator(h.value)


def apply_ns2(op, tree, stream=None):
    """mra_apply_ns2 (Algorithm 3 in d = 2, FP64): (ns-form Tree2, stats)."""
    st = ApplyStats()
    h = _P()
    _check(lib().mra_apply_ns2(op.h, tree.h, _stream(stream), ctypes.byref(h), ctypes.byref(st)))
    return Tree2(h.value), st.as_dict()


def reconstruct2(tree, truncate=False, eps=0.0, stream=None):
    rem = ctypes.c_double(0.0)
    _check(lib().mra_reconstruct2(tree.h, int(truncate), eps, _stream(stream), ctypes.byref(rem)))
    return rem.value


COMPRESS_NORMS, COMPRESS_STORE_D, COMPRESS_SCALING = 0, 1, 2


def compress(tree, store_d=False, stream=None, norms=True):
    """mra_compress: store_d keeps the wavelet cubes (mode MRA_COMPRESS_STORE_D);
    norms=False computes the scaling blocks only (MRA_COMPRESS_SCALING), all that
    apply_ns reads of its input."""
    mode = COMPRESS_STORE_D if store_d else (COMPRESS_NORMS if norms else COMPRESS_SCALING)
    _check(lib().mra_compress(tree.h, mode, _stream(stream)))


def make_operator(mu, alpha, eps, k, max_level, stream=None, allocator="torch"):
    h = _P()
    _check(lib().mra_make_operator(mu, alpha, eps, k, max_level, _alloc_ptr(allocator), _stream(stream),
                                   ctypes.byref(h)))
    return Operator(h.value)


def apply_ns(op, tree, precision="fp64", block_screen=False, unscreened=False, itemwise=False, stream=None,
             stats=True, screen="static", schedule=None, margin=2, wait_limit=0, test_flags=0):
    """mra_apply_ns.  screen: "static" (Sec. 4's ranges), "pair" (exact
    per-pair ranges) or "learned" (the network ``schedule``'s cut-offs, judged
    by the exact test).  wait_limit / test_flags: the tensor-core apply's
    bounded completion waits (0 = defaults)."""
    o = ApplyOpts(PREC[precision], int(block_screen), int(unscreened), int(itemwise), SCREEN[screen], int(margin),
                  int(wait_limit), int(test_flags))
    if schedule is not None:
        o.schedule = schedule.h
    st = ApplyStats()
    h = _P()
    _check(lib().mra_apply_ns(op.h, tree.h, ctypes.byref(o), _stream(stream), ctypes.byref(h),
                              ctypes.byref(st) if stats else None))
    return Tree(h.value), (st.as_dict() if stats else None)


class OpCache:
    """An operator handle kept between Kalos steps (mra_kalos_step's
    op_cache); freed with the object."""

    def __init__(self):
        self.h = _P()

    def free(self):
        if self.h.value:
            lib().mra_free(self.h)
            self.h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def op_retune(op, mu, stream=None):
    """mra_op_retune: new weights for mu on op's term grid."""
    _check(lib().mra_op_retune(op.h, float(mu), _stream(stream)))


def kalos_step(phi, potential, length, mu, eps, max_level, precision="fp64", screen="static", op_cache=None,
               stream=None):
    """mra_kalos_step: one pass of phi = -2 G_mu V phi; returns (phi_next,
    info dict with energy, mu_next, norm_new, n_terms, op_rebuilt, n_items,
    ms_apply).  op_cache: an OpCache reused across steps, or None."""
    v = potential.c_struct()
    o = ApplyOpts(PREC[precision], 0, 0, 0, SCREEN[screen], 2, 0, 0)
    info = KalosInfo()
    h = _P()
    _check(lib().mra_kalos_step(phi.h, ctypes.byref(v), float(length), float(mu), float(eps), int(max_level),
                                ctypes.byref(o), ctypes.byref(op_cache.h) if op_cache is not None else None,
                                _stream(stream), ctypes.byref(h), ctypes.byref(info)))
    return Tree(h.value), {f: getattr(info, f) for f, _ in KalosInfo._fields_}


def apply_ns_noalloc(op, tree, out_ptr, precision="fp64", stream=None):
    """mra_apply_ns_noalloc: writes ghat into caller-owned device memory at
    out_ptr (n_nodes * k^3 doubles); returns the item count."""
    n = ctypes.c_int64(0)
    _check(lib().mra_apply_ns_noalloc(op.h, tree.h, PREC[precision], out_ptr, _stream(stream), ctypes.byref(n)))
    return n.value


class Plan:
    """Batched apply of one operator to many trees (mra_plan_*).  Keeps the
    operator and the trees alive for its own lifetime."""

    def __init__(self, handle, op, trees):
        self.h = handle
        self._op = op
        self._trees = list(trees)

    def execute(self, stream=None):
        _check(lib().mra_plan_execute(self.h, _stream(stream)))

    def autotune(self, reps=3, stream=None):
        _check(lib().mra_plan_autotune(self.h, int(reps), _stream(stream)))
        return self.info(stream)

    def set_variant(self, terms_per_chunk=8, ctas_per_sm=2, heavy_first=False):
        _check(lib().mra_plan_set_variant(self.h, int(terms_per_chunk), int(ctas_per_sm), int(heavy_first)))

    def output(self, b, stream=None):
        h = _P()
        _check(lib().mra_plan_output(self.h, int(b), _stream(stream), ctypes.byref(h)))
        return Tree(h.value)

    def info(self, stream=None):
        inf = PlanInfo()
        _check(lib().mra_plan_get_info(self.h, ctypes.byref(inf), _stream(stream)))
        return inf.as_dict()

    def tree_stats(self, b, stream=None):
        st = ApplyStats()
        _check(lib().mra_plan_tree_stats(self.h, int(b), _stream(stream), ctypes.byref(st)))
        return st.as_dict()

    def free(self):
        if self.h:
            lib().mra_free_plan(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def plan_create(op, trees, precision=None, use_graph=True, stream=None, screen="static", schedule=None, margin=2):
    """mra_plan_create over compressed trees (all of op's order k); screen
    "static", "pair" (exact per-pair ranges fixed at creation) or "learned"
    (the network ``schedule``'s ranges, every miss restored at creation)."""
    arr = (_P * len(trees))(*[t.h for t in trees])
    opts = None
    if precision is not None or not use_graph or screen != "static":
        k = op.info().k
        prec = PREC[precision] if precision is not None else (PREC["tc"] if k <= 8 else PREC["fp64"])
        po = PlanOpts(prec, int(use_graph), SCREEN[screen], int(margin))
        if schedule is not None:
            po.schedule = schedule.h
        opts = ctypes.byref(po)
    h = _P()
    _check(lib().mra_plan_create(op.h, arr, len(trees), opts, _stream(stream), ctypes.byref(h)))
    return Plan(h.value, op, trees)


class Mlp:
    """The learned schedule's network (mra_mlp_*).  Device arrays are passed
    as torch CUDA float32 tensors (contiguous, row-major)."""

    def __init__(self, handle):
        self.h = handle

    @property
    def n_params(self):
        n = ctypes.c_int64(0)
        _check(lib().mra_mlp_num_params(self.h, ctypes.byref(n)))
        return n.value

    def get_params(self, stream=None):
        out = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().mra_mlp_get_params(self.h, out.ctypes.data_as(_FP), _stream(stream)))
        return out

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().mra_mlp_set_params(self.h, p.ctypes.data_as(_FP), _stream(stream)))

    def forward(self, x, y, stream=None):
        _check(lib().mra_mlp_forward(self.h, x.data_ptr(), x.shape[0], y.data_ptr(), _stream(stream)))

    def loss_grad(self, x, target, stream=None):
        g = np.zeros(self.n_params, dtype=np.float32)
        L = ctypes.c_double(0.0)
        _check(lib().mra_mlp_loss_grad(self.h, x.data_ptr(), target.data_ptr(), x.shape[0], g.ctypes.data_as(_FP),
                                       ctypes.byref(L), _stream(stream)))
        return L.value, g

    def train_step(self, x, target, lr, stream=None, want_loss=False):
        L = ctypes.c_double(0.0)
        _check(lib().mra_mlp_train_step(self.h, x.data_ptr(), target.data_ptr(), x.shape[0], float(lr),
                                        _stream(stream), ctypes.byref(L) if want_loss else None))
        return L.value if want_loss else None

    def free(self):
        if self.h:
            lib().mra_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mlp_create(n_in=16, n_out=12, params=None, seed=0, stream=None, allocator="torch"):
    p = None
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float32)
        p = params.ctypes.data_as(_FP)
    h = _P()
    _check(lib().mra_mlp_create(int(n_in), int(n_out), p, int(seed), _alloc_ptr(allocator), _stream(stream),
                                ctypes.byref(h)))
    return Mlp(h.value)


def screen_data(op, tree, inputs=None, targets=None, stream=None):
    """mra_screen_data into torch CUDA float32 tensors [n, 16] / [n, 12]
    (allocated when not given); returns (inputs, targets)."""
    import torch
    n = tree.n
    if inputs is None:
        inputs = torch.empty((n, 16), dtype=torch.float32, device="cuda")
    if targets is None:
        targets = torch.empty((n, 12), dtype=torch.float32, device="cuda")
    _check(lib().mra_screen_data(op.h, tree.h, inputs.data_ptr(), targets.data_ptr(), _stream(stream)))
    return inputs, targets


def reconstruct(tree, mode="assemble", truncate=False, eps=0.0, stream=None):
    rem = ctypes.c_double(0.0)
    m = {"assemble": 0, "inverse": 1}[mode]
    _check(lib().mra_reconstruct(tree.h, m, int(truncate), eps, _stream(stream), ctypes.byref(rem)))
    return rem.value


def free(handle):
    """mra_free on a handle object (Tree, Operator, Plan, Mlp) or a raw
    handle pointer; the object forgets its handle."""
    h = getattr(handle, "h", handle)
    if h:
        _check(lib().mra_free(h))
    if hasattr(handle, "h"):
        handle.h = None


def kernel_launches():
    return int(lib().mra_kernel_launches())


def release_cached():
    """mra_release_cached: return the library's cached device blocks to their
    allocator hooks; the number of bytes released."""
    return int(lib().mra_release_cached())


def version():
    return lib().mra_version().decode()


def last_error():
    return lib().mra_last_error().decode()
