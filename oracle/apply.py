"""Oracle: Algorithm 3 -- adaptive modified ns-form apply in d = 3 -- and the
adaptive projection of eq. g_assemble (Secs. 2.3, 4, 5).

Test infrastructure only (see ``oracle/__init__``).

Notation: output box a at level j, input box b = a - t, translation t in Z^3,
terms m = 0..M-1 (tau increasing with m).  For each kept item (a, t, m),
    ghat^j_a += w_m (F^{j;m,t1} x F^{j;m,t2} x F^{j;m,t3}) f^j_{a-t}
(eqs. KernelApproxByGaussians2 / sep_apply and the sum of Algorithm 3, Step 3).

Band (eq. fine_scale_band with b_j = 3, per direction): t_d in [-3, 2] when
a_d is even and [-2, 3] when a_d is odd -- the fine translations whose coarse
parents lie in the coarse core |L| <= 1 = floor(b_j / 2) (eq. down_band).
Translations whose input box leaves [0, 2^j)^3 are dropped (f = 0 outside B).

Readings of the passages the paper leaves open:

* Threshold scale.  The paper's thresholds are "below eps"; here they are
  relative: eta = eps * ||T_0 f_0|| / ||f||, where T_0 f_0 is the level-0
  apply of all M terms to the root block (a one-block pilot of ||g||), so the
  dropped contributions are a fraction eps of the output's scale.
* Term activity across scales (Sec. 4, eq. sep_apply): J_m is the finest
  scale j >= 1 at which w_m * max_{L in {-1,0,1}^3} Est(j, m, L) > eta / M
  (Est: eq. NormEstimateUsing1DBlocks), or 0.  Term m is applied at scales
  j <= J_m only.  At an internal node of scale j < J_m the core |t|_inf <= 1
  is left to the finer scale (outer band, eq. apply_algo); at a leaf, or at
  j = J_m, the whole band is applied.  This keeps the telescoping exact per
  term: a term whose scale-to-scale differences are negligible below J_m is
  applied once, whole-band, at J_m and reaches finer scales through the
  projection of eq. g_assemble.
* Subset ranges (Sec. 4, Core / Boundary-1/2/3 by the number of directions
  with |t_d| <= 1): for each scale j and subset S, e_m = w_m * prod_d
  max_{t_d in class} nF(j, m, t_d) over the terms with J_m >= j; [m1, m2]
  trims from each end the terms whose cumulative e_m stays <= eta / (2 * 216).
* Optional per-block screen (``block_screen=True``, the per-block check the
  paper avoids): an item is also dropped when w_m prod_d nF(j,m,t_d)
  ||f_{a-t}|| <= eps ||T_0 f_0|| / sqrt(N_nodes * 216 * M).
* Optional per-pair screen (``pair_screen=True``): the same per-item test
  decides a term range per (output box, translation) pair -- from the first
  to the last term that passes it -- and every term of the static schedule
  inside that range is applied (a pair with no passing term is dropped).
  This is the exact norm screen that judges the learned schedule's per-box
  cut-offs, and ``screen_data`` returns its per-box targets.
* Step 2: a missing input block is refined from its ancestor leaf with the
  d = 0 half of eqs. recon_even / recon_odd and cached.
* Output skeleton: a copy of the input's redundant tree (Algorithm 2/3,
  Initialization).
* Final truncation: after assembly and compression, an internal node whose 8
  children are leaves is merged when ||d|| < eps ||g|| / sqrt(N_nodes),
  repeated bottom-up; the removed l2 mass is reported.
"""
import itertools

import numpy as np

from . import tree as T

BAND_EVEN = (-3, -2, -1, 0, 1, 2)
BAND_ODD = (-2, -1, 0, 1, 2, 3)


def band(a):
    return itertools.product(*[(BAND_EVEN if a[d] % 2 == 0 else BAND_ODD) for d in range(3)])


class Schedule:
    """Per-apply screening tables (J_m and [m1, m2] per scale and subset)."""

    def __init__(self, op, sigma, fnorm, nlev, screen=True):
        M = op.M
        self.eta = op.eps * sigma / fnorm if fnorm > 0 else 0.0
        if not screen:
            # every term at every scale, whole ranges: band truncation only
            self.Jm = np.full(M, nlev - 1, dtype=np.int64)
            self.m1 = np.zeros((nlev, 4), dtype=np.int64)
            self.m2 = np.full((nlev, 4), M - 1, dtype=np.int64)
            return
        self.Jm = np.zeros(M, dtype=np.int64)
        for m in range(M):
            for j in range(1, nlev):
                if op.w[m] * op.est_core[j, m] > self.eta / M:
                    self.Jm[m] = j
        nFc = op.nF[:, :, 2:5].max(axis=2)                       # |t| <= 1
        nFb = np.maximum(op.nF[:, :, [0, 1, 5, 6]].max(axis=2), 0.0)  # 2 <= |t| <= 3
        self.m1 = np.zeros((nlev, 4), dtype=np.int64)
        self.m2 = np.full((nlev, 4), -1, dtype=np.int64)
        budget = self.eta / (2.0 * 216.0)
        for j in range(nlev):
            cand = [m for m in range(M) if self.Jm[m] >= j]
            for S in range(4):                                    # S = number of core dims
                if not cand:
                    continue
                e = [op.w[m] * nFc[j, m] ** S * nFb[j, m] ** (3 - S) for m in cand]
                lo, acc = 0, 0.0
                while lo < len(cand) and acc + e[lo] <= budget:
                    acc += e[lo]
                    lo += 1
                hi, acc = len(cand) - 1, 0.0
                while hi >= lo and acc + e[hi] <= budget:
                    acc += e[hi]
                    hi -= 1
                if hi >= lo:
                    self.m1[j, S] = cand[lo]
                    self.m2[j, S] = cand[hi]

    def terms(self, j, t, leaf):
        S = sum(1 for v in t if abs(v) <= 1)
        core = S == 3
        out = []
        for m in range(self.m1[j, S], self.m2[j, S] + 1):
            if self.Jm[m] < j:
                continue
            if core and not leaf and self.Jm[m] > j:
                continue
            out.append(m)
        return out


def separated_apply(w, F1, F2, F3, x):
    """sum_m w_m (F1_m x F2_m x F3_m) x as three mode products (direction 3,
    then 2, then 1, the last one also summing over m).  Shapes: w (M,),
    F* (M, k, k), x (k, k, k)."""
    k = x.shape[0]
    M = len(w)
    z = x.reshape(k * k, k) @ F3.transpose(0, 2, 1)            # (M, k*k, k): [m, (i,j), c]
    z = F2[:, None] @ z.reshape(M, k, k, k)                     # (M, k, k, k): [m, i, b, c]
    wF1 = (w[:, None, None] * F1).transpose(1, 0, 2).reshape(k, M * k)
    return (wF1 @ z.reshape(M * k, k * k)).reshape(k, k, k)


def pilot_sigma(op, tree):
    s0 = tree[(0, 0, 0, 0)].s
    F0 = op.F[0, :, 3]                                            # (M, k, k), t = 0
    g0 = separated_apply(op.w, F0, F0, F0, s0)
    return float(np.linalg.norm(g0))


class _Inputs:
    """Step 2 of Algorithm 3: input blocks at any level, refined on demand."""

    def __init__(self, tree, k):
        self.tree, self.k, self.cache = tree, k, {}
        self.n_refined = 0

    def get(self, j, b):
        key = (j,) + tuple(b)
        if key in self.tree:
            return self.tree[key].s
        if key in self.cache:
            return self.cache[key]
        for jj in range(j - 1, -1, -1):
            anc = (jj,) + tuple(v >> (j - jj) for v in b)
            if anc in self.tree:
                break
        s = self.tree[anc].s
        for lev in range(jj, j):
            sh = j - lev - 1
            p = tuple((v >> sh) & 1 for v in b)
            s = T.upsample(self.k, s, p)
        self.cache[key] = s
        self.n_refined += 1
        return s


def _pair_terms(op, j, t, ms, xn, eta_blk):
    # terms of ms whose bound w_m prod_d nF(j,m,t_d) ||x|| exceeds eta_blk
    return [m for m in ms if op.w[m] * op.nF[j, m, t[0] + 3] * op.nF[j, m, t[1] + 3]
            * op.nF[j, m, t[2] + 3] * xn > eta_blk]


def apply_ns(op, tree, block_screen=False, stats=None, nodes=None, screen=True, pair_screen=False):
    """Algorithm 3, Steps 1-3: returns ghat (dict key -> (k,k,k)) on the
    skeleton of the compressed input tree.  ``nodes`` restricts the output
    boxes (for sampled checks); all nodes by default."""
    k = op.k
    nlev = T.levels(tree)
    if nlev - 1 > op.max_level:
        raise ValueError("tree deeper than the operator tables")
    fnorm = T.norm2(tree)
    sigma = pilot_sigma(op, tree)
    sch = Schedule(op, sigma, fnorm, nlev, screen=screen)
    eta_blk = op.eps * sigma / np.sqrt(len(tree) * 216.0 * op.M) if (block_screen or pair_screen) else -1.0
    inp = _Inputs(tree, k)
    ghat = {}
    n_items = 0
    n_pairs = 0
    keys = sorted(tree.keys()) if nodes is None else list(nodes)
    for key in keys:
        j, a = key[0], key[1:]
        leaf = tree[key].leaf
        y = np.zeros((k, k, k))
        for t in band(a):
            b = tuple(a[d] - t[d] for d in range(3))
            if min(b) < 0 or max(b) >= 2 ** j:
                continue
            ms = sch.terms(j, t, leaf)
            if not ms:
                continue
            x = inp.get(j, b)
            if block_screen or pair_screen:
                keep = _pair_terms(op, j, t, ms, float(np.linalg.norm(x)), eta_blk)
                if not keep:
                    continue
                ms = keep if block_screen else [m for m in ms if keep[0] <= m <= keep[-1]]
            ms = np.array(ms)
            y += separated_apply(op.w[ms], op.F[j, ms, t[0] + 3], op.F[j, ms, t[1] + 3],
                                 op.F[j, ms, t[2] + 3], x)
            n_items += len(ms)
            n_pairs += 1
        ghat[key] = y
    if stats is not None:
        stats.update(dict(n_items=n_items, n_pairs=n_pairs, n_refined=inp.n_refined,
                          eta=sch.eta, sigma=sigma, fnorm=fnorm, Jm=sch.Jm.copy(),
                          m1=sch.m1.copy(), m2=sch.m2.copy()))
    return ghat


def screen_data(op, tree, J=None):
    """Per-box inputs and targets of the learned schedule, from the static
    screen and the exact per-pair screen on a compressed tree.

    Features (16 per box, in this order): j / J; leaf flag;
    log10(||s_a|| / eta_blk) / 10; for each class S = 0..3 the maximum and
    the sum of ||x_b|| / eta_blk over the box's static pairs of that class,
    each as log10(.) / 10 (0 when the class has no pair); the number of such
    pairs / 64 per class; mu / 2.  eta_blk = eps ||T_0 f_0|| / sqrt(N 216 M).
    Targets (12 per box): per class S, [E_S, LO_S, HI_S] with E_S = 1 when no
    term of any pair of the class passes the exact test, else 0 and the first
    / last passing term over the class's pairs divided by (M - 1) (0, 0 when
    empty).  Returns (keys, X (n, 16), Y (n, 12)) in sorted key order."""
    k, M = op.k, op.M
    J = op.max_level if J is None else J
    nlev = T.levels(tree)
    fnorm = T.norm2(tree)
    sigma = pilot_sigma(op, tree)
    sch = Schedule(op, sigma, fnorm, nlev)
    eta_blk = op.eps * sigma / np.sqrt(len(tree) * 216.0 * M)
    inp = _Inputs(tree, k)
    keys = sorted(tree.keys())
    X = np.zeros((len(keys), 16))
    Y = np.zeros((len(keys), 12))

    def lg(v):
        return np.log10(max(v, 1e-300)) / 10.0
    for r, key in enumerate(keys):
        j, a = key[0], key[1:]
        leaf = tree[key].leaf
        mx = np.zeros(4)
        sm = np.zeros(4)
        cnt = np.zeros(4)
        lo = np.full(4, M)
        hi = np.full(4, -1)
        for t in band(a):
            b = tuple(a[d] - t[d] for d in range(3))
            if min(b) < 0 or max(b) >= 2 ** j:
                continue
            ms = sch.terms(j, t, leaf)
            if not ms:
                continue
            S = sum(1 for v in t if abs(v) <= 1)
            xn = float(np.linalg.norm(inp.get(j, b)))
            mx[S] = max(mx[S], xn / eta_blk)
            sm[S] += xn / eta_blk
            cnt[S] += 1
            keep = _pair_terms(op, j, t, ms, xn, eta_blk)
            if keep:
                lo[S] = min(lo[S], keep[0])
                hi[S] = max(hi[S], keep[-1])
        X[r, 0] = j / J
        X[r, 1] = 1.0 if leaf else 0.0
        X[r, 2] = lg(float(np.linalg.norm(tree[key].s)) / eta_blk)
        for S in range(4):
            X[r, 3 + S] = lg(mx[S]) if cnt[S] else 0.0
            X[r, 7 + S] = lg(sm[S]) if cnt[S] else 0.0
            X[r, 11 + S] = cnt[S] / 64.0
            if hi[S] >= 0:
                Y[r, 3 * S + 1] = lo[S] / (M - 1)
                Y[r, 3 * S + 2] = hi[S] / (M - 1)
            else:
                Y[r, 3 * S] = 1.0
        X[r, 15] = op.mu / 2.0
    return keys, X, Y


def assemble(op, tree, ghat):
    """Eq. g_assemble: top-down, each child adds the upsampled (d = 0)
    output of its parent; returns the output tree with g on its leaves."""
    k = op.k
    out = {key: T.Node(n.leaf, ghat[key].copy()) for key, n in tree.items()}
    for j in range(T.levels(tree) - 1):
        for key, node in out.items():
            if key[0] != j or node.leaf:
                continue
            for p, ck in zip(T.OCTS, T.children(key)):
                out[ck].s += T.upsample(k, node.s, p)
    return out


def truncate(g, k, eps):
    """Discard unnecessary blocks (Algorithm 3, Step 4): compress, then merge
    leaf siblings whose parent's wavelet norm is below eps ||g|| / sqrt(N)."""
    T.compress(g, k)
    thr = eps * T.norm2(g) / np.sqrt(len(g))
    removed2 = 0.0
    for j in range(T.levels(g) - 2, -1, -1):
        for key in [kk for kk in g if kk[0] == j]:
            node = g[key]
            if node.leaf:
                continue
            ch = T.children(key)
            if all(g[c].leaf for c in ch) and node.dnorm < thr:
                removed2 += node.dnorm ** 2
                for c in ch:
                    del g[c]
                node.leaf = True
                node.d = None
    return g, float(np.sqrt(removed2))


def apply_full(op, tree, truncate_out=False, block_screen=False, stats=None, screen=True):
    """compress -> Algorithm 3 -> eq. g_assemble [-> truncation]."""
    t = T.copy_tree(tree)
    T.compress(t, op.k)
    ghat = apply_ns(op, t, block_screen=block_screen, stats=stats, screen=screen)
    g = assemble(op, t, ghat)
    if truncate_out:
        g, rem = truncate(g, op.k, op.eps)
        if stats is not None:
            stats["truncation_l2"] = rem
    return g
