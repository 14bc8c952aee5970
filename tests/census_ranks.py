"""Census of the numerical rank of the operator blocks F^{j;m,t} that the
static screen's items use (the evidence for leaving a rank-structured apply
out): per item (a, t, m), sum_d sigma_2/sigma_1 of its three 1-D blocks
bounds the relative error of replacing each block by its best rank-one
approximation, and the script prints the share of items below several
tolerances.  Oracle only (FP64 numpy); a few minutes for the small workloads.

    python tests/census_ranks.py poisson_small
    python tests/census_ranks.py helmholtz_slater
"""
import sys

import numpy as np

sys.path.insert(0, __file__.rsplit("/tests/", 1)[0])

from oracle import apply as OA  # noqa: E402
from oracle import operator as OO  # noqa: E402
from oracle import tree as OT  # noqa: E402
from paper_0706_0747_gb300 import workloads as W  # noqa: E402


def census(name):
    cfg, dens = getattr(W, name)()
    op = OO.Operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    od = OT.Density(dens.coef, dens.expo, dens.centers, dens.r2coef)
    tree, _ = OT.build_tree(od, cfg.k, cfg.eps, cfg.max_level, uniform_level=cfg.uniform_level,
                            init_level=cfg.init_level)
    OT.compress(tree, cfg.k)
    sv = np.linalg.svd(op.F, compute_uv=False)                  # (J+1, M, 7, k)
    r1 = sv[..., 1] / np.maximum(sv[..., 0], 1e-300)            # sigma_2 / sigma_1
    sch = OA.Schedule(op, OA.pilot_sigma(op, tree), OT.norm2(tree), OT.levels(tree))
    tols = (1e-2, 1e-4, 1e-6, 1e-8)
    below = dict.fromkeys(tols, 0)
    total = 0
    for key in tree:
        j, a = key[0], key[1:]
        for t in OA.band(a):
            b = tuple(a[d] - t[d] for d in range(3))
            if min(b) < 0 or max(b) >= 2 ** j:
                continue
            for m in sch.terms(j, t, tree[key].leaf):
                e = r1[j, m, t[0] + 3] + r1[j, m, t[1] + 3] + r1[j, m, t[2] + 3]
                total += 1
                for tol in tols:
                    below[tol] += e <= tol
    return cfg, op, total, below


if __name__ == "__main__":
    for name in sys.argv[1:] or ["poisson_small"]:
        cfg, op, total, below = census(name)
        share = ", ".join(f"<= {tol:g}: {below[tol] / total:.4f}" for tol in sorted(below, reverse=True))
        print(f"{cfg.name}: M = {op.M}, {total} items; share of items whose rank-one error bound is {share}")
