"""Profiling driver (not a test): two applies on the 3-D Poisson k = 8 tree
through the C ABI, each followed by assembly and truncation; ncu captures the
second apply's kernel.  Usage: python tests/profile_apply.py [precision] [screen]."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_0706_0747_gb300 import mra, workloads as W  # noqa: E402


def main(prec="tc", screen="static"):
    cfg, dens = W.poisson_k8()
    op = mra.make_operator(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    tree, _ = mra.build_tree(dens, cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    mra.compress(tree, norms=False)
    st = None
    for _ in range(2):
        g, st = mra.apply_ns(op, tree, precision=prec, screen=screen)
        mra.reconstruct(g, mode="assemble", truncate=True, eps=cfg.eps)
        g.free()
    torch.cuda.synchronize()
    print("ok", st["n_items"], st["ms_apply"])


if __name__ == "__main__":
    main(*sys.argv[1:3])
