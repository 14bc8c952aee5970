"""Profiling driver (not a test): two steps of the d = 2 variant on the
full-size workload (poisson2d: k = 8, eps = 1e-6, 64 Gaussians) through the
C ABI: compress2, apply_ns2, reconstruct2 with truncation; ncu captures the
second apply's kernel.  Usage: python tests/profile_d2.py."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_0706_0747_gb300 import mra, workloads as W  # noqa: E402


def main():
    cfg, dens = W.poisson2d()
    op = mra.make_operator2(cfg.mu, cfg.alpha, cfg.eps, cfg.k, cfg.max_level)
    t, _ = mra.build_tree2(dens, cfg.k, cfg.eps, cfg.max_level, init_level=cfg.init_level)
    st = None
    for _ in range(2):
        mra.compress2(t)
        g, st = mra.apply_ns2(op, t)
        mra.reconstruct2(g, truncate=True, eps=cfg.eps)
        g.free()
    torch.cuda.synchronize()
    print("ok", st["n_items"], st["ms_apply"])


if __name__ == "__main__":
    main()
