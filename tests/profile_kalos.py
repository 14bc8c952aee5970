"""Profiling driver (not a test): the hydrogen ground-state iteration of
Sec. 6.2 at full size (k = 8, eps = 1e-6, depth 12, a 32-bohr cube) through
the C ABI, `steps` Kalos steps with the operator kept in a cache and
re-weighted each step; prints per-step wall time and energy.  Usage:
python tests/profile_kalos.py [precision] [steps]."""
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import torch  # noqa: E402

from paper_0706_0747_gb300 import mra, workloads as W  # noqa: E402


def main(prec="tc", steps="6"):
    hc = W.hydrogen()
    phi, _ = mra.build_tree(hc.start_density(), hc.k, hc.eps, hc.max_level, init_level=hc.init_level)
    mra.tree_scale(phi, 1.0 / math.sqrt(mra.tree_dot(phi, phi) * hc.L ** 3))
    pot = mra.Potential(charges=[-1.0 / hc.L], positions=[hc.u0])
    mu, cache = hc.mu0, mra.OpCache()
    for it in range(int(steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phi, info = mra.kalos_step(phi, pot, hc.L, mu, hc.eps, hc.max_level, precision=prec, op_cache=cache)
        torch.cuda.synchronize()
        print(it, "ms %.3f" % (1e3 * (time.perf_counter() - t0)), "E %.10f" % info["energy"], flush=True)
        mu = info["mu_next"]


if __name__ == "__main__":
    main(*sys.argv[1:3])
