"""Training and evaluation of the learned schedule.

The network (mra_mlp_*, 16 inputs -> 3 x 128 ReLU -> 12 outputs) learns, per
output box, the term cut-offs of the exact per-pair screen; the apply uses
them with the exact test as the judge of every miss (MRA_SCREEN_LEARNED).
Everything here is orchestration: trees are built, screened and applied by
the CUDA library, the inputs and targets come from mra_screen_data on the
GPU, and the network is trained by the library's own forward, backward and
Adam kernels.  Data stay on the GPU as torch tensors.

    python -m paper_0706_0747_gb300.schedule --train 2000 --heldout 200 \\
        --out paper_0706_0747_gb300/schedule_net_k8_eps1e-6.npy

trains on the seeded learned-schedule densities (16-128 unit-mass Gaussians,
log10 exponent U[2, 5], Poisson or Helmholtz mu = 1.5; seeds 5000 + i) and
evaluates on held-out seeds (5000 + 2000 + i).
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import mra, workloads as W

K, EPS, MAX_LEVEL, INIT_LEVEL = 8, 1e-6, 7, 2
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "schedule_net_k8_eps1e-6.npy")


def operators(k=K, eps=EPS, max_level=MAX_LEVEL):
    return {mu: mra.make_operator(mu, 1.0, eps, k, max_level) for mu in (0.0, 1.5)}


def dataset(ops, items, k=K, eps=EPS, max_level=MAX_LEVEL, init_level=INIT_LEVEL):
    """Inputs and targets of every node of every density's tree (torch CUDA
    float32 [n, 16] and [n, 12])."""
    import torch
    xs, ys = [], []
    for mu, d in items:
        t, _ = mra.build_tree(d, k, eps, max_level, init_level=init_level)
        mra.compress(t)
        x, y = mra.screen_data(ops[mu], t)
        xs.append(x)
        ys.append(y)
        t.free()
    return torch.cat(xs), torch.cat(ys)


def train(X, Y, epochs=4, batch=4096, lr=2e-3, seed=0, log_every=0):
    """Adam on shuffled mini-batches; the learning rate halves each epoch."""
    import torch
    net = mra.mlp_create(seed=seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = X.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=gen)
        rate = lr * 0.5 ** ep
        for s0 in range(0, n - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            want = log_every and (s0 // batch) % log_every == 0
            L = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), rate, want_loss=bool(want))
            if want:
                hist.append((ep, s0 // batch, L))
    return net, hist


def evaluate(net, ops, items, k=K, eps=EPS, max_level=MAX_LEVEL, init_level=INIT_LEVEL, precision="tc"):
    """Per held-out density: items of the static, exact-pair and learned
    screens, misses, and the apply times (device, from the library's stats)."""
    rows = []
    for mu, d in items:
        t, _ = mra.build_tree(d, k, eps, max_level, init_level=init_level)
        mra.compress(t)
        op = ops[mu]
        r = {"mu": mu, "n_gauss": int(d.n), "nodes": t.n}
        outs = {}
        for name, kw in (("static", {}), ("pair", {"screen": "pair"}),
                         ("learned", {"screen": "learned", "schedule": net})):
            g, st = mra.apply_ns(op, t, precision=precision, **kw)
            outs[name] = g.export()[2]
            g.free()
            r[f"items_{name}"] = int(st["n_items"])
            r[f"ms_apply_{name}"] = float(st["ms_apply"])
            r[f"ms_screen_{name}"] = float(st["ms_screen"] + st["ms_ghost"])
            if name == "learned":
                r["misses"] = int(st["n_misses"])
        ref = outs["static"]
        den = float((ref ** 2).sum())
        r["rel_l2_learned_vs_static"] = math.sqrt(float(((outs["learned"] - ref) ** 2).sum()) / den)
        r["rel_l2_pair_vs_static"] = math.sqrt(float(((outs["pair"] - ref) ** 2).sum()) / den)
        rows.append(r)
        t.free()
    return rows


def summary(rows):
    tot = {key: sum(r[key] for r in rows) for key in ("items_static", "items_pair", "items_learned", "misses")}
    ms = {key: sum(r[key] for r in rows) for key in ("ms_apply_static", "ms_apply_pair", "ms_apply_learned",
                                                     "ms_screen_static", "ms_screen_pair", "ms_screen_learned")}
    return {"densities": len(rows), **tot, **ms,
            "items_saved_vs_static": 1.0 - tot["items_learned"] / max(1, tot["items_static"]),
            "max_rel_l2_learned_vs_static": max(r["rel_l2_learned_vs_static"] for r in rows),
            "max_rel_l2_pair_vs_static": max(r["rel_l2_pair_vs_static"] for r in rows)}


def load(path=DEFAULT_WEIGHTS):
    return mra.mlp_create(params=np.load(path))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default="")
    args = ap.parse_args()
    import torch
    ops = operators()
    t0 = time.time()
    X, Y = dataset(ops, W.schedule_set(args.train, 0))
    torch.cuda.synchronize()
    t1 = time.time()
    net, hist = train(X, Y, epochs=args.epochs, batch=args.batch, lr=args.lr, log_every=200)
    torch.cuda.synchronize()
    t2 = time.time()
    loss_train = net.loss_grad(X[:200000].contiguous(), Y[:200000].contiguous())[0]
    del X, Y
    Xh, Yh = dataset(ops, W.schedule_set(args.heldout, 2000))
    loss_held = net.loss_grad(Xh[:200000].contiguous(), Yh[:200000].contiguous())[0]
    del Xh, Yh
    rows = evaluate(net, ops, W.schedule_set(args.heldout, 2000))
    t3 = time.time()
    np.save(args.out, net.get_params())
    rep = {"train_densities": args.train, "heldout_densities": args.heldout, "epochs": args.epochs,
           "batch": args.batch, "lr": args.lr, "s_data": t1 - t0, "s_train": t2 - t1, "s_eval": t3 - t2,
           "loss_train": loss_train, "loss_heldout": loss_held, "loss_log": hist[-20:],
           "heldout": summary(rows)}
    print(json.dumps(rep))
    if args.report:
        with open(args.report, "w") as f:
            json.dump({"report": rep, "rows": rows}, f)


if __name__ == "__main__":
    main()
