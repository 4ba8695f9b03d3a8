"""Learned warm start vs the plain FBP-seeded initialisation (one B300).

    python -m paper_2411_04844_b300.learned_bench [--side 128] [--views 50]
        [--train 256] [--test 16] [--ns 100000] [--fit-iters 300] [--epochs 4]

1. training phantoms (seeded, 40 ellipsoids), their projections (+ noise) and
   FDK-style inputs;
2. the plain method fits every training problem from the FBP-seeded
   initialisation (batched, CUDA graph) -> targets (fitted density, mean
   log-scale per voxel);
3. the network is trained on (FDK input -> targets) with the project's own
   kernels (forward, backward, loss, Adam);
4. held-out problems are fitted twice -- plain initialisation and learned
   initialisation -- and compared on the iterations and the wall time each
   needs to reach the plain fit's final PSNR (within 0.1 dB).
Prints one JSON line.
"""
import argparse
import json
import math
import sys
import time

import numpy as np
import torch

from . import dgr, synth, warmstart as W

CONFIG = 5  # seed family of the warm-start study


def problems(gs, geo, ids, dev):
    out = []
    for i in ids:
        ph = synth.ellipsoid_phantom_torch(synth.rng_for(CONFIG, i), gs, 40, dev)
        out.append(W.make_problem(gs, geo, ph, 0.01, 10_000_000 + i, dev))
    return out


def batched_fits(probs, inits, iters, lr0, lr1, batch, record=None):
    """Fits in batches; returns the states (and PSNR curves every `record` iterations)."""
    states, curves = [], []
    for b0 in range(0, len(probs), batch):
        F = W.Fit(probs[b0:b0 + batch], inits[b0:b0 + batch], lr0, lr1, iters)
        curve = [F.psnrs()] if record else None
        done = 0
        while done < iters:
            k = min(record or iters, iters - done)
            F.step(k)
            done += k
            if record:
                curve.append(F.psnrs())
        if F.status():
            raise RuntimeError(f"device status {F.status():#x} in a fit")
        states += F.states
        if record:
            curves += list(map(list, zip(*curve)))
    return states, curves


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--views", type=int, default=50)
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--ns", type=int, default=100000)
    ap.add_argument("--fit-iters", type=int, default=300)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr0", type=float, default=3e-3)
    ap.add_argument("--lr1", type=float, default=3e-4)
    ap.add_argument("--net-lr", type=float, default=1e-3)
    ap.add_argument("--record", type=int, default=10)
    a = ap.parse_args(argv)
    dev = "cuda"
    gs, geo = synth.learned_workload(a.side, a.views)
    t0 = time.time()
    log = {}
    # 1-2: training problems and their plain fits
    train = problems(gs, geo, range(a.train), dev)
    rng = np.random.default_rng(1)
    inits = [W.plain_init(p, a.ns, rng) for p in train]
    states, _ = batched_fits(train, inits, a.fit_iters, a.lr0, a.lr1, a.batch)
    targets = [W.targets_from_fit(p, st) for p, st in zip(train, states)]
    del states, inits
    torch.cuda.synchronize()
    log["fit_train_s"] = round(time.time() - t0, 1)
    # 3: train the network
    net = W.Net(a.side, seed=0)
    t1 = time.time()
    order = np.random.default_rng(2)
    losses = []
    for ep in range(a.epochs):
        for i in order.permutation(len(train)):
            losses.append(net.train_step(train[i].fdk, targets[i], a.net_lr).clone())
    torch.cuda.synchronize()
    log["train_net_s"] = round(time.time() - t1, 1)
    log["train_steps"] = len(losses)
    log["net_loss_first_last"] = [float(losses[0]), float(torch.stack(losses[-len(train):]).mean())]
    del targets
    # 4: held-out comparison
    test = problems(gs, geo, range(100_000, 100_000 + a.test), dev)
    rng_p, rng_l = np.random.default_rng(3), np.random.default_rng(3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    plain0 = [W.plain_init(p, a.ns, rng_p) for p in test]
    ev[1].record()
    learned0 = [W.learned_init(p, net, a.ns, rng_l) for p in test]
    ev[2].record()
    torch.cuda.synchronize()
    init_ms_plain = ev[0].elapsed_time(ev[1]) / a.test
    init_ms_learned = ev[1].elapsed_time(ev[2]) / a.test
    t2 = time.time()
    _, cp = batched_fits(test, plain0, a.fit_iters, a.lr0, a.lr1, a.batch, record=a.record)
    _, cl = batched_fits(test, learned0, a.fit_iters, a.lr0, a.lr1, a.batch, record=a.record)
    torch.cuda.synchronize()
    log["fit_test_s"] = round(time.time() - t2, 1)
    # per-iteration time of a fit of one problem (batched graph over the test set / test count)
    F = W.Fit(test[:1], [W.plain_init(test[0], a.ns, np.random.default_rng(9))], a.lr0, a.lr1, a.fit_iters)
    F.step(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(); F.step(20); e1.record(); torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / 20
    reach, gains = [], []
    for p_curve, l_curve in zip(cp, cl):
        target = p_curve[-1] - 0.1
        it_plain = a.record * next(i for i, v in enumerate(p_curve) if v >= target)
        hit = [i for i, v in enumerate(l_curve) if v >= target]
        it_learned = a.record * hit[0] if hit else None
        reach.append((it_plain, it_learned))
        gains.append(l_curve[0] - p_curve[0])
    ok = [r for r in reach if r[1] is not None]
    iters_plain = float(np.mean([r[0] for r in reach]))
    iters_learned = float(np.mean([r[1] for r in ok])) if ok else None
    wall_plain = init_ms_plain + iters_plain * ms_iter
    wall_learned = (init_ms_learned + iters_learned * ms_iter) if ok else None
    out = {
        "workload": f"{a.side}^3 grid, cone {a.views} views x {a.side}^2, {a.ns} Gaussians, "
                    f"{a.train} training / {a.test} held-out phantoms (40 ellipsoids, N(0,0.01^2))",
        "fit": {"iters": a.fit_iters, "lr": [a.lr0, a.lr1], "ms_per_iter_single": ms_iter},
        "plain_final_psnr_mean": float(np.mean([c[-1] for c in cp])),
        "learned_final_psnr_mean": float(np.mean([c[-1] for c in cl])),
        "initial_psnr_gain_db_mean": float(np.mean(gains)),
        "iters_to_plain_final_plain": iters_plain,
        "iters_to_plain_final_learned": iters_learned,
        "reached": f"{len(ok)}/{len(reach)}",
        "wall_ms_to_plain_final_plain": wall_plain,
        "wall_ms_to_plain_final_learned": wall_learned,
        "init_ms": {"plain": init_ms_plain, "learned": init_ms_learned},
        "log": log,
    }
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
