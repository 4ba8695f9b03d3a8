"""Learned warm start (and batching) vs the plain FBP-seeded initialisation
(one B300).

    python -m paper_2411_04844_b300.learned_bench [--side 128] [--views 50]
        [--train 256] [--test 16] [--ns 100000] [--train-iters 300]
        [--fit-iters 2000] [--epochs 4] [--record 10]

1. training phantoms (seeded, 40 ellipsoids), their projections (+ noise) and
   FDK-style inputs;
2. the plain method fits every training problem from the FBP-seeded
   initialisation (batched, CUDA graph) -> targets (fitted density, mean
   log-scale per voxel).  These fits only make targets: they run the short
   schedule --train-lr0 -> --train-lr1 over --train-iters iterations;
3. the network is trained on (FDK input -> targets) with the project's own
   kernels (forward, backward, loss, Adam);
4. held-out problems, fitted with the method's schedule (Adam, lr --lr0 ->
   --lr1 = 3e-4 -> 3e-5 over --fit-iters, Sec. 5.1):
   * plain: each problem alone, FBP-seeded initialisation, its PSNR recorded
     every --record iterations; its target is its final PSNR - 0.1 dB;
   * learned: the same problems, initialised by the network, the same way;
   * learned + batched: all held-out problems in one dgr_step_batched graph
     from the learned initialisation; after every block of --record
     iterations the instances at their target leave the batch (re-planned,
     graph captured again, both timed), until none is left.
   Wall times are CUDA-event times of the initialisation and of the steps up
   to (and including) the block of --record iterations in which the target
   is reached; PSNR evaluations between blocks are outside the timed
   intervals.
Prints one JSON line.
"""
import argparse
import json
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


def batched_fits(probs, inits, iters, lr0, lr1, batch):
    """Fits in batches of `batch` instances; returns the final states."""
    states = []
    for b0 in range(0, len(probs), batch):
        F = W.Fit(probs[b0:b0 + batch], inits[b0:b0 + batch], lr0, lr1, iters)
        F.step(iters)
        if F.status():
            raise RuntimeError(f"device status {F.status():#x} in a fit")
        states += F.states
    return states


class Timer:
    def __init__(self):
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def __enter__(self):
        self.e0.record()
        return self

    def __exit__(self, *exc):
        self.e1.record()
        torch.cuda.synchronize()
        self.ms = self.e0.elapsed_time(self.e1)


def timed_fit(probs, init_fn, iters, lr0, lr1, record, targets=None):
    """Initialise (timed) and fit the problems together (one instance: a
    single fit), recording PSNR every `record` iterations.  Returns the init
    time, per-block step times and the PSNR curves (index 0 = initial)."""
    with Timer() as ti:
        inits = [init_fn(p) for p in probs]
    F = W.Fit(probs, inits, lr0, lr1, iters)
    curves = [[v] for v in F.psnrs()]
    blocks = []
    done = 0
    while done < iters:
        k = min(record, iters - done)
        with Timer() as tb:
            F.step(k)
        blocks.append(tb.ms)
        done += k
        for c, v in zip(curves, F.psnrs()):
            c.append(v)
        if targets is not None and all(max(c) >= t for c, t in zip(curves, targets)):
            break
    if F.status():
        raise RuntimeError(f"device status {F.status():#x} in a fit")
    return ti.ms, blocks, curves


def retiring_fit(probs, init_fn, iters, lr0, lr1, record, targets):
    """All problems in one batched fit (one graph replay per iteration); after
    every block of `record` iterations the instances that reached their
    target leave the batch (its workspace is planned again and the next block
    captures a new graph).  Returns the total wall time (initialisation, step
    blocks and the re-planning, each CUDA-event timed) until the last
    instance reaches its target (None if one never does), and the iteration
    at which each instance reached it."""
    with Timer() as ti:
        inits = [init_fn(p) for p in probs]
    F = W.Fit(probs, inits, lr0, lr1, iters)
    active = list(range(len(probs)))
    hit = [None] * len(probs)
    total = ti.ms
    done = 0
    for i, v in zip(active, F.psnrs()):
        if v >= targets[i]:
            hit[i] = 0
    while done < iters:
        keep = [j for j, i in enumerate(active) if hit[i] is None]
        if not keep:
            break
        if len(keep) < len(active):
            with Timer() as tr:
                F.keep(keep)
            total += tr.ms
            active = [active[j] for j in keep]
        k = min(record, iters - done)
        with Timer() as tb:
            F.step(k)
        total += tb.ms
        done += k
        if F.status():
            raise RuntimeError(f"device status {F.status():#x} in a fit")
        for i, v in zip(active, F.psnrs()):
            if hit[i] is None and v >= targets[i]:
                hit[i] = done
    return (total if all(h is not None for h in hit) else None), hit, ti.ms


def reach(curve, target):
    """Index of the first record at or above target (None if never)."""
    return next((i for i, v in enumerate(curve) if v >= target), None)


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--views", type=int, default=50)
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=16)
    ap.add_argument("--ns", type=int, default=100000)
    ap.add_argument("--train-iters", type=int, default=300)
    ap.add_argument("--train-lr0", type=float, default=3e-3)
    ap.add_argument("--train-lr1", type=float, default=3e-4)
    ap.add_argument("--fit-iters", type=int, default=2000)
    ap.add_argument("--lr0", type=float, default=3e-4)
    ap.add_argument("--lr1", type=float, default=3e-5)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--net-lr", type=float, default=1e-3)
    ap.add_argument("--record", type=int, default=10)
    return ap.parse_args(argv)


def study(a) -> dict:
    """Steps 1-4 of the module doc with the options a; returns the record."""
    dev = "cuda"
    gs, geo = synth.learned_workload(a.side, a.views)
    t0 = time.time()
    log = {}
    # 1-2: training problems and their plain fits
    train = problems(gs, geo, range(a.train), dev)
    rng = np.random.default_rng(1)
    inits = [W.plain_init(p, a.ns, rng) for p in train]
    states = batched_fits(train, inits, a.train_iters, a.train_lr0, a.train_lr1, a.batch)
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
    del targets, train
    # 4: held-out comparison
    test = problems(gs, geo, range(100_000, 100_000 + a.test), dev)
    t2 = time.time()
    rng_p = np.random.default_rng(3)
    plain = [timed_fit([p], lambda q: W.plain_init(q, a.ns, rng_p), a.fit_iters, a.lr0, a.lr1,
                       a.record) for p in test]
    tgt = [c[0][-1] - 0.1 for _, _, c in plain]
    rng_l = np.random.default_rng(3)
    learned = [timed_fit([p], lambda q: W.learned_init(q, net, a.ns, rng_l), a.fit_iters, a.lr0,
                         a.lr1, a.record, [t]) for p, t in zip(test, tgt)]
    rng_b = np.random.default_rng(3)
    batched_ms, hit_b, b_init = retiring_fit(test, lambda q: W.learned_init(q, net, a.ns, rng_b),
                                             a.fit_iters, a.lr0, a.lr1, a.record, tgt)
    log["fit_test_s"] = round(time.time() - t2, 1)

    def cost(init_ms, blocks, curve, target):
        i = reach(curve, target)
        if i is None:
            return None, None
        return i * a.record, init_ms + sum(blocks[:i])

    rp = [cost(im, bl, c[0], t) for (im, bl, c), t in zip(plain, tgt)]
    rl = [cost(im, bl, c[0], t) for (im, bl, c), t in zip(learned, tgt)]
    ok = [r for r in rl if r[0] is not None]
    out = {
        "workload": f"{a.side}^3 grid, cone {a.views} views x {a.side}^2, {a.ns} Gaussians, "
                    f"{a.train} training / {a.test} held-out phantoms (40 ellipsoids, N(0,0.01^2))",
        "schedule": {"held_out": {"iters": a.fit_iters, "lr": [a.lr0, a.lr1]},
                     "training_fits": {"iters": a.train_iters, "lr": [a.train_lr0, a.train_lr1]}},
        "plain_final_psnr_mean": float(np.mean([c[0][-1] for _, _, c in plain])),
        "initial_psnr_mean": {"plain": float(np.mean([c[0][0] for _, _, c in plain])),
                              "learned": float(np.mean([c[0][0] for _, _, c in learned]))},
        "reached_learned": f"{len(ok)}/{len(rl)}",
        "reached_learned_batched": f"{sum(h is not None for h in hit_b)}/{len(hit_b)}",
        "iters_to_target_mean": {"plain": float(np.mean([r[0] for r in rp])),
                                 "learned": float(np.mean([r[0] for r in ok])) if ok else None,
                                 "learned_batched": float(np.mean([h for h in hit_b if h is not None]))
                                 if any(h is not None for h in hit_b) else None},
        "wall_ms_to_target_per_problem_mean": {
            "plain": float(np.mean([r[1] for r in rp])),
            "learned": float(np.mean([r[1] for r in ok])) if ok else None},
        "wall_ms_all_problems": {
            "plain_sequential": float(sum(r[1] for r in rp)),
            "learned_sequential": float(sum(r[1] for r in rl)) if len(ok) == len(rl) else None,
            "learned_batched": batched_ms},
        "init_ms_mean": {"plain": float(np.mean([im for im, _, _ in plain])),
                         "learned": float(np.mean([im for im, _, _ in learned])),
                         "learned_batched_all": b_init},
        "log": log,
    }
    return out


def main(argv=None):
    print(json.dumps(study(parse(argv))))
    return 0


if __name__ == "__main__":
    sys.exit(main())
