"""Batched reconstructions vs sequential plain runs (one B300).

    python -m paper_2411_04844_b300.batch_bench [--inst 16] [--steps 10] [--warmup 3]
        [--sizes 64 128 192 256] [--n-range 5000 200000]

16 independent reconstructions (synth.batched_workload: grids of 64^3 ..
256^3, 5K..200K Gaussians, 25..100 cone-beam views, detector N x N): one
iteration of all of them as
  * sequential: dgr_step of each instance in turn (its own workspace), and
  * batched:    one dgr_step_batched (one launch per phase over all
                instances), captured once in a CUDA graph and replayed,
with the voxelizer tile depth chosen by the autotuner for the batch.  Both
paths compute the same numbers (bit for bit in deterministic mode).  Prints
one JSON line: ms per iteration of all instances for each path.
"""
import argparse
import json
import sys

import numpy as np
import torch

from . import autotune, dgr, graph, synth


def build(insts, dev):
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    B = {"grids": [], "geoms": [], "angs": [], "probs": [], "meas": [], "states": [], "ns": [],
         "fields": [f.field for f in insts]}
    for i, ins in enumerate(insts):
        grid = dgr.Grid.of(ins.grid)
        ang = T(ins.geom.angles)
        geom = dgr.Geom.of(ins.geom, ang)
        phantom = synth.ellipsoid_phantom(synth.rng_for(4, 100 + i), ins.grid, 10)
        noise = synth.rng_for(4, 200 + i).normal(0.0, ins.noise_sigma, ins.geom.shape).astype(np.float32)
        wsp = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, geom))
        meas = torch.empty(ins.geom.shape, device=dev)
        dgr.dgr_project(grid, geom, T(phantom), meas, wsp)
        meas += T(noise)
        torch.cuda.synchronize()
        wsp.close()
        f = ins.field
        st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
        prob = dgr.make_problem(grid, geom, 3.0, 3e-4, 3e-5, 1000)
        dgr.dgr_params_init(prob, st)
        for k, v in (("grids", grid), ("geoms", geom), ("angs", ang), ("probs", prob), ("meas", meas),
                     ("states", st), ("ns", f.n)):
            B[k].append(v)
    return B


def counts(B, dev):
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    pairs, items = [], []
    for g, f in zip(B["grids"], B["fields"]):
        ws0 = dgr.Workspace(dgr.make_plan(g, f.n))
        p, it = dgr.dgr_voxelize_count(g, T(f.mu), T(f.s), T(f.q), 3.0, ws0)
        ws0.close()
        pairs.append(int(p * 1.3) + 1024)
        items.append(int(it * 1.3) + 1024)
    return pairs, items


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--inst", type=int, default=16)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--sizes", type=int, nargs="+", default=[64, 128, 192, 256],
                    help="grid sides the instances draw from")
    ap.add_argument("--n-range", type=int, nargs=2, default=[5000, 200000],
                    help="Gaussian counts, log-uniform")
    a = ap.parse_args(argv)
    dev = "cuda"
    insts = synth.batched_workload(a.inst, sizes=tuple(a.sizes), n_range=tuple(a.n_range))
    B = build(insts, dev)
    n_inst = len(insts)
    loss = torch.zeros(n_inst, device=dev)

    def make_batched():
        pairs, items = counts(B, dev)
        ws = dgr.Workspace(dgr.make_batch_plan(B["grids"], B["geoms"], B["ns"], pairs, items))
        return lambda: dgr.dgr_step_batched(B["probs"], B["states"], B["meas"], loss, ws)

    key = "batched/" + "/".join(f"{g.nx}:{n}" for g, n in zip(B["grids"], B["ns"]))
    depth = 32 if a.no_tune else autotune.tune(key, make_batched, reps=2)
    dgr.dgr_set_tile_depth(depth)
    pairs, items = counts(B, dev)
    ws_b = dgr.Workspace(dgr.make_batch_plan(B["grids"], B["geoms"], B["ns"], pairs, items))
    ws_s = [dgr.Workspace(dgr.make_plan(g, n, p, it, ge, step=True))
            for g, ge, n, p, it in zip(B["grids"], B["geoms"], B["ns"], pairs, items)]

    def sequential():
        for i in range(n_inst):
            dgr.dgr_step(B["probs"][i], B["states"][i], B["meas"][i], loss[i:i + 1], ws_s[i])

    g = graph.batched_step_graph(B["probs"], B["states"], B["meas"], loss, ws_b, warmup=a.warmup)
    flush = torch.empty(64 * 1024 * 1024, device=dev)

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(a.steps)]
        for _ in range(a.warmup):
            fn()
        torch.cuda.synchronize()
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
        return float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))

    ms_seq = timed(sequential)
    ms_bat = timed(g.replay)
    # each instance's step alone (L2 flushed before it): where the sequential
    # time goes, and how much of it batching can reach (the small instances'
    # idle SMs and launch gaps; a large instance fills the GPU on its own)
    ms_inst = [timed(lambda i=i: dgr.dgr_step(B["probs"][i], B["states"][i], B["meas"][i],
                                              loss[i:i + 1], ws_s[i]))
               for i in range(n_inst)]
    status = dgr.dgr_status(ws_b)
    out = {"workload": f"{n_inst} instances: grids {sorted(set(x.nx for x in B['grids']))}^3, "
                       f"Gaussians {min(B['ns'])}..{max(B['ns'])}, views "
                       f"{min(x.n_views for x in B['geoms'])}..{max(x.n_views for x in B['geoms'])}",
           "tile_depth": depth, "ms_per_iteration_sequential": ms_seq,
           "ms_per_iteration_batched_graph": ms_bat, "speedup": ms_seq / ms_bat,
           "iterations_per_s_all_instances_batched": 1000.0 / ms_bat, "status": status,
           "ms_per_instance_alone": [round(x, 4) for x in ms_inst],
           "instances": [{"side": x.nx, "gaussians": n, "views": ge.n_views}
                         for x, n, ge in zip(B["grids"], B["ns"], B["geoms"])],
           "total_gaussians": int(sum(B["ns"])), "l2": "flushed before every iteration (256 MiB write)"}
    print(json.dumps(out))
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
