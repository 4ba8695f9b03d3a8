#!/usr/bin/env python
"""Benchmark of the DGR hot path on one B300: one optimisation iteration
(voxelize -> project -> L1 residual -> backproject -> voxelize adjoint ->
Adam) of 50,000 anisotropic Gaussians in a 256^3 grid against 50 cone-beam
views of 256 x 256 pixels (source-origin 1000 mm, source-detector 1500 mm,
1.5 mm pitch), synthetic ellipsoid phantom with N(0, 0.01^2) noise.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is DGR iterations/s with every input resident
in HBM (CUDA events around each step on the launching stream, L2 flushed by a
256 MiB write before every step, outside the events); `e2e` is the same
metric through the C ABI with every step's measured projections copied host
-> device from pinned memory (on a copy stream, overlapping the previous
step) and the loss copied back every step, timed as one interval over all
steps with the L2 flushes inside it.  Under torchrun each
rank runs an independent replica (the workload does not shard; no collective
touches the data path) and rank 0 prints the aggregate.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

METRIC = "FVR Gvoxel-evals/s & DGR iters/s at 256³; time-to-PSNR, learned+batched vs plain"
UNIT = "iter/s"
WORKLOAD = 2  # 50,000 Gaussians, 256^3, cone 50 x 256^2
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 148


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--objective", choices=["l1", "paper"], default="l1",
                    help="l1: the L1 data term (the hot path); paper: 0.6 L1 + 0.2 SSIM + 1 TV")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--split", choices=["replicas", "slab"], default="replicas",
                    help="replicas: one independent reconstruction per GPU (weak scaling); slab: "
                         "one reconstruction split into z-slabs over the GPUs (strong scaling, "
                         "NCCL reduce-scatter / all-gather / all-reduce)")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            P = json.load(f)
        return {"hbm_gbs": float(P["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(P.get("sm_max_mhz", 2032))}
    except Exception:
        return {"hbm_gbs": 6400.0, "src": "fallback", "sm_max_mhz": 2032.0}


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist
    return None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def setup_problem(rank, dev, objective="l1"):
    import torch
    from paper_2411_04844_b300 import dgr, synth
    wl = synth.workload(WORKLOAD)
    rng = synth.rng_for(WORKLOAD, rank)
    f = synth.gaussian_field(rng, wl.n_gauss, wl.grid, wl.scale)
    f.rho = np.clip(f.rho, 0.02, 1.0).astype(np.float32)
    phantom = synth.ellipsoid_phantom(synth.rng_for(WORKLOAD, 100 + rank), wl.grid, wl.phantom_m)
    noise = synth.rng_for(WORKLOAD, 200 + rank).normal(0.0, wl.noise_sigma, wl.geom.shape).astype(np.float32)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    grid = dgr.Grid.of(wl.grid)
    ang = T(wl.geom.angles)
    geom = dgr.Geom.of(wl.geom, ang)
    # measured projections: the phantom through the projector, plus noise
    ws_p = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, geom))
    meas = torch.empty(wl.geom.shape, device=dev)
    dgr.dgr_project(grid, geom, T(phantom), meas, ws_p)
    meas += T(noise)
    torch.cuda.synchronize()
    ws_p.close()
    mu, s, q, rho = T(f.mu), T(f.s), T(f.q), T(f.rho)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, wl.k_trunc, ws0)
    # in-box (Gaussian, voxel) pairs: the algorithmic work of voxelize
    an = torch.empty((f.n, 3), dtype=torch.int32, device=dev)
    bx = torch.empty((f.n, 6), dtype=torch.int32, device=dev)
    dgr.dgr_footprint(grid, mu, s, q, wl.k_trunc, an, bx)
    ext = (bx[:, 3:] - bx[:, :3] + 1).clamp(min=0).to(torch.float64)
    inbox = float(ext.prod(1).sum())
    ws0.close()
    plan = dgr.make_plan(grid, f.n, int(pairs * 1.5) + 1024, int(items * 1.5) + 1024, geom, step=True)
    ws = dgr.Workspace(plan)
    weights = dgr.PAPER_WEIGHTS if objective == "paper" else (1.0, 0.0, 0.0)
    prob = dgr.make_problem(grid, geom, wl.k_trunc, 3e-4, 3e-5, wl.n_iters, weights=weights)
    st = dgr.State(mu, s, q, rho)
    dgr.dgr_params_init(prob, st)
    return dict(wl=wl, grid=grid, geom=geom, ang=ang, meas=meas, ws=ws, prob=prob, st=st,
                pairs=pairs, items=items, inbox=inbox, f=f)


def run_ours(args, dist, rank, local):
    import torch
    from paper_2411_04844_b300 import dgr
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    P = setup_problem(rank, dev, args.objective)
    wl, ws, prob, st, meas = P["wl"], P["ws"], P["prob"], P["st"], P["meas"]
    # the exp2 and FMA pipes' rates per SM clock on this GPU (the voxelizer's
    # and its adjoint's roofline peaks), measured before the timed region
    from paper_2411_04844_b300 import peaks as pipe_peaks
    rates = pipe_peaks.pipe_rates()
    rates["l2"] = pipe_peaks.l2_rates()
    stream = torch.cuda.current_stream()
    loss = torch.zeros(1, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    K, W = args.steps, args.warmup
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(dgr.DGR_STEP_KERNEL_EVENTS)]
          for _ in range(K)]
    for row in ev:
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    for _ in range(W):
        flush.zero_()
        dgr.dgr_step(prob, st, meas, loss, ws)
    torch.cuda.synchronize()
    status = dgr.dgr_status(ws)
    if status:
        raise RuntimeError(f"device status {status:#x} after warm-up")

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    barrier(dist)
    torch.cuda.synchronize()
    l0 = dgr.dgr_launch_count()
    t_wall0 = time.perf_counter()
    for k in range(K):
        flush.zero_()
        dgr.dgr_step_timed(prob, st, meas, loss, ws, ev[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = dgr.dgr_launch_count() - l0
    barrier(dist)
    step_ms = [ev[k][0].elapsed_time(ev[k][6]) for k in range(K)]
    phase_ms = {name: [ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(K)]
                for i, name in enumerate(dgr.STEP_PHASES)}
    # the main kernels of the two projector phases, timed on their own stream
    kernel_ms = {"backproject": [ev[k][7].elapsed_time(ev[k][8]) for k in range(K)],
                 "project": [ev[k][9].elapsed_time(ev[k][10]) for k in range(K)],
                 "voxelize": [ev[k][11].elapsed_time(ev[k][12]) for k in range(K)],
                 "voxelize_backward": [ev[k][13].elapsed_time(ev[k][14]) for k in range(K)]}

    # end to end through the C ABI: every step's measured projections copied
    # pinned host -> device on a copy stream (into one of two device buffers,
    # overlapping the previous step), the step on the compute stream after
    # that copy, the loss copied back every step; one interval from the first
    # copy to the last loss read, L2 flushes included
    meas_host = meas.cpu().pin_memory()
    loss_host = torch.zeros(max(K, W, 2)).pin_memory()
    meas_dev = [meas.clone() for _ in range(2)]
    # the step as a CUDA graph (graph.step_graph, the library's replayable
    # iteration), one per input buffer: one launch per step, so the host's
    # enqueue time (about 0.1 ms per eager dgr_step, more on a slower host)
    # cannot limit the loop
    from paper_2411_04844_b300 import graph as dgr_graph
    g_e2e = [dgr_graph.step_graph(prob, st, meas_dev[b], loss, ws, warmup=1) for b in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(k):
        b = k & 1
        with torch.cuda.stream(copy_stream):
            if k >= 2:
                copy_stream.wait_event(used[b])  # step k - 2 read this buffer
            meas_dev[b].copy_(meas_host, non_blocking=True)
            copied[b].record(copy_stream)

    def e2e_steps(n, first):
        # n steps of the loop: the first step's copy is not overlapped (it
        # waits for `first`), every later one overlaps the step before it
        copy_stream.wait_event(first)
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            flush.zero_()
            stream.wait_event(copied[k & 1])
            g_e2e[k & 1].replay()
            used[k & 1].record(stream)
            loss_host[k:k + 1].copy_(loss, non_blocking=True)

    # untimed warm-up of the loop itself (each graph's first launch uploads
    # it to the device; the copies and the pinned buffers are touched once)
    e_warm = torch.cuda.Event()
    e_warm.record(stream)
    e2e_steps(max(W, 2), e_warm)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    e_start.record(stream)
    e2e_steps(K, e_start)
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    e2e_ms = [e_start.elapsed_time(e_end)]
    status = dgr.dgr_status(ws)
    if status:
        raise RuntimeError(f"device status {status:#x} after timed steps")
    if not bool(torch.isfinite(loss_host).all()):
        raise RuntimeError("non-finite loss")

    tot_s = max_over_ranks(dist, sum(step_ms) / 1000.0)
    tot_e2e = max_over_ranks(dist, sum(e2e_ms) / 1000.0)
    N = args.gpus
    value = N * K / tot_s
    e2e_value = N * K / tot_e2e
    phases = {k: statistics.mean(v) for k, v in phase_ms.items()}
    kernels = {k: statistics.mean(v) for k, v in kernel_ms.items()}
    return dict(P=P, value=value, e2e=e2e_value, step_ms=statistics.mean(step_ms), phases=phases,
                kernels=kernels, rates=rates,
                launches=launches, clocks=clk, t_wall=t_wall, loss=float(loss_host[K - 1].item()))


KERNEL_NAMES = {"project": "k_path_n<0, 2> (projector walk, two rays per thread)",
                "backproject": "k_path_n<1, 2> (backprojector walk + fixed-point scatter, two rays per thread)",
                "voxelize": "k_voxelize (tile evaluation)",
                "voxelize_backward": "k_bwd_items (per-item moments of the FVR adjoint)"}


def roofline(P, phases, clk, pk, kernels=None, rates=None):
    """Roofline of the dominant kernel of one iteration.  Each of the four
    heavy phases is represented by its main kernel, timed by its own pair of
    events (the phase time is kept beside it); the others by the phase time.
    The exp2 and FMA peaks are the rates measured on this GPU (per SM clock)
    x SMs x the SM clock sampled during the timed region."""
    kernels = kernels or {}
    rates = rates or {}
    wl = P["wl"]
    nvox = wl.grid.dims[0] * wl.grid.dims[1] * wl.grid.dims[2]
    nrays = wl.geom.n_views * wl.geom.nu * wl.geom.nv
    proj_bytes = 4.0 * nvox * wl.geom.n_views + 4.0 * nrays
    mhz = clk.get("sm_mhz") or pk["sm_max_mhz"]
    sms = rates.get("sms", SMS)
    ex2_clk = rates.get("ex2")
    fma_clk = max(rates.get("ffma", 0.0), rates.get("ffma2", 0.0)) or None
    sfu_peak = sms * ex2_clk * mhz * 1e6 / 1e9 if ex2_clk else None  # G ex2 / s
    ffma_peak = sms * fma_clk * mhz * 1e6 / 1e9 if fma_clk else None  # G FFMA / s
    per = {}
    for name, ph_ms in phases.items():
        ms = kernels.get(name, ph_ms)
        s = ms / 1000.0
        if name in ("project", "backproject"):
            a = proj_bytes / s / 1e9
            per[name] = {"bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": a / pk["hbm_gbs"], "ms": ms}
            # the volume and the integer sums stay in L2 between views: the L2
            # traffic per launch (ncu lts__t_bytes) against the L2 read bandwidth
            # measured in this run
            l2b = l2_bytes_for(name)
            l2peak = (rates.get("l2") or {}).get("read_gbs")
            if l2b and l2peak:
                per[name]["l2"] = {"achieved": l2b / s / 1e9, "peak": l2peak, "unit": "GB/s",
                                   "frac": l2b / s / 1e9 / l2peak, "bytes_per_launch": l2b}
        elif name == "voxelize" and sfu_peak:
            a = P["inbox"] / s / 1e9
            per[name] = {"bound": "alu", "achieved": a, "peak": sfu_peak, "unit": "Gex2/s",
                         "frac": a / sfu_peak, "ms": ms,
                         "frac_phase": P["inbox"] / (ph_ms / 1000.0) / 1e9 / sfu_peak}
        elif name == "voxelize_backward" and ffma_peak:
            a = 12.0 * P["inbox"] / s / 1e9
            per[name] = {"bound": "alu", "achieved": a, "peak": ffma_peak, "unit": "GFFMA/s",
                         "frac": a / ffma_peak, "ms": ms,
                         "frac_phase": 12.0 * P["inbox"] / (ph_ms / 1000.0) / 1e9 / ffma_peak}
        else:
            per[name] = {"ms": ms}
        per[name]["phase_ms"] = ph_ms
    dom = max(per, key=lambda k: per[k]["ms"])
    r = dict(per[dom])
    r["kernel_ms"] = r.pop("ms")
    r.pop("phase_ms")
    r["kernel"] = KERNEL_NAMES.get(dom, dom)
    r["phase"] = dom
    r["peak_src"] = (pk["src"] if r.get("unit") == "GB/s" else
                     f"measured pipe rate per clock x {sms} SMs x {mhz:.0f} MHz")
    r["traffic"] = traffic_for(dom)
    return r, per


def l2_bytes_for(phase):
    """L2 bytes (lts__t_bytes.sum) per launch from the committed ncu record,
    if the kernel's source is unchanged since; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            T = json.load(f)
        ent = T[phase]
        src = os.path.join(ROOT, "paper_2411_04844_b300", "csrc", ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return float(ent["l2_bytes_per_launch"]) if h == ent["source_sha256_16"] else None
    except Exception:
        return None


def traffic_for(phase):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source is unchanged since the counters were taken; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            T = json.load(f)
        ent = T[phase]
        src = os.path.join(ROOT, "paper_2411_04844_b300", "csrc", ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return float(ent["dram_bytes_per_launch"]) if h == ent["source_sha256_16"] else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(frac_gauss, n_views_sample, seed_rank=0):
    """Time the FP64 oracle on a bounded sample of one iteration of the
    workload and scale to a full iteration.  Returns (iters/s, threads,
    description, seconds spent)."""
    import oracle as O
    from paper_2411_04844_b300 import synth
    wl = synth.workload(WORKLOAD)
    f = synth.gaussian_field(synth.rng_for(WORKLOAD, seed_rank), wl.n_gauss, wl.grid, wl.scale)
    ng = max(1, int(round(wl.n_gauss * frac_gauss)))
    og = O.Grid(wl.grid.dims, wl.grid.h, wl.grid.org)
    geo = wl.geom
    idx = np.linspace(0, geo.n_views - 1, n_views_sample).round().astype(int)
    oo = O.Geom(geo.beam, geo.angles[idx], geo.nu, geo.nv, geo.pu, geo.pv, geo.dso, geo.dsd)
    t0 = time.perf_counter()
    vol = O.voxelize(og, f.mu[:ng], f.s[:ng], f.q[:ng], f.rho[:ng], wl.k_trunc)
    t1 = time.perf_counter()
    sino = O.project(og, oo, vol)
    t2 = time.perf_counter()
    gv = O.backproject(og, oo, np.sign(sino) / sino.size)
    t3 = time.perf_counter()
    O.voxelize_backward(og, f.mu[:ng], f.s[:ng], f.q[:ng], f.rho[:ng], gv, wl.k_trunc)
    t4 = time.perf_counter()
    sg = wl.n_gauss / ng
    sv = geo.n_views / n_views_sample
    t_iter = (t1 - t0) * sg + (t2 - t1) * sv + (t3 - t2) * sv + (t4 - t3) * sg
    desc = (f"FP64 oracle on {O.num_threads()} threads: voxelize + adjoint of {ng} of "
            f"{wl.n_gauss} Gaussians, project + backproject of {n_views_sample} of "
            f"{geo.n_views} views, 256^3 grid; scaled to one full iteration")
    parts = ((t1 - t0) + (t4 - t3), (t2 - t1) + (t3 - t2))  # Gaussian part, view part
    return 1.0 / t_iter, O.num_threads(), desc, t4 - t0, parts


def sample_size(target_s, frac0=0.01):
    """Calibrate on a small sample (a fraction frac0 of the Gaussians, one
    view), then size (fraction of Gaussians, views) so that one sample takes
    about target_s seconds: half for the views (at most all of them), the
    rest for the Gaussians (at most all of them), and what the Gaussians
    leave back to the views."""
    *_, (tg, tv) = oracle_sample(frac0, 1)
    tg, tv = max(tg, 1e-3), max(tv, 1e-3)
    nv = int(max(1, min(50, round(0.5 * target_s / tv))))
    fg = min(1.0, frac0 * max(0.5 * target_s, target_s - nv * tv) / tg)
    nv = int(max(nv, min(50, round((target_s - fg / frac0 * tg) / tv))))
    return fg, nv


def cpu_baseline(target_s):
    """The oracle's iterations/s on a bounded sample; when even the whole
    iteration is shorter than the target, it is repeated (at most 4 times)
    and the times summed."""
    fg, nv = sample_size(target_s)
    times, spent, th, desc = [], 0.0, None, None
    while not times or (spent < 0.66 * target_s and len(times) < 4):
        v, th, desc, t, _ = oracle_sample(fg, nv)
        times.append(1.0 / v)
        spent += t
    if len(times) > 1:
        desc += f" (x{len(times)})"
    return {"value": len(times) / sum(times), "unit": UNIT, "cores": th, "kind": "oracle",
            "sample": desc, "seconds": round(spent, 2)}


def run_reference(args, rank, ws_n):
    """The reference arm: the FP64 oracle as it stands, on the host cores,
    each step a bounded sample of one iteration."""
    if rank != 0:
        return
    W, K = args.warmup, args.steps
    # each step a bounded sample: about 2 minutes for the whole run, at most 5 s a step
    fg, nv = sample_size(min(5.0, max(0.1, 120.0 / (W + K))), frac0=0.002)
    per = []
    desc = th = None
    for k in range(W + K):
        v, th, desc, spent, _ = oracle_sample(fg, nv, seed_rank=k % 3)
        if k >= W:
            per.append(1.0 / v)
    value = K / sum(per)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": 1000.0 * sum(per) / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                             "sample": desc + " (per step)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_block():
    return {"workload": "cone256_50k: 50,000 anisotropic Gaussians (log-uniform scales 0.5-6 "
                        "voxels, 3-sigma boxes) -> 256^3 grid, cone beam 50 views x 256^2 "
                        "(dso 1000, dsd 1500, pitch 1.5 mm), 40-ellipsoid phantom + N(0,0.01^2)",
            "grid": [256, 256, 256], "n_gauss": 50000, "views": 50, "detector": [256, 256],
            "l2": "flushed before every step by a 256 MiB write (outside the timed events)",
            "parallelism": "replicas (one independent reconstruction per GPU)"}


def run_slab(args, rank, world, local):
    """One reconstruction of the workload split into z-slabs over the ranks
    (paper_2411_04844_b300.slab): per-step CUDA events around each rank's
    iteration, max over ranks; iterations of the one reconstruction per
    second."""
    import torch
    import torch.distributed as dist
    from paper_2411_04844_b300 import dgr, slab
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if "MASTER_ADDR" not in os.environ:  # one GPU without torchrun: a group of one rank
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(sk.getsockname()[1]),
                              RANK="0", WORLD_SIZE="1")
    dist.init_process_group("nccl", device_id=torch.device(dev))
    P = setup_problem(0, dev, "l1")  # every rank builds the same reconstruction
    wl, prob, st, meas = P["wl"], P["prob"], P["st"], P["meas"]
    spec = slab.slab_spec(wl.grid.dims[2], wl.geom.n_views, wl.geom.nu * wl.geom.nv, rank, world)
    R = slab.SlabRank(spec, slab.CudaBackend(prob, st, spec, dev))
    comm = slab.TorchComm()
    meas_mine = meas[spec.v0:spec.v0 + spec.nv].contiguous()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup
    for _ in range(W):
        slab.run_step(R, comm, meas_mine)
    torch.cuda.synchronize()
    if R.be.status():
        raise RuntimeError(f"device status {R.be.status():#x} after warm-up")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    dist.barrier()
    torch.cuda.synchronize()
    loss = None
    for k in range(K):
        flush.zero_()
        ev[k][0].record()
        loss = slab.run_step(R, comm, meas_mine)
        ev[k][1].record()
    torch.cuda.synchronize()
    dist.barrier()
    tot = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    t = torch.tensor([tot], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = float(t.item())
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": K / tot, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": 1000.0 * tot / K, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {**config_block(), "parallelism": f"z-slab split of one reconstruction over {world} GPUs"},
            "loss": float(loss.item()), "split": "slab"}))
    dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.split == "slab":
        run_slab(args, rank, world, local)
        return
    dist = dist_init(world)
    R = run_ours(args, dist, rank, local)
    if rank != 0:
        return
    pk = peaks()
    roof, per = roofline(R["P"], R["phases"], R["clocks"], pk, R["kernels"], R["rates"])
    P = R["P"]
    wl = P["wl"]
    fvr_ms = R["phases"]["voxelize"]
    line = {
        "metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": R["step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_block(),
        "fvr_gvoxel_evals_per_s": P["inbox"] / (fvr_ms / 1000.0) / 1e9,
        "fvr_kernel_gvoxel_evals_per_s": P["inbox"] / (R["kernels"]["voxelize"] / 1000.0) / 1e9,
        "pipe_rates_per_clk_sm": {k: (round(v, 3) if isinstance(v, float) else v)
                                  for k, v in R["rates"].items()},
        "phases_ms": {k: round(v, 4) for k, v in R["phases"].items()},
        "phase_roofline": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                               for kk, vv in v.items()} for k, v in per.items()},
        "work": {"inbox_pairs": P["inbox"], "tile_pairs": P["pairs"], "items": P["items"]},
        "roofline": roof,
        "e2e": {"value": R["e2e"], "unit": UNIT, "h2d_bytes_per_step": int(P["meas"].numel() * 4),
                "d2h_bytes_per_step": 4,
                "launch": "CUDA graph of dgr_step (graph.step_graph), one replay per step"},
        "gpu_launches": R["launches"],
        "clocks": R["clocks"],
        "loss": R["loss"],
        "objective": args.objective,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
