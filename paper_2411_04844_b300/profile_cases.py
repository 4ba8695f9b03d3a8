"""Run one entry point of the C ABI a few times on a synthetic workload, with
every input already in HBM -- a fixed, small command for profilers.

    python -m paper_2411_04844_b300.profile_cases OP [--workload 2] [--reps 3] [--views N]
        [--backprojector 0|1|2] [--isotropic] [--no-separable] [--staged]

OP: voxelize | voxelize_backward | project | backproject | step | net_forward |
net_backward (the warm-start network on a --side^3 grid, default 128, with
--conv-engine as dgr_set_conv_engine, default 2; also prints the four
tensor-core convolutions' forward GEMM FLOPs).
Workload numbers are those of synth.workload (2: 50,000 Gaussians, 256^3,
cone 50 views x 256^2).  --views keeps only the first N views (smaller
captures).  Prints the mean CUDA-event time per call.
"""
import argparse
import sys

import numpy as np
import torch

from . import dgr, synth


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["voxelize", "voxelize_backward", "project", "backproject", "step",
                                   "net_forward", "net_backward"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--views", type=int, default=0)
    ap.add_argument("--backprojector", type=int, default=0, help="0: ray scatter, 1: column gather, 2: brick scatter")
    ap.add_argument("--isotropic", action="store_true", help="one scale per Gaussian (separable FVR)")
    ap.add_argument("--no-separable", action="store_true", help="general voxelizer even when separable")
    ap.add_argument("--staged", action="store_true", help="path walks staged through shared memory (off by default, as in the library)")
    ap.add_argument("--side", type=int, default=128, help="network grid side")
    ap.add_argument("--conv-engine", type=int, default=2, help="2: tcgen05, several taps per MMA; 3: tcgen05 halo tiles, one tap per MMA; 1: tcgen05 gathered tiles; 0: mma.sync")
    a = ap.parse_args(argv)
    if a.op.startswith("net"):
        return net_case(a)
    dgr.dgr_set_backprojector(a.backprojector)
    dgr.dgr_set_separable(not a.no_separable)
    dgr.dgr_set_staged_walk(a.staged)
    wl = synth.workload(a.workload)
    geo_spec = wl.geom
    if a.views:
        geo_spec = synth.GeomSpec(geo_spec.beam, geo_spec.angles[:a.views], geo_spec.nu,
                                  geo_spec.nv, geo_spec.pu, geo_spec.pv, geo_spec.dso, geo_spec.dsd)
    dev = "cuda"
    T = lambda x: torch.as_tensor(np.ascontiguousarray(x), device=dev)
    grid = dgr.Grid.of(wl.grid)
    ang = T(geo_spec.angles)
    geom = dgr.Geom.of(geo_spec, ang)
    f = synth.gaussian_field(synth.rng_for(a.workload, 0), wl.n_gauss, wl.grid, wl.scale, isotropic=a.isotropic)
    f.rho = np.clip(f.rho, 0.02, 1.0).astype(np.float32)
    mu, s, q, rho = T(f.mu), T(f.s), T(f.q), T(f.rho)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, wl.k_trunc, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, int(pairs * 1.5) + 1024, int(items * 1.5) + 1024,
                                     geom, step=True))
    rng = np.random.default_rng(0)
    vol = T(rng.uniform(0, 1, wl.grid.shape).astype(np.float32))
    sino = T(rng.standard_normal(geo_spec.shape).astype(np.float32))
    outs = [torch.empty(sh, device=dev) for sh in ((f.n, 3), (f.n, 3), (f.n, 4), (f.n,))]
    prob = dgr.make_problem(grid, geom, wl.k_trunc, 3e-4, 3e-5, max(wl.n_iters, 2))
    st = dgr.State(mu, s, q, rho)
    dgr.dgr_params_init(prob, st)
    loss = torch.zeros(1, device=dev)
    out_vol = torch.empty(wl.grid.shape, device=dev)
    out_sino = torch.empty(geo_spec.shape, device=dev)

    def once():
        if a.op == "voxelize":
            dgr.dgr_voxelize(grid, mu, s, q, rho, wl.k_trunc, out_vol, ws)
        elif a.op == "voxelize_backward":
            dgr.dgr_voxelize_backward(grid, mu, s, q, rho, wl.k_trunc, vol, *outs, ws)
        elif a.op == "project":
            dgr.dgr_project(grid, geom, vol, out_sino, ws)
        elif a.op == "backproject":
            dgr.dgr_backproject(grid, geom, sino, out_vol, ws)
        else:
            dgr.dgr_step(prob, st, sino, loss, ws)

    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    status = dgr.dgr_status(ws)
    print(f"{a.op}: {e0.elapsed_time(e1) / a.reps:.4f} ms per call (status {status})")
    return 0 if status == 0 else 1


def net_case(a):
    """forward (or forward + backward) of the warm-start network"""
    dev, n = "cuda", a.side
    rng = np.random.default_rng(0)
    npar = dgr.dgr_net_param_count()
    params = torch.as_tensor(rng.standard_normal(npar).astype(np.float32) * 0.05, device=dev)
    x = torch.as_tensor(rng.uniform(0, 1, (n, n, n)).astype(np.float32), device=dev)
    gy = torch.as_tensor(rng.standard_normal((n, n, n, 2)).astype(np.float32), device=dev)
    out = torch.empty((n, n, n, 2), device=dev)
    gp = torch.empty(npar, device=dev)
    ws = torch.empty(dgr.dgr_net_ws_bytes(n), dtype=torch.uint8, device=dev)
    dgr.dgr_set_conv_engine(a.conv_engine)

    def once():
        dgr.dgr_net_forward(n, params, x, out, ws)
        if a.op == "net_backward":
            dgr.dgr_net_backward(n, params, x, gy, gp, ws)

    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    status = dgr.dgr_net_status(n, ws)
    h3, q3, n3 = (n // 2) ** 3, (n // 4) ** 3, n ** 3
    # GEMM FLOPs of the four tensor-core convolutions (forward)
    fl = 2 * 27 * (h3 * 16 * 32 + q3 * 32 * 64 + h3 * 64 * 32 + n3 * 32 * 16)
    print(f"{a.op} n={n} engine={a.conv_engine}: {ms:.4f} ms per call (status {status}); "
          f"forward conv GEMMs {fl / 1e9:.1f} GFLOP")
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
