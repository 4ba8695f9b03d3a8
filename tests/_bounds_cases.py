"""Cases run by tests/test_gpu_bounds.py, once with the default library and
once (in a child process, DGR_CHECK_BOUNDS=1) with the bounds-checked one:
the projector and backprojector on geometries that take each walk kernel
(two-ray walks with 256-, 128- and 64-row CTAs, the one-ray walk of steep
cone rays), the voxelizer and its adjoint on a ragged grid, and full
optimisation steps.  Returns every output and every status word."""
import os
import sys

import numpy as np
import torch

from paper_2411_04844_b300 import dgr, synth

DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


GEOMS = [
    ("cone256rows", synth.GridSpec((40, 36, 44), 1.0, (-20.0, -18.0, -22.0)),
     synth.cone_geom(9, 48, 200, 1.0, 0.35, 90.0, 140.0)),
    ("cone128rows", synth.GridSpec((40, 36, 44), 1.0, (-20.0, -18.0, -22.0)),
     synth.cone_geom(7, 48, 100, 1.0, 0.7, 90.0, 140.0)),
    ("parallel64rows", synth.GridSpec((33, 29, 21), 0.8, (-13.0, -12.0, -8.0)),
     synth.parallel_geom(11, 44, 30, 1.0, 0.9)),
    ("steep_cone", synth.GridSpec((16, 16, 16), 1.0, (-8.0, -8.0, -8.0)),
     synth.cone_geom(6, 40, 60, 1.0, 1.5, 24.0, 40.0)),
]


def run_cases() -> dict:
    out = {}
    rng = np.random.default_rng(7)
    for name, gs, geo in GEOMS:
        grid = dgr.Grid.of(gs)
        ang = T(geo.angles)
        gg = dgr.Geom.of(geo, ang)
        f = synth.gaussian_field(synth.rng_for(1, 300 + len(out)), 300, gs, ("loguniform", 0.6, 3.0))
        f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
        ws = dgr.Workspace(dgr.make_plan(grid, f.n, 1 << 22, 1 << 20, gg, step=True))
        vol = T(rng.uniform(0, 1, gs.shape).astype(np.float32))
        sino = torch.empty(geo.shape, device=DEV)
        dgr.dgr_project(grid, gg, vol, sino, ws)
        out[f"{name}/sino"] = sino.cpu().numpy()
        out[f"{name}/status_project"] = np.int64(dgr.dgr_status(ws))
        r = T(rng.standard_normal(geo.shape).astype(np.float32))
        bp = torch.empty(gs.shape, device=DEV)
        dgr.dgr_backproject(grid, gg, r, bp, ws)
        out[f"{name}/bp"] = bp.cpu().numpy()
        out[f"{name}/status_backproject"] = np.int64(dgr.dgr_status(ws))
        # voxelize and its adjoint, then three optimisation steps
        v = torch.empty(gs.shape, device=DEV)
        dgr.dgr_voxelize(grid, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, v, ws)
        out[f"{name}/vox"] = v.cpu().numpy()
        g = [torch.empty((f.n, w), device=DEV) for w in (3, 3, 4)] + [torch.empty(f.n, device=DEV)]
        dgr.dgr_voxelize_backward(grid, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, vol, *g, ws)
        for k, t in zip(("g_mu", "g_s", "g_q", "g_rho"), g):
            out[f"{name}/{k}"] = t.cpu().numpy()
        out[f"{name}/status_fvr"] = np.int64(dgr.dgr_status(ws))
        prob = dgr.make_problem(grid, gg, 3.0, 1e-2, 1e-3, 10)
        st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
        dgr.dgr_params_init(prob, st)
        loss = torch.zeros(1, device=DEV)
        for _ in range(3):
            dgr.dgr_step(prob, st, sino, loss, ws)
        out[f"{name}/theta"] = st.theta[:11 * f.n].cpu().numpy()
        out[f"{name}/loss"] = loss.cpu().numpy()
        out[f"{name}/status_step"] = np.int64(dgr.dgr_status(ws))
    torch.cuda.synchronize()
    return out


def loaded_libraries() -> list:
    with open("/proc/self/maps") as fh:
        return sorted({line.split()[-1] for line in fh if "libdgr" in line})


if __name__ == "__main__":
    res = run_cases()
    res["libs"] = np.array(loaded_libraries())
    np.savez(sys.argv[1], **{k.replace("/", "__"): v for k, v in res.items()})
