"""Learned warm start of DGR reconstructions (on top of the method; the paper
initialises Gaussians from FBP or at random).

Pipeline, every numerical step in libdgr kernels:
  1. input: an FDK-style volume -- cosine-weighted, ramp-filtered projections
     (dgr_fdk_filter) backprojected with the exact adjoint (dgr_backproject)
     and scaled by pi / n_views;
  2. the network (dgr_net_forward; BF16 tensor cores) proposes per voxel a
     density and a log-scale (in voxels);
  3. seeding (dgr_seed): Gaussians drawn with probability proportional to the
     proposed density, isotropic scale from the proposed log-scale, intensity
     refined by a few fixed-point steps (dgr_voxelize + dgr_seed_rescale) so
     their voxelized field matches the proposal;
  4. the plain method continues from there (dgr_step / dgr_step_batched).
The fallback (and the yardstick for the network's error) is the plain FBP-seeded
initialisation: the same seeding with the clipped FDK volume as density and a
fixed scale.  Training targets come from fits of the plain method itself: the
voxelized fitted field (density) and the intensity-weighted mean log-scale of
the fitted Gaussians at each voxel.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import dgr, graph, synth

PLAIN_LOG_SCALE = math.log(1.5)


def psnr(vol, ref, peak=1.0):
    """10 log10(peak^2 / MSE) over the whole volume."""
    mse = float(((vol.double() - ref.double()) ** 2).mean())
    return 10.0 * math.log10(peak * peak / max(mse, 1e-30))


class Net:
    """Parameters (FP32 master copy), Adam state and activation workspace."""

    def __init__(self, n: int, seed: int = 0, device="cuda"):
        self.n = n
        rng = np.random.default_rng(seed)
        parts = []
        for ci, co, taps in ((1, 16, 27), (16, 32, 27), (32, 64, 27), (64, 32, 27), (32, 16, 27), (16, 2, 1)):
            parts.append(rng.standard_normal(taps * ci * co) * math.sqrt(2.0 / (taps * ci)))
            parts.append(np.zeros(co))
        p = np.concatenate(parts).astype(np.float32)
        assert p.size == dgr.dgr_net_param_count()
        self.params = torch.as_tensor(p, device=device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.ws = torch.empty(dgr.dgr_net_ws_bytes(n), dtype=torch.uint8, device=device)
        self.out = torch.empty((n, n, n, 2), device=device)
        self.gout = torch.empty_like(self.out)
        self.loss = torch.zeros(1, device=device)
        self.t = 0

    def forward(self, x):
        dgr.dgr_net_forward(self.n, self.params, x.contiguous(), self.out, self.ws)
        return self.out

    def train_step(self, x, target, lr, w_density=1.0, w_scale=0.1):
        x = x.contiguous()
        dgr.dgr_net_forward(self.n, self.params, x, self.out, self.ws)
        dgr.dgr_net_loss(self.n, self.out, target.contiguous(), w_density, w_scale, self.gout,
                         self.loss, self.ws)
        dgr.dgr_net_backward(self.n, self.params, x, self.gout, self.grads, self.ws)
        self.t += 1
        dgr.dgr_adam_flat(self.params, self.grads, self.m, self.v, self.t, lr)
        return self.loss

    def state(self):
        return {"params": self.params.cpu().numpy(), "t": self.t}


@dataclass
class Problem:
    """One reconstruction: grid, geometry, measured projections, phantom."""
    gs: synth.GridSpec
    geo: synth.GeomSpec
    phantom: torch.Tensor
    meas: torch.Tensor
    grid: dgr.Grid
    geom: dgr.Geom
    ang: torch.Tensor
    fdk: torch.Tensor = None


def make_problem(gs, geo, phantom_np, noise_sigma, noise_seed, device="cuda") -> Problem:
    grid = dgr.Grid.of(gs)
    ang = torch.as_tensor(geo.angles, device=device)
    geom = dgr.Geom.of(geo, ang)
    ph = torch.as_tensor(phantom_np, device=device)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, geom))
    meas = torch.empty(geo.shape, device=device)
    dgr.dgr_project(grid, geom, ph, meas, ws)
    if noise_sigma > 0:
        noise = np.random.default_rng(noise_seed).normal(0, noise_sigma, geo.shape).astype(np.float32)
        meas += torch.as_tensor(noise, device=device)
    P = Problem(gs, geo, ph, meas, grid, geom, ang)
    P.fdk = fdk_volume(P, ws)
    ws.close()
    return P


def fdk_volume(P: Problem, ws=None):
    """Cosine-weighted ramp-filtered backprojection with the FBP constant
    pi / N x pu pv / (M h^3) (M = dsd / dso; a ramp at detector pitch) folded
    into the filter."""
    own = ws is None
    if own:
        ws = dgr.Workspace(dgr.make_plan(P.grid, 0, 0, 0, P.geom))
    filt = torch.empty_like(P.meas)
    mag = P.geo.dsd / P.geo.dso if P.geo.beam == dgr.DGR_CONE else 1.0
    scale = math.pi / P.geo.n_views * (P.geo.pu * P.geo.pv) / (mag * P.gs.h ** 3)
    dgr.dgr_fdk_filter(P.geom, P.meas, filt, scale)
    vol = torch.empty(P.gs.shape, device=P.meas.device)
    dgr.dgr_backproject(P.grid, P.geom, filt, vol, ws)
    if own:
        ws.close()
    return vol


def seed(P: Problem, density, log_scale, ns, rng, rescale_iters=3):
    """Gaussians from proposals (see module doc).  Returns (mu, s, q, rho)."""
    dev = density.device
    n = P.gs.dims[0]
    u = torch.as_tensor(rng.uniform(0, 1, ns).astype(np.float32), device=dev)
    jit = torch.as_tensor(rng.uniform(-0.5, 0.5, (ns, 3)).astype(np.float32), device=dev)
    mu = torch.empty((ns, 3), device=dev); s = torch.empty((ns, 3), device=dev)
    q = torch.empty((ns, 4), device=dev); rho = torch.empty(ns, device=dev)
    vox = torch.empty(ns, dtype=torch.int32, device=dev)
    scratch = torch.empty(dgr.dgr_seed_bytes(n), dtype=torch.uint8, device=dev)
    dens = density.contiguous()
    dgr.dgr_seed(P.grid, dens, log_scale.contiguous(), u, jit, mu, s, q, rho, vox, scratch)
    ws0 = dgr.Workspace(dgr.make_plan(P.grid, ns))
    pairs, items = dgr.dgr_voxelize_count(P.grid, mu, s, q, 3.0, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(P.grid, ns, pairs + 64, items + 64))
    vol = torch.empty(P.gs.shape, device=dev)
    for _ in range(rescale_iters):
        dgr.dgr_voxelize(P.grid, mu, s, q, rho, 3.0, vol, ws)
        dgr.dgr_seed_rescale(vox, dens, vol, rho)
    ws.close()
    return mu, s, q, rho


def plain_init(P: Problem, ns, rng):
    """The fallback: FBP-seeded Gaussians of a fixed scale (1.5 voxels)."""
    dens, logs = torch.empty_like(P.fdk), torch.empty_like(P.fdk)
    dgr.dgr_proposals(P.fdk, 1, PLAIN_LOG_SCALE, dens, logs)
    return seed(P, dens, logs, ns, rng)


def learned_init(P: Problem, net: Net, ns, rng):
    out = net.forward(P.fdk)
    dens, logs = torch.empty_like(P.fdk), torch.empty_like(P.fdk)
    dgr.dgr_proposals(out, 2, PLAIN_LOG_SCALE, dens, logs)
    return seed(P, dens, logs, ns, rng)


class Fit:
    """Batched fits of several problems (one dgr_step_batched per iteration,
    captured in a CUDA graph)."""

    def __init__(self, probs: list, inits: list, lr0=3e-3, lr1=3e-4, n_iters=300):
        self.P = probs
        self.states = [dgr.State(*init) for init in inits]
        self.problems = [dgr.make_problem(p.grid, p.geom, 3.0, lr0, lr1, n_iters) for p in probs]
        for pr, st in zip(self.problems, self.states):
            dgr.dgr_params_init(pr, st)
        self.loss = torch.zeros(len(probs), device=probs[0].meas.device)
        self._plan(slack=1.6)
        self.g = None
        self.vol_ws = None

    def _plan(self, slack):
        pairs, items = [], []
        for p, st in zip(self.P, self.states):
            ws0 = dgr.Workspace(dgr.make_plan(p.grid, st.n))
            pp, it = dgr.dgr_voxelize_count(p.grid, st.mu, st.s, st.q, 3.0, ws0)
            ws0.close()
            pairs.append(int(pp * slack) + 1024); items.append(int(it * slack) + 1024)
        self.ws = dgr.Workspace(dgr.make_batch_plan([p.grid for p in self.P], [p.geom for p in self.P],
                                                    [st.n for st in self.states], pairs, items))

    def keep(self, idx):
        """Restrict the batch to the instances at positions idx: their states
        (parameters, Adam moments, step counters) carry on; the workspace is
        planned again for them and the next step captures a new graph."""
        self.g = None
        self.ws.close()
        self.P = [self.P[i] for i in idx]
        self.states = [self.states[i] for i in idx]
        self.problems = [self.problems[i] for i in idx]
        self.loss = torch.zeros(len(idx), device=self.loss.device)
        self._plan(slack=1.6)

    def step(self, k=1):
        if self.g is None:
            self.g = graph.batched_step_graph(self.problems, self.states, [p.meas for p in self.P],
                                              self.loss, self.ws, warmup=1)
            k -= 1
        for _ in range(k):
            self.g.replay()

    def volumes(self):
        out = []
        for p, st in zip(self.P, self.states):
            ws0 = dgr.Workspace(dgr.make_plan(p.grid, st.n))
            pp, it = dgr.dgr_voxelize_count(p.grid, st.mu, st.s, st.q, 3.0, ws0)
            ws0.close()
            ws = dgr.Workspace(dgr.make_plan(p.grid, st.n, pp + 64, it + 64))
            v = torch.empty(p.gs.shape, device=p.meas.device)
            dgr.dgr_voxelize(p.grid, st.mu, st.s, st.q, st.rho, 3.0, v, ws)
            out.append(v)
        return out

    def psnrs(self):
        return [psnr(v, p.phantom) for v, p in zip(self.volumes(), self.P)]

    def status(self):
        return dgr.dgr_status(self.ws)


def targets_from_fit(P: Problem, st: dgr.State):
    """[n,n,n,2]: voxelized fitted density; intensity-weighted mean log-scale
    (geometric mean of the axis scales, in voxels) where the density is
    significant, the plain log-scale elsewhere."""
    dev = P.meas.device
    ws0 = dgr.Workspace(dgr.make_plan(P.grid, st.n))
    pp, it = dgr.dgr_voxelize_count(P.grid, st.mu, st.s, st.q, 3.0, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(P.grid, st.n, pp + 64, it + 64))
    mu, s, q, rho = st.view()
    dens = torch.empty(P.gs.shape, device=dev)
    dgr.dgr_voxelize(P.grid, mu, s, q, rho, 3.0, dens, ws)
    w = torch.empty_like(rho)
    dgr.dgr_logscale_weight(s, rho, P.gs.h, w)
    wsum = torch.empty_like(dens)
    dgr.dgr_voxelize(P.grid, mu, s, q, w, 3.0, wsum, ws)
    out = torch.empty(P.gs.shape + (2,), device=dev)
    dgr.dgr_fit_targets(dens, wsum, 1e-3, math.log(0.3), math.log(8.0), PLAIN_LOG_SCALE, out)
    ws.close()
    return out
