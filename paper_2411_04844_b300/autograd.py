"""torch.autograd.Function wrappers of the C ABI (differentiation of the hot path).

    vox = Voxelizer(grid_spec, k_trunc=3.0)
    proj = Projector(grid_spec, geom_spec)
    vol = voxelize(vox, mu, s, q, rho)          # dgr_voxelize
    sino = project(proj, vol)                   # dgr_project
    loss = (sino - meas).abs().mean()
    loss.backward()                             # dgr_backproject, dgr_voxelize_backward

Only the inputs (mu, s, q, rho) are saved for backward: the exponentials of
every (Gaussian, voxel) pair are recomputed in dgr_voxelize_backward instead
of being stored (the paper's Gamma tensor would take 4 bytes per pair, ~24 GB
for 500K Gaussians at 512^3).  Workspaces grow on demand: before each call
the exact work-list sizes are counted (one small synchronising launch).
"""
from __future__ import annotations

import torch

from . import dgr


class Voxelizer:
    """A voxel grid, a truncation factor and a workspace that grows with the
    Gaussian count and the work lists."""

    def __init__(self, grid_spec, k_trunc: float = 3.0, slack: float = 1.25):
        self.grid = dgr.Grid.of(grid_spec)
        self.shape = self.grid.shape
        self.k = float(k_trunc)
        self.slack = slack
        self.ws = None

    def _ensure(self, mu, s, q):
        n = mu.shape[0]
        if self.ws is None or n > self.ws.plan.max_n:
            self.ws = dgr.Workspace(dgr.make_plan(self.grid, max(n, 1)))
        pairs, items = dgr.dgr_voxelize_count(self.grid, mu, s, q, self.k, self.ws)
        p = self.ws.plan
        if pairs > p.max_pairs or items > p.max_items:
            self.ws.close()
            self.ws = dgr.Workspace(dgr.make_plan(self.grid, max(n, 1), int(pairs * self.slack) + 64,
                                                  int(items * self.slack) + 64))
        return self.ws


class _VoxelizeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vox: Voxelizer, mu, s, q, rho):
        mu, s, q, rho = (t.contiguous() for t in (mu, s, q, rho))
        ws = vox._ensure(mu, s, q)
        vol = torch.empty(vox.shape, device=mu.device, dtype=torch.float32)
        dgr.dgr_voxelize(vox.grid, mu, s, q, rho, vox.k, vol, ws)
        ctx.vox = vox
        ctx.save_for_backward(mu, s, q, rho)
        return vol

    @staticmethod
    def backward(ctx, grad_vol):
        mu, s, q, rho = ctx.saved_tensors
        vox = ctx.vox
        ws = vox._ensure(mu, s, q)
        g = [torch.empty_like(t) for t in (mu, s, q, rho)]
        dgr.dgr_voxelize_backward(vox.grid, mu, s, q, rho, vox.k, grad_vol.contiguous(), *g, ws)
        return (None, *g)


def voxelize(vox: Voxelizer, mu, s, q, rho):
    """Differentiable FVR forward: [nz, ny, nx] volume."""
    return _VoxelizeFn.apply(vox, mu, s, q, rho)


class Projector:
    """A grid, a scan geometry (angles kept on the device) and a workspace."""

    def __init__(self, grid_spec, geom_spec, device="cuda"):
        self.grid = dgr.Grid.of(grid_spec)
        self.angles = torch.as_tensor(geom_spec.angles, dtype=torch.float32, device=device).contiguous()
        self.geom = dgr.Geom.of(geom_spec, self.angles)
        self.vol_shape = self.grid.shape
        self.sino_shape = self.geom.shape
        self.ws = dgr.Workspace(dgr.make_plan(self.grid, 0, 0, 0, self.geom))


class _ProjectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, proj: Projector, vol):
        vol = vol.contiguous()
        sino = torch.empty(proj.sino_shape, device=vol.device, dtype=torch.float32)
        dgr.dgr_project(proj.grid, proj.geom, vol, sino, proj.ws)
        ctx.proj = proj
        return sino

    @staticmethod
    def backward(ctx, grad_sino):
        proj = ctx.proj
        g = torch.empty(proj.vol_shape, device=grad_sino.device, dtype=torch.float32)
        dgr.dgr_backproject(proj.grid, proj.geom, grad_sino.contiguous(), g, proj.ws)
        return None, g


def project(proj: Projector, vol):
    """Differentiable projector: [n_views, nv, nu] line integrals."""
    return _ProjectFn.apply(proj, vol)
