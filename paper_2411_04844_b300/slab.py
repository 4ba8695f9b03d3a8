"""Z-slab split of one reconstruction over several GPUs (one process each).

The voxel sum is additive over Gaussians (Eq. 4) and the line integral over
path segments (Sec. 4.3, P_hat = T(V)), so one optimisation iteration splits
over G ranks that each own a z-slab of the volume:

  rank r: layers [z0_r, z0_r + nz_r) (boundaries on multiples of 32, the
          voxelizer's tile depth, so a slab's values are bit-identical to the
          whole grid's), every Gaussian's parameters (replicated: Gaussians
          whose boxes cross a boundary contribute to both slabs), and the
          views [v0_r, v0_r + nv_r) of the measured projections.

  1. voxelize the slab                          (dgr_voxelize, slab grid)
  2. project the slab: every ray's segment sum  (dgr_project, slab grid)
  3. reduce-scatter the partial sinograms by views: rank r gets the whole
     prediction of its views
  4. L1 loss and residual of its views, weighted by (its rays / all rays)
  5. all-gather the residual
  6. backproject it onto the slab               (dgr_backproject, slab grid)
  7. voxelize adjoint on the slab: each Gaussian's gradient from the slab's
     voxels                                     (dgr_voxelize_backward)
  8. all-reduce the gradients and the loss (sums)
  9. Adam on every Gaussian, identical on every rank (dgr_adam)

The arithmetic of every step runs in libdgr kernels; the collectives are
torch.distributed's (NCCL on GPUs).  Views are padded with zeros to a
multiple of G for the equal-chunk collectives.  The compute of steps 1, 2, 4,
6, 7 and 9 goes through a backend object (CudaBackend: libdgr on the rank's
GPU); the orchestration -- partition, padding, weights and the order of the
exchanges -- is this module's.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import dgr

SLAB_ALIGN = 32  # the voxelizer's tile depth


def partition(nz: int, world: int, align: int = SLAB_ALIGN):
    """Contiguous z-slabs [(z0, nz_r)] of a grid of nz layers over `world`
    ranks: blocks of `align` layers (the last one ragged) dealt out as evenly
    as possible, lower ranks first.  A rank gets no layers (nz_r = 0) only if
    there are fewer blocks than ranks."""
    if nz < 1 or world < 1 or align < 1:
        raise ValueError("partition: nz, world and align must be positive")
    blocks = -(-nz // align)
    out, z = [], 0
    for r in range(world):
        nb = blocks // world + (1 if r < blocks % world else 0)
        z1 = min(nz, z + nb * align)
        out.append((z, z1 - z))
        z = z1
    assert z == nz
    return out


def view_split(n_views: int, world: int):
    """Views [(v0, nv_r)] of each rank for the reduce-scatter: chunks of
    ceil(n_views / world) (the last ones shorter or empty) and the padded
    view count world x chunk."""
    chunk = -(-n_views // world)
    out = [(min(r * chunk, n_views), max(0, min(chunk, n_views - r * chunk))) for r in range(world)]
    return out, chunk * world


class TorchComm:
    """The collectives of the split over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def reduce_scatter(self, full: torch.Tensor) -> torch.Tensor:
        """full [world x chunk, ...] summed over ranks; returns this rank's chunk."""
        out = torch.empty((full.shape[0] // self.world,) + tuple(full.shape[1:]), dtype=full.dtype,
                          device=full.device)
        self.dist.reduce_scatter_tensor(out, full.contiguous(), group=self.group)
        return out

    def all_gather(self, mine: torch.Tensor) -> torch.Tensor:
        out = torch.empty((mine.shape[0] * self.world,) + tuple(mine.shape[1:]), dtype=mine.dtype,
                          device=mine.device)
        self.dist.all_gather_into_tensor(out, mine.contiguous(), group=self.group)
        return out

    def all_reduce(self, t: torch.Tensor) -> torch.Tensor:
        self.dist.all_reduce(t, group=self.group)
        return t


@dataclass
class SlabSpec:
    """What one rank of the split owns."""
    rank: int
    world: int
    z0: int
    nz: int
    v0: int
    nv: int
    chunk: int       # views per rank in the padded collectives
    n_views: int     # all views
    rays_per_view: int

    @property
    def weight(self) -> float:
        """This rank's share of the L1 mean: its rays / all rays."""
        return self.nv / self.n_views


def slab_spec(nz: int, n_views: int, rays_per_view: int, rank: int, world: int) -> SlabSpec:
    z0, nzr = partition(nz, world)[rank]
    views, padded = view_split(n_views, world)
    v0, nvr = views[rank]
    return SlabSpec(rank, world, z0, nzr, v0, nvr, padded // world, n_views, rays_per_view)


class SlabRank:
    """One rank's part of one optimisation iteration, phase by phase, on a
    backend (see the module doc).  Between the phases the caller runs the
    collectives:

        part = r.forward()                        # [padded views, nv, nu]
        pred = reduce_scatter(part)               # [chunk, nv, nu]
        resid, loss = r.residual(pred, meas_mine)
        resid_all = all_gather(resid)             # [padded views, nv, nu]
        grads = r.backward(resid_all)             # [11 n] (mu 3n | s 3n | q 4n | rho n)
        grads = all_reduce(grads); loss = all_reduce(loss)
        r.update(grads)
    """

    def __init__(self, spec: SlabSpec, backend):
        self.spec = spec
        self.be = backend

    def forward(self):
        S = self.spec
        part = self.be.zeros_sino(S.chunk * S.world)
        if S.nz > 0:
            vol = self.be.voxelize(S.z0, S.nz)
            self.be.project(S.z0, S.nz, vol, part[:S.n_views])
        return part

    def residual(self, pred_chunk, meas_mine):
        """pred_chunk: this rank's views of the summed prediction (padded
        chunk); meas_mine: the measured projections of its nv views."""
        S = self.spec
        resid = self.be.zeros_sino(S.chunk)
        loss = self.be.zeros_scalar()
        if S.nv > 0:
            self.be.l1(pred_chunk[:S.nv], meas_mine, S.weight, resid[:S.nv], loss)
        return resid, loss

    def backward(self, resid_all):
        S = self.spec
        if S.nz == 0:
            return self.be.zeros_grads()
        gvol = self.be.backproject(S.z0, S.nz, resid_all[:S.n_views])
        return self.be.voxelize_backward(S.z0, S.nz, gvol)

    def update(self, grads):
        self.be.adam(grads)


def run_step(rank: SlabRank, comm, meas_mine):
    """One iteration of one rank with its collectives; returns the loss (the
    whole objective's, identical on every rank)."""
    part = rank.forward()
    pred = comm.reduce_scatter(part)
    resid, loss = rank.residual(pred, meas_mine)
    resid_all = comm.all_gather(resid)
    grads = rank.backward(resid_all)
    comm.all_reduce(grads)
    comm.all_reduce(loss)
    rank.update(grads)
    return loss


def run_step_emulated(ranks, meas_parts):
    """One iteration of all ranks of a split in one process (one GPU): each
    phase runs to completion on every rank, then the collectives are sums on
    the device between phases.  Returns the loss."""
    W = len(ranks)
    parts = [r.forward() for r in ranks]
    total = torch.stack(parts).sum(0)
    chunk = ranks[0].spec.chunk
    res = [r.residual(total[i * chunk:(i + 1) * chunk], m) for i, (r, m) in enumerate(zip(ranks, meas_parts))]
    resid_all = torch.cat([x for x, _ in res])
    loss = torch.stack([l for _, l in res]).sum(0)
    grads = torch.stack([r.backward(resid_all) for r in ranks]).sum(0)
    for r in ranks:
        r.update(grads.clone())
    return loss


class CudaBackend:
    """libdgr on the rank's GPU: the whole grid (z0 = 0) and its geometry,
    every Gaussian's optimiser state (replicated), slab workspaces."""

    def __init__(self, prob: dgr.Problem, state: dgr.State, spec: SlabSpec, device="cuda"):
        self.prob = prob
        self.state = state
        self.spec = spec
        self.dev = device
        g = prob.grid
        geo = prob.geom
        self.k = prob.k_trunc
        self.sino_shape = (geo.nv, geo.nu)
        n = state.n
        if spec.nz > 0:
            sg = g.slab(spec.z0, spec.nz)
            self.sgrid = sg
            mu, s, q, rho = state.view()
            ws0 = dgr.Workspace(dgr.make_plan(sg, n))
            pairs, items = dgr.dgr_voxelize_count(sg, mu, s, q, self.k, ws0)
            ws0.close()
            self.ws = dgr.Workspace(dgr.make_plan(sg, n, int(pairs * 1.5) + 1024,
                                                  int(items * 1.5) + 1024, geo))
        else:
            self.ws = dgr.Workspace(dgr.make_plan(g, 0))
        self.grads = torch.zeros(11 * n, device=device)

    def zeros_sino(self, views):
        return torch.zeros((views,) + self.sino_shape, device=self.dev)

    def zeros_scalar(self):
        return torch.zeros(1, device=self.dev)

    def zeros_grads(self):
        return torch.zeros(11 * self.state.n, device=self.dev)

    def voxelize(self, z0, nz):
        vol = torch.empty((nz, self.sgrid.ny, self.sgrid.nx), device=self.dev)
        dgr.dgr_voxelize(self.sgrid, *self.state.view(), self.k, vol, self.ws)
        return vol

    def project(self, z0, nz, vol, out):
        dgr.dgr_project(self.sgrid, self.prob.geom, vol, out, self.ws)

    def l1(self, pred, meas, weight, resid, loss):
        dgr.dgr_l1_residual(pred.contiguous(), meas, resid, loss, self.ws, weight)

    def backproject(self, z0, nz, resid):
        gvol = torch.empty((nz, self.sgrid.ny, self.sgrid.nx), device=self.dev)
        dgr.dgr_backproject(self.sgrid, self.prob.geom, resid.contiguous(), gvol, self.ws)
        return gvol

    def voxelize_backward(self, z0, nz, gvol):
        n = self.state.n
        g = torch.empty(11 * n, device=self.dev)
        gm, gs, gq, gr = (g[:3 * n].view(n, 3), g[3 * n:6 * n].view(n, 3), g[6 * n:10 * n].view(n, 4),
                          g[10 * n:])
        dgr.dgr_voxelize_backward(self.sgrid, *self.state.view(), self.k, gvol, gm, gs, gq, gr, self.ws)
        return g

    def adam(self, grads):
        n = self.state.n
        dgr.dgr_adam(self.prob, self.state, grads[:3 * n].view(n, 3), grads[3 * n:6 * n].view(n, 3),
                     grads[6 * n:10 * n].view(n, 4), grads[10 * n:])

    def status(self):
        return dgr.dgr_status(self.ws)
