"""The z-slab split of one reconstruction over several ranks (one process per
GPU in production), checked on CPU: the partition, and the whole exchange
arithmetic -- slab voxelization, per-slab projection of every ray, the
reduce-scatter of the partial sinograms by views, the weighted L1 residual of
each rank's views, the all-gather of the residual, per-slab backprojection and
voxelize adjoint, the all-reduce of the gradients, replicated Adam -- as 2 and
3 gloo ranks whose compute is the FP64 oracle, against the oracle's own
iteration of the whole problem in one process.

The split rests on two additivities: the voxel sum over Gaussians (Eq. 4;
each slab holds the whole grid's values on its layers) and the line integral
over the segments of a ray (Sec. 4.3, P_hat = T(V); the slabs' partial
projections add up to the whole one).  In FP64 the split and the whole agree
to rounding (relative 1e-10 here)."""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import slab, synth
from tests._common import oracle_geom, oracle_grid

LR0, LR1, N_ITERS, STEPS = 3e-3, 3e-4, 10, 2


def test_partition_covers_the_grid_on_tile_boundaries():
    for nz in (1, 31, 32, 33, 80, 256, 1000):
        for world in (1, 2, 3, 4, 8):
            P = slab.partition(nz, world)
            assert len(P) == world
            z = 0
            for z0, n in P:
                assert z0 == z and n >= 0
                if n > 0 and z0 + n < nz:
                    assert (z0 + n) % slab.SLAB_ALIGN == 0
                z += n
            assert z == nz
            sizes = [n for _, n in P if n > 0 and _ + n < nz]
            assert not sizes or max(sizes) - min(sizes) <= slab.SLAB_ALIGN
    for nv in (1, 5, 9, 10, 50):
        for world in (1, 2, 3, 4):
            views, padded = slab.view_split(nv, world)
            assert padded % world == 0 and padded >= nv
            assert sum(n for _, n in views) == nv
            assert all(v0 == r * (padded // world) or n == 0 for r, (v0, n) in enumerate(views))


def _problem():
    gs = synth.GridSpec((40, 36, 80), 1.0, (-20.0, -18.0, -40.0))
    geo = synth.cone_geom(10, 48, 88, 1.5, 1.5, 150.0, 225.0)
    f = synth.gaussian_field(synth.rng_for(1, 41), 200, gs, ("loguniform", 0.5, 3.0))
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    phantom = synth.ellipsoid_phantom(synth.rng_for(1, 42), gs, 5)
    og, oo = oracle_grid(gs), oracle_geom(geo)
    meas = O.project(og, oo, phantom)
    return gs, geo, f, og, oo, meas


class OracleBackend:
    """One rank's compute in FP64 by the oracle, the slab semantics taken
    from their definitions: a slab's volume is the whole grid's on its
    layers; its projection is the exact line integral over the slab's box;
    its adjoint gradient is the whole grid's with G_V zero outside it."""

    def __init__(self, gs, geo, f, og, oo):
        self.gs, self.og, self.oo = gs, og, oo
        self.shape = (geo.nv, geo.nu)
        self.th = O.to_opt(og, *(a.astype(np.float64) for a in (f.mu, f.s, f.q, f.rho)))
        self.m = {k: np.zeros_like(a) for k, a in self.th.items()}
        self.v = {k: np.zeros_like(a) for k, a in self.th.items()}
        self.t = 1
        self.n = f.n

    def _params(self):
        p64 = O.from_opt(self.og, self.th)
        p32 = [a.astype(np.float32) for a in p64]
        _, box = O.footprint(self.og, p32[0], p32[1], p32[2], 3.0)
        return p64, box

    def _slab_grid(self, z0, nz):
        nx, ny, _ = self.gs.dims
        ox, oy, oz = self.gs.org
        return O.Grid((nx, ny, nz), self.gs.h, (ox, oy, oz + z0 * self.gs.h))

    def zeros_sino(self, views):
        return torch.zeros((views,) + self.shape, dtype=torch.float64)

    def zeros_scalar(self):
        return torch.zeros(1, dtype=torch.float64)

    def zeros_grads(self):
        return torch.zeros(11 * self.n, dtype=torch.float64)

    def voxelize(self, z0, nz):
        p64, box = self._params()
        return O.voxelize_core(self.og, *p64, box)[z0:z0 + nz]

    def project(self, z0, nz, vol, out):
        out.copy_(torch.from_numpy(O.project(self._slab_grid(z0, nz), self.oo, vol)))

    def l1(self, pred, meas, weight, resid, loss):
        lo, r = O.l1_loss(pred.numpy(), np.asarray(meas))
        resid.copy_(torch.from_numpy(weight * r))
        loss.fill_(weight * lo)

    def backproject(self, z0, nz, resid):
        return O.backproject(self._slab_grid(z0, nz), self.oo, resid.numpy())

    def voxelize_backward(self, z0, nz, gvol):
        p64, box = self._params()
        full = np.zeros(self.gs.shape)
        full[z0:z0 + nz] = gvol
        g = O.voxelize_backward_core(self.og, *p64, box, full)
        return torch.from_numpy(np.concatenate([a.reshape(-1) for a in g]))

    def adam(self, grads):
        n = self.n
        g = grads.numpy()
        parts = (g[:3 * n].reshape(n, 3), g[3 * n:6 * n].reshape(n, 3), g[6 * n:10 * n].reshape(n, 4),
                 g[10 * n:])
        self.th, _ = O.optimiser_step(self.og, self.th, self.m, self.v, self.t, parts, LR0, LR1, N_ITERS)
        self.t += 1


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        gs, geo, f, og, oo, meas = _problem()
        spec = slab.slab_spec(gs.dims[2], geo.n_views, geo.nu * geo.nv, rank, world)
        be = OracleBackend(gs, geo, f, og, oo)
        r = slab.SlabRank(spec, be)
        comm = slab.TorchComm()
        losses = []
        for _ in range(STEPS):
            meas_mine = torch.from_numpy(meas[spec.v0:spec.v0 + spec.nv].copy())
            losses.append(float(slab.run_step(r, comm, meas_mine)))
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), losses=np.array(losses),
                 **{k: a for k, a in be.th.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_split_iterations_on_gloo_ranks_match_the_whole_problem(world, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    gs, geo, f, og, oo, meas = _problem()
    th = O.to_opt(og, *(a.astype(np.float64) for a in (f.mu, f.s, f.q, f.rho)))
    m = {k: np.zeros_like(a) for k, a in th.items()}
    v = {k: np.zeros_like(a) for k, a in th.items()}
    ref_losses = []
    for t in range(1, STEPS + 1):
        p32 = [a.astype(np.float32) for a in O.from_opt(og, th)]
        lo, th, _ = O.step(og, oo, *p32, th, m, v, t, meas, 3.0, LR0, LR1, N_ITERS)
        ref_losses.append(lo)
    for rank in range(world):
        got = np.load(tmp_path / f"rank{rank}.npz")
        assert np.allclose(got["losses"], ref_losses, rtol=1e-10, atol=0)
        for k in th:
            # every rank holds the same parameters (replicated Adam on summed gradients)
            assert np.allclose(got[k], th[k], rtol=1e-10, atol=1e-12), (rank, k)
