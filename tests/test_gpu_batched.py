"""Batching (row a10): dgr_step_batched over heterogeneous instances equals the
same instances stepped one by one with dgr_step, bit for bit (deterministic
mode; one instance dense enough that the voxelizer splits its tile lists);
a CUDA-graph replay equals eager steps; every voxelizer tile depth the
autotuner may pick gives the oracle's volume."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, graph, synth
from tests._common import guard_field, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _instances():
    specs = [
        (synth.GridSpec((24, 24, 24), 1.0, (-12.0, -12.0, -12.0)), synth.parallel_geom(10, 30, 26), 150),
        (synth.GridSpec((33, 29, 21), 0.8, (-12.0, -13.0, -9.0)),
         synth.cone_geom(13, 41, 31, 1.1, 1.3, 60.0, 95.0, arc=1.3), 300),
        (synth.GridSpec((40, 40, 40), 1.0, (-20.0, -20.0, -20.0)),
         synth.cone_geom(20, 50, 44, 1.5, 1.5, 120.0, 180.0), 500),
        # few tiles holding thousands of Gaussians each: the voxelizer splits
        # their lists over several CTAs (the same way alone and in the batch)
        (synth.GridSpec((16, 16, 32), 1.0, (-8.0, -8.0, -16.0)), synth.parallel_geom(8, 24, 34), 4000),
    ]
    out = []
    for i, (gs, geo, n) in enumerate(specs):
        scale = ("loguniform", 0.5, 1.5) if n > 1000 else ("loguniform", 0.5, 3.0)
        f = synth.gaussian_field(synth.rng_for(4, 50 + i), n, gs, scale)
        f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
        meas = np.abs(np.random.default_rng(i).normal(3.0, 1.0, geo.shape)).astype(np.float32)
        out.append((gs, geo, f, meas))
    return out


class Built:
    def __init__(self, insts, batched_ws=True):
        self.grids = [dgr.Grid.of(gs) for gs, _, _, _ in insts]
        self.angs = [T(geo.angles) for _, geo, _, _ in insts]
        self.geoms = [dgr.Geom.of(geo, a) for (_, geo, _, _), a in zip(insts, self.angs)]
        self.probs = [dgr.make_problem(g, ge, 3.0, 3e-4, 3e-5, 20) for g, ge in zip(self.grids, self.geoms)]
        self.meas = [T(m) for _, _, _, m in insts]
        self.states = [dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho)) for _, _, f, _ in insts]
        for p, st in zip(self.probs, self.states):
            dgr.dgr_params_init(p, st)
        pairs, items = [], []
        for g, (_, _, f, _) in zip(self.grids, insts):
            ws0 = dgr.Workspace(dgr.make_plan(g, f.n))
            pp, it = dgr.dgr_voxelize_count(g, T(f.mu), T(f.s), T(f.q), 3.0, ws0)
            ws0.close()
            pairs.append(2 * pp + 64); items.append(2 * it + 64)
        self.pairs, self.items = pairs, items
        self.ns = [f.n for _, _, f, _ in insts]
        self.ws = dgr.Workspace(dgr.make_batch_plan(self.grids, self.geoms, self.ns, pairs, items))
        self.single_ws = [dgr.Workspace(dgr.make_plan(g, n, p, it, ge, step=True))
                          for g, ge, n, p, it in zip(self.grids, self.geoms, self.ns, pairs, items)]
        self.loss = torch.zeros(len(insts), device=DEV)

    def batched(self):
        dgr.dgr_step_batched(self.probs, self.states, self.meas, self.loss, self.ws)

    def sequential(self):
        for i in range(len(self.probs)):
            dgr.dgr_step(self.probs[i], self.states[i], self.meas[i], self.loss[i:i + 1], self.single_ws[i])

    def snapshot(self):
        torch.cuda.synchronize()
        return [torch.cat([st.theta, st.m, st.v, st.mu.flatten(), st.s.flatten(), st.q.flatten(),
                           st.rho.flatten(), st.step.float()]).clone() for st in self.states] + \
               [self.loss.clone()]


def test_batched_step_equals_sequential_steps_bitwise():
    insts = _instances()
    a, b = Built(insts), Built(insts)
    for _ in range(2):
        a.batched()
        b.sequential()
    assert dgr.dgr_status(a.ws) == 0
    for x, y in zip(a.snapshot(), b.snapshot()):
        assert torch.equal(x, y)


def test_graph_replay_equals_eager():
    insts = _instances()
    a, b = Built(insts), Built(insts)
    g = graph.batched_step_graph(a.probs, a.states, a.meas, a.loss, a.ws, warmup=1)
    b.batched()  # the capture's warm-up step
    for _ in range(2):
        g.replay()
        b.batched()
    for x, y in zip(a.snapshot(), b.snapshot()):
        assert torch.equal(x, y)


@pytest.mark.parametrize("depth", [8, 16])
def test_voxelize_parity_every_tile_depth(depth):
    gs = synth.GridSpec((45, 37, 29), 0.7, (-13.3, 2.1, -40.0))
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 2), 700, gs, ("loguniform", 0.4, 4.0),
                                         unnormalised_q=True), gs)
    try:
        dgr.dgr_set_tile_depth(depth)
        grid = dgr.Grid.of(gs)
        ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
        pairs, items = dgr.dgr_voxelize_count(grid, T(f.mu), T(f.s), T(f.q), 3.0, ws0)
        ws = dgr.Workspace(dgr.make_plan(grid, f.n, pairs + 64, items + 64))
        vol = torch.empty(gs.shape, device=DEV)
        dgr.dgr_voxelize(grid, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, vol, ws)
        torch.cuda.synchronize()
        assert dgr.dgr_status(ws) == 0
    finally:
        dgr.dgr_set_tile_depth(32)
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)
    assert rel_l2(vol.cpu().numpy(), vo) <= 1e-5
    assert np.max(np.abs(vol.cpu().numpy() - vo)) <= 1e-5 * float(f.rho.max())
