"""The z-slab split on one GPU, through the C ABI: slab grids (dgr_grid.z0)
for voxelize, project, backproject and the voxelize adjoint against the whole
grid, and whole split iterations of 2 and 3 ranks emulated in one process
(each phase runs to completion on every rank; the collectives are sums on the
device between phases -- no kernel waits on another) against dgr_step of the
whole problem and the FP64 oracle.  A single-rank NCCL group runs the same
per-rank code through torch.distributed's collectives.

Tolerances: slab volumes bit-identical to the whole grid's layers when the
slab starts on a multiple of the tile depth (32), else the volume bounds of
the parity tests (relative L2 <= 1e-5, max-abs <= 1e-5 max rho); projections and backprojections (non-negative data)
relative L2 <= 1e-5; gradients relative L2 <= 1e-5 per kind against the whole
grid's (the same FP32 moments, split differently); a split step vs dgr_step
and the oracle: loss within 1e-5 of the mean measured projection (the loss is
a mean of margins, its error that of the prediction) for three steps; after
the first, m and v relative L2 <= 2e-4 and the moves of entries with a
non-negligible gradient within 1e-2 lr."""
import datetime
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, slab, synth
from tests._common import guard_field, margin_measurement, oracle_geom, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _setup(guard=False):
    gs = synth.GridSpec((64, 48, 96), 1.0, (-32.0, -24.0, -48.0))
    geo = synth.cone_geom(16, 72, 100, 1.5, 1.5, 200.0, 300.0)
    f = synth.gaussian_field(synth.rng_for(1, 61), 2000, gs, ("loguniform", 0.5, 4.0))
    if guard:
        # several steps against the oracle: keep every footprint integer off
        # its rounding edge while the parameters move
        f = guard_field(f, gs, band=0.03)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    geom = dgr.Geom.of(geo, ang)
    return gs, geo, f, grid, ang, geom


def _ws(grid, f, geom=None):
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, T(f.mu), T(f.s), T(f.q), 3.0, ws0)
    ws0.close()
    return dgr.Workspace(dgr.make_plan(grid, f.n, pairs + 1024, items + 1024, geom))


def _vox(grid, f, shape):
    ws = _ws(grid, f)
    v = torch.empty(shape, device=DEV)
    dgr.dgr_voxelize(grid, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, v, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) == 0
    return v


def test_slab_voxelize_is_the_whole_grid_on_its_layers():
    gs, geo, f, grid, ang, geom = _setup()
    whole = _vox(grid, f, gs.shape)
    for z0, nz in slab.partition(gs.dims[2], 3):
        part = _vox(grid.slab(z0, nz), f, (nz, gs.dims[1], gs.dims[0]))
        assert torch.equal(part, whole[z0:z0 + nz]), (z0, nz)
    # a slab off the tile boundaries: other tiles, other summation chunks
    part = _vox(grid.slab(20, 37), f, (37, gs.dims[1], gs.dims[0]))
    ref = whole[20:57].double()
    assert rel_l2(part.cpu().numpy(), ref.cpu().numpy()) <= 1e-5
    assert float((part.double() - ref).abs().max()) <= 1e-5 * float(f.rho.max())
    # footprint integers of a slab: the whole grid's, shifted and clipped
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)[20:57]
    assert rel_l2(part.cpu().numpy(), vo) <= 1e-5


def test_slab_projections_add_up_and_backprojections_restrict():
    gs, geo, f, grid, ang, geom = _setup()
    rng = np.random.default_rng(5)
    vol = rng.uniform(0, 1, gs.shape).astype(np.float32)
    y = np.abs(rng.standard_normal(geo.shape)).astype(np.float32)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, geom))
    whole_p = torch.empty(geo.shape, device=DEV)
    dgr.dgr_project(grid, geom, T(vol), whole_p, ws)
    whole_b = torch.empty(gs.shape, device=DEV)
    dgr.dgr_backproject(grid, geom, T(y), whole_b, ws)
    tot = torch.zeros(geo.shape, device=DEV, dtype=torch.float64)
    for z0, nz in slab.partition(gs.dims[2], 3):
        sg = grid.slab(z0, nz)
        wss = dgr.Workspace(dgr.make_plan(sg, 0, 0, 0, geom))
        p = torch.empty(geo.shape, device=DEV)
        dgr.dgr_project(sg, geom, T(vol[z0:z0 + nz]), p, wss)
        tot += p.double()
        b = torch.empty((nz, gs.dims[1], gs.dims[0]), device=DEV)
        dgr.dgr_backproject(sg, geom, T(y), b, wss)
        torch.cuda.synchronize()
        assert rel_l2(b.cpu().numpy(), whole_b[z0:z0 + nz].cpu().numpy()) <= 1e-5, (z0, nz)
    so = O.project(oracle_grid(gs), oracle_geom(geo), vol)
    assert rel_l2(tot.cpu().numpy(), whole_p.cpu().numpy()) <= 1e-5
    assert rel_l2(tot.cpu().numpy(), so) <= 1e-5


def test_slab_adjoints_add_up_to_the_whole_grids():
    gs, geo, f, grid, ang, geom = _setup()
    GV = np.random.default_rng(6).standard_normal(gs.shape).astype(np.float32)
    n = f.n

    def adj(g, gv):
        ws = _ws(g, f)
        out = [torch.empty(sh, device=DEV) for sh in ((n, 3), (n, 3), (n, 4), (n,))]
        dgr.dgr_voxelize_backward(g, T(f.mu), T(f.s), T(f.q), T(f.rho), 3.0, T(gv), *out, ws)
        torch.cuda.synchronize()
        assert dgr.dgr_status(ws) == 0
        return [o.double() for o in out]

    whole = adj(grid, GV)
    tot = [torch.zeros_like(w) for w in whole]
    for z0, nz in slab.partition(gs.dims[2], 3):
        for t, p in zip(tot, adj(grid.slab(z0, nz), GV[z0:z0 + nz])):
            t += p
    for t, w, name in zip(tot, whole, ("mu", "s", "q", "rho")):
        assert rel_l2(t.cpu().numpy(), w.cpu().numpy()) <= 1e-5, name


def _split_problem():
    gs, geo, f, grid, ang, geom = _setup(guard=True)
    og, oo = oracle_grid(gs), oracle_geom(geo)
    th = O.to_opt(og, *(a.astype(np.float64) for a in (f.mu, f.s, f.q, f.rho)))
    # a residual of one sign: two FP32 paths (whole grid, slabs) round their
    # chords differently, and a residual of random signs would cancel in the
    # backprojection and leave that rounding exposed (reading R1)
    meas, _ = margin_measurement(og, oo, th, np.random.default_rng(7), signs="positive")
    prob = dgr.make_problem(grid, geom, 3.0, 1e-4, 1e-5, 10)
    return gs, geo, f, grid, ang, geom, og, oo, th, meas, prob


KINDS = (("mu", 3), ("s", 3), ("q", 4), ("rho", 1))


def _split(flat, n):
    out, o = {}, 0
    for k, w in KINDS:
        out[k] = flat[o:o + w * n].reshape((n, w) if w > 1 else (n,))
        o += w * n
    return out


@pytest.mark.parametrize("world", [2, 3])
def test_emulated_split_steps_match_dgr_step_and_the_oracle(world):
    """Step 1: the split's Adam moments (they carry the gradients in optimiser
    variables) and its moves on entries with a non-negligible gradient against
    dgr_step and the oracle.  Steps 2 and 3: the loss, and every replica
    identical.  (Beyond step 1 two correct FP32 paths drift apart on entries
    whose gradient is near Adam's eps: lr g / (|g| + eps) turns their rounding
    differences into different moves -- the multi-step optimiser parity lives
    in test_gpu_step_multi, on a field without such entries.)"""
    gs, geo, f, grid, ang, geom, og, oo, th, meas, prob = _split_problem()
    n = f.n
    ranks, states = [], []
    for r in range(world):
        st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
        dgr.dgr_params_init(prob, st)
        spec = slab.slab_spec(gs.dims[2], geo.n_views, geo.nu * geo.nv, r, world)
        ranks.append(slab.SlabRank(spec, slab.CudaBackend(prob, st, spec)))
        states.append(st)
    parts = [T(meas[R.spec.v0:R.spec.v0 + R.spec.nv]) for R in ranks]
    # the whole problem by dgr_step
    st1 = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
    dgr.dgr_params_init(prob, st1)
    ws1 = _ws(grid, f, geom)
    ws1 = dgr.Workspace(dgr.make_plan(grid, n, 2 * ws1.plan.max_pairs, 2 * ws1.plan.max_items, geom,
                                      step=True))
    loss1 = torch.zeros(1, device=DEV)
    th0 = {k: a.copy() for k, a in th.items()}
    m = {k: np.zeros_like(a) for k, a in th.items()}
    v = {k: np.zeros_like(a) for k, a in th.items()}
    # the loss is a mean of |pred - meas| ~ the margin; its error is that of
    # the prediction (sinogram tolerance 1e-5 of the projection's scale)
    tol = 1e-5 * float(np.abs(meas).mean())
    for t in range(1, 4):
        p32 = [a.astype(np.float32) for a in O.from_opt(og, th)]
        lo, th, _ = O.step(og, oo, *p32, th, m, v, t, meas, 3.0, 1e-4, 1e-5, 10)
        ls = float(slab.run_step_emulated(ranks, parts))
        dgr.dgr_step(prob, st1, T(meas), loss1, ws1)
        torch.cuda.synchronize()
        assert all(R.be.status() == 0 for R in ranks) and dgr.dgr_status(ws1) == 0
        assert abs(ls - lo) <= tol and abs(ls - float(loss1)) <= tol, (t, ls, lo, float(loss1))
        for st in states[1:]:  # replicas stay identical
            assert torch.equal(st.theta, states[0].theta) and torch.equal(st.v, states[0].v)
        if t > 1:
            continue
        mg, vg = _split(states[0].m.cpu().numpy(), n), _split(states[0].v.cpu().numpy(), n)
        tg = _split(states[0].theta.cpu().numpy().astype(np.float64), n)
        refs = (("dgr_step", _split(st1.m.cpu().numpy(), n), _split(st1.v.cpu().numpy(), n),
                 _split(st1.theta.cpu().numpy().astype(np.float64), n)),
                ("oracle", m, v, th))
        for which, mr, vr, thr in refs:
            for k, _ in KINDS:
                assert rel_l2(mg[k], mr[k]) <= 2e-4, (which, k, "m", rel_l2(mg[k], mr[k]))
                assert rel_l2(vg[k], vr[k]) <= 2e-4, (which, k, "v", rel_l2(vg[k], vr[k]))
                live = np.sqrt(vr[k]) >= 1e-3 * np.max(np.sqrt(vr[k]))
                d = np.abs((tg[k] - th0[k]) - (thr[k] - th0[k]))
                assert np.all(d[live] <= 1e-2 * 1e-4), (which, k, float(d[live].max()))


def test_split_step_through_a_single_rank_nccl_group():
    import torch.distributed as dist
    gs, geo, f, grid, ang, geom, og, oo, th, meas, prob = _split_problem()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=60))
    try:
        st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
        dgr.dgr_params_init(prob, st)
        spec = slab.slab_spec(gs.dims[2], geo.n_views, geo.nu * geo.nv, 0, 1)
        R = slab.SlabRank(spec, slab.CudaBackend(prob, st, spec))
        loss = float(slab.run_step(R, slab.TorchComm(), T(meas)))
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    p32 = [a.astype(np.float32) for a in O.from_opt(og, th)]
    m = {k: np.zeros_like(a) for k, a in th.items()}
    v = {k: np.zeros_like(a) for k, a in th.items()}
    lo, _, _ = O.step(og, oo, *p32, th, m, v, 1, meas, 3.0, 1e-4, 1e-5, 10)
    assert abs(loss - lo) <= 1e-5 * lo
    mg = _split(st.m.cpu().numpy(), f.n)
    for k, _ in KINDS:
        assert rel_l2(mg[k], m[k]) <= 2e-4, k
