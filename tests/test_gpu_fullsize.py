"""Parity at the full size of the benchmark workload (50,000 Gaussians, 256^3,
cone beam 50 views x 256^2), in the launch configuration bench.py times:
sampled voxels, sampled views, sampled Gaussians, the adjoint identity at full
size, and the loss of one full optimisation step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import oracle_geom, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


@pytest.fixture(scope="module")
def problem():
    wl = synth.workload(2)
    f = synth.gaussian_field(synth.rng_for(2, 0), wl.n_gauss, wl.grid, wl.scale)
    f.rho = np.clip(f.rho, 0.02, 1.0).astype(np.float32)
    grid = dgr.Grid.of(wl.grid)
    ang = T(wl.geom.angles)
    geom = dgr.Geom.of(wl.geom, ang)
    mu, s, q, rho = T(f.mu), T(f.s), T(f.q), T(f.rho)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, 3.0, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, int(pairs * 1.5) + 1024, int(items * 1.5) + 1024,
                                     geom, step=True))
    return dict(wl=wl, f=f, grid=grid, ang=ang, geom=geom, ws=ws, t=(mu, s, q, rho))


def test_fullsize_voxelize_sampled(problem):
    P = problem
    wl, f = P["wl"], P["f"]
    vol = torch.empty(wl.grid.shape, device=DEV)
    dgr.dgr_voxelize(P["grid"], *P["t"], 3.0, vol, P["ws"])
    torch.cuda.synchronize()
    assert dgr.dgr_status(P["ws"]) == 0
    rng = np.random.default_rng(41)
    pts = np.stack([rng.integers(0, 256, 400) for _ in range(3)], 1)
    vo = O.voxelize_points(oracle_grid(wl.grid), f.mu, f.s, f.q, f.rho, pts, 3.0)
    vg = vol[pts[:, 2], pts[:, 1], pts[:, 0]].cpu().numpy()
    assert rel_l2(vg, vo) <= 1e-5
    assert np.max(np.abs(vg - vo)) <= 1e-5 * float(f.rho.max()) * max(1.0, float(np.abs(vo).max()))


def test_fullsize_project_sampled_views_and_adjoint(problem):
    P = problem
    wl = P["wl"]
    rng = np.random.default_rng(42)
    vol = rng.uniform(0, 1, wl.grid.shape).astype(np.float32)
    y = rng.standard_normal(wl.geom.shape).astype(np.float32)
    sg = torch.empty(wl.geom.shape, device=DEV)
    bg = torch.empty(wl.grid.shape, device=DEV)
    dgr.dgr_project(P["grid"], P["geom"], T(vol), sg, P["ws"])
    dgr.dgr_backproject(P["grid"], P["geom"], T(y), bg, P["ws"])
    torch.cuda.synchronize()
    views = np.array([0, 13, 29, 41])
    g = wl.geom
    sub = O.Geom(g.beam, g.angles[views], g.nu, g.nv, g.pu, g.pv, g.dso, g.dsd)
    so = O.project(oracle_grid(wl.grid), sub, vol)
    assert rel_l2(sg[torch.as_tensor(views, device=DEV)].cpu().numpy(), so) <= 1e-5
    lhs = float((sg.double() * T(y).double()).sum())
    rhs = float((T(vol).double() * bg.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


def test_fullsize_voxelize_backward_sampled(problem):
    P = problem
    wl, f = P["wl"], P["f"]
    rng = np.random.default_rng(43)
    GV = rng.standard_normal(wl.grid.shape, dtype=np.float32)
    n = f.n
    out = [torch.empty(sh, device=DEV) for sh in ((n, 3), (n, 3), (n, 4), (n,))]
    dgr.dgr_voxelize_backward(P["grid"], *P["t"], 3.0, T(GV), *out, P["ws"])
    torch.cuda.synchronize()
    assert dgr.dgr_status(P["ws"]) == 0
    idx = np.concatenate([rng.choice(n, 80, replace=False), np.argsort(-f.s.max(1))[:4]])
    ref = O.voxelize_backward(oracle_grid(wl.grid), f.mu[idx], f.s[idx], f.q[idx], f.rho[idx], GV, 3.0)
    for o, r, name in zip(out, ref, ("mu", "s", "q", "rho")):
        assert rel_l2(o[torch.as_tensor(idx, device=DEV)].cpu().numpy(), r) <= 1e-4, name


def test_fullsize_step_loss(problem):
    """Loss of one optimisation step at full size vs the oracle's FP64 loss
    (its volume, its projection, the same measured data)."""
    P = problem
    wl, f = P["wl"], P["f"]
    phantom = synth.ellipsoid_phantom(synth.rng_for(2, 100), wl.grid, wl.phantom_m)
    og, oo = oracle_grid(wl.grid), oracle_geom(wl.geom)
    meas = O.project(og, oo, phantom).astype(np.float32)
    prob = dgr.make_problem(P["grid"], P["geom"], 3.0, 3e-4, 3e-5, wl.n_iters)
    st = dgr.State(*P["t"])
    dgr.dgr_params_init(prob, st)
    loss = torch.zeros(1, device=DEV)
    dgr.dgr_step(prob, st, T(meas), loss, P["ws"])
    torch.cuda.synchronize()
    assert dgr.dgr_status(P["ws"]) == 0
    vo = O.voxelize(og, f.mu, f.s, f.q, f.rho, 3.0)
    lo, _ = O.l1_loss(O.project(og, oo, vo), meas)
    assert abs(float(loss) - lo) <= 1e-5 * lo
    assert bool(torch.isfinite(st.theta).all())


def test_fullsize_step_timed_kernel_events(problem):
    """dgr_step_timed with the kernel events does the same step as dgr_step
    (same loss, same parameters, bit for bit), and the two kernel intervals
    lie inside their phases."""
    P = problem
    wl = P["wl"]
    meas = T(np.random.default_rng(43).uniform(0, 50, wl.geom.shape).astype(np.float32))
    prob = dgr.make_problem(P["grid"], P["geom"], 3.0, 3e-4, 3e-5, wl.n_iters)
    out = []
    for timed in (False, True):
        st = dgr.State(*[t.clone() for t in P["t"]])
        dgr.dgr_params_init(prob, st)
        loss = torch.zeros(1, device=DEV)
        if timed:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(dgr.DGR_STEP_KERNEL_EVENTS)]
            for e in ev:
                e.record()
            dgr.dgr_step_timed(prob, st, meas, loss, P["ws"], ev)
        else:
            dgr.dgr_step(prob, st, meas, loss, P["ws"])
        torch.cuda.synchronize()
        assert dgr.dgr_status(P["ws"]) == 0
        out.append((float(loss), st.theta.clone()))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    assert ev[7].elapsed_time(ev[8]) > 0 and ev[9].elapsed_time(ev[10]) > 0
    assert ev[3].elapsed_time(ev[7]) >= 0 and ev[8].elapsed_time(ev[4]) >= 0  # backproject phase
    assert ev[1].elapsed_time(ev[9]) >= 0 and ev[10].elapsed_time(ev[2]) >= 0  # project phase
    assert ev[7].elapsed_time(ev[8]) <= ev[3].elapsed_time(ev[4])
