"""Parity at the full size of the benchmark workload (50,000 Gaussians, 256^3,
cone beam 50 views x 256^2), in the launch configuration bench.py times,
element by element against the FP64 oracle: the whole volume (Eq. 4 with
3-sigma confinement, Sec. 4.1), all 50 views of the projection and the whole
backprojection (Sec. 4.3), the gradients of all 50,000 Gaussians, the
adjoint identity at full size, and the loss of one full optimisation step.

Tolerances as in the small parity tests: volume relative L2 <= 1e-5 and
max |diff| <= 1e-5 max(rho); sinogram relative L2 <= 1e-5; backprojection of
non-negative data relative L2 <= 1e-5, of signed data |diff| <= 1e-5 |BP(|y|)|
(the FP32 chord lengths' error does not cancel with the data's signs);
gradients relative L2 <= 1e-4 per parameter kind."""
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


def test_fullsize_voxelize_whole_volume(problem):
    P = problem
    wl, f = P["wl"], P["f"]
    vol = torch.empty(wl.grid.shape, device=DEV)
    dgr.dgr_voxelize(P["grid"], *P["t"], 3.0, vol, P["ws"])
    torch.cuda.synchronize()
    assert dgr.dgr_status(P["ws"]) == 0
    vo = O.voxelize(oracle_grid(wl.grid), f.mu, f.s, f.q, f.rho, 3.0)
    vg = vol.cpu().numpy().astype(np.float64)
    err = np.max(np.abs(vg - vo))
    print(f"256^3 volume: rel-L2 {rel_l2(vg, vo):.3e}, max-abs {err:.3e}, max V {vo.max():.3f}")
    assert rel_l2(vg, vo) <= 1e-5
    assert err <= 1e-5 * float(f.rho.max()), err


def test_fullsize_project_all_views_backproject_and_adjoint(problem):
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
    og, oo = oracle_grid(wl.grid), oracle_geom(wl.geom)
    so = O.project(og, oo, vol)
    assert rel_l2(sg.cpu().numpy(), so) <= 1e-5, rel_l2(sg.cpu().numpy(), so)
    # backprojection: of non-negative data, relative L2 <= 1e-5; of signed data
    # (random signs cancel in every voxel's sum) the error is bounded relative
    # to the backprojection of |y| -- each FP32 chord length is a difference
    # of plane-crossing parameters along a ray ~360 voxels long (relative
    # error ~1e-5 per chord), so a cancelling sum keeps that error per term
    ya = np.abs(y)
    ba = torch.empty(wl.grid.shape, device=DEV)
    dgr.dgr_backproject(P["grid"], P["geom"], T(ya), ba, P["ws"])
    torch.cuda.synchronize()
    boa = O.backproject(og, oo, ya)
    assert rel_l2(ba.cpu().numpy(), boa) <= 1e-5, rel_l2(ba.cpu().numpy(), boa)
    bo = O.backproject(og, oo, y)
    err = np.linalg.norm(bg.cpu().numpy().astype(np.float64) - bo)
    print(f"backprojection of signed data: rel-L2 {rel_l2(bg.cpu().numpy(), bo):.3e}, "
          f"relative to |BP(|y|)| {err / np.linalg.norm(boa):.3e}")
    assert err <= 1e-5 * np.linalg.norm(boa)
    lhs = float((sg.double() * T(y).double()).sum())
    rhs = float((T(vol).double() * bg.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


def test_fullsize_voxelize_backward_all_gaussians(problem):
    P = problem
    wl, f = P["wl"], P["f"]
    rng = np.random.default_rng(43)
    GV = rng.standard_normal(wl.grid.shape, dtype=np.float32)
    n = f.n
    out = [torch.empty(sh, device=DEV) for sh in ((n, 3), (n, 3), (n, 4), (n,))]
    dgr.dgr_voxelize_backward(P["grid"], *P["t"], 3.0, T(GV), *out, P["ws"])
    torch.cuda.synchronize()
    assert dgr.dgr_status(P["ws"]) == 0
    ref = O.voxelize_backward(oracle_grid(wl.grid), f.mu, f.s, f.q, f.rho, GV, 3.0)
    for o, r, name in zip(out, ref, ("mu", "s", "q", "rho")):
        assert rel_l2(o.cpu().numpy(), r) <= 1e-4, (name, rel_l2(o.cpu().numpy(), r))


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
    (same loss, same parameters, bit for bit), and the four kernel intervals
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
    assert ev[0].elapsed_time(ev[11]) >= 0 and ev[12].elapsed_time(ev[1]) >= 0  # voxelize phase
    assert ev[4].elapsed_time(ev[13]) >= 0 and ev[14].elapsed_time(ev[5]) >= 0  # adjoint phase
    assert ev[11].elapsed_time(ev[12]) > 0 and ev[13].elapsed_time(ev[14]) > 0
