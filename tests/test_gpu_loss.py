"""The paper's full objective on the GPU (SSIM of the projections, TV of the
volume; Sec. 4.3, App. D.1) against the FP64 oracle: each term and its
gradient through the C ABI, and one optimisation step with the paper's
weights 0.6 / 0.2 / 1.

Tolerances (FP32 statistics through an 11-tap separable window; an FP32
emulation of the same formula differs from FP64 by ~3e-7 relative on these
inputs): SSIM loss within 1e-6 absolute, its gradient within 1e-5 relative L2;
TV loss within 1e-6 relative (FP32 partial sums of |differences|), its gradient
exact up to the final scaling (signs of FP32 differences are exact)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import guard_field, oracle_geom, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def H(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("data_range", [1.0, 2.5])
def test_ssim_loss_and_gradient_match_oracle(data_range):
    rng = np.random.default_rng(21)
    geo = synth.parallel_geom(3, 53, 37)  # ragged 32 x 16 tiles
    x = rng.uniform(0, 2, geo.shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.3, geo.shape), 0, None).astype(np.float32)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    plan = dgr.make_plan(None, 0, 0, 0, gg)
    plan.max_rays = int(np.prod(geo.shape))
    ws = dgr.Workspace(plan)
    grad = torch.full(geo.shape, float("nan"), device=DEV)
    loss = torch.zeros(1, device=DEV)
    dgr.dgr_ssim_loss(gg, T(x), T(y), grad, loss, ws, data_range=data_range)
    torch.cuda.synchronize()
    lo, go = O.ssim_loss(x, y, data_range)
    assert abs(float(loss) - lo) <= 1e-6, (float(loss), lo)
    assert rel_l2(H(grad), go) <= 1e-5, rel_l2(H(grad), go)


def test_ssim_of_identical_projections_is_zero_loss():
    geo = synth.parallel_geom(2, 40, 20)
    x = np.random.default_rng(22).uniform(0, 3, geo.shape).astype(np.float32)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    plan = dgr.make_plan(None, 0, 0, 0, gg)
    plan.max_rays = int(np.prod(geo.shape))
    ws = dgr.Workspace(plan)
    grad = torch.empty(geo.shape, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dgr.dgr_ssim_loss(gg, T(x), T(x), grad, loss, ws)
    torch.cuda.synchronize()
    assert abs(float(loss)) <= 1e-6
    assert float(grad.abs().max()) <= 1e-6 * 3 / x.size * 100


@pytest.mark.parametrize("dims", [(31, 29, 37), (64, 48, 1)])
def test_tv_loss_and_gradient_match_oracle(dims):
    gs = synth.GridSpec(dims, 1.0, tuple(-0.5 * d for d in dims))
    vol = np.random.default_rng(23).standard_normal(gs.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    plan = dgr.make_plan(grid)
    plan.max_vox = int(np.prod(dims))
    ws = dgr.Workspace(plan)
    grad = torch.full(gs.shape, float("nan"), device=DEV)
    loss = torch.zeros(1, device=DEV)
    dgr.dgr_tv_loss(grid, T(vol), grad, loss, ws)
    torch.cuda.synchronize()
    lo, go = O.tv_loss(vol)
    assert abs(float(loss) - lo) <= 1e-6 * lo
    assert np.max(np.abs(H(grad) - go)) <= 1e-6 * np.max(np.abs(go))


def _problem(which):
    if which == "parallel3d":
        gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
        geo = synth.parallel_geom(12, 40, 32, 1.0, 1.0)
    else:
        gs = synth.slice_grid(48, 1.0)
        geo = synth.fan_geom(40, 72, 1.5, 150.0, 240.0)
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 31), 300, gs, ("loguniform", 0.5, 3.0)), gs)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    phantom = synth.ellipsoid_phantom(synth.rng_for(1, 32), gs, 6)
    meas = O.project(oracle_grid(gs), oracle_geom(geo), phantom).astype(np.float32)
    return gs, geo, f, meas


@pytest.mark.parametrize("which", ["parallel3d", "fan"])
def test_step_with_the_paper_objective_matches_oracle(which):
    gs, geo, f, meas = _problem(which)
    w = dgr.PAPER_WEIGHTS
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    prob = dgr.make_problem(grid, gg, 3.0, 3e-4, 3e-5, 50, weights=w, ssim_range=4.0)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, T(f.mu), T(f.s), T(f.q), 3.0, ws0)
    ws0.close()
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, pairs * 2 + 64, items * 2 + 64, gg, step=True))
    st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
    dgr.dgr_params_init(prob, st)
    loss = torch.zeros(1, device=DEV)
    dgr.dgr_step(prob, st, T(meas), loss, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) == 0
    og = oracle_grid(gs)
    th = O.to_opt(og, f.mu.astype(np.float64), f.s.astype(np.float64), f.q.astype(np.float64),
                  f.rho.astype(np.float64))
    m = {k: np.zeros_like(v) for k, v in th.items()}
    v = {k: np.zeros_like(v) for k, v in th.items()}
    lo, th1, grads = O.step(og, oracle_geom(geo), f.mu, f.s, f.q, f.rho, th, m, v, 1, meas, 3.0,
                            3e-4, 3e-5, 50, weights=w, data_range=4.0)
    assert abs(float(loss) - lo) <= 1e-5 * abs(lo), (float(loss), lo)
    n = f.n
    theta = H(st.theta).astype(np.float64)
    parts = {"mu": theta[:3 * n].reshape(n, 3), "s": theta[3 * n:6 * n].reshape(n, 3),
             "q": theta[6 * n:10 * n].reshape(n, 4), "rho": theta[10 * n:]}
    for k in parts:
        # the first Adam step moves each variable by lr * g / (|g| + eps)
        mv_g = parts[k] - th[k]
        mv_o = th1[k] - th[k]
        small = np.abs(grads[k]) < 1e-3 * np.max(np.abs(grads[k]))
        diff = np.abs(mv_g - mv_o)
        assert np.all(diff[~small] <= 1e-2 * 3e-4), (k, diff[~small].max())
