"""GPU (sm_103a, through the C ABI) vs the FP64 oracle, element by element.

Tolerances (FP32 arithmetic against FP64):
  volumes:    relative L2 <= 1e-5 and max |diff| <= 1e-5 * max(rho)
  sinograms:  relative L2 <= 1e-5 (also backprojections)
  gradients:  per parameter kind, relative L2 <= 1e-4 against the oracle's
              analytic gradient (itself pinned to FP64 central differences);
              against FP64 central differences directly: per element
              |g - g_fd| <= 1e-3 * max(|g_fd|, 1e-2 * max|g_fd| of that kind)
  footprint integers: bit-exact.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import guard_field, oracle_geom, oracle_grid, rel_l2

pytestmark = pytest.mark.gpu

DEV = "cuda"


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def H(t):
    return t.detach().cpu().numpy()


def field_t(f):
    return T(f.mu), T(f.s), T(f.q), T(f.rho)


def workspace_for(grid, f=None, geom=None, k=3.0, step=False, slack=1.25):
    n = 0 if f is None else f.n
    plan = dgr.make_plan(grid, n, 0, 0, geom, step)
    if f is not None and n > 0:
        # size the work lists exactly with a counting pass
        ws0 = dgr.Workspace(dgr.make_plan(grid, n))
        mu, s, q, _ = field_t(f)
        pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, k, ws0)
        ws0.close()
        plan.max_pairs = int(pairs * slack) + 64
        plan.max_items = int(items * slack) + 64
    return dgr.Workspace(plan)


def gpu_voxelize(gspec, f, k=3.0, ws=None):
    grid = dgr.Grid.of(gspec)
    ws = ws or workspace_for(grid, f, k=k)
    mu, s, q, rho = field_t(f)
    vol = torch.full(gspec.shape, float("nan"), device=DEV)
    dgr.dgr_voxelize(grid, mu, s, q, rho, k, vol, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) == 0
    return vol


def check_volume(vg, vo, rho_max):
    vg = H(vg).astype(np.float64)
    assert np.isfinite(vg).all()
    assert rel_l2(vg, vo) <= 1e-5, rel_l2(vg, vo)
    assert np.max(np.abs(vg - vo)) <= 1e-5 * rho_max, np.max(np.abs(vg - vo))


# ---------------------------------------------------------------------------
# footprint integers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [3.0, 2.5, -17.0, -5.0])
def test_footprint_integers_bit_exact_unguarded(k):
    gs = synth.GridSpec((45, 37, 29), 0.7, (-13.3, 2.1, -40.0))
    rng = synth.rng_for(1, 11)
    f = synth.gaussian_field(rng, 20000, gs, ("loguniform", 0.3, 8.0), unnormalised_q=True)
    # some Gaussians far outside or straddling the grid
    f.mu[:500] *= 3.0
    grid = dgr.Grid.of(gs)
    mu, s, q, _ = field_t(f)
    an = torch.zeros((f.n, 3), dtype=torch.int32, device=DEV)
    bx = torch.zeros((f.n, 6), dtype=torch.int32, device=DEV)
    dgr.dgr_footprint(grid, mu, s, q, k, an, bx)
    torch.cuda.synchronize()
    a_o, b_o = O.footprint(oracle_grid(gs), f.mu, f.s, f.q, k)
    assert np.array_equal(H(an), a_o)
    assert np.array_equal(H(bx), b_o)


# ---------------------------------------------------------------------------
# voxelize
# ---------------------------------------------------------------------------
def test_voxelize_small_workload_parity():
    """2,000 Gaussians in 64^3 (log-uniform scales 0.5..3 voxels)."""
    wl = synth.workload(1)
    f = guard_field(synth.gaussian_field(synth.rng_for(1), wl.n_gauss, wl.grid, wl.scale), wl.grid)
    vg = gpu_voxelize(wl.grid, f)
    vo = O.voxelize(oracle_grid(wl.grid), f.mu, f.s, f.q, f.rho, 3.0)
    check_volume(vg, vo, f.rho.max())


@pytest.mark.parametrize("k", [3.0, -17.0])
def test_voxelize_ragged_grid_and_box_modes(k):
    """Grid not a multiple of the 8x16x8 tile, off-centre origin, h != 1,
    Gaussians straddling the border, both truncation modes."""
    gs = synth.GridSpec((45, 37, 29), 0.7, (-13.3, 2.1, -40.0))
    rng = synth.rng_for(1, 2)
    f = synth.gaussian_field(rng, 700, gs, ("loguniform", 0.4, 4.0), unnormalised_q=True)
    f = guard_field(f, gs, k=abs(k))
    vg = gpu_voxelize(gs, f, k)
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, k)
    check_volume(vg, vo, f.rho.max())


def test_voxelize_edge_cases():
    gs = synth.GridSpec((16, 16, 16), 1.0, (-8.0, -8.0, -8.0))
    grid = dgr.Grid.of(gs)
    ws = dgr.Workspace(dgr.make_plan(grid, 8, 1000, 1000))
    # n = 0: the volume is all zeros
    z = torch.zeros((0, 3), device=DEV)
    vol = torch.full(gs.shape, 7.0, device=DEV)
    dgr.dgr_voxelize(grid, z, z, torch.zeros((0, 4), device=DEV), torch.zeros(0, device=DEV), 3.0,
                     vol, ws)
    torch.cuda.synchronize()
    assert float(vol.abs().max()) == 0.0
    # one Gaussian entirely outside, one huge (box = whole grid), one tiny
    f = synth.Field(np.array([[100., 0, 0], [0.3, -0.2, 0.1], [1.7, 2.2, -3.1]], np.float32),
                    np.array([[1., 1, 1], [40., 30, 50], [0.05, 0.05, 0.05]], np.float32),
                    np.array([[1., 0, 0, 0], [0.2, 0.3, -0.5, 0.7], [1., 2, 3, 4]], np.float32),
                    np.array([1., 0.5, 2.0], np.float32))
    vg = gpu_voxelize(gs, f, ws=ws)
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)
    check_volume(vg, vo, 2.0)
    # non-finite parameters are skipped and reported
    bad = synth.Field(f.mu.copy(), f.s.copy(), f.q.copy(), f.rho.copy())
    bad.mu[1, 0] = np.nan
    mu, s, q, rho = field_t(bad)
    dgr.dgr_voxelize(grid, mu, s, q, rho, 3.0, vol, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) & dgr.DGR_STATUS_NONFINITE
    assert torch.isfinite(vol).all()


def test_voxelize_overflow_is_reported():
    gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
    f = synth.gaussian_field(synth.rng_for(1, 3), 300, gs, ("loguniform", 0.5, 3.0))
    grid = dgr.Grid.of(gs)
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, 10, 10))
    mu, s, q, rho = field_t(f)
    vol = torch.zeros(gs.shape, device=DEV)
    dgr.dgr_voxelize(grid, mu, s, q, rho, 3.0, vol, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) & dgr.DGR_STATUS_PAIR_OVERFLOW
    assert torch.isfinite(vol).all()


@pytest.mark.parametrize("depth", [32, 8])
def test_voxelize_long_tile_lists(depth):
    """9,000 small Gaussians in a 16 x 16 x 32 grid: every tile's list holds
    more than 4,096 Gaussians, so the chunked sort + merge path runs."""
    gs = synth.GridSpec((16, 16, 32), 1.0, (-8.0, -8.0, -16.0))
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 31), 9000, gs, ("loguniform", 0.5, 1.5)), gs)
    try:
        dgr.dgr_set_tile_depth(depth)
        grid = dgr.Grid.of(gs)
        ws = workspace_for(grid, f)
        a = gpu_voxelize(gs, f, ws=ws)
        b = gpu_voxelize(gs, f, ws=ws)
    finally:
        dgr.dgr_set_tile_depth(32)
    assert torch.equal(a, b)
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)
    check_volume(a, vo, f.rho.max())


def test_voxelize_deterministic_bitwise():
    wl = synth.workload(1)
    f = synth.gaussian_field(synth.rng_for(1, 5), 6000, wl.grid, ("loguniform", 0.5, 6.0))
    grid = dgr.Grid.of(wl.grid)
    ws = workspace_for(grid, f)
    a = gpu_voxelize(wl.grid, f, ws=ws)
    b = gpu_voxelize(wl.grid, f, ws=ws)
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------
def _projector_cases():
    par = synth.workload(1)
    cone_g = synth.GridSpec((40, 44, 36), 1.0, (-20.0, -22.0, -18.0))
    cone = synth.cone_geom(24, 70, 50, 1.5, 1.5, 120.0, 180.0)
    odd = synth.GridSpec((33, 29, 21), 0.8, (-12.0, -13.0, -9.0))
    odd_geom = synth.parallel_geom(17, 45, 27, 0.9, 0.7)
    odd_cone = synth.cone_geom(13, 41, 31, 1.1, 1.3, 60.0, 95.0, arc=1.3)
    # a wide cone: rays cross several z planes inside one (x, y) cell
    steep_g = synth.GridSpec((24, 24, 24), 1.0, (-12.0, -12.0, -12.0))
    steep = synth.cone_geom(8, 40, 64, 1.5, 1.5, 30.0, 45.0)
    # 2D fan beam on a slice; 90-degree limited-angle scans (fan and 3D parallel)
    fan_g = synth.slice_grid(64, 1.0)
    fan = synth.fan_geom(36, 96, 1.4, 160.0, 260.0)
    fan90 = synth.fan_geom(24, 96, 1.4, 160.0, 260.0, arc=np.pi / 2)
    par90 = synth.parallel_geom(20, 56, 44, 1.0, 1.0, arc=np.pi / 2)
    return [("parallel64", par.grid, par.geom), ("cone", cone_g, cone),
            ("parallel_odd", odd, odd_geom), ("cone_odd", odd, odd_cone), ("cone_steep", steep_g, steep),
            ("fan2d", fan_g, fan), ("fan2d_limited90", fan_g, fan90),
            ("parallel_limited90", cone_g, par90)]


@pytest.mark.parametrize("case", _projector_cases(), ids=lambda c: c[0])
def test_project_and_backproject_parity(case):
    _, gs, geo = case
    rng = np.random.default_rng(3)
    vol = rng.uniform(0, 1, gs.shape).astype(np.float32)
    sino = rng.standard_normal(geo.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
    sg = torch.full(geo.shape, float("nan"), device=DEV)
    dgr.dgr_project(grid, gg, T(vol), sg, ws)
    bg = torch.full(gs.shape, float("nan"), device=DEV)
    dgr.dgr_backproject(grid, gg, T(sino), bg, ws)
    torch.cuda.synchronize()
    so = O.project(oracle_grid(gs), oracle_geom(geo), vol)
    bo = O.backproject(oracle_grid(gs), oracle_geom(geo), sino)
    assert rel_l2(H(sg), so) <= 1e-5, rel_l2(H(sg), so)
    assert rel_l2(H(bg), bo) <= 1e-5, rel_l2(H(bg), bo)
    # adjoint identity of the device pair
    lhs = float((H(sg).astype(np.float64) * sino).sum())
    rhs = float((vol.astype(np.float64) * H(bg)).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("variant", [0, 2])
def test_backproject_several_view_groups(variant):
    """300 views: the fixed-point scatters run three groups of views (128,
    128, 44), each with its own step from its own largest residual (the
    residual scale differs by 10^4 between groups), and the fold adds the
    groups."""
    gs = synth.GridSpec((32, 28, 24), 1.0, (-16.0, -14.0, -12.0))
    geo = synth.cone_geom(300, 40, 32, 1.5, 1.5, 300.0, 450.0)
    y = np.random.default_rng(19).standard_normal(geo.shape).astype(np.float32)
    y[128:256] *= 1e-4
    y[256:] *= 30.0
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
    try:
        dgr.dgr_set_backprojector(variant)
        a = torch.empty(gs.shape, device=DEV)
        dgr.dgr_backproject(grid, gg, T(y), a, ws)
        torch.cuda.synchronize()
        assert dgr.dgr_status(ws) == 0
    finally:
        dgr.dgr_set_backprojector(0)
    bo = O.backproject(oracle_grid(gs), oracle_geom(geo), y)
    assert rel_l2(H(a), bo) <= 1e-5, rel_l2(H(a), bo)
    # the small group alone is still resolved (its own step)
    b = torch.empty(gs.shape, device=DEV)
    ymid = np.zeros_like(y)
    ymid[128:256] = y[128:256]
    dgr.dgr_backproject(grid, gg, T(ymid), b, ws)
    torch.cuda.synchronize()
    bmid = O.backproject(oracle_grid(gs), oracle_geom(geo), ymid)
    assert rel_l2(H(b), bmid) <= 1e-5, rel_l2(H(b), bmid)


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_backproject_variants_agree_and_are_deterministic(variant):
    """Every backprojector (ray scatter, column gather, brick scatter) gives the oracle's
    transpose on the workload's cone geometry at reduced size, bit-identically
    run to run."""
    gs = synth.GridSpec((64, 48, 40), 1.0, (-32.0, -24.0, -20.0))
    geo = synth.cone_geom(20, 96, 64, 1.5, 1.5, 1000.0, 1500.0)
    y = np.random.default_rng(13).standard_normal(geo.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
    try:
        dgr.dgr_set_backprojector(variant)
        a = torch.empty(gs.shape, device=DEV); b = torch.empty(gs.shape, device=DEV)
        dgr.dgr_backproject(grid, gg, T(y), a, ws)
        dgr.dgr_backproject(grid, gg, T(y), b, ws)
        torch.cuda.synchronize()
    finally:
        dgr.dgr_set_backprojector(0)
    assert torch.equal(a, b)
    bo = O.backproject(oracle_grid(gs), oracle_geom(geo), y)
    assert rel_l2(H(a), bo) <= 1e-5


@pytest.mark.parametrize("case", [c for c in _projector_cases() if c[1].dims[2] % 4 == 0], ids=lambda c: c[0])
def test_staged_walks_match_direct_walks(case):
    """The bulk-copy staged walks (shared-memory windows of each cell's z
    column) give the direct walks' projections and the same backprojection
    bits (integer sums do not depend on the order of the additions)."""
    _, gs, geo = case
    rng = np.random.default_rng(8)
    vol = rng.uniform(0, 1, gs.shape).astype(np.float32)
    sino = rng.standard_normal(geo.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
    out = {}
    try:
        for staged in (False, True):
            dgr.dgr_set_staged_walk(staged)
            sg = torch.empty(geo.shape, device=DEV)
            bg = torch.empty(gs.shape, device=DEV)
            dgr.dgr_project(grid, gg, T(vol), sg, ws)
            dgr.dgr_backproject(grid, gg, T(sino), bg, ws)
            torch.cuda.synchronize()
            assert dgr.dgr_status(ws) == 0
            out[staged] = (sg, bg)
    finally:
        dgr.dgr_set_staged_walk(False)
    assert rel_l2(H(out[True][0]), H(out[False][0])) <= 1e-6
    assert torch.equal(out[True][1], out[False][1])


def test_ray_and_brick_scatter_agree_bitwise():
    """The two fixed-point scatters add the same integer contributions (same
    chord lengths, same step per group of views) and fold them in the same
    order, so they return the same bits; a workspace without room for the
    integer sums falls back to the brick scatter."""
    gs = synth.GridSpec((40, 56, 36), 1.0, (-20.0, -28.0, -18.0))
    geo = synth.cone_geom(19, 80, 50, 1.4, 1.3, 400.0, 650.0)
    y = np.random.default_rng(17).standard_normal(geo.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
    out = []
    try:
        for variant in (0, 2):
            dgr.dgr_set_backprojector(variant)
            v = torch.empty(gs.shape, device=DEV)
            dgr.dgr_backproject(grid, gg, T(y), v, ws)
            out.append(v)
        dgr.dgr_set_backprojector(0)
        plan = dgr.make_plan(grid, 0, 0, 0, gg)
        plan.max_vox = 0  # no room for the integer sums
        ws2 = dgr.Workspace(plan)
        v = torch.empty(gs.shape, device=DEV)
        dgr.dgr_backproject(grid, gg, T(y), v, ws2)
        out.append(v)
        torch.cuda.synchronize()
    finally:
        dgr.dgr_set_backprojector(0)
    assert torch.equal(out[0], out[1])
    assert torch.equal(out[0], out[2])


# ---------------------------------------------------------------------------
# voxelize adjoint
# ---------------------------------------------------------------------------
def _gpu_backward(gs, f, W, k=3.0):
    grid = dgr.Grid.of(gs)
    ws = workspace_for(grid, f, k=k)
    mu, s, q, rho = field_t(f)
    n = f.n
    out = [torch.full(sh, float("nan"), device=DEV) for sh in ((n, 3), (n, 3), (n, 4), (n,))]
    dgr.dgr_voxelize_backward(grid, mu, s, q, rho, k, T(W), *out, ws)
    torch.cuda.synchronize()
    assert dgr.dgr_status(ws) == 0
    return [H(o).astype(np.float64) for o in out]


def test_voxelize_backward_matches_oracle_gradient():
    gs = synth.GridSpec((48, 40, 44), 0.9, (-20.0, -17.0, -21.0))
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 7), 800, gs, ("loguniform", 0.5, 5.0),
                                         unnormalised_q=True), gs)
    W = np.random.default_rng(4).standard_normal(gs.shape).astype(np.float32)
    gg = _gpu_backward(gs, f, W)
    go = O.voxelize_backward(oracle_grid(gs), f.mu, f.s, f.q, f.rho, W, 3.0)
    for name, a, b in zip(("mu", "s", "q", "rho"), gg, go):
        assert rel_l2(a, b) <= 1e-4, (name, rel_l2(a, b))


def test_voxelize_backward_large_boxes():
    """Gaussians whose boxes hold more than 256 work items (over 512K voxels:
    scales of 12-20 voxels in a 96 x 96 x 88 grid) are summed by a CTA each;
    with small ones around them, every gradient matches the oracle."""
    gs = synth.GridSpec((96, 96, 88), 1.0, (-48.0, -48.0, -44.0))
    big = synth.gaussian_field(synth.rng_for(1, 71), 6, gs, ("loguniform", 12.0, 20.0), unnormalised_q=True)
    big.mu = (0.25 * big.mu).astype(np.float32)  # near the centre: boxes mostly inside the grid
    small = synth.gaussian_field(synth.rng_for(1, 72), 300, gs, ("loguniform", 0.5, 4.0), unnormalised_q=True)
    f = synth.Field(np.concatenate([big.mu, small.mu]), np.concatenate([big.s, small.s]),
                            np.concatenate([big.q, small.q]), np.concatenate([big.rho, small.rho]))
    f = guard_field(f, gs)
    og = oracle_grid(gs)
    _, box = O.footprint(og, f.mu, f.s, f.q, 3.0)
    vox = np.prod(np.maximum(box[:, 3:6] - box[:, 0:3] + 1, 0), axis=1)
    assert (vox[:6] > 256 * 2048).sum() >= 3  # several Gaussians take the large-box path
    W = np.random.default_rng(6).standard_normal(gs.shape).astype(np.float32)
    gg = _gpu_backward(gs, f, W)
    go = O.voxelize_backward(og, f.mu, f.s, f.q, f.rho, W, 3.0)
    for name, a, b in zip(("mu", "s", "q", "rho"), gg, go):
        assert rel_l2(a, b) <= 1e-4, (name, rel_l2(a, b))
        assert rel_l2(a[:6], b[:6]) <= 1e-4, (name, "large", rel_l2(a[:6], b[:6]))


def test_voxelize_backward_vs_fp64_finite_differences():
    """16 Gaussians in 16^3 with the 512^3 workload's heavy-tailed scale law."""
    gs = synth.GridSpec((16, 16, 16), 1.0, (-8.0, -8.0, -8.0))
    f = synth.gaussian_field(synth.rng_for(3, 16), 16, gs, ("lognormal", 1.5, 0.894),
                             unnormalised_q=True)
    f.s = np.clip(f.s, 0.6, 6.0).astype(np.float32)
    f = guard_field(f, gs)
    W = np.random.default_rng(5).standard_normal(gs.shape).astype(np.float32)
    gg = _gpu_backward(gs, f, W)
    og = oracle_grid(gs)
    _, box = O.footprint(og, f.mu, f.s, f.q, 3.0)
    d = lambda a: np.asarray(a, np.float64)
    base = [d(f.mu), d(f.s), d(f.q), d(f.rho)]
    W64 = W.astype(np.float64)
    for kind in range(4):
        fd = np.zeros_like(base[kind]).reshape(-1)
        for j in range(fd.size):
            p = [b.copy() for b in base]
            eps = 1e-6 * max(1.0, abs(p[kind].reshape(-1)[j]))
            p[kind].reshape(-1)[j] += eps
            lp = (O.voxelize_core(og, *p, box) * W64).sum()
            p[kind].reshape(-1)[j] -= 2 * eps
            lm = (O.voxelize_core(og, *p, box) * W64).sum()
            fd[j] = (lp - lm) / (2 * eps)
        g = gg[kind].reshape(-1)
        floor = 1e-2 * np.max(np.abs(fd))
        err = np.abs(g - fd) / np.maximum(np.abs(fd), floor)
        assert err.max() <= 1e-3, (kind, err.max())


# ---------------------------------------------------------------------------
# loss and one full optimisation step
# ---------------------------------------------------------------------------
def test_l1_residual_parity():
    rng = np.random.default_rng(6)
    p = rng.standard_normal((7, 33, 41)).astype(np.float32)
    m = rng.standard_normal((7, 33, 41)).astype(np.float32)
    m[0, 0, :5] = p[0, 0, :5]  # ties -> sign 0
    grid = dgr.Grid(8, 8, 8, 1.0, 0, 0, 0)
    ws = dgr.Workspace(dgr.make_plan(grid, 0))
    r = torch.empty(p.shape, device=DEV)
    loss = torch.empty(1, device=DEV)
    dgr.dgr_l1_residual(T(p), T(m), r, loss, ws)
    torch.cuda.synchronize()
    lo, ro = O.l1_loss(p, m)
    assert abs(float(loss) - lo) <= 1e-6 * lo
    assert np.max(np.abs(H(r) - ro)) <= 1e-7 * np.max(np.abs(ro))


def _step_problem():
    gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
    geo = synth.parallel_geom(12, 40, 32, 1.0, 1.0)
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 9), 300, gs, ("loguniform", 0.5, 3.0)), gs)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    phantom = synth.ellipsoid_phantom(synth.rng_for(1, 10), gs, 6)
    meas = O.project(oracle_grid(gs), oracle_geom(geo), phantom).astype(np.float32)
    return gs, geo, f, meas


def _fan_step_problem(arc):
    """2D fan beam over a one-voxel-thick slice (full scan or 90 degrees)."""
    gs = synth.slice_grid(48, 1.0)
    geo = synth.fan_geom(40, 72, 1.5, 150.0, 240.0, arc)
    f = guard_field(synth.gaussian_field(synth.rng_for(1, 11), 250, gs, ("loguniform", 0.5, 3.0)), gs)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    phantom = synth.ellipsoid_phantom(synth.rng_for(1, 12), gs, 6)
    meas = O.project(oracle_grid(gs), oracle_geom(geo), phantom).astype(np.float32)
    return gs, geo, f, meas


@pytest.mark.parametrize("which", ["parallel3d", "fan", "fan_limited90"])
def test_step_parity_with_oracle(which):
    if which == "parallel3d":
        gs, geo, f, meas = _step_problem()
    else:
        gs, geo, f, meas = _fan_step_problem(2 * np.pi if which == "fan" else np.pi / 2)
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    prob = dgr.make_problem(grid, gg, 3.0, 3e-4, 3e-5, 50)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    pairs, items = dgr.dgr_voxelize_count(grid, *field_t(f)[:3], 3.0, ws0)
    ws0.close()
    plan = dgr.make_plan(grid, f.n, pairs * 2 + 64, items * 2 + 64, gg, step=True)
    ws = dgr.Workspace(plan)
    st = dgr.State(*field_t(f))
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
                            3e-4, 3e-5, 50)
    assert abs(float(loss) - lo) <= 1e-5 * lo
    n = f.n
    theta = H(st.theta).astype(np.float64)
    parts = {"mu": theta[:3 * n].reshape(n, 3), "s": theta[3 * n:6 * n].reshape(n, 3),
             "q": theta[6 * n:10 * n].reshape(n, 4), "rho": theta[10 * n:]}
    for k in parts:
        # the first Adam step moves each variable by lr * g / (|g| + eps): compare
        # the move, allowing sign flips only where the gradient is negligible
        mv_g = parts[k] - th[k]
        mv_o = th1[k] - th[k]
        small = np.abs(grads[k]) < 1e-3 * np.max(np.abs(grads[k]))
        diff = np.abs(mv_g - mv_o)
        assert np.all(diff[~small] <= 1e-2 * 3e-4), (k, diff[~small].max())
    assert int(H(st.step)[0]) == 1
