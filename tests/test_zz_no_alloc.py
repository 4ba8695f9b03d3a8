"""dgr_project_noalloc: the projector for callers that cannot allocate device
memory (its scratch is a fixed device array, not a workspace).  Through the C
ABI it must give what dgr_project gives -- same tolerance as the projector
parity tests (relative L2 <= 1e-5) -- on two calls in a row with different
geometries, refuse a geometry whose ray tables exceed the fixed array, and
leave the device's free memory unchanged over repeated calls.  Collected last so that a failure here stops a -x run after everything else."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_04844_b300 import dgr, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def rel_l2(a, b):
    a = a.double(); b = b.double()
    return float((a - b).norm() / b.norm())


def _case(gs, geo, seed):
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    vol = T(np.random.default_rng(seed).uniform(0, 1, gs.shape).astype(np.float32))
    return grid, gg, ang, vol


def test_noalloc_projector_matches_workspace_projector_twice():
    cases = [
        (synth.GridSpec((40, 44, 36), 1.0, (-20.0, -22.0, -18.0)),
         synth.cone_geom(24, 70, 50, 1.5, 1.5, 120.0, 180.0), 1),
        (synth.GridSpec((33, 29, 21), 0.8, (-12.0, -13.0, -9.0)),
         synth.parallel_geom(17, 45, 27, 0.9, 0.7), 2),
    ]
    for gs, geo, seed in cases:
        grid, gg, ang, vol = _case(gs, geo, seed)
        ws = dgr.Workspace(dgr.make_plan(grid, 0, 0, 0, gg))
        ref = torch.empty(geo.shape, device=DEV)
        dgr.dgr_project(grid, gg, vol, ref, ws)
        out = torch.full(geo.shape, float("nan"), device=DEV)
        dgr.dgr_project_noalloc(grid, gg, vol, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert rel_l2(out, ref) <= 1e-5
        ws.close()


def test_noalloc_projector_refuses_oversized_geometry():
    gs = synth.GridSpec((16, 16, 16), 1.0, (-8.0, -8.0, -8.0))
    # 600 views x 512 detector columns x 32 bytes of tables > the fixed scratch
    geo = synth.parallel_geom(600, 512, 4, 1.0, 1.0)
    assert 600 * 512 * 32 > dgr.NOALLOC_SCRATCH_BYTES
    grid, gg, ang, vol = _case(gs, geo, 3)
    out = torch.zeros(geo.shape, device=DEV)
    with pytest.raises(dgr.DgrError, match="workspace plan too small"):
        dgr.dgr_project_noalloc(grid, gg, vol, out)


def test_noalloc_projector_leaves_free_memory_unchanged():
    """After a first call (which loads the kernels and looks up the scratch
    address), further calls take no device memory: the driver's free-memory
    count is the same before and after them."""
    gs = synth.GridSpec((32, 32, 32), 1.0, (-16.0, -16.0, -16.0))
    geo = synth.cone_geom(16, 48, 40, 1.5, 1.5, 100.0, 150.0)
    grid, gg, ang, vol = _case(gs, geo, 4)
    out = torch.empty(geo.shape, device=DEV)
    dgr.dgr_project_noalloc(grid, gg, vol, out)
    torch.cuda.synchronize()
    first = out.clone()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        dgr.dgr_project_noalloc(grid, gg, vol, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(out, first)
