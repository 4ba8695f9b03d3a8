"""Separable voxelizer (the paper's isotropic representation,
Sec. 4.1): when every Gaussian has a diagonal A (isotropic scales under any
rotation, or the identity rotation) FVR becomes a sum of outer products of two
small exponential tables per tile.  Same tolerances as the general voxelizer
(relative L2 <= 1e-5, max-abs <= 1e-5 max rho) against the FP64 oracle, on
ragged grids and long per-tile lists; a call with one rotated anisotropic
Gaussian falls back to the general kernel bit for bit; the adjoint of FVR with
isotropic Gaussians matches the oracle's analytic gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2411_04844_b300 import dgr, synth
from tests._common import guard_field, oracle_grid, rel_l2
from tests.test_gpu_parity import check_volume, gpu_voxelize, field_t, H

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _voxelize(gs, f, separable):
    dgr.dgr_set_separable(separable)
    try:
        return gpu_voxelize(gs, f)
    finally:
        dgr.dgr_set_separable(True)


@pytest.mark.parametrize("case", ["isotropic", "axis_aligned", "long_lists"])
def test_separable_voxelize_matches_oracle(case):
    if case == "long_lists":
        gs = synth.GridSpec((24, 20, 40), 1.0, (-12.0, -10.0, -20.0))
        f = synth.gaussian_field(synth.rng_for(6, 1), 6000, gs, ("loguniform", 1.0, 4.0), isotropic=True)
    else:
        gs = synth.GridSpec((70, 50, 45), 0.9, (-31.0, -22.0, -20.0))  # ragged 8 x 16 x 32 tiles
        f = synth.gaussian_field(synth.rng_for(6, 2), 3000, gs, ("loguniform", 0.5, 4.0),
                                 isotropic=case == "isotropic")
        if case == "axis_aligned":
            f.q[:] = np.array([1.0, 0.0, 0.0, 0.0], np.float32)
    f = guard_field(f, gs)
    sep = _voxelize(gs, f, True)
    gen = _voxelize(gs, f, False)
    vo = O.voxelize(oracle_grid(gs), f.mu, f.s, f.q, f.rho, 3.0)
    check_volume(sep, vo, float(f.rho.max()))
    check_volume(gen, vo, float(f.rho.max()))
    assert not torch.equal(sep, gen)  # the separable kernel did run
    assert torch.equal(sep, _voxelize(gs, f, True))  # bit-reproducible


def test_one_rotated_anisotropic_gaussian_selects_the_general_kernel():
    gs = synth.GridSpec((40, 40, 40), 1.0, (-20.0, -20.0, -20.0))
    f = guard_field(synth.gaussian_field(synth.rng_for(6, 3), 800, gs, ("loguniform", 0.5, 3.0),
                                         isotropic=True), gs)
    f.s[5] = np.array([1.0, 2.0, 3.0], np.float32)  # rotated, anisotropic
    f = guard_field(f, gs)
    assert torch.equal(_voxelize(gs, f, True), _voxelize(gs, f, False))


def test_isotropic_adjoint_matches_oracle():
    gs = synth.GridSpec((32, 28, 36), 1.0, (-16.0, -14.0, -18.0))
    f = guard_field(synth.gaussian_field(synth.rng_for(6, 4), 400, gs, ("loguniform", 0.5, 3.0),
                                         isotropic=True), gs)
    gv = np.random.default_rng(5).standard_normal(gs.shape).astype(np.float32)
    grid = dgr.Grid.of(gs)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n))
    mu, s, q, rho = field_t(f)
    pairs, items = dgr.dgr_voxelize_count(grid, mu, s, q, 3.0, ws0)
    ws = dgr.Workspace(dgr.make_plan(grid, f.n, pairs + 64, items + 64))
    outs = [torch.empty((f.n, 3), device=DEV), torch.empty((f.n, 3), device=DEV),
            torch.empty((f.n, 4), device=DEV), torch.empty(f.n, device=DEV)]
    dgr.dgr_voxelize_backward(grid, mu, s, q, rho, 3.0, torch.as_tensor(gv, device=DEV), *outs, ws)
    torch.cuda.synchronize()
    ref = O.voxelize_backward(oracle_grid(gs), f.mu, f.s, f.q, f.rho, gv, 3.0)
    for name, got, want in zip(("mu", "s", "rho"), (outs[0], outs[1], outs[3]), (ref[0], ref[1], ref[3])):
        assert rel_l2(H(got), want) <= 1e-4, (name, rel_l2(H(got), want))
    # an isotropic Gaussian does not depend on its rotation: dL/dq is 0 up to
    # FP32 rounding of the chain rule (whose terms are of size |dL/ds| s)
    scale = float(np.max(np.abs(ref[1]) * f.s))
    assert float(np.max(np.abs(H(outs[2])))) <= 1e-4 * scale
    assert float(np.max(np.abs(ref[2]))) <= 1e-12 * scale
