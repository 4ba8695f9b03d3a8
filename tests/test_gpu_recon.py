"""Checkpoint / resume of a reconstruction on the GPU: in deterministic mode a
fit interrupted after k iterations, saved, loaded into a new state and
workspace and continued, ends bit for bit where the uninterrupted fit ends
(theta, Adam's m and v, the step counter, the world-space parameters and the
per-iteration losses), for the L1 objective and the paper's full objective;
the log's PSNR is that of the voxelized state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_04844_b300 import dgr, recon, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _problem(weights):
    gs = synth.GridSpec((28, 24, 20), 1.0, (-14.0, -12.0, -10.0))
    geo = synth.cone_geom(12, 40, 32, 1.5, 1.5, 80.0, 120.0)
    f = synth.gaussian_field(synth.rng_for(1, 91), 400, gs, ("loguniform", 0.6, 3.0))
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    phantom = T(synth.ellipsoid_phantom(synth.rng_for(1, 92), gs, 6).astype(np.float32))
    grid = dgr.Grid.of(gs)
    ang = T(geo.angles)
    gg = dgr.Geom.of(geo, ang)
    ws0 = dgr.Workspace(dgr.make_plan(grid, f.n, 1 << 22, 1 << 20, gg, step=True))
    meas = torch.empty(geo.shape, device=DEV)
    dgr.dgr_project(grid, gg, phantom, meas, ws0)
    prob = dgr.make_problem(grid, gg, 3.0, 1e-2, 1e-3, 12, weights=weights)
    return f, grid, gg, ang, prob, meas, phantom


def _fresh(prob, f):
    st = dgr.State(T(f.mu), T(f.s), T(f.q), T(f.rho))
    dgr.dgr_params_init(prob, st)
    return st


def _ws(grid, gg, n):
    return dgr.Workspace(dgr.make_plan(grid, n, 1 << 22, 1 << 20, gg, step=True))


@pytest.mark.parametrize("weights", [(1.0, 0.0, 0.0), dgr.PAPER_WEIGHTS], ids=["l1", "paper"])
def test_resume_equals_uninterrupted_bitwise(tmp_path, weights):
    dgr.dgr_set_deterministic(True)
    f, grid, gg, ang, prob, meas, phantom = _problem(weights)
    # uninterrupted: 8 iterations
    st_a = _fresh(prob, f)
    with recon.IterLog(str(tmp_path / "a.jsonl")) as log:
        recon.fit(prob, st_a, meas, _ws(grid, gg, f.n), 8, log=log)
    # interrupted after 3, resumed from the checkpoint in a new state and workspace
    ck = str(tmp_path / "ck.npz")
    st_b = _fresh(prob, f)
    with recon.IterLog(str(tmp_path / "b.jsonl")) as log:
        recon.fit(prob, st_b, meas, _ws(grid, gg, f.n), 3, log=log, checkpoint=ck)
    del st_b
    assert recon.problem_settings_match(prob, ck)
    st_c = recon.load_checkpoint(ck, device=DEV)
    assert int(st_c.step.item()) == 3
    with recon.IterLog(str(tmp_path / "b.jsonl"), append=True) as log:
        recon.fit(prob, st_c, meas, _ws(grid, gg, f.n), 5, log=log)
    torch.cuda.synchronize()
    n = f.n
    assert int(st_c.step.item()) == int(st_a.step.item()) == 8
    for name in ("theta", "m", "v"):
        assert torch.equal(getattr(st_c, name)[:11 * n], getattr(st_a, name)[:11 * n]), name
    for name in ("mu", "s", "q", "rho"):
        assert torch.equal(getattr(st_c, name)[:n], getattr(st_a, name)[:n]), name
    la, lb = recon.read_log(str(tmp_path / "a.jsonl")), recon.read_log(str(tmp_path / "b.jsonl"))
    assert [r["iter"] for r in lb] == list(range(1, 9)) == [r["iter"] for r in la]
    assert [r["loss"] for r in lb] == [r["loss"] for r in la]



def test_log_psnr_is_the_voxelized_state(tmp_path):
    dgr.dgr_set_deterministic(True)
    f, grid, gg, ang, prob, meas, phantom = _problem((1.0, 0.0, 0.0))
    st = _fresh(prob, f)
    ws = _ws(grid, gg, f.n)
    path = str(tmp_path / "p.jsonl")
    with recon.IterLog(path) as log:
        recon.fit(prob, st, meas, ws, 4, log=log, log_every=2, reference=phantom, psnr_every=2)
    recs = recon.read_log(path)
    assert [r["iter"] for r in recs] == [2, 4]
    assert all("psnr" in r and r["ms"] > 0 and r["n_gauss"] == f.n for r in recs)
    vol = torch.empty(phantom.shape, device=DEV)
    dgr.dgr_voxelize(grid, *st.view(), prob.k_trunc, vol, ws)
    assert recs[-1]["psnr"] == recon.psnr(vol, phantom)
