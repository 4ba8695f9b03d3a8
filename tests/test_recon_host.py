"""Checkpoint / resume and the per-iteration log of the reconstruction driver
(host logic, no GPU): a checkpoint restores every array of the optimiser state
bit for bit and records the problem's scalar settings; malformed checkpoints
are refused; the JSON-lines log round-trips."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2411_04844_b300 import dgr, recon


def _state(n=37, cap=50, accumulate=True, seed=3):
    rng = np.random.default_rng(seed)
    T = lambda a: torch.as_tensor(a.astype(np.float32))
    st = dgr.State(T(rng.normal(size=(n, 3))), T(rng.uniform(0.5, 3, (n, 3))), T(rng.normal(size=(n, 4))),
                   T(rng.uniform(0, 1, n)), accumulate=accumulate, capacity=cap)
    # optimiser state with bits that a float round trip through text would lose
    st.theta[:11 * n] = T(rng.normal(size=11 * n) * 1e-7 + 1.0)
    st.m[:11 * n] = T(rng.normal(size=11 * n) * 1e-3)
    st.v[:11 * n] = T(rng.uniform(0, 1e-6, 11 * n))
    st.step.fill_(123)
    if accumulate:
        st.grad_accum[:n] = T(rng.uniform(0, 5, n))
    return st


def _problem(lr0=3e-4):
    grid = dgr.Grid(16, 16, 16, 1.0, -8.0, -8.0, -8.0)
    geom = dgr.Geom(dgr.DGR_CONE, 10, 20, 20, 1.5, 1.5, 100.0, 150.0, None)
    return dgr.make_problem(grid, geom, 3.0, lr0, 3e-5, 2000, weights=dgr.PAPER_WEIGHTS)


@pytest.mark.parametrize("accumulate", [True, False])
def test_checkpoint_round_trip_bitwise(tmp_path, accumulate):
    st = _state(accumulate=accumulate)
    prob = _problem()
    path = str(tmp_path / "ck.npz")
    recon.save_checkpoint(path, st, prob, {"iter": 123})
    r = recon.load_checkpoint(path, device="cpu")
    n = st.n
    assert r.n == n and r.cap == st.cap
    for name in ("mu", "s", "q", "rho"):
        assert torch.equal(getattr(r, name)[:n], getattr(st, name)[:n]), name
    for name in ("theta", "m", "v"):
        assert torch.equal(getattr(r, name)[:11 * n], getattr(st, name)[:11 * n]), name
    assert int(r.step.item()) == 123 and r.step.dtype == torch.int32
    assert (r.grad_accum is not None) == accumulate
    if accumulate:
        assert torch.equal(r.grad_accum[:n], st.grad_accum[:n])
    h = recon.read_header(path)
    assert h["meta"] == {"iter": 123} and h["n"] == n
    assert recon.problem_settings_match(prob, path)
    assert not recon.problem_settings_match(_problem(lr0=1e-3), path)
    # more room for densification on resume
    assert recon.load_checkpoint(path, device="cpu", capacity=80).cap == 80


def test_checkpoint_refuses_malformed(tmp_path):
    st = _state(accumulate=False)
    path = str(tmp_path / "ck.npz")
    recon.save_checkpoint(path, st)
    with np.load(path) as z:
        a = {k: z[k] for k in z.files}
    bad = dict(a)
    bad["theta"] = a["theta"][:-1]
    np.savez(str(tmp_path / "bad.npz"), **bad)
    with pytest.raises(dgr.DgrError):
        recon.load_checkpoint(str(tmp_path / "bad.npz"), device="cpu")
    old = dict(a)
    old["header"] = np.frombuffer(b'{"version": 0, "n": 37}', dtype=np.uint8)
    np.savez(str(tmp_path / "old.npz"), **old)
    with pytest.raises(dgr.DgrError):
        recon.load_checkpoint(str(tmp_path / "old.npz"), device="cpu")


def test_iter_log_round_trip(tmp_path):
    path = str(tmp_path / "log.jsonl")
    with recon.IterLog(path) as log:
        log.write({"iter": 1, "loss": 2.5, "ms": 0.1, "n_gauss": 10})
        log.write({"iter": 2, "loss": 2.25, "ms": 0.1, "n_gauss": 10, "psnr": 20.0})
    with recon.IterLog(path, append=True) as log:
        log.write({"iter": 3, "loss": 2.0, "ms": 0.1, "n_gauss": 12})
    recs = recon.read_log(path)
    assert [r["iter"] for r in recs] == [1, 2, 3]
    assert recs[1]["psnr"] == 20.0 and recs[2]["n_gauss"] == 12


def test_psnr_closed_form():
    ref = torch.zeros(4, 4, 4)
    vol = ref + 0.1  # MSE 0.01 -> 20 dB at peak 1
    assert abs(recon.psnr(vol, ref) - 20.0) < 1e-6  # 0.1 rounded to FP32
