"""Reconstruction driver around dgr_step: the optimisation loop of the method
(paper Sec. 4.3, global optimisation with Adam, Sec. 5.1 schedule) with a
per-iteration JSON-lines log and checkpoint / resume of the whole optimiser
state.

A checkpoint holds everything a step reads or writes that outlives the step:
the optimiser variables theta (mu normalised to [-1, 1] per axis, log s, q,
inverse-softplus rho), Adam's first and second moments m and v, the step
counter t (the learning-rate schedule and Adam's bias corrections are
functions of t alone), the world-space parameters (mu, s, q, rho) the step
derived from theta, the densification statistic when present, and the
problem's scalar settings.  Arrays are stored bit for bit (.npz), so resuming
in deterministic mode continues exactly as the uninterrupted run would: the
step itself is order-independent and bit-reproducible there.

Nothing here computes any part of the method: every iteration is one
dgr_step through the C ABI; the log's PSNR is a metric of the voxelized state
against a reference volume, evaluated between iterations.
"""
import json
import math
import os

import numpy as np
import torch

from . import dgr

CKPT_VERSION = 1
# the Problem fields a checkpoint records (the grid and geometry are the
# caller's: a checkpoint resumes the same problem)
_PROB_FIELDS = ("k_trunc", "lr0", "lr1", "n_iters", "beta1", "beta2", "eps", "w_l1", "w_ssim", "w_tv",
                "ssim_range")


def _cpu(t: torch.Tensor) -> np.ndarray:
    return t.detach().to("cpu").numpy().copy()


def save_checkpoint(path: str, st: "dgr.State", prob: "dgr.Problem" = None, meta: dict = None) -> None:
    """Write the optimiser state of `st` (and the scalar settings of `prob`) to
    `path` (.npz).  Synchronises with the device (the state is copied to the
    host).  The file is written under a temporary name and renamed, so a
    checkpoint is either complete or absent."""
    n = st.n
    arrays = {
        "mu": _cpu(st.mu[:n]), "s": _cpu(st.s[:n]), "q": _cpu(st.q[:n]), "rho": _cpu(st.rho[:n]),
        # theta, m and v are laid out in blocks of n ([mu 3n][log s 3n][q 4n][rho n])
        "theta": _cpu(st.theta[:11 * n]), "m": _cpu(st.m[:11 * n]), "v": _cpu(st.v[:11 * n]),
        "step": _cpu(st.step),
    }
    if st.grad_accum is not None:
        arrays["grad_accum"] = _cpu(st.grad_accum[:n])
    head = {"version": CKPT_VERSION, "n": n, "capacity": st.cap, "meta": meta or {}}
    if prob is not None:
        head["problem"] = {f: getattr(prob, f) for f in _PROB_FIELDS}
    arrays["header"] = np.frombuffer(json.dumps(head).encode(), dtype=np.uint8)
    tmp = path + ".tmp.npz"
    np.savez(tmp, **arrays)
    os.replace(tmp, path)


def read_header(path: str) -> dict:
    with np.load(path) as z:
        return json.loads(bytes(z["header"]).decode())


def load_checkpoint(path: str, device="cuda", capacity: int = None) -> "dgr.State":
    """A new dgr.State on `device` holding the checkpoint's optimiser state.
    capacity: room for densification (default: the saved capacity)."""
    with np.load(path) as z:
        head = json.loads(bytes(z["header"]).decode())
        if head.get("version") != CKPT_VERSION:
            raise dgr.DgrError(f"checkpoint version {head.get('version')} (expected {CKPT_VERSION})")
        n = int(head["n"])
        a = {k: z[k] for k in z.files if k != "header"}
    for k, w in (("mu", 3), ("s", 3), ("q", 4), ("rho", 1)):
        if a[k].shape != ((n, w) if w > 1 else (n,)):
            raise dgr.DgrError(f"checkpoint array {k} has shape {a[k].shape} for n = {n}")
    for k in ("theta", "m", "v"):
        if a[k].shape != (11 * n,):
            raise dgr.DgrError(f"checkpoint array {k} has shape {a[k].shape} for n = {n}")
    T = lambda x: torch.as_tensor(x, device=device)
    st = dgr.State(T(a["mu"]), T(a["s"]), T(a["q"]), T(a["rho"]), accumulate="grad_accum" in a,
                   capacity=max(n, capacity or int(head.get("capacity", n))))
    st.theta[:11 * n] = T(a["theta"])
    st.m[:11 * n] = T(a["m"])
    st.v[:11 * n] = T(a["v"])
    st.step.copy_(T(a["step"]))
    if "grad_accum" in a:
        st.grad_accum[:n] = T(a["grad_accum"])
    return st


def problem_settings_match(prob: "dgr.Problem", path: str) -> bool:
    """Whether `prob` has the scalar settings recorded in the checkpoint (the
    schedule continues only if they agree)."""
    saved = read_header(path).get("problem")
    if saved is None:
        return True
    return all(float(getattr(prob, f)) == float(saved[f]) for f in _PROB_FIELDS)


class IterLog:
    """Per-iteration JSON-lines log: one object per logged iteration with the
    iteration number, the loss, the step's device time, the Gaussian count and,
    when a reference volume is given, the PSNR of the voxelized state."""

    def __init__(self, path: str, append: bool = False):
        self.path = path
        self.f = open(path, "a" if append else "w")

    def write(self, rec: dict) -> None:
        self.f.write(json.dumps(rec) + "\n")
        self.f.flush()

    def close(self) -> None:
        if self.f:
            self.f.close()
            self.f = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_log(path: str) -> list:
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def psnr(vol: torch.Tensor, ref: torch.Tensor, peak: float = 1.0) -> float:
    """10 log10(peak^2 / MSE) over the whole volume (App. B's metric)."""
    mse = float(((vol.double() - ref.double()) ** 2).mean())
    return 10.0 * math.log10(peak * peak / max(mse, 1e-30))


def fit(prob: "dgr.Problem", st: "dgr.State", measured: torch.Tensor, ws: "dgr.Workspace", iters: int, *,
        log: IterLog = None, log_every: int = 1, reference: torch.Tensor = None, psnr_every: int = 0,
        checkpoint: str = None, checkpoint_every: int = 0, stream=None) -> float:
    """Run `iters` optimisation steps (dgr_step) from the state as it stands
    (a fresh state after dgr_params_init, or one from load_checkpoint).

    log / log_every: every log_every-th iteration writes {"iter", "loss",
    "ms", "n_gauss"} (+ "psnr" every psnr_every-th iteration when `reference`,
    a volume of the grid's shape, is given; "iter" counts from the state's own
    step counter, so a resumed run continues the numbering).  Logging reads the
    loss back, i.e. synchronises at each logged iteration; log_every = 0 logs
    nothing.  checkpoint / checkpoint_every: save_checkpoint every
    checkpoint_every-th iteration and after the last.  Returns the last loss."""
    dev = measured.device
    loss = torch.zeros(1, device=dev)
    t0 = int(st.step.item())
    vol = torch.empty(reference.shape, device=dev) if reference is not None else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    logging = log is not None and log_every > 0
    for k in range(iters):
        it = t0 + k + 1
        logged = logging and (it % log_every == 0 or k == iters - 1)
        if logged:
            ev[0].record()
        dgr.dgr_step(prob, st, measured, loss, ws, stream)
        if logged:
            ev[1].record()
            ev[1].synchronize()
            rec = {"iter": it, "loss": float(loss.item()), "ms": ev[0].elapsed_time(ev[1]), "n_gauss": st.n}
            if reference is not None and psnr_every > 0 and (it % psnr_every == 0 or k == iters - 1):
                dgr.dgr_voxelize(prob.grid, *st.view(), prob.k_trunc, vol, ws, stream)
                rec["psnr"] = psnr(vol, reference)
            log.write(rec)
        if checkpoint and ((checkpoint_every > 0 and it % checkpoint_every == 0) or k == iters - 1):
            save_checkpoint(checkpoint, st, prob, {"iter": it})
    last = float(loss.item())
    status = dgr.dgr_status(ws)
    if status != 0:
        raise dgr.DgrError(f"fit: device status {status}")
    return last
