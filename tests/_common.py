"""Shared test helpers: matching oracle / device descriptions of one problem."""
import math

import numpy as np

import oracle as O
from paper_2411_04844_b300 import synth


def oracle_grid(spec: synth.GridSpec) -> O.Grid:
    return O.Grid(spec.dims, spec.h, spec.org)


def oracle_geom(spec: synth.GeomSpec) -> O.Geom:
    return O.Geom(spec.beam, spec.angles, spec.nu, spec.nv, spec.pu, spec.pv, spec.dso, spec.dsd)


def guard_field(field: synth.Field, grid: synth.GridSpec, k=3.0, band=1e-3, rng=None):
    """Resample Gaussians whose voxel-unit centre u_a or k sigma_a lies within
    `band` of an integer (FP64 check), so no footprint decision sits on an
    FP32 rounding edge.  Returns a new field with the same size."""
    rng = rng or np.random.default_rng(12345)
    f = synth.Field(field.mu.copy(), field.s.copy(), field.q.copy(), field.rho.copy())
    for _ in range(100):
        bad = _near_integer(f, grid, k, band)
        if not bad.any():
            return f
        idx = np.nonzero(bad)[0]
        lo = np.array(grid.org); hi = lo + np.array(grid.extent)
        f.mu[idx] = rng.uniform(lo, hi, (len(idx), 3)).astype(np.float32)
        # one factor per Gaussian: isotropic Gaussians stay isotropic
        f.s[idx] = (f.s[idx] * rng.uniform(0.97, 1.03, (len(idx), 1))).astype(np.float32)
    raise RuntimeError("guard band not reached")


def _near_integer(f, grid, k, band):
    q = f.q.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    var = np.einsum("nak,nk->na", R ** 2, f.s.astype(np.float64) ** 2)
    ks = k * np.sqrt(var) / grid.h
    u = (f.mu.astype(np.float64) - np.array(grid.org)) / grid.h - 0.5
    near = lambda a: np.abs(a - np.round(a)) < band
    return (near(u) | near(ks)).any(1)


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def margin_measurement(og, oo, th, rng, k=3.0, lo=0.02, hi=0.06, signs="random"):
    """Measured projections for an oracle-vs-GPU step comparison: the FP64
    oracle's own prediction at optimiser variables th plus +-U[lo, hi] per
    ray, so no L1 residual sits near its kink (both sides take every sign
    decision alike).  signs="random": a random sign per ray; "positive": the
    prediction always above the measurement (a residual of one sign, whose
    backprojection does not cancel).  Also returns the FP32 parameters that
    decide the box integers (mu, s, q, rho)."""
    p32 = tuple(a.astype(np.float32) for a in O.from_opt(og, th))
    _, box = O.footprint(og, p32[0], p32[1], p32[2], k)
    pred = O.project(og, oo, O.voxelize_core(og, *O.from_opt(og, th), box))
    sg = rng.choice([-1.0, 1.0], pred.shape) if signs == "random" else -np.ones(pred.shape)
    meas = pred + sg * rng.uniform(lo, hi, pred.shape)
    return meas.astype(np.float32), p32
