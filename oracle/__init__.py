"""FP64 CPU oracle for the DGR hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU arms of ``bench.py``
may import this package.  It shares no code with the CUDA path and never
imports it.  The arithmetic of the voxelizer, projector and their adjoints is
plain C in ``oracle.c`` (FP64, OpenMP); the loss, the parameter transforms
and the Adam step are plain numpy below.

Paper passages followed (arxiv 2411.04844):
  * Gaussian and volume sum: Eq. 3, Eq. 4 (Sec. 4.1)
  * local box and floored anchor: Sec. 4.1 "Gaussian Effect Confinement",
    "Discretize and Align" (Eq. 6-7); valid mask of Algorithm 1
  * projection P_hat = T(V): Sec. 4.3 (Eq. 12); line integrals of the voxel
    image (Siddon's method)
  * L1 data term: Sec. 4.3 (Eq. 13, first term); Adam with lr 3e-4 -> 3e-5:
    Sec. 5.1 "Implementation Details"

Parity status per function (pins live in tests/test_oracle_pins.py):
  footprint, voxelize, voxelize_backward, project, backproject, l1_loss: pinned
  adam_update / step lr schedule: "parity unpinned" beyond the textbook Adam
  recurrence (the paper fixes neither betas, epsilon nor the decay law).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        f = ctypes.c_float
        d = ctypes.c_double
        L.oracle_footprint.argtypes = [P, f, P, i, P, P, P, f, P, P]
        L.oracle_footprint.restype = None
        L.oracle_voxelize_core.argtypes = [P, d, P, i, P, P, P, P, P, i, P]
        L.oracle_voxelize_core.restype = None
        L.oracle_voxelize_points.argtypes = [P, d, P, i, P, P, P, P, P, i, P, P]
        L.oracle_voxelize_points.restype = None
        L.oracle_voxelize_backward_core.argtypes = [P, d, P, i, P, P, P, P, P, P, P, P, P, P]
        L.oracle_voxelize_backward_core.restype = None
        proj = [P, d, P, i, i, i, i, d, d, d, d, P, P, P]
        L.oracle_project.argtypes = proj
        L.oracle_project.restype = None
        L.oracle_backproject.argtypes = proj
        L.oracle_backproject.restype = None
        L.oracle_ray.argtypes = [i, d, i, i, i, i, d, d, d, d, P, P]
        L.oracle_ray.restype = None
        L.oracle_num_threads.restype = i
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ---------------------------------------------------------------------------
# grid / geometry helpers (plain descriptions, no method arithmetic)
# ---------------------------------------------------------------------------
class Grid:
    """Voxel grid: dims (nx, ny, nz), voxel size h, min corner org.  Volumes are
    stored [nz][ny][nx] (x fastest); voxel i has centre org + (i + 1/2) h."""

    def __init__(self, dims, h, org):
        self.dims = tuple(int(x) for x in dims)
        self.h = float(np.float32(h))
        self.org = tuple(float(np.float32(x)) for x in org)

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)


class Geom:
    """Detector geometry: beam 0 = parallel, 1 = cone; angles in radians."""

    def __init__(self, beam, angles, nu, nv, pu, pv, dso=0.0, dsd=0.0):
        self.beam = int(beam)
        self.angles = np.asarray(angles, dtype=np.float32)
        self.nu, self.nv = int(nu), int(nv)
        self.pu, self.pv = float(np.float32(pu)), float(np.float32(pv))
        self.dso, self.dsd = float(np.float32(dso)), float(np.float32(dsd))

    @property
    def n_views(self):
        return int(self.angles.shape[0])

    @property
    def shape(self):
        return (self.n_views, self.nv, self.nu)


# ---------------------------------------------------------------------------
# voxelizer
# ---------------------------------------------------------------------------
def footprint(grid: Grid, mu, s, q, k_trunc: float):
    """Integer anchor a = floor(u) and clipped box per Gaussian, from the FP32
    operation sequence of the oracle (Sec. 4.1 confinement + Eq. 6)."""
    mu = _c(mu, np.float32).reshape(-1, 3)
    s = _c(s, np.float32).reshape(-1, 3)
    q = _c(q, np.float32).reshape(-1, 4)
    n = mu.shape[0]
    anchor = np.zeros((n, 3), np.int32)
    box = np.zeros((n, 6), np.int32)
    dims = np.array(grid.dims, np.int32)
    org = np.array(grid.org, np.float32)
    lib().oracle_footprint(_p(dims), ctypes.c_float(grid.h), _p(org), n, _p(mu), _p(s), _p(q),
                           ctypes.c_float(k_trunc), _p(anchor), _p(box))
    return anchor, box


def voxelize_core(grid: Grid, mu, s, q, rho, box, brute: bool = False):
    """FP64 volume for given FP64 parameters and fixed integer boxes."""
    mu = _c(mu, np.float64).reshape(-1, 3)
    s = _c(s, np.float64).reshape(-1, 3)
    q = _c(q, np.float64).reshape(-1, 4)
    rho = _c(rho, np.float64).reshape(-1)
    box = _c(box, np.int32).reshape(-1, 6)
    n = mu.shape[0]
    vol = np.zeros(grid.shape, np.float64)
    dims = np.array(grid.dims, np.int32)
    org = np.array(grid.org, np.float64)
    lib().oracle_voxelize_core(_p(dims), grid.h, _p(org), n, _p(mu), _p(s), _p(q), _p(rho),
                               _p(box), 1 if brute else 0, _p(vol))
    return vol


def voxelize(grid: Grid, mu, s, q, rho, k_trunc: float = 3.0, brute: bool = False):
    """V = sum_g rho_g exp(-1/2 d^T A_g d) over each Gaussian's box (Eq. 4)."""
    _, box = footprint(grid, mu, s, q, k_trunc)
    return voxelize_core(grid, np.asarray(mu, np.float32).astype(np.float64),
                         np.asarray(s, np.float32).astype(np.float64),
                         np.asarray(q, np.float32).astype(np.float64),
                         np.asarray(rho, np.float32).astype(np.float64), box, brute)


def voxelize_points(grid: Grid, mu, s, q, rho, pts, k_trunc: float = 3.0):
    """V at voxels pts [m, 3] = (x, y, z) (brute force over all Gaussians)."""
    _, box = footprint(grid, mu, s, q, k_trunc)
    f = lambda a, c: np.ascontiguousarray(np.asarray(a, np.float32).astype(np.float64).reshape(-1, c))
    mu64, s64, q64 = f(mu, 3), f(s, 3), f(q, 4)
    rho64 = np.ascontiguousarray(np.asarray(rho, np.float32).astype(np.float64))
    pts = _c(pts, np.int32).reshape(-1, 3)
    out = np.zeros(pts.shape[0])
    dims = np.array(grid.dims, np.int32)
    org = np.array(grid.org, np.float64)
    lib().oracle_voxelize_points(_p(dims), grid.h, _p(org), mu64.shape[0], _p(mu64), _p(s64),
                                 _p(q64), _p(rho64), _p(box), pts.shape[0], _p(pts), _p(out))
    return out


def voxelize_backward_core(grid: Grid, mu, s, q, rho, box, grad_vol):
    mu = _c(mu, np.float64).reshape(-1, 3)
    s = _c(s, np.float64).reshape(-1, 3)
    q = _c(q, np.float64).reshape(-1, 4)
    rho = _c(rho, np.float64).reshape(-1)
    box = _c(box, np.int32).reshape(-1, 6)
    gv = _c(grad_vol, np.float64)
    assert gv.shape == grid.shape
    n = mu.shape[0]
    g_mu = np.zeros((n, 3)); g_s = np.zeros((n, 3)); g_q = np.zeros((n, 4)); g_rho = np.zeros(n)
    dims = np.array(grid.dims, np.int32)
    org = np.array(grid.org, np.float64)
    lib().oracle_voxelize_backward_core(_p(dims), grid.h, _p(org), n, _p(mu), _p(s), _p(q),
                                        _p(rho), _p(box), _p(gv), _p(g_mu), _p(g_s), _p(g_q),
                                        _p(g_rho))
    return g_mu, g_s, g_q, g_rho


def voxelize_backward(grid: Grid, mu, s, q, rho, grad_vol, k_trunc: float = 3.0):
    _, box = footprint(grid, mu, s, q, k_trunc)
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    return voxelize_backward_core(grid, f(mu), f(s), f(q), f(rho), box, grad_vol)


# ---------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------
def _proj_args(grid: Grid, geom: Geom):
    dims = np.array(grid.dims, np.int32)
    org = np.array(grid.org, np.float64)
    ang = geom.angles.astype(np.float64)
    return dims, org, ang


def project(grid: Grid, geom: Geom, vol):
    """P_hat[view][iv][iu] = sum over voxels of (chord length) x V (Sec. 4.3)."""
    vol = _c(vol, np.float64)
    assert vol.shape == grid.shape
    dims, org, ang = _proj_args(grid, geom)
    sino = np.zeros(geom.shape, np.float64)
    lib().oracle_project(_p(dims), grid.h, _p(org), geom.beam, geom.n_views, geom.nu, geom.nv,
                         geom.pu, geom.pv, geom.dso, geom.dsd, _p(ang), _p(vol), _p(sino))
    return sino


def backproject(grid: Grid, geom: Geom, sino):
    """Exact transpose of project."""
    sino = _c(sino, np.float64)
    assert sino.shape == geom.shape
    dims, org, ang = _proj_args(grid, geom)
    vol = np.zeros(grid.shape, np.float64)
    lib().oracle_backproject(_p(dims), grid.h, _p(org), geom.beam, geom.n_views, geom.nu, geom.nv,
                             geom.pu, geom.pv, geom.dso, geom.dsd, _p(ang), _p(sino), _p(vol))
    return vol


def ray(geom: Geom, view: int, iu: int, iv: int):
    S = np.zeros(3); D = np.zeros(3)
    lib().oracle_ray(geom.beam, float(geom.angles[view]), iu, iv, geom.nu, geom.nv, geom.pu,
                     geom.pv, geom.dso, geom.dsd, _p(S), _p(D))
    return S, D


# ---------------------------------------------------------------------------
# loss, parameter transforms, Adam, one optimisation step
# ---------------------------------------------------------------------------
def l1_loss(pred, meas):
    """L1 data term mean|P_hat - P| and its gradient sign(P_hat - P)/M
    (sign(0) = 0)."""
    diff = np.asarray(pred, np.float64) - np.asarray(meas, np.float64)
    M = diff.size
    return float(np.abs(diff).sum() / M), np.sign(diff) / M


def grid_centre_half(grid: Grid):
    c = np.array([grid.org[a] + 0.5 * grid.dims[a] * grid.h for a in range(3)])
    half = np.array([0.5 * grid.dims[a] * grid.h for a in range(3)])
    return c, half


def to_opt(grid: Grid, mu, s, q, rho):
    """Optimiser variables: mu in [-1,1]^3 box coordinates, log s, raw q,
    inverse-softplus rho (keeps s > 0 and rho > 0, Sec. 4.1 I in R+)."""
    c, half = grid_centre_half(grid)
    mu = np.asarray(mu, np.float64); s = np.asarray(s, np.float64)
    rho = np.asarray(rho, np.float64)
    return {"mu": (mu - c) / half, "s": np.log(s), "q": np.asarray(q, np.float64).copy(),
            "rho": rho + np.log(-np.expm1(-rho))}


def from_opt(grid: Grid, th):
    c, half = grid_centre_half(grid)
    t = th["rho"]
    rho = np.maximum(t, 0) + np.log1p(np.exp(-np.abs(t)))
    return c + half * th["mu"], np.exp(th["s"]), th["q"].copy(), rho


def lr_at(t: int, lr0: float, lr1: float, n_iters: int) -> float:
    """Exponential decay from lr0 at step 1 to lr1 at step n_iters."""
    if n_iters <= 1:
        return lr0
    return lr0 * (lr1 / lr0) ** ((t - 1) / (n_iters - 1))


def adam_update(th, grads, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Textbook Adam (Kingma & Ba 2015) on every array of the dict."""
    out = {}
    for k in th:
        g = grads[k]
        m[k] = b1 * m[k] + (1 - b1) * g
        v[k] = b2 * v[k] + (1 - b2) * g * g
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        out[k] = th[k] - lr * mh / (np.sqrt(vh) + eps)
    return out


def step(grid: Grid, geom: Geom, mu, s, q, rho, th, m, v, t, meas, k_trunc, lr0, lr1, n_iters):
    """One optimisation iteration in FP64: voxelize -> project -> L1 ->
    backproject -> voxelize adjoint -> chain to optimiser variables -> Adam.
    mu, s, q, rho are the FP32 parameters used for the box integers."""
    _, box = footprint(grid, mu, s, q, k_trunc)
    mu64, s64, q64, rho64 = from_opt(grid, th)
    vol = voxelize_core(grid, mu64, s64, q64, rho64, box)
    pred = project(grid, geom, vol)
    loss, r = l1_loss(pred, meas)
    gv = backproject(grid, geom, r)
    g_mu, g_s, g_q, g_rho = voxelize_backward_core(grid, mu64, s64, q64, rho64, box, gv)
    _, half = grid_centre_half(grid)
    sig = 1.0 / (1.0 + np.exp(-th["rho"]))
    grads = {"mu": g_mu * half, "s": g_s * s64, "q": g_q, "rho": g_rho * sig}
    th_new = adam_update(th, grads, m, v, t, lr_at(t, lr0, lr1, n_iters))
    return loss, th_new, grads
