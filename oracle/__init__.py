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
  * full objective w1 L1 + w2 L_SSIM + w3 L_TV (Sec. 4.3, weights 0.6 / 0.2 /
    1; App. D.1): SSIM of Wang et al. 2004 on every projection image with an
    11 x 11 Gaussian window (sigma 1.5), anisotropic TV of the volume

Parity status per function (pins live in tests/test_oracle_pins.py):
  footprint, voxelize, voxelize_backward, project, backproject, l1_loss,
  ssim_loss, tv_loss: pinned
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


def gaussian_window(size: int = 11, sigma: float = 1.5):
    """1D Gaussian weights exp(-(i - c)^2 / (2 sigma^2)), c the middle tap,
    normalised to sum 1; the SSIM window is their outer product (Wang et al.
    2004, cited by the paper for SSIM)."""
    i = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-i * i / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(img, g):
    """Correlation of each [nv][nu] image with the separable window, zero
    outside the image ("same" size)."""
    from scipy.ndimage import correlate1d
    out = correlate1d(np.asarray(img, np.float64), g, axis=-1, mode="constant", cval=0.0)
    return correlate1d(out, g, axis=-2, mode="constant", cval=0.0)


def ssim_terms(x, y, data_range: float = 1.0):
    """Local SSIM statistics of x against y (arrays [views][nv][nu], each view
    an image): windowed means, variances and covariance with an 11 x 11
    Gaussian window (sigma 1.5, zero outside the image), C1 = (0.01 L)^2,
    C2 = (0.03 L)^2.  Returns the SSIM map and the dict of statistics."""
    g = gaussian_window()
    x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
    mx, my = _blur(x, g), _blur(y, g)
    sxx = _blur(x * x, g) - mx * mx
    syy = _blur(y * y, g) - my * my
    sxy = _blur(x * y, g) - mx * my
    c1 = (0.01 * data_range) ** 2
    c2 = (0.03 * data_range) ** 2
    n1, n2 = 2 * mx * my + c1, 2 * sxy + c2
    d1, d2 = mx * mx + my * my + c1, sxx + syy + c2
    smap = n1 * n2 / (d1 * d2)
    return smap, dict(mx=mx, my=my, sxx=sxx, syy=syy, sxy=sxy, n1=n1, n2=n2, d1=d1, d2=d2, g=g)


def ssim_loss(pred, meas, data_range: float = 1.0):
    """L_SSIM = 1 - mean SSIM map over every pixel of every view (paper
    Sec. 4.3 / App. D.1: SSIM computed in the projection domain), and its
    gradient with respect to pred.  With S = N1 N2 / (D1 D2) per pixel p and
    the local statistics linear or quadratic in pred:
        dS/dmu_x = 2 mu_y N2 / (D1 D2) - 2 mu_x S / D1,
        dS/dsig_xx = -S / D2,   dS/dsig_xy = 2 N1 / (D1 D2),
    and with A = dS/dmu_x - 2 mu_x dS/dsig_xx - mu_y dS/dsig_xy,
    B = dS/dsig_xx, C = dS/dsig_xy, the chain through the window gives
        d mean(S) / d x(q) = [ (w*A)(q) + 2 x(q) (w*B)(q) + y(q) (w*C)(q) ] / N
    (w symmetric, zero outside the image)."""
    x = np.asarray(pred, np.float64); y = np.asarray(meas, np.float64)
    smap, t = ssim_terms(x, y, data_range)
    N = smap.size
    dd = t["d1"] * t["d2"]
    dmx = 2 * t["my"] * t["n2"] / dd - 2 * t["mx"] * smap / t["d1"]
    dsxx = -smap / t["d2"]
    dsxy = 2 * t["n1"] / dd
    A = dmx - 2 * t["mx"] * dsxx - t["my"] * dsxy
    g = t["g"]
    grad = (_blur(A, g) + 2 * x * _blur(dsxx, g) + y * _blur(dsxy, g)) / N
    return float(1.0 - smap.mean()), -grad


def tv_loss(vol):
    """Anisotropic total variation of the volume [nz][ny][nx]: the sum over
    axes of |forward differences| where both voxels exist, divided by the
    number of voxels (the paper names TV without a formula; this is the
    reading), and its gradient (sign(0) = 0)."""
    v = np.asarray(vol, np.float64)
    total = 0.0
    grad = np.zeros_like(v)
    for ax in range(3):
        d = np.diff(v, axis=ax)
        total += np.abs(d).sum()
        sg = np.sign(d)
        lo = [slice(None)] * 3; hi = [slice(None)] * 3
        lo[ax] = slice(0, -1); hi[ax] = slice(1, None)
        grad[tuple(lo)] -= sg
        grad[tuple(hi)] += sg
    return total / v.size, grad / v.size


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


def step(grid: Grid, geom: Geom, mu, s, q, rho, th, m, v, t, meas, k_trunc, lr0, lr1, n_iters,
         weights=(1.0, 0.0, 0.0), data_range: float = 1.0):
    """One optimisation iteration in FP64: voxelize -> project -> loss ->
    backproject -> voxelize adjoint -> chain to optimiser variables -> Adam.
    The loss is w1 L1(P_hat, P) + w2 L_SSIM(P_hat, P) + w3 L_TV(V) (paper
    Sec. 4.3, weights 0.6 / 0.2 / 1 there; (1, 0, 0) is the L1 term alone).
    mu, s, q, rho are the FP32 parameters used for the box integers."""
    w1, w2, w3 = weights
    _, box = footprint(grid, mu, s, q, k_trunc)
    mu64, s64, q64, rho64 = from_opt(grid, th)
    vol = voxelize_core(grid, mu64, s64, q64, rho64, box)
    pred = project(grid, geom, vol)
    l1, r = l1_loss(pred, meas)
    loss, r = w1 * l1, w1 * r
    if w2:
        ls, gs = ssim_loss(pred, meas, data_range)
        loss += w2 * ls
        r = r + w2 * gs
    gv = backproject(grid, geom, r)
    if w3:
        lt, gt = tv_loss(vol)
        loss += w3 * lt
        gv = gv + w3 * gt
    g_mu, g_s, g_q, g_rho = voxelize_backward_core(grid, mu64, s64, q64, rho64, box, gv)
    th_new, grads = optimiser_step(grid, th, m, v, t, (g_mu, g_s, g_q, g_rho), lr0, lr1, n_iters)
    return loss, th_new, grads


def optimiser_step(grid: Grid, th, m, v, t, param_grads, lr0, lr1, n_iters):
    """The last link of an iteration (Sec. 5.1): the gradients with respect
    to (mu, s, q, rho) chained to the optimiser variables -- d/d((mu-c)/half)
    = half d/dmu, d/dlog s = s d/ds, q raw, d/d(softplus^-1 rho) =
    sigmoid(theta_rho) d/drho -- then one Adam step at lr(t).  Returns the new
    variables and the chained gradients (m, v updated in place)."""
    g_mu, g_s, g_q, g_rho = param_grads
    _, half = grid_centre_half(grid)
    s64 = np.exp(th["s"])
    sig = 1.0 / (1.0 + np.exp(-th["rho"]))
    grads = {"mu": g_mu * half, "s": g_s * s64, "q": g_q, "rho": g_rho * sig}
    return adam_update(th, grads, m, v, t, lr_at(t, lr0, lr1, n_iters)), grads
