"""Thin Python binding of libdgr (include/dgr.h): argument marshalling only.

Every function named ``dgr_*`` maps one-to-one onto the C entry point of the
same name; tensors are passed as device pointers, the stream is torch's
current stream unless given.  No computation happens here and there is no
fallback: if the library is missing or fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_LIB = None

DGR_OK = 0
DGR_ERR_ARG = 1
DGR_ERR_WS_TOO_SMALL = 2
DGR_ERR_CUDA = 3
DGR_STATUS_NONFINITE = 0x10
DGR_STATUS_PAIR_OVERFLOW = 0x20
DGR_STATUS_ITEM_OVERFLOW = 0x40
DGR_STATUS_BOUNDS = 0x100  # bounds-checked build only (DGR_CHECK_BOUNDS=1)
DGR_PARALLEL = 0
DGR_CONE = 1

# voxel tile of the forward voxelizer (x, y, default z depth)
TILE = (8, 16, 32)

EXPORTS = [
    "dgr_ws_bytes", "dgr_ws_create", "dgr_ws_destroy", "dgr_tile_count", "dgr_status",
    "dgr_strerror", "dgr_set_deterministic", "dgr_footprint", "dgr_voxelize_count",
    "dgr_voxelize", "dgr_voxelize_backward", "dgr_project", "dgr_backproject",
    "dgr_l1_residual", "dgr_params_init", "dgr_adam", "dgr_step", "dgr_step_timed", "dgr_launch_count",
    "dgr_project_noalloc", "dgr_step_batched", "dgr_set_tile_depth", "dgr_set_backprojector",
    "dgr_net_param_count", "dgr_net_ws_bytes", "dgr_net_forward", "dgr_net_backward",
    "dgr_net_loss", "dgr_adam_flat", "dgr_fdk_filter", "dgr_seed_bytes", "dgr_seed",
    "dgr_seed_rescale", "dgr_ssim_loss", "dgr_tv_loss", "dgr_densify", "dgr_set_separable", "dgr_set_staged_walk",
    "dgr_set_conv_engine", "dgr_net_status", "dgr_pipe_rate", "dgr_l2_rate", "dgr_test_bounded_wait", "dgr_proposals",
    "dgr_logscale_weight", "dgr_fit_targets",
]
# size of the fixed device scratch of dgr_project_noalloc (DGR_NOALLOC_SCRATCH_BYTES)
NOALLOC_SCRATCH_BYTES = 4 << 20
DGR_STEP_EVENTS = 7
# with 15 events, [7]/[8] bracket the backprojector's path scatter kernel,
# [9]/[10] the projector's main kernel, [11]/[12] the voxelizer's tile kernel
# and [13]/[14] the voxelize adjoint's item kernel
DGR_STEP_KERNEL_EVENTS = 15
STEP_PHASES = ("voxelize", "project", "l1", "backproject", "voxelize_backward", "adam")


class DgrError(RuntimeError):
    pass


class Grid(ctypes.Structure):
    """dgr_grid; z0 > 0: the z-slab of layers [z0, z0 + nz) of a larger grid
    with the same origin (see include/dgr.h)."""
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_float), ("ox", ctypes.c_float), ("oy", ctypes.c_float),
                ("oz", ctypes.c_float), ("z0", ctypes.c_int)]

    @staticmethod
    def of(spec) -> "Grid":
        """From any object with dims (nx, ny, nz), h and org."""
        nx, ny, nz = spec.dims
        return Grid(nx, ny, nz, spec.h, *spec.org, 0)

    def slab(self, z0: int, nz: int) -> "Grid":
        """Layers [z0, z0 + nz) of this (whole) grid."""
        if self.z0 != 0 or z0 < 0 or nz < 1 or z0 + nz > self.nz:
            raise DgrError(f"slab [{z0}, {z0 + nz}) of a grid of {self.nz} layers")
        return Grid(self.nx, self.ny, nz, self.h, self.ox, self.oy, self.oz, z0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


class Geom(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int), ("n_views", ctypes.c_int), ("nu", ctypes.c_int),
                ("nv", ctypes.c_int), ("pu", ctypes.c_float), ("pv", ctypes.c_float),
                ("dso", ctypes.c_float), ("dsd", ctypes.c_float), ("angles", ctypes.c_void_p)]

    @staticmethod
    def of(spec, angles_dev: torch.Tensor) -> "Geom":
        """From a geometry description and its angles already on the device
        (the tensor must outlive every call made with this descriptor)."""
        _check(angles_dev, "angles")
        return Geom(spec.beam, spec.n_views, spec.nu, spec.nv, spec.pu, spec.pv, spec.dso,
                    spec.dsd, angles_dev.data_ptr())

    @property
    def shape(self):
        return (self.n_views, self.nv, self.nu)


class WsPlan(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_int), ("max_tiles", ctypes.c_int),
                ("max_pairs", ctypes.c_longlong), ("max_items", ctypes.c_longlong),
                ("max_vox", ctypes.c_longlong), ("max_rays", ctypes.c_longlong),
                ("max_views", ctypes.c_int), ("max_nu", ctypes.c_int), ("max_nv", ctypes.c_int),
                ("max_inst", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("grid", Grid), ("geom", Geom), ("k_trunc", ctypes.c_float),
                ("lr0", ctypes.c_float), ("lr1", ctypes.c_float), ("n_iters", ctypes.c_int),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("w_l1", ctypes.c_float), ("w_ssim", ctypes.c_float), ("w_tv", ctypes.c_float),
                ("ssim_range", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("mu", ctypes.c_void_p), ("s", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("m", ctypes.c_void_p), ("v", ctypes.c_void_p), ("step", ctypes.c_void_p),
                ("grad_accum", ctypes.c_void_p)]


class DensifyCfg(ctypes.Structure):
    """Algorithm 2 constants (paper defaults)."""
    _fields_ = [("tau", ctypes.c_float), ("theta_frac", ctypes.c_float), ("size", ctypes.c_float),
                ("n_max", ctypes.c_int)]

    @classmethod
    def paper(cls, n_max=500_000):
        return cls(2e-4, 0.005, 17.0, int(n_max))


def checked_build() -> bool:
    """DGR_CHECK_BOUNDS=1 in the environment: load the bounds-checked library
    (libdgr_checked.so; indices outside their buffers are reported as
    DGR_STATUS_BOUNDS instead of faulting)."""
    return os.environ.get("DGR_CHECK_BOUNDS", "") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked_build() else _build.LIB


def lib():
    """Load libdgr.so (building it if its sources are newer).  Raises if the
    library cannot be built or loaded -- there is no CPU fallback."""
    global _LIB
    if _LIB is None:
        path = _build.build(checked=checked_build())
        if not os.path.exists(path):
            raise DgrError(f"libdgr not found at {path}")
        L = ctypes.CDLL(path)
        P, i, f, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
        sig = {
            "dgr_ws_bytes": [ctypes.POINTER(WsPlan), ctypes.POINTER(ctypes.c_size_t)],
            "dgr_ws_create": [ctypes.POINTER(P), ctypes.POINTER(WsPlan)],
            "dgr_ws_destroy": [P],
            "dgr_tile_count": [ctypes.POINTER(Grid), ctypes.POINTER(i)],
            "dgr_status": [P, P, ctypes.POINTER(i)],
            "dgr_set_deterministic": [i],
            "dgr_set_tile_depth": [i],
            "dgr_set_separable": [i],
            "dgr_set_staged_walk": [i],
            "dgr_set_backprojector": [i],
            "dgr_set_conv_engine": [i],
            "dgr_net_status": [i, P, ctypes.c_size_t, ctypes.POINTER(i)],
            "dgr_footprint": [ctypes.POINTER(Grid), i, P, P, P, f, P, P, P],
            "dgr_voxelize_count": [ctypes.POINTER(Grid), i, P, P, P, f, ctypes.POINTER(ll),
                                   ctypes.POINTER(ll), P, P],
            "dgr_voxelize": [ctypes.POINTER(Grid), i, P, P, P, P, f, P, P, P],
            "dgr_voxelize_backward": [ctypes.POINTER(Grid), i, P, P, P, P, f, P, P, P, P, P, P, P],
            "dgr_project": [ctypes.POINTER(Grid), ctypes.POINTER(Geom), P, P, P, P],
            "dgr_backproject": [ctypes.POINTER(Grid), ctypes.POINTER(Geom), P, P, P, P],
            "dgr_l1_residual": [P, P, ll, f, P, P, P, P],
            "dgr_adam": [ctypes.POINTER(Problem), ctypes.POINTER(Params), P, P, P, P, P],
            "dgr_ssim_loss": [ctypes.POINTER(Geom), P, P, f, P, P, P, P],
            "dgr_tv_loss": [ctypes.POINTER(Grid), P, P, P, P, P],
            "dgr_densify": [ctypes.POINTER(Grid), ctypes.POINTER(DensifyCfg), i, ctypes.POINTER(Params),
                            P, ctypes.POINTER(Params), ctypes.POINTER(i), P, P],
            "dgr_params_init": [ctypes.POINTER(Problem), ctypes.POINTER(Params), P],
            "dgr_step": [ctypes.POINTER(Problem), ctypes.POINTER(Params), P, P, P, P],
            "dgr_step_timed": [ctypes.POINTER(Problem), ctypes.POINTER(Params), P, P, P, P,
                               ctypes.POINTER(P), i],
            "dgr_project_noalloc": [ctypes.POINTER(Grid), ctypes.POINTER(Geom), P, P, P],
            "dgr_pipe_rate": [i, i, i, P, P, P],
            "dgr_test_bounded_wait": [i, P, P, P],
            "dgr_l2_rate": [i, ll, i, i, P, P, P],
            "dgr_step_batched": [i, ctypes.POINTER(Problem), ctypes.POINTER(Params),
                                 ctypes.POINTER(P), P, P, P],
            "dgr_net_ws_bytes": [i, ctypes.POINTER(ctypes.c_size_t)],
            "dgr_net_forward": [i, P, P, P, P, ctypes.c_size_t, P],
            "dgr_net_backward": [i, P, P, P, P, P, ctypes.c_size_t, P],
            "dgr_net_loss": [i, P, P, f, f, P, P, P, ctypes.c_size_t, P],
            "dgr_adam_flat": [ll, P, P, P, P, i, f, f, f, f, P],
            "dgr_fdk_filter": [ctypes.POINTER(Geom), f, P, P, P],
            "dgr_proposals": [ll, P, i, f, P, P, P],
            "dgr_logscale_weight": [i, P, P, f, P, P],
            "dgr_fit_targets": [ll, P, P, f, f, f, f, P, P],
            "dgr_seed_bytes": [i, ctypes.POINTER(ctypes.c_size_t)],
            "dgr_seed": [ctypes.POINTER(Grid), P, P, i, P, P, P, P, P, P, P, P,
                         ctypes.c_size_t, P],
            "dgr_seed_rescale": [i, P, P, P, P, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.dgr_net_param_count.argtypes = []
        L.dgr_net_param_count.restype = ctypes.c_longlong
        L.dgr_launch_count.argtypes = []
        L.dgr_launch_count.restype = ctypes.c_longlong
        L.dgr_strerror.argtypes = [i]
        L.dgr_strerror.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def _rc(code: int, what: str):
    if code != DGR_OK:
        msg = lib().dgr_strerror(code).decode()
        raise DgrError(f"{what}: {msg} ({code})")


def _check(t: torch.Tensor, name: str, dtype=torch.float32):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a tensor")
    if not t.is_cuda:
        raise DgrError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise DgrError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise DgrError(f"{name} must be contiguous")


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


# ---------------------------------------------------------------------------
# workspace
# ---------------------------------------------------------------------------
class Workspace:
    """Owns one dgr_ws (a single cudaMalloc made by dgr_ws_create)."""

    def __init__(self, plan: WsPlan):
        self.plan = plan
        h = ctypes.c_void_p()
        _rc(lib().dgr_ws_create(ctypes.byref(h), ctypes.byref(plan)), "dgr_ws_create")
        self.handle = h

    @property
    def ptr(self):
        return self.handle

    def close(self):
        if self.handle:
            lib().dgr_ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgr_ws_bytes(plan: WsPlan) -> int:
    b = ctypes.c_size_t()
    _rc(lib().dgr_ws_bytes(ctypes.byref(plan), ctypes.byref(b)), "dgr_ws_bytes")
    return int(b.value)


def dgr_tile_count(grid: Grid) -> int:
    t = ctypes.c_int()
    _rc(lib().dgr_tile_count(ctypes.byref(grid), ctypes.byref(t)), "dgr_tile_count")
    return int(t.value)


def make_plan(grid: Grid = None, n: int = 0, max_pairs: int = 0, max_items: int = 0,
              geom=None, step: bool = False) -> WsPlan:
    p = WsPlan()
    p.max_n = int(n)
    p.max_tiles = dgr_tile_count(grid) if grid is not None else 0
    p.max_pairs = int(max_pairs)
    p.max_items = int(max_items)
    if geom is not None:
        p.max_views, p.max_nu, p.max_nv = int(geom.n_views), int(geom.nu), int(geom.nv)
        if grid is not None:  # room for dgr_project's z-fastest copy of the volume
            p.max_vox = grid.nx * grid.ny * grid.nz
    if step:
        p.max_vox = grid.nx * grid.ny * grid.nz
        p.max_rays = geom.n_views * geom.nu * geom.nv
    return p


def dgr_status(ws: Workspace, stream=None) -> int:
    v = ctypes.c_int()
    _rc(lib().dgr_status(ws.ptr, _stream(stream), ctypes.byref(v)), "dgr_status")
    return int(v.value)


def dgr_set_backprojector(variant: int):
    """0: ray scatter (default); 1: column gather; 2: brick scatter."""
    _rc(lib().dgr_set_backprojector(int(variant)), "dgr_set_backprojector")


def dgr_set_separable(on: bool):
    """Separable voxelizer for all-diagonal-A calls (default on)."""
    _rc(lib().dgr_set_separable(1 if on else 0), "dgr_set_separable")


def dgr_set_staged_walk(on: bool):
    """Bulk-copy staging of the path walks through shared memory (default off)."""
    _rc(lib().dgr_set_staged_walk(1 if on else 0), "dgr_set_staged_walk")


def dgr_set_tile_depth(tz: int):
    _rc(lib().dgr_set_tile_depth(int(tz)), "dgr_set_tile_depth")


def dgr_set_deterministic(on: bool):
    _rc(lib().dgr_set_deterministic(1 if on else 0), "dgr_set_deterministic")


# ---------------------------------------------------------------------------
# voxelizer
# ---------------------------------------------------------------------------
def dgr_footprint(grid: Grid, mu, s, q, k_trunc, anchor, box, stream=None):
    for t, nm in ((mu, "mu"), (s, "s"), (q, "q")):
        _check(t, nm)
    _check(anchor, "anchor", torch.int32)
    _check(box, "box", torch.int32)
    n = mu.shape[0]
    _rc(lib().dgr_footprint(ctypes.byref(grid), n, _ptr(mu), _ptr(s), _ptr(q), float(k_trunc),
                            _ptr(anchor), _ptr(box), _stream(stream)), "dgr_footprint")


def dgr_voxelize_count(grid: Grid, mu, s, q, k_trunc, ws: Workspace, stream=None):
    for t, nm in ((mu, "mu"), (s, "s"), (q, "q")):
        _check(t, nm)
    pairs, items = ctypes.c_longlong(), ctypes.c_longlong()
    _rc(lib().dgr_voxelize_count(ctypes.byref(grid), mu.shape[0], _ptr(mu), _ptr(s), _ptr(q),
                                 float(k_trunc), ctypes.byref(pairs), ctypes.byref(items),
                                 ws.ptr, _stream(stream)), "dgr_voxelize_count")
    return int(pairs.value), int(items.value)


def dgr_voxelize(grid: Grid, mu, s, q, rho, k_trunc, vol, ws: Workspace, stream=None):
    for t, nm in ((mu, "mu"), (s, "s"), (q, "q"), (rho, "rho"), (vol, "vol")):
        _check(t, nm)
    _rc(lib().dgr_voxelize(ctypes.byref(grid), mu.shape[0], _ptr(mu), _ptr(s), _ptr(q),
                           _ptr(rho), float(k_trunc), _ptr(vol), ws.ptr, _stream(stream)),
        "dgr_voxelize")


def dgr_voxelize_backward(grid: Grid, mu, s, q, rho, k_trunc, grad_vol, g_mu, g_s, g_q, g_rho,
                          ws: Workspace, stream=None):
    for t, nm in ((mu, "mu"), (s, "s"), (q, "q"), (rho, "rho"), (grad_vol, "grad_vol"),
                  (g_mu, "g_mu"), (g_s, "g_s"), (g_q, "g_q"), (g_rho, "g_rho")):
        _check(t, nm)
    _rc(lib().dgr_voxelize_backward(ctypes.byref(grid), mu.shape[0], _ptr(mu), _ptr(s), _ptr(q),
                                    _ptr(rho), float(k_trunc), _ptr(grad_vol), _ptr(g_mu),
                                    _ptr(g_s), _ptr(g_q), _ptr(g_rho), ws.ptr, _stream(stream)),
        "dgr_voxelize_backward")


# ---------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------
def dgr_project(grid: Grid, geom: Geom, vol, sino, ws: Workspace, stream=None):
    _check(vol, "vol"); _check(sino, "sino")
    _rc(lib().dgr_project(ctypes.byref(grid), ctypes.byref(geom), _ptr(vol), _ptr(sino), ws.ptr,
                          _stream(stream)), "dgr_project")


def dgr_backproject(grid: Grid, geom: Geom, sino, vol, ws: Workspace, stream=None):
    _check(vol, "vol"); _check(sino, "sino")
    _rc(lib().dgr_backproject(ctypes.byref(grid), ctypes.byref(geom), _ptr(sino), _ptr(vol),
                              ws.ptr, _stream(stream)), "dgr_backproject")


def dgr_project_noalloc(grid: Grid, geom: Geom, vol, sino, stream=None):
    """dgr_project without a workspace: scratch in a fixed device array (for
    callers that cannot allocate).  Raises DgrError if the geometry's ray
    tables do not fit NOALLOC_SCRATCH_BYTES."""
    _check(vol, "vol"); _check(sino, "sino")
    _rc(lib().dgr_project_noalloc(ctypes.byref(grid), ctypes.byref(geom), _ptr(vol), _ptr(sino),
                                  _stream(stream)), "dgr_project_noalloc")


def dgr_l1_residual(pred, meas, resid, loss, ws: Workspace, weight=1.0, stream=None):
    """loss = weight mean|pred - meas|, resid = weight sign(pred - meas) / m."""
    for t, nm in ((pred, "pred"), (meas, "meas"), (resid, "resid"), (loss, "loss")):
        _check(t, nm)
    _rc(lib().dgr_l1_residual(_ptr(pred), _ptr(meas), pred.numel(), float(weight), _ptr(resid),
                              _ptr(loss), ws.ptr, _stream(stream)), "dgr_l1_residual")


def dgr_ssim_loss(geom: Geom, pred, meas, grad, loss, ws: Workspace, data_range=1.0, stream=None):
    """loss = 1 - SSIM(pred, meas) over every projection image, grad = dloss/dpred."""
    for t, nm in ((pred, "pred"), (meas, "meas"), (grad, "grad"), (loss, "loss")):
        _check(t, nm)
    _rc(lib().dgr_ssim_loss(ctypes.byref(geom), _ptr(pred), _ptr(meas), float(data_range), _ptr(grad),
                            _ptr(loss), ws.ptr, _stream(stream)), "dgr_ssim_loss")


def dgr_tv_loss(grid: Grid, vol, grad, loss, ws: Workspace, stream=None):
    """loss = anisotropic TV of vol / voxels, grad = dloss/dvol."""
    for t, nm in ((vol, "vol"), (grad, "grad"), (loss, "loss")):
        _check(t, nm)
    _rc(lib().dgr_tv_loss(ctypes.byref(grid), _ptr(vol), _ptr(grad), _ptr(loss), ws.ptr,
                          _stream(stream)), "dgr_tv_loss")


# ---------------------------------------------------------------------------
# optimisation step
# ---------------------------------------------------------------------------
PAPER_WEIGHTS = (0.6, 0.2, 1.0)  # L1, SSIM, TV (paper Sec. 4.3)


def make_problem(grid: Grid, geom: Geom, k_trunc=3.0, lr0=3e-4, lr1=3e-5, n_iters=2000,
                 beta1=0.9, beta2=0.999, eps=1e-8, weights=(1.0, 0.0, 0.0),
                 ssim_range=1.0) -> Problem:
    """weights: (w_l1, w_ssim, w_tv) of the objective; PAPER_WEIGHTS for the
    paper's full loss.  ssim_range: the data range L of the SSIM constants."""
    return Problem(grid, geom, k_trunc, lr0, lr1, n_iters, beta1, beta2, eps,
                   float(weights[0]), float(weights[1]), float(weights[2]), float(ssim_range))


class State:
    """Device tensors of the optimiser state (dgr_params).  With accumulate=True
    every step adds |dL/dmu| per Gaussian to grad_accum (densification).
    capacity >= n reserves room for densification (arrays hold capacity
    Gaussians, the first n in use)."""

    def __init__(self, mu, s, q, rho, accumulate=False, capacity=None):
        n = mu.shape[0]
        cap = max(n, capacity or n)
        dev = mu.device
        self.n = n
        self.cap = cap

        def buf(t, w):
            b = torch.zeros((cap, w) if w > 1 else (cap,), device=dev)
            b[:n] = t
            return b
        self.mu, self.s, self.q = buf(mu, 3), buf(s, 3), buf(q, 4)
        self.rho = buf(rho, 1)
        self.theta = torch.zeros(11 * cap, device=dev)
        self.m = torch.zeros(11 * cap, device=dev)
        self.v = torch.zeros(11 * cap, device=dev)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.grad_accum = torch.zeros(cap, device=dev) if accumulate else None

    def params(self) -> Params:
        """The dgr_params descriptor (the tensors never move; rebuilt when n changes)."""
        c = getattr(self, "_params", None)
        if c is None or c.n != self.n:
            c = Params(self.n, _ptr(self.mu), _ptr(self.s), _ptr(self.q), _ptr(self.rho),
                       _ptr(self.theta), _ptr(self.m), _ptr(self.v), _ptr(self.step),
                       _ptr(self.grad_accum) if self.grad_accum is not None else None)
            self._params = c
        return c

    def view(self):
        """(mu, s, q, rho) of the n Gaussians in use."""
        return self.mu[:self.n], self.s[:self.n], self.q[:self.n], self.rho[:self.n]


def dgr_densify(grid: Grid, cfg: DensifyCfg, iters: int, src: State, normals, dst: State,
                ws: Workspace, stream=None) -> int:
    """Algorithm 2 from src into dst (dst.cap >= cfg.n_max); returns the new n
    (dst.n is updated).  normals: device [src.n, 2, 3] standard normals."""
    if dst.cap < cfg.n_max:
        raise DgrError("dgr_densify: destination capacity below n_max")
    _check(normals, "normals")
    pin, pout = src.params(), dst.params()
    n_out = ctypes.c_int(0)
    _rc(lib().dgr_densify(ctypes.byref(grid), ctypes.byref(cfg), int(iters), ctypes.byref(pin),
                          _ptr(normals), ctypes.byref(pout), ctypes.byref(n_out), ws.ptr, _stream(stream)),
        "dgr_densify")
    dst.n = int(n_out.value)
    return dst.n


def dgr_params_init(prob: Problem, st: State, stream=None):
    p = st.params()
    _rc(lib().dgr_params_init(ctypes.byref(prob), ctypes.byref(p), _stream(stream)),
        "dgr_params_init")


def dgr_adam(prob: Problem, st: State, g_mu, g_s, g_q, g_rho, stream=None):
    """One Adam step of the optimiser state from given parameter gradients."""
    for t, nm in ((g_mu, "g_mu"), (g_s, "g_s"), (g_q, "g_q"), (g_rho, "g_rho")):
        _check(t, nm)
    p = st.params()
    _rc(lib().dgr_adam(ctypes.byref(prob), ctypes.byref(p), _ptr(g_mu), _ptr(g_s), _ptr(g_q),
                       _ptr(g_rho), _stream(stream)), "dgr_adam")


def dgr_step(prob: Problem, st: State, measured, loss_out, ws: Workspace, stream=None):
    _check(measured, "measured"); _check(loss_out, "loss_out")
    p = st.params()
    _rc(lib().dgr_step(ctypes.byref(prob), ctypes.byref(p), _ptr(measured), _ptr(loss_out),
                       ws.ptr, _stream(stream)), "dgr_step")


def dgr_step_timed(prob: Problem, st: State, measured, loss_out, ws: Workspace, events,
                   stream=None):
    """dgr_step recording torch.cuda.Events (already created, i.e. recorded
    once) at the 7 phase boundaries; given 15, also around the main kernels of
    the backprojector, the projector, the voxelizer and its adjoint."""
    _check(measured, "measured"); _check(loss_out, "loss_out")
    if len(events) < DGR_STEP_EVENTS:
        raise DgrError(f"dgr_step_timed needs {DGR_STEP_EVENTS} events")
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    p = st.params()
    _rc(lib().dgr_step_timed(ctypes.byref(prob), ctypes.byref(p), _ptr(measured), _ptr(loss_out),
                             ws.ptr, _stream(stream), arr, len(events)), "dgr_step_timed")


def dgr_launch_count() -> int:
    return int(lib().dgr_launch_count())


DGR_PIPE_EX2, DGR_PIPE_FFMA, DGR_PIPE_FFMA2 = 0, 1, 2
DGR_STATUS_TIMEOUT = 0x80


def dgr_test_bounded_wait(polls: int, status, gave_up, stream=None):
    """One CTA whose bounded mbarrier wait runs out (see include/dgr.h)."""
    _check(status, "status", torch.int32); _check(gave_up, "gave_up", torch.int32)
    _rc(lib().dgr_test_bounded_wait(int(polls), _ptr(status), _ptr(gave_up), _stream(stream)),
        "dgr_test_bounded_wait")


def dgr_l2_rate(kind: int, buf, passes: int, n_blocks: int, sink, stream=None):
    """Launch the L2 bandwidth kernel over the whole of buf (see include/dgr.h)."""
    _check(sink, "sink")
    if not buf.is_cuda or not buf.is_contiguous():
        raise DgrError("dgr_l2_rate: buf must be a contiguous device tensor")
    _rc(lib().dgr_l2_rate(int(kind), buf.numel() * buf.element_size(), int(passes), int(n_blocks),
                          ctypes.c_void_p(buf.data_ptr()), _ptr(sink), _stream(stream)),
        "dgr_l2_rate")


def dgr_pipe_rate(kind: int, iters: int, n_blocks: int, rec, sink, stream=None):
    """Launch the pipe-rate kernel (see include/dgr.h); rec: int64 device
    tensor [4 n_blocks], sink: float32 device tensor [256 n_blocks]."""
    _check(rec, "rec", torch.int64)
    _check(sink, "sink")
    if rec.numel() < 4 * n_blocks or sink.numel() < 256 * n_blocks:
        raise DgrError("dgr_pipe_rate: rec needs 4 n_blocks entries, sink 256 n_blocks")
    _rc(lib().dgr_pipe_rate(kind, iters, n_blocks, ctypes.c_void_p(rec.data_ptr()), _ptr(sink),
                            _stream(stream)), "dgr_pipe_rate")


def dgr_step_batched(probs, states, measured, loss_out, ws: Workspace, stream=None):
    """One optimisation step of every instance: probs [Problem], states
    [State], measured [device tensors], loss_out device tensor [n_inst]."""
    n = len(probs)
    if not (len(states) == n == len(measured)):
        raise DgrError("dgr_step_batched: mismatched instance lists")
    for t in measured:
        _check(t, "measured")
    _check(loss_out, "loss_out")
    P = (Problem * n)(*probs)
    Q = (Params * n)(*[st.params() for st in states])
    M = (ctypes.c_void_p * n)(*[t.data_ptr() for t in measured])
    _rc(lib().dgr_step_batched(n, P, Q, M, _ptr(loss_out), ws.ptr, _stream(stream)),
        "dgr_step_batched")


def make_batch_plan(grids, geoms, ns, pairs, items) -> WsPlan:
    """Workspace plan for dgr_step_batched over these instances."""
    p = WsPlan()
    p.max_n = int(sum(ns))
    p.max_tiles = int(sum(dgr_tile_count(g) for g in grids))
    p.max_pairs = int(sum(pairs))
    p.max_items = int(sum(items))
    p.max_vox = int(sum(g.nx * g.ny * g.nz for g in grids))
    p.max_rays = int(sum(ge.n_views * ge.nu * ge.nv for ge in geoms))
    p.max_views = int(sum(ge.n_views for ge in geoms))
    p.max_nu = int(max(ge.nu for ge in geoms))
    p.max_nv = int(max(ge.nv for ge in geoms))
    p.max_inst = len(grids)
    return p


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------
def dgr_net_param_count() -> int:
    return int(lib().dgr_net_param_count())


def dgr_net_ws_bytes(n: int) -> int:
    b = ctypes.c_size_t()
    _rc(lib().dgr_net_ws_bytes(int(n), ctypes.byref(b)), "dgr_net_ws_bytes")
    return int(b.value)


def dgr_set_conv_engine(engine: int):
    """Convolutions: 2 tcgen05 on TMA-loaded halo blocks with several taps
    per MMA (default), 3 tcgen05 halo blocks with one MMA per tap, 1 tcgen05
    gathered tiles for forward / data gradient, 0 mma.sync."""
    _rc(lib().dgr_set_conv_engine(int(engine)), "dgr_set_conv_engine")


def dgr_net_status(n, ws) -> int:
    """The network's device status word (synchronous read)."""
    v = ctypes.c_int()
    _rc(lib().dgr_net_status(int(n), _ptr(ws), ws.numel() * ws.element_size(), ctypes.byref(v)),
        "dgr_net_status")
    return int(v.value)


def dgr_net_forward(n, params, inp, out, ws, stream=None):
    for t, nm in ((params, "params"), (inp, "input"), (out, "output")):
        _check(t, nm)
    _rc(lib().dgr_net_forward(int(n), _ptr(params), _ptr(inp), _ptr(out), _ptr(ws),
                              ws.numel() * ws.element_size(), _stream(stream)), "dgr_net_forward")


def dgr_net_backward(n, params, inp, grad_out, grad_params, ws, stream=None):
    for t, nm in ((params, "params"), (inp, "input"), (grad_out, "grad_output"),
                  (grad_params, "grad_params")):
        _check(t, nm)
    _rc(lib().dgr_net_backward(int(n), _ptr(params), _ptr(inp), _ptr(grad_out), _ptr(grad_params),
                               _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)),
        "dgr_net_backward")


def dgr_net_loss(n, out, target, w_density, w_scale, grad_out, loss, ws, stream=None):
    for t, nm in ((out, "output"), (target, "target"), (grad_out, "grad_output"), (loss, "loss")):
        _check(t, nm)
    _rc(lib().dgr_net_loss(int(n), _ptr(out), _ptr(target), float(w_density), float(w_scale),
                           _ptr(grad_out), _ptr(loss), _ptr(ws), ws.numel() * ws.element_size(),
                           _stream(stream)), "dgr_net_loss")


def dgr_adam_flat(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    for x, nm in ((params, "params"), (grads, "grads"), (m, "m"), (v, "v")):
        _check(x, nm)
    _rc(lib().dgr_adam_flat(params.numel(), _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(t),
                            float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
        "dgr_adam_flat")


def dgr_fdk_filter(geom: Geom, sino, out, scale=1.0, stream=None):
    _check(sino, "sino"); _check(out, "out")
    _rc(lib().dgr_fdk_filter(ctypes.byref(geom), float(scale), _ptr(sino), _ptr(out),
                             _stream(stream)), "dgr_fdk_filter")


def dgr_proposals(src, channels: int, log_scale_default: float, density, log_scale, stream=None):
    """density = max(src[..., 0], 0); log_scale = src[..., 1] (channels 2) or
    the default (channels 1)."""
    for t, nm in ((src, "src"), (density, "density"), (log_scale, "log_scale")):
        _check(t, nm)
    _rc(lib().dgr_proposals(density.numel(), _ptr(src), int(channels), float(log_scale_default),
                            _ptr(density), _ptr(log_scale), _stream(stream)), "dgr_proposals")


def dgr_logscale_weight(s, rho, h: float, w, stream=None):
    for t, nm in ((s, "s"), (rho, "rho"), (w, "w")):
        _check(t, nm)
    _rc(lib().dgr_logscale_weight(rho.numel(), _ptr(s), _ptr(rho), float(h), _ptr(w),
                                  _stream(stream)), "dgr_logscale_weight")


def dgr_fit_targets(density, wsum, min_density, log_lo, log_hi, log_default, out, stream=None):
    for t, nm in ((density, "density"), (wsum, "wsum"), (out, "out")):
        _check(t, nm)
    _rc(lib().dgr_fit_targets(density.numel(), _ptr(density), _ptr(wsum), float(min_density),
                              float(log_lo), float(log_hi), float(log_default), _ptr(out),
                              _stream(stream)), "dgr_fit_targets")


def dgr_seed(grid: Grid, density, log_scale, u, jitter, mu, s, q, rho, voxel, scratch, stream=None):
    for t, nm in ((density, "density"), (log_scale, "log_scale"), (u, "u"), (jitter, "jitter"),
                  (mu, "mu"), (s, "s"), (q, "q"), (rho, "rho")):
        _check(t, nm)
    _check(voxel, "voxel", torch.int32)
    _rc(lib().dgr_seed(ctypes.byref(grid), _ptr(density), _ptr(log_scale), u.numel(), _ptr(u),
                       _ptr(jitter), _ptr(mu), _ptr(s), _ptr(q), _ptr(rho), _ptr(voxel),
                       _ptr(scratch), scratch.numel() * scratch.element_size(), _stream(stream)),
        "dgr_seed")


def dgr_seed_bytes(n_side: int) -> int:
    b = ctypes.c_size_t()
    _rc(lib().dgr_seed_bytes(int(n_side), ctypes.byref(b)), "dgr_seed_bytes")
    return int(b.value)


def dgr_seed_rescale(voxel, density, vol, rho, stream=None):
    _check(voxel, "voxel", torch.int32)
    for t, nm in ((density, "density"), (vol, "vol"), (rho, "rho")):
        _check(t, nm)
    _rc(lib().dgr_seed_rescale(rho.numel(), _ptr(voxel), _ptr(density), _ptr(vol), _ptr(rho),
                               _stream(stream)), "dgr_seed_rescale")
