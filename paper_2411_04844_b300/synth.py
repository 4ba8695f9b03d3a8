"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and describes grids/geometries; it holds
none of the method's arithmetic (no Gaussian evaluation, no projection), so
both the CUDA path and the oracle may use it.

The paper evaluates on FIPS, AAPM-Mayo LDCT and FUMPE (Sec. 5.1); those
datasets are not available, so seeded ellipsoid phantoms and random Gaussian
fields of the same sizes stand in for them: 64^3..512^3 volumes, 25-100
cone-beam views, 150K-class Gaussian counts (Sec. 5.1 "Implementation
Details": 150K Gaussians initialised).

Seed recipe: numpy PCG64 seeded with 20241107 + 1000 * config + instance.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PARALLEL = 0
CONE = 1


def seed_for(config: int, instance: int = 0) -> int:
    return 20241107 + 1000 * int(config) + int(instance)


def rng_for(config: int, instance: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, instance)))


@dataclass
class GridSpec:
    """dims = (nx, ny, nz); voxel size h; org = min corner.  Volumes are
    [nz][ny][nx], x fastest; voxel i has centre org + (i + 1/2) h."""
    dims: tuple
    h: float
    org: tuple

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    @property
    def extent(self):
        return tuple(self.dims[a] * self.h for a in range(3))

    @staticmethod
    def centred(n, h=1.0):
        if isinstance(n, int):
            n = (n, n, n)
        return GridSpec(tuple(int(x) for x in n), float(h),
                        tuple(-0.5 * n[a] * h for a in range(3)))


@dataclass
class GeomSpec:
    """beam PARALLEL or CONE; angles [n_views] radians (float32); detector
    nu x nv pixels of pitch (pu, pv) in world units; cone: source-origin and
    source-detector distances dso, dsd."""
    beam: int
    angles: np.ndarray
    nu: int
    nv: int
    pu: float
    pv: float
    dso: float = 0.0
    dsd: float = 0.0

    @property
    def n_views(self):
        return int(len(self.angles))

    @property
    def shape(self):
        return (self.n_views, self.nv, self.nu)


def parallel_geom(n_views, nu, nv, pu=1.0, pv=1.0, arc=math.pi):
    ang = (np.arange(n_views, dtype=np.float64) * (arc / n_views)).astype(np.float32)
    return GeomSpec(PARALLEL, ang, nu, nv, pu, pv)


def cone_geom(n_views, nu, nv, pu, pv, dso, dsd, arc=2 * math.pi):
    ang = (np.arange(n_views, dtype=np.float64) * (arc / n_views)).astype(np.float32)
    return GeomSpec(CONE, ang, nu, nv, pu, pv, dso, dsd)


def fan_geom(n_views, nu, pu, dso, dsd, arc=2 * math.pi):
    """2D fan beam: a cone beam with one detector row through z = 0, for a
    volume one voxel thick centred on that plane.  A limited-angle scan is
    the same with arc < pi (the paper's 90 degree case: arc = pi / 2)."""
    return cone_geom(n_views, nu, 1, pu, 1.0, dso, dsd, arc)


def slice_grid(n, h=1.0):
    """n x n x 1 voxels centred on the origin (z = 0 in the middle of the slice)."""
    return GridSpec((n, n, 1), h, (-0.5 * n * h, -0.5 * n * h, -0.5 * h))


# ---------------------------------------------------------------------------
# Gaussian fields
# ---------------------------------------------------------------------------
def random_quaternions(rng, n):
    """Uniform random rotations: normalised N(0, I_4) draws, (w, x, y, z)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


@dataclass
class Field:
    mu: np.ndarray   # [n,3] float32, world units
    s: np.ndarray    # [n,3] float32, world units
    q: np.ndarray    # [n,4] float32, (w,x,y,z), not necessarily normalised
    rho: np.ndarray  # [n]   float32

    @property
    def n(self):
        return int(self.mu.shape[0])


def gaussian_field(rng, n, grid: GridSpec, scale=("loguniform", 0.5, 3.0), rho=(0.0, 1.0),
                   unnormalised_q=False, isotropic=False):
    """n Gaussians: centres uniform in the volume, uniform random rotations,
    rho ~ U[rho], per-axis scales (in voxels, times h) from
    ("loguniform", lo, hi) or ("lognormal", median, sigma_log); isotropic:
    one scale per Gaussian for all three axes (the paper's representation)."""
    lo = np.array(grid.org)
    hi = lo + np.array(grid.extent)
    mu = rng.uniform(lo, hi, (n, 3))
    if scale[0] == "loguniform":
        s = log_uniform(rng, scale[1], scale[2], (n, 3))
    elif scale[0] == "lognormal":
        s = np.exp(rng.normal(math.log(scale[1]), scale[2], (n, 3)))
    elif scale[0] == "fixed":
        s = np.full((n, 3), float(scale[1]))
    else:
        raise ValueError(scale)
    if isotropic:
        s = np.repeat(s[:, :1], 3, axis=1)
    s = s * grid.h
    q = random_quaternions(rng, n)
    if unnormalised_q:
        q = q * rng.uniform(0.5, 2.0, (n, 1)).astype(np.float32)
    r = rng.uniform(rho[0], rho[1], n)
    return Field(mu.astype(np.float32), s.astype(np.float32), q.astype(np.float32),
                 r.astype(np.float32))


# ---------------------------------------------------------------------------
# ellipsoid phantoms
# ---------------------------------------------------------------------------
def _rot(qn):
    w, x, y, z = qn
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def ellipsoid_phantom(rng, grid: GridSpec, m: int):
    """m random ellipsoids rasterised at voxel centres: centres uniform in a
    ball of radius 0.6 x half-extent, semi-axes U[0.05, 0.35] x extent,
    uniform random rotation, density U[0,1]; values added, then clipped to
    [0, 1].  Returns float32 [nz][ny][nx]."""
    nx, ny, nz = grid.dims
    ext = np.array(grid.extent)
    org = np.array(grid.org)
    centre = org + 0.5 * ext
    vol = np.zeros(grid.shape, np.float32)
    for _ in range(m):
        while True:
            p = rng.uniform(-1, 1, 3)
            if p @ p <= 1:
                break
        c = centre + 0.6 * 0.5 * ext * p
        ax = rng.uniform(0.05, 0.35, 3) * ext
        qn = random_quaternions(rng, 1)[0].astype(np.float64)
        R = _rot(qn)
        dens = rng.uniform(0, 1)
        # bounding box of the ellipsoid: half-widths sqrt(sum_k (R_ak ax_k)^2)
        hw = np.sqrt(((R * ax[None, :]) ** 2).sum(1))
        lo = np.maximum(np.floor((c - hw - org) / grid.h - 0.5).astype(int), 0)
        hi = np.minimum(np.ceil((c + hw - org) / grid.h - 0.5).astype(int), [nx - 1, ny - 1, nz - 1])
        if np.any(hi < lo):
            continue
        xs = org[0] + (np.arange(lo[0], hi[0] + 1) + 0.5) * grid.h - c[0]
        ys = org[1] + (np.arange(lo[1], hi[1] + 1) + 0.5) * grid.h - c[1]
        zs = org[2] + (np.arange(lo[2], hi[2] + 1) + 0.5) * grid.h - c[2]
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        P = np.stack([X, Y, Z], -1) @ R  # body-frame coordinates (R^T p)
        inside = ((P / ax) ** 2).sum(-1) <= 1.0
        vol[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += dens * inside
    np.clip(vol, 0.0, 1.0, out=vol)
    return vol


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    grid: GridSpec
    geom: GeomSpec
    n_gauss: int
    scale: tuple
    phantom_m: int
    noise_sigma: float = 0.0
    k_trunc: float = 3.0
    n_iters: int = 1


def workload(config: int) -> Workload:
    """Synthetic workloads numbered 1..3 (sizes of the paper's Sec. 5 settings):
    1: 2,000 Gaussians, 64^3, parallel 32 views; 2: 50,000 Gaussians, 256^3,
    cone 50 views; 3: 500,000 Gaussians, 512^3, cone 75 views."""
    if config == 1:
        g = GridSpec.centred(64, 1.0)
        return Workload("parallel64_2k", g, parallel_geom(32, 64, 64, 1.0, 1.0), 2000,
                        ("loguniform", 0.5, 3.0), 10)
    if config == 2:
        g = GridSpec.centred(256, 1.0)
        return Workload("cone256_50k", g, cone_geom(50, 256, 256, 1.5, 1.5, 1000.0, 1500.0),
                        50000, ("loguniform", 0.5, 6.0), 40, noise_sigma=0.01, n_iters=2000)
    if config == 3:
        g = GridSpec.centred(512, 1.0)
        return Workload("cone512_500k", g, cone_geom(75, 512, 512, 1.5, 1.5, 1000.0, 1500.0),
                        500000, ("lognormal", 1.5, 0.894), 40)
    raise ValueError(config)


@dataclass
class Instance:
    grid: GridSpec
    geom: GeomSpec
    field: Field
    phantom_m: int = 40
    noise_sigma: float = 0.01


def batched_workload(n_inst: int = 16, config: int = 4, sizes=(64, 128, 192, 256),
                     n_range=(5000, 200000), views_range=(25, 100), scale=("loguniform", 0.5, 6.0)):
    """Independent reconstructions of uneven size: grid side drawn from `sizes`
    (h = 1 mm, centred), Gaussian count log-uniform in n_range, cone beam with
    views uniform in views_range over 360 deg, an N x N detector of pitch 1.5 h
    (source-origin 1000 mm, source-detector 1500 mm)."""
    out = []
    for i in range(n_inst):
        rng = rng_for(config, i)
        N = int(rng.choice(sizes))
        n = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        views = int(rng.integers(views_range[0], views_range[1] + 1))
        grid = GridSpec.centred(N, 1.0)
        geom = cone_geom(views, N, N, 1.5, 1.5, 1000.0, 1500.0)
        f = gaussian_field(rng, n, grid, scale)
        f.rho = np.clip(f.rho, 0.02, 1.0).astype(np.float32)
        out.append(Instance(grid, geom, f))
    return out


def ellipsoid_phantom_torch(rng, grid: GridSpec, m: int, device="cuda"):
    """ellipsoid_phantom with the same random draws, rasterised with torch on
    the device (for large training sets).  Returns a float32 tensor."""
    import torch
    nx, ny, nz = grid.dims
    ext = np.array(grid.extent)
    org = np.array(grid.org)
    centre = org + 0.5 * ext
    vol = torch.zeros(grid.shape, dtype=torch.float32, device=device)
    for _ in range(m):
        while True:
            p = rng.uniform(-1, 1, 3)
            if p @ p <= 1:
                break
        c = centre + 0.6 * 0.5 * ext * p
        ax = rng.uniform(0.05, 0.35, 3) * ext
        qn = random_quaternions(rng, 1)[0].astype(np.float64)
        R = _rot(qn)
        dens = rng.uniform(0, 1)
        hw = np.sqrt(((R * ax[None, :]) ** 2).sum(1))
        lo = np.maximum(np.floor((c - hw - org) / grid.h - 0.5).astype(int), 0)
        hi = np.minimum(np.ceil((c + hw - org) / grid.h - 0.5).astype(int), [nx - 1, ny - 1, nz - 1])
        if np.any(hi < lo):
            continue
        ar = lambda a: torch.arange(lo[a], hi[a] + 1, device=device, dtype=torch.float64)
        xs = org[0] + (ar(0) + 0.5) * grid.h - c[0]
        ys = org[1] + (ar(1) + 0.5) * grid.h - c[1]
        zs = org[2] + (ar(2) + 0.5) * grid.h - c[2]
        Z, Y, X = torch.meshgrid(zs, ys, xs, indexing="ij")
        P = torch.stack([X, Y, Z], -1) @ torch.as_tensor(R, device=device)
        inside = ((P / torch.as_tensor(ax, device=device)) ** 2).sum(-1) <= 1.0
        vol[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += float(dens) * inside.float()
    return vol.clamp_(0.0, 1.0)


def learned_workload(side=128, views=50):
    """Warm-start study: side^3 grid (h = 1 mm, centred), cone beam with `views`
    views over 360 deg, side x side detector of pitch 1.5 mm (source-origin 1000 mm,
    source-detector 1500 mm), 40-ellipsoid phantoms, N(0, 0.01^2) noise."""
    grid = GridSpec.centred(side, 1.0)
    geom = cone_geom(views, side, side, 1.5, 1.5, 1000.0, 1500.0)
    return grid, geom
