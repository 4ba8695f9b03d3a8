"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle with something other than itself: closed forms,
invariants, special cases that reduce to textbook or library routines, brute
force on tiny inputs, and finite differences.  A plausible slip anywhere in
the oracle (dropped term, wrong sign or index, transposed rotation, wrong
voxel-centre convention, wrong cone magnification) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_04844_b300 import synth

LOG2PI = math.log(2 * math.pi)


def grid_of(n, h=1.0, org=None):
    if isinstance(n, int):
        n = (n, n, n)
    if org is None:
        org = tuple(-0.5 * n[a] * h for a in range(3))
    return O.Grid(n, h, org)


def quat_axis_angle(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.array([math.cos(ang / 2), *(math.sin(ang / 2) * axis)], np.float32)


# ---------------------------------------------------------------------------
# voxelizer values
# ---------------------------------------------------------------------------
def test_axis_aligned_is_separable_product():
    """q = identity: the Gaussian factorises, V = rho * prod_a exp(-(i_a-u_a)^2/(2 sig_a^2))
    on the box (Eq. 3 with diagonal Sigma)."""
    g = grid_of((20, 18, 16), h=0.75, org=(-3.0, 1.0, 2.5))
    rng = np.random.default_rng(1)
    mu = np.array([[4.1, 7.3, 8.9]], np.float32)
    s = np.array([[1.3, 0.9, 2.1]], np.float32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    rho = np.array([0.7], np.float32)
    vol = O.voxelize(g, mu, s, q, rho, 3.0)
    _, box = O.footprint(g, mu, s, q, 3.0)
    lo, hi = box[0, :3], box[0, 3:]
    fac = []
    for a in range(3):
        i = np.arange(g.dims[a])
        u = (float(mu[0, a]) - g.org[a]) / g.h - 0.5
        sig = float(s[0, a]) / g.h
        f = np.exp(-(i - u) ** 2 / (2 * sig * sig))
        f[(i < lo[a]) | (i > hi[a])] = 0
        fac.append(f)
    ref = float(rho[0]) * fac[2][:, None, None] * fac[1][None, :, None] * fac[0][None, None, :]
    assert np.max(np.abs(vol - ref)) < 1e-14


def test_isotropic_matches_paper_decomposed_D2():
    """Isotropic Gaussian in the paper's fixed 17^3 box: every voxel value is
    I * exp(-1/2 D^2) with D^2 from the four decomposed sums of Eq. 9
    (cross terms subtracted) over B' = meshgrid(-8..8) anchored at floor(mu)
    (Algorithm 1, Eq. 6-7)."""
    g = grid_of(40)
    mu = np.array([[1.37, -4.61, 3.02]], np.float32)
    sig = float(np.float32(2.2))
    s = np.full((1, 3), sig, np.float32)
    q = np.array([[0.3, -0.5, 0.2, 0.8]], np.float32)  # irrelevant for isotropic
    rho = np.array([1.25], np.float32)
    vol = O.voxelize(g, mu, s, q, rho, -17.0)
    u = (mu[0].astype(np.float64) - np.array(g.org)) / g.h - 0.5
    fl = np.floor(u)
    dmu = u - fl
    b = np.arange(-8, 9, dtype=np.float64)
    Bz, By, Bx = np.meshgrid(b, b, b, indexing="ij")
    B = np.stack([Bx, By, Bz], -1)
    Cinv = 1.0 / sig ** 2
    BCB = (B * Cinv * B).sum(-1)
    BCd = (B * Cinv * dmu).sum(-1)
    dCB = (dmu * Cinv * B).sum(-1)
    dCd = (dmu * Cinv * dmu).sum()
    D2 = BCB - BCd - dCB + dCd
    gam = rho[0] * np.exp(-0.5 * D2)
    z0, y0, x0 = int(fl[2]) - 8, int(fl[1]) - 8, int(fl[0]) - 8
    block = vol[z0:z0 + 17, y0:y0 + 17, x0:x0 + 17]
    assert np.max(np.abs(block - gam)) < 1e-13
    # nothing outside the 17^3 box (confinement, Sec. 4.1)
    assert abs(vol.sum() - block.sum()) < 1e-13
    assert np.count_nonzero(vol) == 17 ** 3


def test_algorithm1_sign_reading():
    """Reading of the sign conflict: Algorithm 1 adds all four terms, Eq. 9
    subtracts the cross terms.  Only Eq. 9 equals the direct D^2 of
    (B' - dmu)^T C^-1 (B' - dmu), so the oracle follows Eq. 9."""
    rng = np.random.default_rng(2)
    B = rng.integers(-8, 9, (100, 3)).astype(float)
    dmu = rng.uniform(0, 1, 3)
    cinv = rng.uniform(0.1, 2.0, 3)
    direct = (((B - dmu) ** 2) * cinv).sum(1)
    eq9 = (B * cinv * B).sum(1) - 2 * (B * cinv * dmu).sum(1) + (dmu * cinv * dmu).sum()
    alg1 = (B * cinv * B).sum(1) + 2 * (B * cinv * dmu).sum(1) + (dmu * cinv * dmu).sum()
    assert np.max(np.abs(direct - eq9)) < 1e-12
    assert np.max(np.abs(direct - alg1)) > 1e-3


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_wide_box_mass_any_rotation(seed):
    """With a wide box the voxel sum of a Gaussian equals its integral
    rho (2 pi)^{3/2} s1 s2 s3 / h^3 (Poisson summation error ~exp(-2 pi^2 sig^2)),
    for any rotation."""
    rng = np.random.default_rng(seed)
    g = grid_of(96, h=0.5)
    mu = rng.uniform(-3, 3, (1, 3)).astype(np.float32)
    s = rng.uniform(1.0, 3.0, (1, 3)).astype(np.float32)  # 2..6 voxels
    q = rng.standard_normal((1, 4)).astype(np.float32)
    rho = np.array([0.8], np.float32)
    vol = O.voxelize(g, mu, s, q, rho, 8.0)
    mass = float(rho[0]) * (2 * math.pi) ** 1.5 * np.prod(s[0].astype(np.float64)) / g.h ** 3
    assert abs(vol.sum() / mass - 1) < 1e-9


def test_default_box_mass_deficit_axis_aligned():
    """3-sigma box on an axis-aligned Gaussian keeps exactly the truncated
    separable sums (the per-axis box, not an ellipsoid)."""
    g = grid_of(64)
    mu = np.array([[0.3, -0.2, 0.45]], np.float32)
    s = np.array([[3.0, 2.5, 4.0]], np.float32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    vol = O.voxelize(g, mu, s, q, np.ones(1, np.float32), 3.0)
    _, box = O.footprint(g, mu, s, q, 3.0)
    tot = 1.0
    for a in range(3):
        i = np.arange(box[0, a], box[0, 3 + a] + 1)
        u = (float(mu[0, a]) - g.org[a]) / g.h - 0.5
        tot *= np.exp(-(i - u) ** 2 / (2 * float(s[0, a]) ** 2)).sum()
    assert abs(vol.sum() - tot) < 1e-12
    full = (2 * math.pi) ** 1.5 * np.prod(s[0].astype(np.float64))
    assert 0.97 < vol.sum() / full < 1.0


def test_moments_pin_rotation_sense_and_centre():
    """A rotation of +30 deg about z (q = (cos 15, 0, 0, sin 15)) turns the long
    axis toward +y: the voxel-weighted covariance equals Rz(30) diag(s^2) Rz(30)^T
    (built from cos/sin, not from a quaternion), and the weighted mean equals mu
    (voxel centres at org + (i + 1/2) h)."""
    g = grid_of(120, h=0.5, org=(-28.0, -33.0, -28.0))
    mu = np.array([[2.3, -3.1, 1.7]], np.float32)
    s = np.array([[3.0, 1.2, 1.6]], np.float32)
    q = quat_axis_angle([0, 0, 1], math.radians(30))[None]
    ang = 2 * math.atan2(float(q[0, 3]), float(q[0, 0]))  # the angle the float32 q encodes
    vol = O.voxelize(g, mu, s, q, np.ones(1, np.float32), 8.0)
    _, box = O.footprint(g, mu, s, q, 8.0)
    assert np.all(box[0, :3] > 0) and np.all(box[0, 3:] < 119)  # no clipping
    nz, ny, nx = vol.shape
    xs = g.org[0] + (np.arange(nx) + 0.5) * g.h
    ys = g.org[1] + (np.arange(ny) + 0.5) * g.h
    zs = g.org[2] + (np.arange(nz) + 0.5) * g.h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    P = np.stack([X, Y, Z], -1).reshape(-1, 3)
    w = vol.reshape(-1)
    keep = w > 0
    P, w = P[keep], w[keep]
    m = (w[:, None] * P).sum(0) / w.sum()
    assert np.max(np.abs(m - mu[0].astype(np.float64))) < 1e-9
    d = P - m
    C = np.einsum("n,ni,nj->ij", w, d, d) / w.sum()
    c, sn = math.cos(ang), math.sin(ang)
    Rz = np.array([[c, -sn, 0], [sn, c, 0], [0, 0, 1]])
    Cref = Rz @ np.diag(s[0].astype(np.float64) ** 2) @ Rz.T
    assert np.max(np.abs(C - Cref)) < 1e-8
    assert C[0, 1] > 0.5  # long axis tilted toward +y


def test_brute_force_equals_footprint_loop():
    g = grid_of((24, 20, 22))
    rng = synth.rng_for(1, 99)
    f = synth.gaussian_field(rng, 60, synth.GridSpec((24, 20, 22), 1.0, g.org), ("loguniform", 0.5, 3.0))
    a = O.voxelize(g, f.mu, f.s, f.q, f.rho, 3.0, brute=True)
    b = O.voxelize(g, f.mu, f.s, f.q, f.rho, 3.0, brute=False)
    assert np.max(np.abs(a - b)) < 1e-13


def test_point_evaluation_equals_full_volume():
    g = grid_of((21, 18, 15))
    rng = synth.rng_for(1, 98)
    f = synth.gaussian_field(rng, 80, synth.GridSpec((21, 18, 15), 1.0, g.org), ("loguniform", 0.5, 3.0))
    vol = O.voxelize(g, f.mu, f.s, f.q, f.rho, 3.0, brute=True)
    pts = np.stack([rng.integers(0, 21, 50), rng.integers(0, 18, 50), rng.integers(0, 15, 50)], 1)
    v = O.voxelize_points(g, f.mu, f.s, f.q, f.rho, pts, 3.0)
    assert np.max(np.abs(v - vol[pts[:, 2], pts[:, 1], pts[:, 0]])) < 1e-14


# ---------------------------------------------------------------------------
# footprint integers
# ---------------------------------------------------------------------------
def test_footprint_box_covers_k_sigma_with_ceiled_radius():
    """k-sigma mode: a = floor(u); the box is [a - R, a + R + 1] with
    R = ceil(k sig_a), sig_a the marginal std sqrt(Sigma_aa) in voxels (FP64
    here, from Sigma = R diag(s^2) R^T), then clipped to the grid; it holds
    the k-sigma interval [u - k sig_a, u + k sig_a]."""
    g = grid_of(48)
    rng = np.random.default_rng(7)
    n = 300
    mu = rng.uniform(-30, 30, (n, 3)).astype(np.float32)
    s = np.exp(rng.uniform(math.log(0.5), math.log(4), (n, 3))).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    anchor, box = O.footprint(g, mu, s, q, 3.0)
    qn = q.astype(np.float64) / np.linalg.norm(q.astype(np.float64), axis=1, keepdims=True)
    bad = checked = 0
    for i in range(n):
        w, x, y, z = qn[i]
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        Sig = R @ np.diag(s[i].astype(np.float64) ** 2) @ R.T
        for a in range(3):
            u = (float(mu[i, a]) - g.org[a]) / g.h - 0.5
            ks = 3 * math.sqrt(Sig[a, a]) / g.h
            # guard band: skip values within 1e-4 of a rounding decision
            if abs(u - round(u)) < 1e-4 or abs(ks - round(ks)) < 1e-4:
                continue
            checked += 1
            an = math.floor(u)
            Rr = math.ceil(ks)
            assert an - Rr <= u - ks and an + Rr + 1 >= u + ks
            lo = max(an - Rr, 0); hi = min(an + Rr + 1, g.dims[a] - 1)
            bad += (anchor[i, a] != an) + (box[i, a] != lo) + (box[i, 3 + a] != hi)
    assert checked > 800 and bad == 0


def test_footprint_fixed_box_mode():
    """k_trunc = -K: the paper's fixed odd box centred on the floored anchor."""
    g = grid_of(40)
    mu = np.array([[0.2, -18.7, 19.4]], np.float32)
    s = np.ones((1, 3), np.float32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    anchor, box = O.footprint(g, mu, s, q, -17.0)
    u = (mu[0].astype(np.float64) - np.array(g.org)) / g.h - 0.5
    a = np.floor(u).astype(int)
    assert list(anchor[0]) == list(a)
    assert list(box[0, :3]) == [max(a[i] - 8, 0) for i in range(3)]
    assert list(box[0, 3:]) == [min(a[i] + 8, 39) for i in range(3)]


# ---------------------------------------------------------------------------
# projector
# ---------------------------------------------------------------------------
def ray_box_length(S, D, lo, hi):
    """Length of the line S + t D inside the axis-aligned box [lo, hi] (slab test)."""
    t0, t1 = -np.inf, np.inf
    for a in range(3):
        if D[a] == 0:
            if not (lo[a] <= S[a] < hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - S[a]) / D[a], (hi[a] - S[a]) / D[a]
        t0 = max(t0, min(ta, tb)); t1 = min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * float(np.linalg.norm(D))


def _geoms():
    par = O.Geom(0, np.array([0.0, 0.3, 1.1, 2.0, math.pi / 2], np.float32), 12, 7, 0.9, 1.1)
    cone = O.Geom(1, np.array([0.0, 0.7, 2.2, 4.0, 5.5], np.float32), 14, 9, 1.3, 1.2, 30.0, 55.0)
    return par, cone


@pytest.mark.parametrize("which", [0, 1])
def test_constant_volume_gives_chord_length(which):
    g = grid_of((9, 7, 5), h=1.1)
    geom = _geoms()[which]
    sino = O.project(g, geom, np.ones(g.shape))
    lo = np.array(g.org); hi = lo + np.array(g.dims) * g.h
    for k in range(geom.n_views):
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                S, D = O.ray(geom, k, iu, iv)
                assert abs(sino[k, iv, iu] - ray_box_length(S, D, lo, hi)) < 1e-11


@pytest.mark.parametrize("which", [0, 1])
def test_chord_matrix_matches_per_voxel_slab_test(which):
    """Each ray's row of the system matrix equals the per-voxel ray/cube
    intersection lengths (dense slab test), built independently of Siddon."""
    g = grid_of((5, 4, 3), h=1.3)
    geom = _geoms()[which]
    geom = O.Geom(geom.beam, geom.angles[:3], 6, 4, geom.pu, geom.pv, geom.dso, geom.dsd)
    nvox = 5 * 4 * 3
    Acols = np.zeros((np.prod(geom.shape), nvox))
    for j in range(nvox):
        e = np.zeros(nvox); e[j] = 1
        Acols[:, j] = O.project(g, geom, e.reshape(g.shape)).reshape(-1)
    r = 0
    for k in range(geom.n_views):
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                S, D = O.ray(geom, k, iu, iv)
                for j in range(nvox):
                    z, rem = divmod(j, 20); y, x = divmod(rem, 5)
                    lo = np.array(g.org) + np.array([x, y, z]) * g.h
                    assert abs(Acols[r, j] - ray_box_length(S, D, lo, lo + g.h)) < 1e-11
                r += 1


@pytest.mark.parametrize("which", [0, 1])
def test_adjoint_identity(which):
    g = grid_of((11, 9, 8), h=0.8)
    geom = _geoms()[which]
    rng = np.random.default_rng(11)
    x = rng.standard_normal(g.shape)
    y = rng.standard_normal(geom.shape)
    lhs = (O.project(g, geom, x) * y).sum()
    rhs = (x * O.backproject(g, geom, y)).sum()
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0) * 10


@pytest.mark.parametrize("arc", [2 * math.pi, math.pi / 2])
def test_fan_beam_slice_chord_lengths(arc):
    """2D fan beam (one detector row through z = 0) over a one-voxel-thick
    slice of ones: every pixel is the 2D chord of its ray through the square,
    computed here from the source/detector positions written out by hand
    (full scan and the 90-degree limited-angle scan)."""
    F = lambda x: float(np.float32(x))  # the geometry is handed over in FP32
    n, h = 10, F(1.2)
    gs = synth.slice_grid(n, h)
    geo = synth.fan_geom(7, 23, F(1.1), 25.0, 41.0, arc)
    g = grid_of((n, n, 1), h=h, org=gs.org)
    sino = O.project(g, O.Geom(geo.beam, geo.angles, geo.nu, geo.nv, geo.pu, geo.pv, geo.dso, geo.dsd),
                     np.ones(g.shape))
    lo = np.array(g.org[:2]); hi = lo + n * g.h  # the FP32 grid as handed over
    for k, th in enumerate(geo.angles.astype(np.float64)):
        c, sn = math.cos(th), math.sin(th)
        src = np.array([-geo.dso * c, -geo.dso * sn])
        for iu in range(geo.nu):
            u = (iu - 0.5 * (geo.nu - 1)) * geo.pu
            det = src + geo.dsd * np.array([c, sn]) + u * np.array([-sn, c])
            d = det - src
            t0, t1 = -np.inf, np.inf
            for a in range(2):
                if d[a] == 0.0:
                    if not (lo[a] <= src[a] < hi[a]):
                        t0, t1 = 1.0, 0.0
                    continue
                ta, tb = (lo[a] - src[a]) / d[a], (hi[a] - src[a]) / d[a]
                t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
            chord = max(0.0, t1 - t0) * float(np.linalg.norm(d))
            assert abs(sino[k, 0, iu] - chord) < 1e-10, (k, iu, sino[k, 0, iu], chord)


def test_axis_aligned_parallel_rays_are_column_sums():
    """theta = 0: rays run along +x at (y, z) = (u, v); each pixel is h times the
    sum of the voxel row it lies in."""
    g = grid_of((8, 6, 4), h=1.0)
    geom = O.Geom(0, np.array([0.0], np.float32), 6, 4, 1.0, 1.0)
    rng = np.random.default_rng(5)
    vol = rng.uniform(0, 1, g.shape)
    sino = O.project(g, geom, vol)
    # u = (iu - 2.5), y index = floor(u + 3); v = iv - 1.5, z index = floor(v + 2)
    for iv in range(4):
        for iu in range(6):
            yi = int(math.floor(iu - 2.5 + 3)); zi = int(math.floor(iv - 1.5 + 2))
            assert abs(sino[0, iv, iu] - vol[zi, yi, :].sum()) < 1e-12


def test_cone_magnification_pins_geometry():
    """A single hot voxel at X projects to u = dsd (X.e_u) / (dso + X.r),
    v = dsd X_z / (dso + X.r): the brightest pixel sits there."""
    g = grid_of(33, h=1.0)
    th = 0.6
    geom = O.Geom(1, np.array([th], np.float32), 101, 81, 0.5, 0.5, 60.0, 100.0)
    vol = np.zeros(g.shape)
    ix, iy, iz = 22, 9, 25
    vol[iz, iy, ix] = 1.0
    X = np.array(g.org) + (np.array([ix, iy, iz]) + 0.5) * g.h
    thf = float(np.float32(th))
    r = np.array([math.cos(thf), math.sin(thf), 0]); eu = np.array([-math.sin(thf), math.cos(thf), 0])
    M = geom.dsd / (geom.dso + X @ r)
    u = M * (X @ eu); v = M * X[2]
    sino = O.project(g, geom, vol)[0]
    iv, iu = np.unravel_index(np.argmax(sino), sino.shape)
    assert abs((iu - 50) * 0.5 - u) <= 0.5
    assert abs((iv - 40) * 0.5 - v) <= 0.5


def test_parallel_projection_of_isotropic_gaussian_is_2d_gaussian():
    """Sanity (not a tight pin): the parallel projection of a voxelised
    isotropic Gaussian approaches rho sqrt(2 pi) sig exp(-r^2 / (2 sig^2)) up to
    the piecewise-constant discretisation error O((h/sig)^2)."""
    g = grid_of(64, h=1.0)
    mu = np.array([[0.4, -1.3, 0.7]], np.float32)
    sig = 5.0
    vol = O.voxelize(g, mu, np.full((1, 3), sig, np.float32), np.array([[1, 0, 0, 0]], np.float32),
                     np.ones(1, np.float32), 6.0)
    th = 0.5
    geom = O.Geom(0, np.array([th], np.float32), 64, 64, 1.0, 1.0)
    sino = O.project(g, geom, vol)[0]
    thf = float(np.float32(th))
    eu = np.array([-math.sin(thf), math.cos(thf)])
    uu = (np.arange(64) - 31.5)
    vv = (np.arange(64) - 31.5)
    du = uu[None, :] - eu @ mu[0, :2].astype(np.float64)
    dv = vv[:, None] - float(mu[0, 2])
    ana = math.sqrt(2 * math.pi) * sig * np.exp(-(du ** 2 + dv ** 2) / (2 * sig * sig))
    assert np.max(np.abs(sino - ana)) / ana.max() < 0.02


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------
def _small_problem(seed=0):
    g = grid_of(16)
    rng = synth.rng_for(3, 500 + seed)
    f = synth.gaussian_field(rng, 16, synth.GridSpec((16, 16, 16), 1.0, g.org), ("lognormal", 1.5, 0.894),
                             unnormalised_q=True)
    f.s = np.clip(f.s, 0.6, 6.0).astype(np.float32)
    _, box = O.footprint(g, f.mu, f.s, f.q, 3.0)
    W = np.random.default_rng(seed).standard_normal(g.shape)
    return g, f, box, W


def test_gradients_match_central_differences():
    g, f, box, W = _small_problem()
    d = lambda a: np.asarray(a, np.float64)
    mu, s, q, rho = d(f.mu), d(f.s), d(f.q), d(f.rho)
    gm, gs, gq, gr = O.voxelize_backward_core(g, mu, s, q, rho, box, W)
    L = lambda *p: (O.voxelize_core(g, *p, box) * W).sum()
    worst = 0.0
    for name, arr, ga in (("mu", mu, gm), ("s", s, gs), ("q", q, gq), ("rho", rho, gr)):
        flat = arr.reshape(-1)
        gflat = ga.reshape(-1)
        scale = np.max(np.abs(gflat))
        for j in range(flat.size):
            eps = 1e-6 * max(1.0, abs(flat[j]))
            p = [mu.copy(), s.copy(), q.copy(), rho.copy()]
            tgt = {"mu": 0, "s": 1, "q": 2, "rho": 3}[name]
            p[tgt].reshape(-1)[j] += eps
            lp = L(*p)
            p[tgt].reshape(-1)[j] -= 2 * eps
            lm = L(*p)
            fd = (lp - lm) / (2 * eps)
            err = abs(fd - gflat[j]) / max(abs(fd), 1e-3 * scale)
            worst = max(worst, err)
    assert worst < 1e-6


def test_rho_adjoint_identity():
    """The volume is linear in rho: <Vox(rho), W> = <rho, dL/drho>."""
    g, f, box, W = _small_problem(1)
    d = lambda a: np.asarray(a, np.float64)
    vol = O.voxelize_core(g, d(f.mu), d(f.s), d(f.q), d(f.rho), box)
    _, _, _, gr = O.voxelize_backward_core(g, d(f.mu), d(f.s), d(f.q), d(f.rho), box, W)
    assert abs((vol * W).sum() - (d(f.rho) * gr).sum()) < 1e-12 * abs((vol * W).sum()) + 1e-13


# ---------------------------------------------------------------------------
# loss and Adam
# ---------------------------------------------------------------------------
def test_l1_gradient_is_sign_over_M():
    rng = np.random.default_rng(8)
    p = rng.standard_normal((3, 4, 5)); m = rng.standard_normal((3, 4, 5))
    loss, r = O.l1_loss(p, m)
    assert abs(loss - np.mean(np.abs(p - m))) < 1e-15
    eps = 1e-7
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 4)]:
        pp = p.copy(); pp[idx] += eps
        lp, _ = O.l1_loss(pp, m)
        pp[idx] -= 2 * eps
        lm, _ = O.l1_loss(pp, m)
        assert abs((lp - lm) / (2 * eps) - r[idx]) < 1e-6
    _, r0 = O.l1_loss(np.zeros(4), np.zeros(4))
    assert np.all(r0 == 0)


def test_adam_matches_torch_optim_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    th = {"a": rng.standard_normal(7)}
    m = {"a": np.zeros(7)}; v = {"a": np.zeros(7)}
    p = torch.nn.Parameter(torch.tensor(th["a"], dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=3e-4, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        gr = rng.standard_normal(7)
        th = O.adam_update(th, {"a": gr}, m, v, t, 3e-4)
        p.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
    assert np.max(np.abs(th["a"] - p.detach().numpy())) < 1e-14


def test_lr_schedule_endpoints_and_transforms():
    assert O.lr_at(1, 3e-4, 3e-5, 2000) == pytest.approx(3e-4, rel=1e-15)
    assert O.lr_at(2000, 3e-4, 3e-5, 2000) == pytest.approx(3e-5, rel=1e-12)
    g = grid_of(32)
    rng = np.random.default_rng(10)
    mu = rng.uniform(-15, 15, (5, 3)); s = rng.uniform(0.5, 4, (5, 3))
    q = rng.standard_normal((5, 4)); rho = rng.uniform(0.01, 1, 5)
    th = O.to_opt(g, mu, s, q, rho)
    assert np.all(np.abs(th["mu"]) <= 1)
    mu2, s2, q2, rho2 = O.from_opt(g, th)
    for a, b in ((mu, mu2), (s, s2), (q, q2), (rho, rho2)):
        assert np.max(np.abs(a - b)) < 1e-12


def _step_fd_problem():
    g = grid_of(16)
    gs = synth.GridSpec((16, 16, 16), 1.0, g.org)
    f = synth.gaussian_field(synth.rng_for(3, 520), 12, gs, ("loguniform", 0.6, 3.0),
                             unnormalised_q=True)
    f.rho = np.clip(f.rho, 0.05, 1.0).astype(np.float32)
    geo = synth.parallel_geom(5, 22, 18, 1.0, 1.0)
    og = O.Geom(geo.beam, geo.angles, geo.nu, geo.nv, geo.pu, geo.pv)
    phantom = synth.ellipsoid_phantom(synth.rng_for(3, 521), gs, 4)
    meas = O.project(g, og, phantom)
    return g, og, f, meas


@pytest.mark.parametrize("weights", [(1.0, 0.0, 0.0), (0.6, 0.2, 1.0)])
def test_step_gradients_in_optimiser_variables_match_central_differences(weights):
    """The gradients oracle.step hands to Adam are d(loss)/d(theta) for the
    optimiser variables theta = ((mu - c)/half, log s, raw q, softplus^-1 rho):
    the chain factors half, s and sigmoid(theta_rho) are checked against FP64
    central differences of the whole objective (Eq. 13 with the given weights,
    box integers fixed) in theta, for every entry."""
    g, og, f, meas = _step_fd_problem()
    d = lambda a: np.asarray(a, np.float64)
    th0 = O.to_opt(g, d(f.mu), d(f.s), d(f.q), d(f.rho))

    def loss_grads(th):
        m = {k: np.zeros_like(a) for k, a in th.items()}
        v = {k: np.zeros_like(a) for k, a in th.items()}
        lo, _, gr = O.step(g, og, f.mu, f.s, f.q, f.rho, th, m, v, 1, meas, 3.0, 3e-4, 3e-5, 10,
                           weights=weights)
        return lo, gr

    # no L1 residual that a Gaussian reaches may sit near its kink (rays no
    # box meets stay at exactly 0 under every perturbation; where the
    # measurement is 0 a positive prediction stays positive)
    mu0, s0, q0, r0 = O.from_opt(g, th0)
    _, box = O.footprint(g, f.mu, f.s, f.q, 3.0)
    pred = O.project(g, og, O.voxelize_core(g, mu0, s0, q0, r0, box))
    assert np.min(np.abs(pred - meas)[(pred > 0) & (meas > 0)]) > 1e-4
    _, grads = loss_grads(th0)
    for k in ("mu", "s", "q", "rho"):
        ga = grads[k].reshape(-1)
        scale = np.max(np.abs(ga))
        assert scale > 0
        worst = 0.0
        for j in range(ga.size):
            th = {kk: a.copy() for kk, a in th0.items()}
            # step near the cube root of FP64 epsilon (central differences)
            eps = 1e-5 * max(1.0, abs(th[k].reshape(-1)[j]))
            th[k].reshape(-1)[j] += eps
            lp, _ = loss_grads(th)
            th[k].reshape(-1)[j] -= 2 * eps
            lm, _ = loss_grads(th)
            fd = (lp - lm) / (2 * eps)
            worst = max(worst, abs(fd - ga[j]) / max(abs(fd), 1e-3 * scale))
        assert worst < 1e-6, (k, worst)


# ---------------------------------------------------------------------------
# full objective: SSIM (projection domain) and TV (volume), Sec. 4.3 / App. D.1
# ---------------------------------------------------------------------------
def test_ssim_window_is_the_normalised_gaussian():
    g = O.gaussian_window()
    ref = np.array([math.exp(-(i - 5) ** 2 / (2 * 1.5 ** 2)) for i in range(11)])
    assert np.allclose(g, ref / ref.sum(), rtol=0, atol=1e-15)


def test_ssim_of_an_image_with_itself_is_one():
    x = np.random.default_rng(1).uniform(0, 3, (2, 17, 23))
    loss, grad = O.ssim_loss(x, x)
    assert abs(loss) < 1e-14
    assert np.abs(grad).max() < 1e-14


def test_ssim_pixel_by_brute_force_window():
    """One interior pixel's SSIM from an explicit 11 x 11 weighted sum
    (exp(-(i^2 + j^2) / (2 sigma^2)) normalised), independent of the
    separable correlation used by the oracle."""
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 2, (1, 21, 25)); y = rng.uniform(0, 2, (1, 21, 25))
    L = 2.0
    smap, _ = O.ssim_terms(x, y, L)
    for (r, c) in [(10, 12), (7, 6), (13, 18)]:
        w = np.array([[math.exp(-(i * i + j * j) / 4.5) for j in range(-5, 6)] for i in range(-5, 6)])
        w /= w.sum()
        px = x[0, r - 5:r + 6, c - 5:c + 6]; py = y[0, r - 5:r + 6, c - 5:c + 6]
        mx, my = (w * px).sum(), (w * py).sum()
        vx, vy = (w * px * px).sum() - mx * mx, (w * py * py).sum() - my * my
        cxy = (w * px * py).sum() - mx * my
        c1, c2 = (0.01 * L) ** 2, (0.03 * L) ** 2
        s = (2 * mx * my + c1) * (2 * cxy + c2) / ((mx * mx + my * my + c1) * (vx + vy + c2))
        assert abs(smap[0, r, c] - s) < 1e-12


def test_ssim_constant_images_closed_form():
    """Away from the border (full window), constant images a and b give
    (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 1.3
    x = np.full((1, 24, 24), a); y = np.full((1, 24, 24), b)
    smap, _ = O.ssim_terms(x, y, 1.0)
    c1 = 1e-4
    assert abs(smap[0, 12, 12] - (2 * a * b + c1) / (a * a + b * b + c1)) < 1e-12


def test_ssim_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (2, 9, 13)); y = rng.uniform(0, 1, (2, 9, 13))
    _, grad = O.ssim_loss(x, y)
    eps = 1e-6
    for idx in [(0, 0, 0), (0, 4, 6), (1, 8, 12), (1, 3, 1), (0, 7, 10)]:
        xp = x.copy(); xp[idx] += eps
        xm = x.copy(); xm[idx] -= eps
        fd = (O.ssim_loss(xp, y)[0] - O.ssim_loss(xm, y)[0]) / (2 * eps)
        assert abs(fd - grad[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (idx, fd, grad[idx])


def test_tv_ramp_closed_form_and_bump():
    nz, ny, nx = 4, 5, 6
    z, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    a, b = 0.3, -0.7
    v = a * xx + b * yy
    t, _ = O.tv_loss(v)
    N = nx * ny * nz
    assert abs(t - ((nx - 1) * ny * nz * abs(a) + nx * (ny - 1) * nz * abs(b)) / N) < 1e-13
    bump = np.zeros((nz, ny, nx)); bump[2, 2, 3] = 0.5
    t, g = O.tv_loss(bump)
    assert abs(t - 6 * 0.5 / N) < 1e-15
    assert abs(g[2, 2, 3] - 6 / N) < 1e-15
    assert abs(g[2, 2, 2] + 1 / N) < 1e-15 and abs(g[1, 2, 3] + 1 / N) < 1e-15


def test_tv_gradient_matches_central_differences():
    v = np.random.default_rng(4).standard_normal((3, 4, 5))
    _, g = O.tv_loss(v)
    eps = 1e-7
    for idx in [(0, 0, 0), (1, 2, 3), (2, 3, 4), (1, 0, 2)]:
        vp = v.copy(); vp[idx] += eps
        vm = v.copy(); vm[idx] -= eps
        fd = (O.tv_loss(vp)[0] - O.tv_loss(vm)[0]) / (2 * eps)
        assert abs(fd - g[idx]) < 1e-8
