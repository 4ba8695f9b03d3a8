// X-ray projector T (a4) and its exact adjoint (a6) on sm_103a.
//
// Ray model (paper Sec. 4.3, P_hat = T(V)): the line integral of the
// piecewise-constant voxel image, i.e. the sum over voxels of (length of the
// ray inside the voxel cube) x value -- Siddon's radiological path.
//
// Both kernels parameterise a ray as X(t) = X0 + t D, with X0 the point of its
// (x, y) projection closest to the grid axis (keeps t small and precise), and
// work in voxel coordinates xi = (X - o)/h.  A plane xi_a = p is crossed at
// t = (p - xi0_a) * inv_e_a.  The forward walks the crossings in order; the
// adjoint, for a voxel, intersects the three slab intervals built from the SAME
// plane crossings, so each chord length is the same FP32 value in both.
//
//   k_ray_tables  per (view, iu): X0, D (FP64 arithmetic, stored FP32)
//   k_project     one thread per ray, incremental plane walk; u-adjacent
//                 rays in a warp read neighbouring voxels
//   k_backproject one thread per (x, y) column and a chunk of z: for each view
//                 it finds the few rays whose pixel footprint can meet the
//                 voxel and gathers length x residual -- no atomics
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr int BP_ZC = 16;        // voxels per backprojector thread along z
constexpr float CAND_EPS = 1e-3f;  // pixel margin of the candidate-ray search

// For an axis the ray runs parallel to, only floor(xi) matters (which voxel
// layer holds the ray).  That decision is taken in FP64 and stored as the
// layer's centre, so a ray lying exactly in a voxel face plane is assigned
// the same way as by an FP64 evaluation of floor((X - o) / h).
__device__ __forceinline__ float snap_layer(double xi) { return (float)(floor(xi) + 0.5); }

__global__ void k_ray_tables(dgr_grid g, dgr_geom geo, RayXY *__restrict__ tab,
                             float2 *__restrict__ view_cs, float *__restrict__ zsnap) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < geo.nv) {
        // z layer of the rays of detector row idx when they run parallel to
        // the z planes (parallel beam, or the cone's v = 0 row)
        const double v = ((double)idx - 0.5 * (double)(geo.nv - 1)) * (double)geo.pv;
        const double X0z = geo.beam == DGR_CONE ? 0.0 : v;
        zsnap[idx] = snap_layer((X0z - (double)g.oz) / (double)g.h);
    }
    if (idx >= geo.n_views * geo.nu) return;
    const int k = idx / geo.nu, iu = idx % geo.nu;
    const double a = (double)geo.angles[k];
    const double c = cos(a), s = sin(a);
    if (iu == 0) view_cs[k] = make_float2((float)c, (float)s);
    const double u = ((double)iu - 0.5 * (double)(geo.nu - 1)) * (double)geo.pu;
    const double h = (double)g.h;
    const double gcx = (double)g.ox + 0.5 * g.nx * h, gcy = (double)g.oy + 0.5 * g.ny * h;
    double Sx, Sy, Dx, Dy;
    if (geo.beam == DGR_CONE) {
        Sx = -(double)geo.dso * c; Sy = -(double)geo.dso * s;
        Dx = (double)geo.dsd * c - u * s; Dy = (double)geo.dsd * s + u * c;
    } else {
        Sx = -u * s; Sy = u * c;
        Dx = c; Dy = s;
    }
    const double d2 = Dx * Dx + Dy * Dy;
    const double tc = ((gcx - Sx) * Dx + (gcy - Sy) * Dy) / d2;
    const double X0x = Sx + tc * Dx, X0y = Sy + tc * Dy;
    RayXY r;
    r.ex = (float)(Dx / h);
    r.ey = (float)(Dy / h);
    r.xi0x = r.ex != 0.f ? (float)((X0x - (double)g.ox) / h) : snap_layer((X0x - (double)g.ox) / h);
    r.xi0y = r.ey != 0.f ? (float)((X0y - (double)g.oy) / h) : snap_layer((X0y - (double)g.oy) / h);
    r.inv_ex = r.ex != 0.f ? (float)(h / Dx) : 0.f;
    r.inv_ey = r.ey != 0.f ? (float)(h / Dy) : 0.f;
    r.tc = (float)tc;
    r.dxy2 = (float)d2;
    tab[idx] = r;
}

struct RayZ {
    float xi0z, ez, inv_ez, dn;
};

// z part of ray (iu, iv); identical FP32 sequence in both kernels.
__device__ __forceinline__ RayZ ray_z(const RayXY &r, const dgr_grid &g, const dgr_geom &geo,
                                      const float *__restrict__ zsnap, int iv) {
    RayZ z;
    const float v = ((float)iv - 0.5f * (float)(geo.nv - 1)) * geo.pv;
    if (geo.beam == DGR_CONE && v != 0.f) {
        z.ez = v / g.h;
        z.dn = sqrtf(r.dxy2 + v * v);
        z.xi0z = (r.tc * v - g.oz) / g.h;
        z.inv_ez = 1.0f / z.ez;
    } else {
        z.ez = 0.f;
        z.dn = sqrtf(geo.beam == DGR_CONE ? r.dxy2 + v * v : r.dxy2);
        z.xi0z = zsnap[iv];
        z.inv_ez = 0.f;
    }
    return z;
}

__device__ __forceinline__ float plane_t(int p, float xi0, float inv) {
    return ((float)p - xi0) * inv;
}

__global__ void __launch_bounds__(128) k_project(dgr_grid g, dgr_geom geo,
                                                 const RayXY *__restrict__ tab,
                                                 const float *__restrict__ zsnap,
                                                 const float *__restrict__ vol,
                                                 float *__restrict__ sino) {
    const long long nrays = (long long)geo.n_views * geo.nv * geo.nu;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrays) return;
    const int iu = (int)(r % geo.nu);
    const int iv = (int)((r / geo.nu) % geo.nv);
    const int k = (int)(r / ((long long)geo.nu * geo.nv));
    const RayXY R = tab[k * geo.nu + iu];
    const RayZ Z = ray_z(R, g, geo, zsnap, iv);
    const float xi0[3] = {R.xi0x, R.xi0y, Z.xi0z};
    const float ev[3] = {R.ex, R.ey, Z.ez};
    const float inv[3] = {R.inv_ex, R.inv_ey, Z.inv_ez};
    const int N[3] = {g.nx, g.ny, g.nz};
    float tmin = -INFINITY, tmax = INFINITY;
    int idx3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ev[a] != 0.f) {
            const float t0 = plane_t(0, xi0[a], inv[a]);
            const float t1 = plane_t(N[a], xi0[a], inv[a]);
            tmin = fmaxf(tmin, fminf(t0, t1));
            tmax = fminf(tmax, fmaxf(t0, t1));
        } else {
            const float f = floorf(xi0[a]);
            if (!(f >= 0.f && f < (float)N[a])) { sino[r] = 0.f; return; }
            idx3[a] = (int)f;
        }
    }
    if (!(tmax > tmin)) { sino[r] = 0.f; return; }
    // entry voxel, made consistent with the plane crossings
    int sgn[3];
    float tn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (ev[a] != 0.f) {
            const int d = ev[a] > 0.f ? 1 : -1;
            sgn[a] = d;
            int i = (int)floorf(fmaf(tmin, ev[a], xi0[a]));
            i = min(max(i, 0), N[a] - 1);
            // upper plane (in the travel direction) must lie after tmin,
            // lower plane at or before it
            for (int it = 0; it < 3; ++it) {
                const float tu = plane_t(d > 0 ? i + 1 : i, xi0[a], inv[a]);
                if (tu <= tmin && i + d >= 0 && i + d < N[a]) i += d; else break;
            }
            for (int it = 0; it < 3; ++it) {
                const float tl = plane_t(d > 0 ? i : i + 1, xi0[a], inv[a]);
                if (tl > tmin && i - d >= 0 && i - d < N[a]) i -= d; else break;
            }
            idx3[a] = i;
            tn[a] = plane_t(d > 0 ? i + 1 : i, xi0[a], inv[a]);
        } else {
            sgn[a] = 0;
            tn[a] = INFINITY;
        }
    }
    const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
    long long idx = idx3[2] * sz + idx3[1] * sy + idx3[0];
    int ix = idx3[0], iy = idx3[1], iz = idx3[2];
    float t = tmin, acc = 0.f;
    const int maxit = g.nx + g.ny + g.nz + 3;
    for (int it = 0; it < maxit; ++it) {
        const float tnext = fminf(tn[0], fminf(tn[1], tn[2]));
        acc = fmaf(tnext - t, __ldg(vol + idx), acc);
        t = tnext;
        if (tnext == tn[0]) {
            ix += sgn[0];
            if (ix < 0 || ix >= g.nx) break;
            idx += sgn[0] * sx;
            tn[0] = plane_t(sgn[0] > 0 ? ix + 1 : ix, xi0[0], inv[0]);
        } else if (tnext == tn[1]) {
            iy += sgn[1];
            if (iy < 0 || iy >= g.ny) break;
            idx += sgn[1] * sy;
            tn[1] = plane_t(sgn[1] > 0 ? iy + 1 : iy, xi0[1], inv[1]);
        } else {
            iz += sgn[2];
            if (iz < 0 || iz >= g.nz) break;
            idx += sgn[2] * sz;
            tn[2] = plane_t(sgn[2] > 0 ? iz + 1 : iz, xi0[2], inv[2]);
        }
    }
    sino[r] = acc * Z.dn;
}

// slab interval of voxel index i along one axis; false if empty
__device__ __forceinline__ bool slab(int i, float xi0, float e, float inv, float &lo, float &hi) {
    if (e != 0.f) {
        const float ta = plane_t(i, xi0, inv), tb = plane_t(i + 1, xi0, inv);
        lo = fminf(ta, tb);
        hi = fmaxf(ta, tb);
        return true;
    }
    lo = -INFINITY;
    hi = INFINITY;
    return floorf(xi0) == (float)i;
}

__global__ void __launch_bounds__(128) k_backproject(dgr_grid g, dgr_geom geo,
                                                     const RayXY *__restrict__ tab,
                                                     const float2 *__restrict__ view_cs,
                                                     const float *__restrict__ zsnap,
                                                     const float *__restrict__ sino,
                                                     float *__restrict__ vol) {
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iy = blockIdx.y * 4 + (threadIdx.x >> 5);
    const int z0 = blockIdx.z * BP_ZC;
    if (ix >= g.nx || iy >= g.ny) return;
    float acc[BP_ZC];
#pragma unroll
    for (int k = 0; k < BP_ZC; ++k) acc[k] = 0.f;
    const float h = g.h;
    const float xl = g.ox + ix * h, xh = xl + h, yl = g.oy + iy * h, yh = yl + h;
    const float cu = 0.5f * (float)(geo.nu - 1), cv = 0.5f * (float)(geo.nv - 1);
    const bool cone = geo.beam == DGR_CONE;
    for (int k = 0; k < geo.n_views; ++k) {
        const float2 cs = view_cs[k];
        // pixel-u range of the column's 4 (x, y) corners, magnification range
        float umin = INFINITY, umax = -INFINITY, mmin = INFINITY, mmax = -INFINITY;
#pragma unroll
        for (int cnr = 0; cnr < 4; ++cnr) {
            const float X = (cnr & 1) ? xh : xl, Y = (cnr & 2) ? yh : yl;
            const float pu_ = -X * cs.y + Y * cs.x;
            const float pr = X * cs.x + Y * cs.y;
            const float M = cone ? geo.dsd / (geo.dso + pr) : 1.f;
            const float uu = M * pu_ / geo.pu + cu;
            umin = fminf(umin, uu); umax = fmaxf(umax, uu);
            mmin = fminf(mmin, M); mmax = fmaxf(mmax, M);
        }
        const int iu0 = max(0, (int)ceilf(umin - CAND_EPS));
        const int iu1 = min(geo.nu - 1, (int)floorf(umax + CAND_EPS));
        for (int iu = iu0; iu <= iu1; ++iu) {
            const RayXY R = tab[k * geo.nu + iu];
            float xlo, xhi, ylo, yhi;
            if (!slab(ix, R.xi0x, R.ex, R.inv_ex, xlo, xhi)) continue;
            if (!slab(iy, R.xi0y, R.ey, R.inv_ey, ylo, yhi)) continue;
            const float tlo = fmaxf(xlo, ylo), thi = fminf(xhi, yhi);
            if (!(thi > tlo)) continue;
            const float *srow = sino + (size_t)k * geo.nv * geo.nu + iu;
#pragma unroll
            for (int zz = 0; zz < BP_ZC; ++zz) {
                const int iz = z0 + zz;
                if (iz >= g.nz) break;
                const float zl = g.oz + iz * h, zh = zl + h;
                float v0, v1;
                if (cone) {
                    v0 = fminf(zl * mmin, zl * mmax);
                    v1 = fmaxf(zh * mmin, zh * mmax);
                } else {
                    v0 = zl; v1 = zh;
                }
                const int iv0 = max(0, (int)ceilf(v0 / geo.pv + cv - CAND_EPS));
                const int iv1 = min(geo.nv - 1, (int)floorf(v1 / geo.pv + cv + CAND_EPS));
                float a = acc[zz];
                for (int iv = iv0; iv <= iv1; ++iv) {
                    const RayZ Z = ray_z(R, g, geo, zsnap, iv);
                    float zlo, zhi;
                    if (!slab(iz, Z.xi0z, Z.ez, Z.inv_ez, zlo, zhi)) continue;
                    const float len = fminf(thi, zhi) - fmaxf(tlo, zlo);
                    if (len > 0.f) a = fmaf(len * Z.dn, __ldg(srow + (size_t)iv * geo.nu), a);
                }
                acc[zz] = a;
            }
        }
    }
    float *col = vol + (size_t)iy * g.nx + ix;
    const size_t zs = (size_t)g.nx * g.ny;
#pragma unroll
    for (int zz = 0; zz < BP_ZC; ++zz)
        if (z0 + zz < g.nz) col[(size_t)(z0 + zz) * zs] = acc[zz];
}

}  // namespace

// table layout: RayXY [n_views * nu] | float2 cos/sin [n_views] | float zsnap [nv]
struct Tables {
    const float2 *view_cs;
    const float *zsnap;
};
static Tables tables_of(const dgr_geom &geo, const RayXY *tab) {
    const int n = geo.n_views * geo.nu;
    const float2 *cs = reinterpret_cast<const float2 *>(tab + n);
    return Tables{cs, reinterpret_cast<const float *>(cs + geo.n_views)};
}

cudaError_t launch_ray_tables(const dgr_grid &g, const dgr_geom &geo, RayXY *tab, cudaStream_t st) {
    const int n = geo.n_views * geo.nu;
    const Tables T = tables_of(geo, tab);
    const int m = n > geo.nv ? n : geo.nv;
    k_ray_tables<<<(m + 127) / 128, 128, 0, st>>>(g, geo, tab, const_cast<float2 *>(T.view_cs),
                                                  const_cast<float *>(T.zsnap));
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_project(const dgr_grid &g, const dgr_geom &geo, const RayXY *tab,
                           const float *vol, float *sino, cudaStream_t st) {
    const long long nrays = (long long)geo.n_views * geo.nv * geo.nu;
    const long long blocks = (nrays + 127) / 128;
    k_project<<<(unsigned)blocks, 128, 0, st>>>(g, geo, tab, tables_of(geo, tab).zsnap, vol, sino);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const dgr_grid &g, const dgr_geom &geo, const RayXY *tab,
                               const float *sino, float *vol, cudaStream_t st) {
    const Tables T = tables_of(geo, tab);
    dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, (g.nz + BP_ZC - 1) / BP_ZC);
    k_backproject<<<grid, 128, 0, st>>>(g, geo, tab, T.view_cs, T.zsnap, sino, vol);
    counted(1);
    return cudaGetLastError();
}

}  // namespace dgr
