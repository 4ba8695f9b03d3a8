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
//   k_ray_tables  per (view, iu): X0, D (FP64 arithmetic, stored FP32);
//                 per detector row: z slope, its reciprocal, FP64 layer snap
//   k_project     one thread per ray, incremental plane walk; u-adjacent
//                 rays in a warp read neighbouring voxels
//   k_scale_dn    residual x |D| per ray (chord lengths are t-intervals x |D|)
//   k_backproject one thread per (x, y) column and a chunk of z: for each view
//                 the candidate detector columns come from the column's four
//                 corners, the candidate rows per voxel in closed form from the
//                 column's slab interval; each candidate costs one slab test
//                 and one load -- no divisions, no atomics
#include <math.h>
#include <string.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr float CAND_EPS = 1e-3f;  // pixel margin of the candidate-ray search

// table layout: RayXY [tot_tab] | float2 cos/sin [tot_views] (padded to 16 B) | RowZ [tot_rows]
struct Tables {
    RayXY *tab;
    float2 *view_cs;
    RowZ *rows;
};
__host__ __device__ inline Tables tables_of(RayXY *tab, int n_tab, int n_views) {
    Tables T;
    T.tab = tab;
    T.view_cs = reinterpret_cast<float2 *>(tab + n_tab);
    const size_t cs_bytes = ((sizeof(float2) * (size_t)n_views + 15) / 16) * 16;
    T.rows = reinterpret_cast<RowZ *>(reinterpret_cast<char *>(T.view_cs) + cs_bytes);
    return T;
}

// For an axis the ray runs parallel to, only floor(xi) matters (which voxel
// layer holds the ray).  That decision is taken in FP64 and stored as the
// layer's centre, so a ray lying exactly in a voxel face plane is assigned
// the same way as by an FP64 evaluation of floor((X - o) / h).
__device__ __forceinline__ float snap_layer(double xi) { return (float)(floor(xi) + 0.5); }

// one thread per global RayXY entry, then per global RowZ entry
__global__ void k_ray_tables(const __grid_constant__ Batch B, RayXY *__restrict__ tab) {
    const Tables T = tables_of(tab, B.tot_tab, B.tot_views);
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B.tot_tab) {
        const int ri = idx - B.tot_tab;
        if (ri >= B.tot_rows) return;
        int i = 0;
        while (i + 1 < B.n && B.in[i + 1].row0 <= ri) ++i;
        const Inst &I = B.in[i];
        const int iv = ri - I.row0;
        const float v = ((float)iv - 0.5f * (float)(I.nv - 1)) * I.pv;
        RowZ R;
        R.v = v;
        R.zv = I.beam == DGR_CONE ? v / I.g.h : 0.f;
        R.izv = R.zv != 0.f ? 1.0f / R.zv : 0.f;
        // z layer of the rays of this row when they run parallel to the z
        // planes (parallel beam, or the cone's v = 0 row)
        const double v64 = ((double)iv - 0.5 * (double)(I.nv - 1)) * (double)I.pv;
        const double X0z = I.beam == DGR_CONE ? 0.0 : v64;
        R.zsnap = snap_layer((X0z - (double)I.g.oz) / (double)I.g.h);
        T.rows[ri] = R;
        return;
    }
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].tab0 <= idx) ++i;
    const Inst &I = B.in[i];
    const dgr_grid &g = I.g;
    const int loc = idx - I.tab0;
    const int k = loc / I.nu, iu = loc % I.nu;
    const double a = (double)I.angles[k];
    const double c = cos(a), s = sin(a);
    if (iu == 0) T.view_cs[I.view0 + k] = make_float2((float)c, (float)s);
    const double u = ((double)iu - 0.5 * (double)(I.nu - 1)) * (double)I.pu;
    const double h = (double)g.h;
    const double gcx = (double)g.ox + 0.5 * g.nx * h, gcy = (double)g.oy + 0.5 * g.ny * h;
    double Sx, Sy, Dx, Dy;
    if (I.beam == DGR_CONE) {
        Sx = -(double)I.dso * c; Sy = -(double)I.dso * s;
        Dx = (double)I.dsd * c - u * s; Dy = (double)I.dsd * s + u * c;
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
    T.tab[idx] = r;
}

struct RayZ {
    float xi0z, ez, inv_ez;
};

// z part of ray (iu, iv); the identical FP32 sequence in every kernel.
// zoff = -oz / h.
__device__ __forceinline__ RayZ ray_z(const RayXY &r, const RowZ &row, float zoff) {
    RayZ z;
    if (row.zv != 0.f) {
        z.ez = row.zv;
        z.inv_ez = row.izv;
        z.xi0z = fmaf(r.tc, row.zv, zoff);
    } else {
        z.ez = 0.f;
        z.inv_ez = 0.f;
        z.xi0z = row.zsnap;
    }
    return z;
}

// |D| of ray (iu, iv): the world length of a unit t-interval
__device__ __forceinline__ float ray_norm(const RayXY &r, const RowZ &row, int beam) {
    return sqrtf(beam == DGR_CONE ? fmaf(row.v, row.v, r.dxy2) : r.dxy2);
}

__device__ __forceinline__ float plane_t(int p, float xi0, float inv) {
    return ((float)p - xi0) * inv;
}

// a4: one thread per global ray; incremental Siddon walk.
__global__ void __launch_bounds__(128) k_project(const __grid_constant__ Batch B,
                                                 RayXY *__restrict__ tab_base) {
    const long long r_g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r_g >= B.tot_rays) return;
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    const Inst &I = B.in[inst_of_ray(B, r_g)];
    const dgr_grid &g = I.g;
    const long long r = r_g - I.ray0;
    const int iu = (int)(r % I.nu);
    const int iv = (int)((r / I.nu) % I.nv);
    const int k = (int)(r / ((long long)I.nu * I.nv));
    const float *__restrict__ vol = I.vol;
    float *__restrict__ sino = I.sino;
    const RayXY R = T.tab[I.tab0 + k * I.nu + iu];
    const RowZ row = T.rows[I.row0 + iv];
    const RayZ Z = ray_z(R, row, I.zoff);
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
    // per-axis state as scalars (selected, never indexed, so it stays in
    // registers); voxel indices 32-bit (the API bounds a volume to < 2^31)
    const int sx = sgn[0], sy = sgn[1] * g.nx, sz = sgn[2] * g.nx * g.ny;  // signed index steps
    int idx = idx3[2] * g.nx * g.ny + idx3[1] * g.nx + idx3[0];
    int ix = idx3[0], iy = idx3[1], iz = idx3[2];
    float tx = tn[0], ty = tn[1], tz = tn[2];
    const float x0 = xi0[0], y0 = xi0[1], z0 = xi0[2];
    const float ivx = inv[0], ivy = inv[1], ivz = inv[2];
    const int ux = sgn[0] > 0, uy = sgn[1] > 0, uz = sgn[2] > 0;
    float t = tmin, acc = 0.f;
    // walk the plane crossings WALK at a time: segment lengths and voxel
    // indices first (ALU only), then their loads together, then the sums in
    // walk order
    constexpr int WALK = 4;
    const int maxgroups = (g.nx + g.ny + g.nz + 3) / WALK + 1;
    bool done = false;
    for (int grp = 0; grp < maxgroups && !done; ++grp) {
        float len[WALK];
        int at[WALK];
#pragma unroll
        for (int j = 0; j < WALK; ++j) {
            at[j] = idx;
            const float tnext = fminf(tx, fminf(ty, tz));
            len[j] = done ? 0.f : tnext - t;
            t = done ? t : tnext;
            if (done) continue;
            if (tnext == tx) {
                const int ni = ix + sx;
                if (ni < 0 || ni >= g.nx) { done = true; continue; }
                ix = ni; idx += sx;
                tx = plane_t(ni + ux, x0, ivx);
            } else if (tnext == ty) {
                const int ni = iy + sgn[1];
                if (ni < 0 || ni >= g.ny) { done = true; continue; }
                iy = ni; idx += sy;
                ty = plane_t(ni + uy, y0, ivy);
            } else {
                const int ni = iz + sgn[2];
                if (ni < 0 || ni >= g.nz) { done = true; continue; }
                iz = ni; idx += sz;
                tz = plane_t(ni + uz, z0, ivz);
            }
        }
        float v[WALK];
#pragma unroll
        for (int j = 0; j < WALK; ++j) v[j] = __ldg(vol + at[j]);
#pragma unroll
        for (int j = 0; j < WALK; ++j) acc = fmaf(len[j], v[j], acc);
    }
    sino[r] = acc * ray_norm(R, row, I.beam);
}

// residual x |D| per ray, written view-major with v fastest ([view][u][v]) so
// that the backprojector's lanes (consecutive z -> consecutive detector rows)
// read it coalesced; the chord lengths are t-intervals x |D|.
// blockIdx.z: global view.
constexpr int TR = 32;
__global__ void k_scale_dn_t(const __grid_constant__ Batch B, RayXY *__restrict__ tab_base,
                             float *__restrict__ out_base) {
    __shared__ float tile[TR][TR + 1];
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    const Inst &I = B.in[inst_of_view(B, blockIdx.z)];
    const int k = blockIdx.z - I.view0;
    const int u0 = blockIdx.x * TR, v0 = blockIdx.y * TR;
    if (u0 >= I.nu || v0 >= I.nv) return;  // block-uniform
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const float *src = I.sino + (size_t)k * I.nv * I.nu;
    for (int j = ty; j < TR; j += 8) {
        const int iv = v0 + j, iu = u0 + tx;
        if (iv < I.nv && iu < I.nu)
            tile[j][tx] = src[(size_t)iv * I.nu + iu] *
                          ray_norm(T.tab[I.tab0 + k * I.nu + iu], T.rows[I.row0 + iv], I.beam);
    }
    __syncthreads();
    float *dst = out_base + I.ray0 + (size_t)k * I.nu * I.nv;
    for (int j = ty; j < TR; j += 8) {
        const int iu = u0 + j, iv = v0 + tx;
        if (iv < I.nv && iu < I.nu) dst[(size_t)iu * I.nv + iv] = tile[tx][j];
    }
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

// a6: backprojector.  A CTA of BP_W warps owns BP_W consecutive x-columns at
// one y and a z-pass of 32 * BP_ZJ voxels of one instance; a warp owns one
// column, its lanes consecutive z (lane + 32 j).  For each view the candidate
// detector columns follow from the column's 4 corners (warp-uniform), the slab
// interval of each candidate ray column is warp-uniform, and each lane finds
// its candidate rows in closed form and gathers length x scaled residual (rows
// contiguous across lanes).  The results leave through shared memory as full
// sectors.  blockIdx.x: global backprojector block.
constexpr int BP_W = 8;
constexpr int BP_ZJ = 8;
constexpr int BP_ZP = 32 * BP_ZJ;

__global__ void __launch_bounds__(32 * BP_W, 3) k_backproject(const __grid_constant__ Batch B,
                                                             RayXY *__restrict__ tab_base,
                                                             const float *__restrict__ sino_t_base) {
    __shared__ float out_tile[BP_ZP][BP_W];
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    const Inst &I = B.in[inst_of_blk(B, blockIdx.x)];
    const dgr_grid &g = I.g;
    const int b = blockIdx.x - I.blk0;
    const int bxi = b % I.nbx, iy = (b / I.nbx) % g.ny, bz = b / (I.nbx * g.ny);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ix = bxi * BP_W + w;
    const int zp = bz * BP_ZP;
    const bool cone = I.beam == DGR_CONE;
    const RayXY *__restrict__ tab = T.tab + I.tab0;
    const float2 *__restrict__ view_cs = T.view_cs + I.view0;
    const RowZ *__restrict__ rows = T.rows + I.row0;
    const float *__restrict__ sino_t = sino_t_base + I.ray0;
    const float zoff = I.zoff;
    const int nu = I.nu, nv = I.nv;
    float acc[BP_ZJ];
#pragma unroll
    for (int j = 0; j < BP_ZJ; ++j) acc[j] = 0.f;
    if (ix < g.nx) {
        const float h = g.h;
        const float xl = g.ox + ix * h, xh = xl + h, yl = g.oy + iy * h, yh = yl + h;
        const float cu = 0.5f * (float)(nu - 1), cv = 0.5f * (float)(nv - 1);
        const float inv_pu = 1.0f / I.pu;
        const float rows_per_zv = g.h / I.pv;  // detector rows per unit of zv
        const float row_of_oz = g.oz / I.pv + cv;
        for (int k = 0; k < I.n_views; ++k) {
            const float2 cs = view_cs[k];
            float umin = INFINITY, umax = -INFINITY;
#pragma unroll
            for (int cnr = 0; cnr < 4; ++cnr) {
                const float X = (cnr & 1) ? xh : xl, Y = (cnr & 2) ? yh : yl;
                const float pu_ = fmaf(-X, cs.y, Y * cs.x);
                float uu;
                if (cone) {
                    const float pr = fmaf(X, cs.x, Y * cs.y);
                    uu = __fdividef(I.dsd * pu_, I.dso + pr) * inv_pu + cu;
                } else {
                    uu = pu_ * inv_pu + cu;
                }
                umin = fminf(umin, uu);
                umax = fmaxf(umax, uu);
            }
            const int iu0 = max(0, (int)ceilf(umin - CAND_EPS));
            const int iu1 = min(nu - 1, (int)floorf(umax + CAND_EPS));
            for (int iu = iu0; iu <= iu1; ++iu) {
                const RayXY R = tab[k * nu + iu];
                float xlo, xhi, ylo, yhi;
                if (!slab(ix, R.xi0x, R.ex, R.inv_ex, xlo, xhi)) continue;
                if (!slab(iy, R.xi0y, R.ey, R.inv_ey, ylo, yhi)) continue;
                const float tlo = fmaxf(xlo, ylo), thi = fminf(xhi, yhi);
                if (!(thi > tlo)) continue;
                const float *scol = sino_t + ((size_t)k * nu + iu) * nv;
                if (cone) {
                    // ray row zv meets layer iz over t in [tlo, thi] only if
                    // z = zv (tc + t) + zoff, with tc + t in [wa, wb] (> 0: between
                    // source and detector), reaches [iz, iz + 1]:
                    //   zv in [min(zr/wa, zr/wb), max((zr+1)/wa, (zr+1)/wb)], zr = iz - zoff
                    const float ia = __fdividef(rows_per_zv, R.tc + tlo);
                    const float ib = __fdividef(rows_per_zv, R.tc + thi);
#pragma unroll
                    for (int j = 0; j < BP_ZJ; ++j) {
                        const int iz = zp + lane + 32 * j;
                        if (iz >= g.nz) break;
                        const float zr = (float)iz - zoff;
                        const float f0 = fminf(fmaf(zr, ia, cv), fmaf(zr, ib, cv));
                        const float f1 = fmaxf(fmaf(zr + 1.0f, ia, cv), fmaf(zr + 1.0f, ib, cv));
                        const int iv0 = max(0, (int)ceilf(f0 - CAND_EPS));
                        const int iv1 = min(nv - 1, (int)floorf(f1 + CAND_EPS));
                        float a = acc[j];
                        for (int iv = iv0; iv <= iv1; ++iv) {
                            const RowZ row = rows[iv];
                            const RayZ Z = ray_z(R, row, zoff);
                            float zlo, zhi;
                            if (!slab(iz, Z.xi0z, Z.ez, Z.inv_ez, zlo, zhi)) continue;
                            const float len = fminf(thi, zhi) - fmaxf(tlo, zlo);
                            if (len > 0.f) a = fmaf(len, __ldg(scol + iv), a);
                        }
                        acc[j] = a;
                    }
                } else {
                    const float len = thi - tlo;
#pragma unroll
                    for (int j = 0; j < BP_ZJ; ++j) {
                        const int iz = zp + lane + 32 * j;
                        if (iz >= g.nz) break;
                        const float f = fmaf((float)iz, rows_per_zv, row_of_oz);
                        const int iv0 = max(0, (int)ceilf(f - CAND_EPS));
                        const int iv1 = min(nv - 1, (int)floorf(f + rows_per_zv + CAND_EPS));
                        float a = acc[j];
                        for (int iv = iv0; iv <= iv1; ++iv) {
                            if (floorf(rows[iv].zsnap) == (float)iz) a = fmaf(len, __ldg(scol + iv), a);
                        }
                        acc[j] = a;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < BP_ZJ; ++j) out_tile[lane + 32 * j][w] = acc[j];
    __syncthreads();
    // write back: 8 consecutive x of one z per 8 threads (one 32-byte sector)
    const size_t zs = (size_t)g.nx * g.ny;
    for (int i = threadIdx.x; i < BP_ZP * BP_W; i += 32 * BP_W) {
        const int zz = i / BP_W, xx = i % BP_W;
        const int x = bxi * BP_W + xx, z = zp + zz;
        if (x < g.nx && z < g.nz) I.vol[(size_t)z * zs + (size_t)iy * g.nx + x] = out_tile[zz][xx];
    }
}

// residual x |D| per ray, natural layout ([view][v][u]), for the brick backprojector
__global__ void k_scale_dn(const __grid_constant__ Batch B, RayXY *__restrict__ tab_base,
                           float *__restrict__ out_base) {
    const long long r_g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r_g >= B.tot_rays) return;
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    const Inst &I = B.in[inst_of_ray(B, r_g)];
    const long long r = r_g - I.ray0;
    const int iu = (int)(r % I.nu);
    const int iv = (int)((r / I.nu) % I.nv);
    const int k = (int)(r / ((long long)I.nu * I.nv));
    out_base[r_g] = I.sino[r] * ray_norm(T.tab[I.tab0 + k * I.nu + iu], T.rows[I.row0 + iv], I.beam);
}

// a6 (brick scatter): a CTA owns a BBX x BBY x BBZ brick of one instance with
// FP32 accumulators in shared memory.  For each view it takes the detector
// rays whose pixel lies in the bounding box of the brick's projected corners,
// in colour classes (iu mod col_u, iv mod col_v): a voxel's footprint is
// narrower than col_u x col_v pixels, so two rays of one class never cross the
// same voxel and each class is added without atomics; classes and views go in
// a fixed order (bit-reproducible).  Each ray walks the brick's plane crossings
// exactly as k_project does (same t values), so every chord length equals the
// projector's.  blockIdx.x: global brick.
constexpr int BBX = 32, BBY = 16, BBZ = 16;
constexpr int BB_THREADS = 128;

__global__ void __launch_bounds__(BB_THREADS) k_bp_brick(const __grid_constant__ Batch B,
                                                          RayXY *__restrict__ tab_base,
                                                          const float *__restrict__ sino_s) {
    __shared__ float acc[BBZ * BBY * BBX];
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    int ii = 0;
    while (ii + 1 < B.n && B.in[ii + 1].bb0 <= (int)blockIdx.x) ++ii;
    const Inst &I = B.in[ii];
    const dgr_grid &g = I.g;
    const int b = blockIdx.x - I.bb0;
    const int bx = b % I.nbbx, by = (b / I.nbbx) % I.nbby, bz = b / (I.nbbx * I.nbby);
    const int x0 = bx * BBX, y0 = by * BBY, z0 = bz * BBZ;
    const int x1 = min(x0 + BBX, g.nx), y1 = min(y0 + BBY, g.ny), z1 = min(z0 + BBZ, g.nz);
    for (int i = threadIdx.x; i < BBZ * BBY * BBX; i += BB_THREADS) acc[i] = 0.f;
    const RayXY *__restrict__ tab = T.tab + I.tab0;
    const float2 *__restrict__ view_cs = T.view_cs + I.view0;
    const RowZ *__restrict__ rows = T.rows + I.row0;
    const float *__restrict__ sview0 = sino_s + I.ray0;
    const bool cone = I.beam == DGR_CONE;
    const float h = g.h;
    const float cu = 0.5f * (float)(I.nu - 1), cv = 0.5f * (float)(I.nv - 1);
    // brick corners (world)
    const float wx0 = g.ox + x0 * h, wx1 = g.ox + x1 * h, wy0 = g.oy + y0 * h, wy1 = g.oy + y1 * h;
    const float wz0 = g.oz + z0 * h, wz1 = g.oz + z1 * h;
    const int N0[3] = {x0, y0, z0}, N1[3] = {x1, y1, z1};
    __syncthreads();
    for (int k = 0; k < I.n_views; ++k) {
        const float2 cs = view_cs[k];
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float X = (c & 1) ? wx1 : wx0, Y = (c & 2) ? wy1 : wy0, Z = (c & 4) ? wz1 : wz0;
            const float pu_ = fmaf(-X, cs.y, Y * cs.x);
            float M = 1.f;
            if (cone) M = __fdividef(I.dsd, I.dso + fmaf(X, cs.x, Y * cs.y));
            const float uu = M * pu_ / I.pu + cu, vv = M * Z / I.pv + cv;
            umin = fminf(umin, uu); umax = fmaxf(umax, uu);
            vmin = fminf(vmin, vv); vmax = fmaxf(vmax, vv);
        }
        const int iu0 = max(0, (int)ceilf(umin - CAND_EPS)), iu1 = min(I.nu - 1, (int)floorf(umax + CAND_EPS));
        const int iv0 = max(0, (int)ceilf(vmin - CAND_EPS)), iv1 = min(I.nv - 1, (int)floorf(vmax + CAND_EPS));
        const float *sview = sview0 + (size_t)k * I.nv * I.nu;
        for (int cls = 0; cls < I.col_u * I.col_v; ++cls) {
            const int cuo = cls % I.col_u, cvo = cls / I.col_u;
            // first iu >= iu0 with iu % col_u == cuo, likewise for iv
            const int ua = iu0 + ((cuo - iu0 % I.col_u) + I.col_u) % I.col_u;
            const int va = iv0 + ((cvo - iv0 % I.col_v) + I.col_v) % I.col_v;
            const int nuc = ua <= iu1 ? (iu1 - ua) / I.col_u + 1 : 0;
            const int nvc = va <= iv1 ? (iv1 - va) / I.col_v + 1 : 0;
            for (int j = threadIdx.x; j < nuc * nvc; j += BB_THREADS) {
                const int iu = ua + (j % nuc) * I.col_u, iv = va + (j / nuc) * I.col_v;
                const float w = sview[(size_t)iv * I.nu + iu];
                if (w == 0.f) continue;
                const RayXY R = tab[k * I.nu + iu];
                const RayZ Z = ray_z(R, rows[iv], I.zoff);
                const float xi0[3] = {R.xi0x, R.xi0y, Z.xi0z};
                const float ev[3] = {R.ex, R.ey, Z.ez};
                const float inv[3] = {R.inv_ex, R.inv_ey, Z.inv_ez};
                // the brick's slab intervals
                float tmin = -INFINITY, tmax = INFINITY;
                int cur[3];
                bool miss = false;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (ev[a] != 0.f) {
                        const float ta = plane_t(N0[a], xi0[a], inv[a]), tb = plane_t(N1[a], xi0[a], inv[a]);
                        tmin = fmaxf(tmin, fminf(ta, tb));
                        tmax = fminf(tmax, fmaxf(ta, tb));
                    } else {
                        const float f = floorf(xi0[a]);
                        miss = miss || !(f >= (float)N0[a] && f < (float)N1[a]);
                        cur[a] = (int)f;
                    }
                }
                if (miss || !(tmax > tmin)) continue;
                int sg[3];
                float tn[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (ev[a] != 0.f) {
                        const int d = ev[a] > 0.f ? 1 : -1;
                        sg[a] = d;
                        int i = (int)floorf(fmaf(tmin, ev[a], xi0[a]));
                        i = min(max(i, N0[a]), N1[a] - 1);
                        for (int it = 0; it < 3; ++it) {
                            const float tu = plane_t(d > 0 ? i + 1 : i, xi0[a], inv[a]);
                            if (tu <= tmin && i + d >= N0[a] && i + d < N1[a]) i += d; else break;
                        }
                        for (int it = 0; it < 3; ++it) {
                            const float tl = plane_t(d > 0 ? i : i + 1, xi0[a], inv[a]);
                            if (tl > tmin && i - d >= N0[a] && i - d < N1[a]) i -= d; else break;
                        }
                        cur[a] = i;
                        tn[a] = plane_t(d > 0 ? i + 1 : i, xi0[a], inv[a]);
                    } else {
                        sg[a] = 0;
                        tn[a] = INFINITY;
                    }
                }
                int ix = cur[0] - x0, iy = cur[1] - y0, iz = cur[2] - z0;
                float t = tmin;
                for (int it = 0; it < BBX + BBY + BBZ + 3; ++it) {
                    const float tnext = fminf(tn[0], fminf(tn[1], tn[2]));
                    const float len = tnext - t;
                    if (len > 0.f) {
                        float *cell = &acc[(iz * BBY + iy) * BBX + ix];
                        *cell = fmaf(len, w, *cell);
                    }
                    t = tnext;
                    if (tnext == tn[0]) {
                        ix += sg[0];
                        if (ix < 0 || ix >= x1 - x0) break;
                        tn[0] = plane_t(x0 + ix + (sg[0] > 0), xi0[0], inv[0]);
                    } else if (tnext == tn[1]) {
                        iy += sg[1];
                        if (iy < 0 || iy >= y1 - y0) break;
                        tn[1] = plane_t(y0 + iy + (sg[1] > 0), xi0[1], inv[1]);
                    } else {
                        iz += sg[2];
                        if (iz < 0 || iz >= z1 - z0) break;
                        tn[2] = plane_t(z0 + iz + (sg[2] > 0), xi0[2], inv[2]);
                    }
                }
            }
            __syncthreads();  // the next class may touch the same voxels
        }
    }
    // write the brick (x fastest)
    const size_t zs = (size_t)g.nx * g.ny;
    for (int i = threadIdx.x; i < BBZ * BBY * BBX; i += BB_THREADS) {
        const int xx = i % BBX, yy = (i / BBX) % BBY, zz = i / (BBX * BBY);
        const int x = x0 + xx, y = y0 + yy, z = z0 + zz;
        if (x < x1 && y < y1 && z < z1) I.vol[(size_t)z * zs + (size_t)y * g.nx + x] = acc[i];
    }
}

}  // namespace

size_t ray_table_bytes(int n_tab, int n_views, int n_rows) {
    return sizeof(RayXY) * (size_t)n_tab + ((sizeof(float2) * (size_t)n_views + 15) / 16) * 16 +
           sizeof(RowZ) * (size_t)n_rows;
}

int bp_bricks(const dgr_grid &g, int &nbx, int &nby, int &nbz) {
    nbx = (g.nx + BBX - 1) / BBX;
    nby = (g.ny + BBY - 1) / BBY;
    nbz = (g.nz + BBZ - 1) / BBZ;
    return nbx * nby * nbz;
}

// Colour classes for the brick backprojector: a voxel's projected footprint,
// bounded over a 5 x 5 x 5 lattice of grid positions and every view (FP64,
// 10% margin), must be narrower than col_u x col_v pixels.
void bp_colours(const dgr_grid &g, const dgr_geom &geo, int &cu, int &cv) {
    double wu = 0.0, wv = 0.0;
    const double h = g.h;
    // the angles live on the device: bound over the full circle instead,
    // sampled every 5 degrees (the 10% margin covers the gaps)
    for (int ia = 0; ia < 72; ++ia) {
        const double a = ia * 3.14159265358979323846 / 36.0;
        const double c = cos(a), s = sin(a);
        for (int lz = 0; lz <= 4; ++lz)
            for (int ly = 0; ly <= 4; ++ly)
                for (int lx = 0; lx <= 4; ++lx) {
                    const double X0 = g.ox + lx * 0.25 * (g.nx - 1) * h;
                    const double Y0 = g.oy + ly * 0.25 * (g.ny - 1) * h;
                    const double Z0 = g.oz + lz * 0.25 * (g.nz - 1) * h;
                    double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
                    for (int cnr = 0; cnr < 8; ++cnr) {
                        const double X = X0 + ((cnr & 1) ? h : 0), Y = Y0 + ((cnr & 2) ? h : 0),
                                     Z = Z0 + ((cnr & 4) ? h : 0);
                        const double M = geo.beam == DGR_CONE ? geo.dsd / (geo.dso + X * c + Y * s) : 1.0;
                        const double u = M * (-X * s + Y * c) / geo.pu, v = M * Z / geo.pv;
                        umin = fmin(umin, u); umax = fmax(umax, u);
                        vmin = fmin(vmin, v); vmax = fmax(vmax, v);
                    }
                    wu = fmax(wu, umax - umin);
                    wv = fmax(wv, vmax - vmin);
                }
    }
    cu = (int)floor(1.1 * wu + 0.05) + 1;
    cv = (int)floor(1.1 * wv + 0.05) + 1;
}

static int g_bp_variant = 0;  // 0: column gather, 1: brick scatter
int backprojector_variant() { return g_bp_variant; }
void set_backprojector_variant(int v) { g_bp_variant = v; }

int bp_blocks(const dgr_grid &g, int &nbx, int &nbz) {
    nbx = (g.nx + BP_W - 1) / BP_W;
    nbz = (g.nz + BP_ZP - 1) / BP_ZP;
    return nbx * g.ny * nbz;
}

cudaError_t launch_ray_tables(const Batch &B, RayXY *tab, cudaStream_t st) {
    const int m = B.tot_tab + B.tot_rows;
    if (m == 0) return cudaSuccess;
    k_ray_tables<<<(m + 127) / 128, 128, 0, st>>>(B, tab);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_project(const Batch &B, const RayXY *tab, cudaStream_t st) {
    const long long blocks = (B.tot_rays + 127) / 128;
    if (blocks == 0) return cudaSuccess;
    k_project<<<(unsigned)blocks, 128, 0, st>>>(B, const_cast<RayXY *>(tab));
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const Batch &B, const RayXY *tab, float *sino_scaled, cudaStream_t st) {
    if (g_bp_variant == 1) {
        k_scale_dn<<<(unsigned)((B.tot_rays + 255) / 256), 256, 0, st>>>(B, const_cast<RayXY *>(tab),
                                                                         sino_scaled);
        k_bp_brick<<<B.tot_bricks, BB_THREADS, 0, st>>>(B, const_cast<RayXY *>(tab), sino_scaled);
        counted(2);
        return cudaGetLastError();
    }
    int max_u = 1, max_v = 1;
    for (int i = 0; i < B.n; ++i) {
        max_u = B.in[i].nu > max_u ? B.in[i].nu : max_u;
        max_v = B.in[i].nv > max_v ? B.in[i].nv : max_v;
    }
    dim3 tgrid((max_u + TR - 1) / TR, (max_v + TR - 1) / TR, B.tot_views);
    k_scale_dn_t<<<tgrid, 256, 0, st>>>(B, const_cast<RayXY *>(tab), sino_scaled);
    k_backproject<<<B.tot_blk, 32 * BP_W, 0, st>>>(B, const_cast<RayXY *>(tab), sino_scaled);
    counted(2);
    return cudaGetLastError();
}

size_t ray_table_bytes_single(const dgr_geom &geo) {
    return ray_table_bytes(geo.n_views * geo.nu, geo.n_views, geo.nv);
}

cudaError_t launch_project_single(const dgr_grid &g, const dgr_geom &geo, RayXY *tab,
                                  const float *vol, float *sino, cudaStream_t st) {
    static thread_local Batch B;
    memset(&B, 0, sizeof(B));
    B.n = 1;
    Inst &I = B.in[0];
    I.g = g;
    I.zoff = -g.oz / g.h;
    I.beam = geo.beam; I.n_views = geo.n_views; I.nu = geo.nu; I.nv = geo.nv;
    I.pu = geo.pu; I.pv = geo.pv; I.dso = geo.dso; I.dsd = geo.dsd; I.angles = geo.angles;
    I.vol = const_cast<float *>(vol);
    I.sino = sino;
    B.tot_tab = geo.n_views * geo.nu;
    B.tot_views = geo.n_views;
    B.tot_rows = geo.nv;
    B.tot_rays = (long long)geo.n_views * geo.nu * geo.nv;
    cudaError_t e = launch_ray_tables(B, tab, st);
    if (e == cudaSuccess) e = launch_project(B, tab, st);
    return e;
}

}  // namespace dgr
