// X-ray projector T (a4) and its exact adjoint (a6) on sm_103a.
//
// Ray model (paper Sec. 4.3, P_hat = T(V)): the line integral of the
// piecewise-constant voxel image, i.e. the sum over voxels of (length of the
// ray inside the voxel cube) x value -- Siddon's radiological path.
//
// Every kernel parameterises a ray as X(t) = X0 + t D, with X0 the point of
// its (x, y) projection closest to the grid axis (keeps t small and precise),
// and works in voxel coordinates xi = (X - o)/h.  A plane xi_a = p is crossed
// at t = (p - xi0_a) * inv_e_a.  The forward walks the crossings in order; the
// default adjoint walks the same crossings (so each chord length is the same
// FP32 value in both), the column gather intersects the three slab intervals
// built from the same plane crossings.
//
//   k_ray_tables    per (view, iu): X0, D (FP64 arithmetic, stored FP32);
//                   per detector row: z slope, its reciprocal, FP64 layer snap
//   k_path_n<0, 2>  a CTA per (view, detector column): the column's (x, y)
//                   path is merged into shared memory once, each thread walks
//                   two detector rows' z crossings along it; z-fastest volume
//                   (k_path<0>: a row per thread, for geometries where a ray
//                   may cross two z planes inside one (x, y) cell, or staged;
//                   k_project_ray: the C ABI's x-fastest layout)
//   k_scale_dn      residual x |D| per ray (chord lengths are t-intervals x |D|)
//   k_path_n<1, 2>  the adjoint as the same walk: integer sums += round(length
//                   x scaled residual) by 32-bit reductions (order-independent,
//                   bit-reproducible); k_bp_fold scales them into the FP32
//                   gradient (k_path<1> as k_path<0>)
//   k_bp_brick      the brick scatter (same integers, summed per brick in
//                   shared memory) and
//   k_backproject   the column gather: one thread per (x, y) column and a
//                   chunk of z; for each view the candidate detector columns
//                   come from the column's four corners, the candidate rows per
//                   voxel in closed form from the column's slab interval --
//                   no divisions, no atomics (selectable variants)
#include <limits.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "async_ops.cuh"
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
    DEP_ENTER();
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

// Entry cell along one axis at t = tmin, made consistent with the plane
// crossings: the plane ahead (in the travel direction) lies after tmin, the
// one behind at or before it.  lo/hi bound the index (a grid axis) or are
// INT_MIN/INT_MAX (the z axis of the row-warp walk, which runs over unbounded
// z layers and masks the ones outside the grid).
__device__ __forceinline__ int entry_cell(float tmin, float e, float xi0, float inv, int d, int lo,
                                          int hi) {
    float f = floorf(fmaf(tmin, e, xi0));
    f = fminf(fmaxf(f, (float)max(lo, -(1 << 24))), (float)min(hi, 1 << 24));
    int i = (int)f;
    for (int it = 0; it < 3; ++it) {
        const float tu = plane_t(d > 0 ? i + 1 : i, xi0, inv);
        if (tu <= tmin && i + d >= lo && i + d <= hi) i += d; else break;
    }
    for (int it = 0; it < 3; ++it) {
        const float tl = plane_t(d > 0 ? i : i + 1, xi0, inv);
        if (tl > tmin && i - d >= lo && i - d <= hi) i -= d; else break;
    }
    return i;
}

// a4 (shared-path projector): a CTA owns one detector column of one view and
// up to PR_ROWS detector rows, a warp 32 consecutive rows.  All rays of a
// column follow the same (x, y) path (rotation about z).  The CTA first lays
// that path out in shared memory -- the x and y plane crossings merged in
// parallel, each crossing's rank found by binary search in the other axis'
// crossings (x first on ties, as a sequential walk would take them) -- and
// every warp then streams through it: per (x, y) cell one shared load, and per
// lane the z planes its own ray crosses inside the cell (one in the common
// case, a bounded loop for more).  Segment lengths are differences of the same
// FP32 plane crossings the backprojector uses.  The volume is z fastest, so
// the lanes of a warp read neighbouring words.  Rows whose rays leave the grid
// through a z face walk with a per-segment mask (MASKZ).
constexpr int PR_THREADS = 256;
constexpr int PR_ROWS = PR_THREADS;
constexpr int SEG_MAX = 2048;  // path segments staged per round
constexpr int WALK = 4;  // segments per unrolled group (at most; the scatter walks 2 at a time)

struct __align__(8) Seg {
    float t1;  // end of the segment (the crossing that leaves its cell)
    int cb;    // element offset of the segment's (x, y) cell
};

// number of i in [0, n) whose crossing plane_t(p0 + sg i) is < T (le: <= T);
// the crossings are non-decreasing in i
__device__ __forceinline__ int count_before(float T, int n, int p0, int sg, float xi0, float inv,
                                            bool le) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float tm = plane_t(p0 + sg * mid, xi0, inv);
        if (le ? tm <= T : tm < T) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// the (x, y) path of a column through the whole grid, shared by every ray of a
// CTA: entry cell (ix0, iy0), the crossings ahead -- x planes px0 + sgx j for
// j < nxe, the last one leaving the grid, likewise y -- and the number of
// segments, which ends at the first leaving crossing
struct PathXY {
    int sgx, sgy, ix0, iy0, nxe, nye, px0, py0, nseg, cb0;
};

__device__ __forceinline__ PathXY xy_path(const RayXY &R, const Inst &I, float tmin, float fx, float fy) {
    const dgr_grid &g = I.g;
    PathXY P;
    P.sgx = R.ex > 0.f ? 1 : (R.ex < 0.f ? -1 : 0);
    P.sgy = R.ey > 0.f ? 1 : (R.ey < 0.f ? -1 : 0);
    P.ix0 = P.sgx ? entry_cell(tmin, R.ex, R.xi0x, R.inv_ex, P.sgx, 0, g.nx - 1) : (int)fx;
    P.iy0 = P.sgy ? entry_cell(tmin, R.ey, R.xi0y, R.inv_ey, P.sgy, 0, g.ny - 1) : (int)fy;
    P.nxe = P.sgx > 0 ? g.nx - P.ix0 : (P.sgx < 0 ? P.ix0 + 1 : 0);
    P.nye = P.sgy > 0 ? g.ny - P.iy0 : (P.sgy < 0 ? P.iy0 + 1 : 0);
    P.px0 = P.sgx > 0 ? P.ix0 + 1 : P.ix0;
    P.py0 = P.sgy > 0 ? P.iy0 + 1 : P.iy0;
    int rend = INT_MAX;
    if (P.nxe > 0) {
        const float te = plane_t(P.px0 + P.sgx * (P.nxe - 1), R.xi0x, R.inv_ex);
        rend = min(rend, P.nxe - 1 + count_before(te, P.nye, P.py0, P.sgy, R.xi0y, R.inv_ey, false));
    }
    if (P.nye > 0) {
        const float te = plane_t(P.py0 + P.sgy * (P.nye - 1), R.xi0y, R.inv_ey);
        rend = min(rend, P.nye - 1 + count_before(te, P.nxe, P.px0, P.sgx, R.xi0x, R.inv_ex, true));
    }
    P.nseg = rend + 1;  // segments 0 .. rend
    P.cb0 = P.ix0 * I.vsx + P.iy0 * I.vsy;
    return P;
}

// segments c0 .. c1 - 1 of the path into seg[0 .. c1 - c0), each with its cell
// and leaving parameter, then WALK copies of the last one (empty segments at
// the last crossing, so groups are whole).  Every crossing finds its rank r in
// the merged x/y order by a binary search of the other axis; NT threads of the
// CTA take the crossings in turn.  Synchronises before (the previous round's
// readers are done) and after.
template <int NT>
__device__ __forceinline__ void stage_segs(Seg *seg, const PathXY &P, const RayXY &R, const Inst &I, int c0,
                                           int c1) {
    __syncthreads();
    if (c0 == 0 && threadIdx.x == 0) seg[0].cb = P.cb0;
    for (int e = threadIdx.x; e < P.nxe + P.nye; e += NT) {
        float te;
        int r, cx, cy;  // rank; cell after the crossing
        if (e < P.nxe) {
            te = plane_t(P.px0 + P.sgx * e, R.xi0x, R.inv_ex);
            r = e + count_before(te, P.nye, P.py0, P.sgy, R.xi0y, R.inv_ey, false);
            cx = P.ix0 + P.sgx * (e + 1);
            cy = P.iy0 + P.sgy * (r - e);
        } else {
            const int i = e - P.nxe;
            te = plane_t(P.py0 + P.sgy * i, R.xi0y, R.inv_ey);
            r = i + count_before(te, P.nxe, P.px0, P.sgx, R.xi0x, R.inv_ex, true);
            cx = P.ix0 + P.sgx * (r - i);
            cy = P.iy0 + P.sgy * (i + 1);
        }
        if (r >= c0 && r < c1) seg[r - c0].t1 = te;
        // r + 1 < c1 <= nseg: the crossing is not the leaving one, the cell is inside
        if (r + 1 >= c0 && r + 1 < c1) seg[r + 1 - c0].cb = cx * I.vsx + cy * I.vsy;
    }
    __syncthreads();
    if (threadIdx.x < WALK) {
        const Seg last = seg[c1 - 1 - c0];
        seg[c1 - c0 + threadIdx.x] = last;
    }
    __syncthreads();
}

// fixed-point step of one group of nkv <= VGROUP views of an instance: the
// largest power of two S with nkv x col_u x col_v x (longest chord in t units) x
// max |scaled residual| x S < 2^30, so that a voxel's integer sum over the
// group cannot overflow (a voxel meets at most col_u x col_v rays per view).
// Returns 0 if a residual of the group is not finite.  Called by whole warps
// (converged): the lanes share the maximum over the group's views.
constexpr int VGROUP = 128;
constexpr int FOLD_Y = 4;  // y rows of 32 x 32 (x, z) tiles per CTA of k_bp_fold
__device__ __forceinline__ float group_step(const Inst &I, const unsigned *view_max, int kv0, int nkv) {
    unsigned m = 0u;
    for (int j = threadIdx.x & 31; j < nkv; j += 32) m = max(m, view_max[I.view0 + kv0 + j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float amax = __uint_as_float(m);
    if (!(amax <= 3.0e38f)) return 0.f;
    // longest chord of a voxel in t units: sqrt(3) h / |D|, |D| >= dsd (cone) or 1 (parallel)
    const float tchord = 1.7320509f * I.g.h / (I.beam == DGR_CONE ? I.dsd : 1.f) * 1.001f;
    const float bound = (float)(nkv * I.col_u * I.col_v) * tchord * amax;
    if (!(bound > 0.f)) return 1.f;
    int ex;
    frexpf(bound, &ex);  // bound < 2^ex
    return ldexpf(1.f, min(30 - ex, 126));
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (the Tensor Memory Accelerator's 1D form) through
// shared memory: a CTA's detector column walks a path of (x, y) cells; with
// the volume z fastest, the part of a cell's z column its rows can reach is
// one contiguous run, so per chunk of cells one thread issues a bulk copy per
// cell (global -> shared, completion counted in bytes on an mbarrier) for the
// projector, or a bulk reduce-add per cell (shared -> global integer sums)
// for the backprojector, and the lanes work on shared memory.  Two stages: the
// next chunk's copies fly while the current one is walked.
// ---------------------------------------------------------------------------
// where the walk reads (MODE 0) or adds (MODE 1): the global volume / integer
// sums at cell offset + z (unstaged), or a shared-memory window of each cell's
// column: [slot][z - zlo] for the segments s0 .. s0 + nslot - 1 (staged)
struct Stage {
    int s0, nslot, zspan, zlo, zhi;
};

// Fast walk for geometries where no ray crosses two z planes inside one
// (x, y) cell (sqrt(2) max|e_z| / min|e_xy| < 1 with margin; checked on the
// host): the crossing is a predicated update and the second segment's length
// is t1 - min(tz_before, t1), zero when nothing was crossed.
template <int MODE, bool MASKZ, bool STAGED>
__device__ __forceinline__ void walk_segs1(const float *__restrict__ vol, int *__restrict__ acci, float wq,
                                           const Seg *seg, int c0, int r0, int r1, int nz, const Stage &G,
                                           float &t, float &acc, int &iz, float &fz, float &tz, int sgz,
                                           float xi0z, float iez, long long nvox, int *status) {
    (void)nvox;
    (void)status;
    // segments per unrolled group: 4 loads in flight for the projector; the
    // scatter keeps 2 (fewer registers, more resident warps)
    constexpr int NW = MODE == 0 ? WALK : 2;
    const unsigned zmax = (unsigned)(nz - 1);
    const int zl = STAGED ? G.zlo : 0, zh = STAGED ? G.zhi : nz - 1;
    // the layer the addresses use: clamped into the volume (unstaged: one
    // unsigned min -- a lane below the volume is clamped to the top layer,
    // harmless since its masked segments have zero length) or the window
    auto layer = [&](int i) { return STAGED ? min(max(i, zl), zh) : (int)min((unsigned)i, zmax); };
    int zc = layer(iz);
    const float fsg = (float)sgz;
    for (int r = r0; r < r1; r += NW) {
        float l0[NW], l1[NW];
        int a0[NW], a1[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const Seg S = seg[r + j - c0];  // past the round's end: padding, empty segments
            const int base = STAGED ? min(r + j - G.s0, G.nslot - 1) * G.zspan - G.zlo : S.cb;
            const float t1 = S.t1;
            const float m = fminf(tz, t1);
            l0[j] = (!MASKZ || (unsigned)iz <= zmax) ? m - t : 0.f;
            a0[j] = base + zc;
            if (tz < t1) {
                iz += sgz;
                fz += fsg;
                tz = (fz - xi0z) * iez;
                zc = layer(iz);
            }
            // at most one z crossing per cell: the next one lies beyond t1, so
            // the second segment is t1 - m (zero without a crossing)
            l1[j] = (!MASKZ || (unsigned)iz <= zmax) ? t1 - m : 0.f;
            a1[j] = base + zc;
            t = t1;
        }
        if (MODE == 0) {
            float v0[NW], v1[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                v0[j] = STAGED ? vol[a0[j]] : ((STAGED || DGR_INB(a0[j], nvox, status)) ? __ldg(vol + a0[j]) : 0.f);
                // the second segment's voxel only after a crossing (else l1 = 0)
                v1[j] = l1[j] != 0.f ? (STAGED ? vol[a1[j]] : ((STAGED || DGR_INB(a1[j], nvox, status)) ? __ldg(vol + a1[j]) : 0.f)) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < NW; ++j) acc = fmaf(l1[j], v1[j], fmaf(l0[j], v0[j], acc));
        } else {
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                // without a crossing the second segment is empty (q1 = 0): one
                // reduction; integer sums do not depend on how they are split
                const float2 lw = __fmul2_rn(make_float2(l0[j], l1[j]), make_float2(wq, wq));
                const int q0 = __float2int_rn(lw.x), q1 = __float2int_rn(lw.y);
                if (STAGED || DGR_INB(a0[j], nvox, status)) atomicAdd(acci + a0[j], q0);
                if (q1 != 0 && (STAGED || DGR_INB(a1[j], nvox, status))) atomicAdd(acci + a1[j], q1);
            }
        }
    }
}

// MODE 0 (project): acc += length x volume value.  MODE 1 (backproject
// scatter): the integer sums at the same voxels += round(length x wq).
template <int MODE, bool MASKZ, bool STAGED>
__device__ __forceinline__ void walk_segs(const float *__restrict__ vol, int *__restrict__ acci, float wq,
                                          const Seg *seg, int c0, int r0, int r1, int nz, const Stage &G,
                                          float &t, float &acc, int &iz, float &fz, float &tz, int sgz,
                                          float xi0z, float iez, long long nvox, int *status) {
    (void)nvox;
    (void)status;
    // segments per unrolled group: 4 loads in flight for the projector; the
    // scatter keeps 2 (fewer registers, more resident warps)
    constexpr int NW = MODE == 0 ? WALK : 2;
    const unsigned zmax = (unsigned)(nz - 1);
    const int zl = STAGED ? G.zlo : 0, zh = STAGED ? G.zhi : nz - 1;
    int zc = min(max(iz, zl), zh);
    const float fsg = (float)sgz;
    for (int r = r0; r < r1; r += NW) {
        float l0[NW], l1[NW];
        int a0[NW], a1[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const Seg S = seg[r + j - c0];  // past the round's end: padding, empty segments
            const int base = STAGED ? min(r + j - G.s0, G.nslot - 1) * G.zspan - G.zlo : S.cb;
            const float t1 = S.t1;
            const float m = fminf(tz, t1);
            const bool in0 = !MASKZ || (unsigned)iz <= zmax;
            l0[j] = in0 ? m - t : 0.f;
            a0[j] = base + zc;
            l1[j] = 0.f;
            a1[j] = a0[j];
            if (tz < t1) {
                float ts = tz;
                iz += sgz;
                fz += fsg;
                tz = (fz - xi0z) * iez;
                zc = min(max(iz, zl), zh);
                const bool in1 = !MASKZ || (unsigned)iz <= zmax;
                l1[j] = in1 ? fminf(tz, t1) - ts : 0.f;
                a1[j] = base + zc;
                // rare: further z planes inside this cell (bounded: a crossing
                // that rounding failed to advance cannot spin)
                for (int rep = 0; rep <= nz && tz < t1; ++rep) {
                    ts = tz;
                    iz += sgz;
                    fz += fsg;
                    tz = (fz - xi0z) * iez;
                    zc = min(max(iz, zl), zh);
                    if (!MASKZ || (unsigned)iz <= zmax) {
                        const float len = fminf(tz, t1) - ts;
                        if (MODE == 0) acc = fmaf(len, STAGED ? vol[base + zc] : ((STAGED || DGR_INB(base + zc, nvox, status)) ? __ldg(vol + base + zc) : 0.f), acc);
                        else if (len != 0.f && (STAGED || DGR_INB(base + zc, nvox, status))) atomicAdd(acci + base + zc, __float2int_rn(len * wq));
                    }
                }
            }
            t = t1;
        }
        if (MODE == 0) {
            float v0[NW], v1[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                v0[j] = STAGED ? vol[a0[j]] : ((STAGED || DGR_INB(a0[j], nvox, status)) ? __ldg(vol + a0[j]) : 0.f);
                v1[j] = STAGED ? vol[a1[j]] : ((STAGED || DGR_INB(a1[j], nvox, status)) ? __ldg(vol + a1[j]) : 0.f);
            }
#pragma unroll
            for (int j = 0; j < NW; ++j) acc = fmaf(l1[j], v1[j], fmaf(l0[j], v0[j], acc));
        } else {
#pragma unroll
            for (int j = 0; j < NW; ++j) {
                if (l0[j] != 0.f && (STAGED || DGR_INB(a0[j], nvox, status))) atomicAdd(acci + a0[j], __float2int_rn(l0[j] * wq));
                if (l1[j] != 0.f && (STAGED || DGR_INB(a1[j], nvox, status))) atomicAdd(acci + a1[j], __float2int_rn(l1[j] * wq));
            }
        }
    }
}

// one walk over segments [r0, r1) of the current round (starting at c0)
template <int MODE, bool STAGED>
__device__ __forceinline__ void walk_any(bool multiz, bool masked, const float *vol, int *acci, float wq,
                                         const Seg *seg, int c0, int r0, int r1, int nz, const Stage &G,
                                         float &t, float &acc, int &iz, float &fz, float &tz, int sgz,
                                         float xi0z, float iez, long long nvox = 0, int *status = nullptr) {
    if (multiz) {
        if (masked)
            walk_segs<MODE, true, STAGED>(vol, acci, wq, seg, c0, r0, r1, nz, G, t, acc, iz, fz, tz, sgz, xi0z, iez, nvox, status);
        else
            walk_segs<MODE, false, STAGED>(vol, acci, wq, seg, c0, r0, r1, nz, G, t, acc, iz, fz, tz, sgz, xi0z, iez, nvox, status);
    } else {
        if (masked)
            walk_segs1<MODE, true, STAGED>(vol, acci, wq, seg, c0, r0, r1, nz, G, t, acc, iz, fz, tz, sgz, xi0z, iez, nvox, status);
        else
            walk_segs1<MODE, false, STAGED>(vol, acci, wq, seg, c0, r0, r1, nz, G, t, acc, iz, fz, tz, sgz, xi0z, iez, nvox, status);
    }
}

// MODE 0: a4, the projector.  MODE 1: a6, the ray-driven backprojector for
// the views [kv0, kv0 + nkv) of every instance: each lane's row adds
// length x scaled residual, in the fixed point of its view group, into
// integer sums laid out like the projector's volume (z fastest); k_bp_fold
// then moves them into the FP32 gradient.  Integer sums do not depend on the
// order of the additions, so the result is bit-reproducible.
// blockIdx.x: global block (instance, view of the launch, row group, column).
template <int MODE, bool TMA>
__global__ void __launch_bounds__(PR_THREADS) k_path(const __grid_constant__ Batch B,
                                                     RayXY *__restrict__ tab_base,
                                                     const float *__restrict__ sino_s,
                                                     const unsigned *__restrict__ view_max) {
    DEP_ENTER();
    __shared__ Seg seg[SEG_MAX + WALK];
    // TMA: two stages of B.tma_ch cell columns of up to B.tma_zcap words each
    extern __shared__ __align__(128) float cols[];
    __shared__ unsigned long long bar[2];
    __shared__ float s_zr[2][PR_THREADS / 32];
    __shared__ int s_abort;  // a bounded wait gave up: leave the staged walk
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    int ii = 0;
    while (ii + 1 < B.n && B.in[ii + 1].pb0 <= (int)blockIdx.x) ++ii;
    const Inst &I = B.in[ii];
    const dgr_grid &g = I.g;
    const int b = blockIdx.x - I.pb0;
    const int iu = b % I.nu, rg = (b / I.nu) % I.npv, k = I.kv0 + b / (I.nu * I.npv);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int iv = rg * PR_ROWS + w * 32 + lane;
    const RayXY R = T.tab[I.tab0 + k * I.nu + iu];
    const RowZ row = T.rows[I.row0 + min(iv, I.nv - 1)];
    const size_t ray = ((size_t)k * I.nv + min(iv, I.nv - 1)) * I.nu + iu;
    // (x, y) interval of the grid and entry cell: the same for the whole CTA
    float tmin = -INFINITY, tmax = INFINITY;
    bool miss = false;
    float fx = 0.f, fy = 0.f;
    if (R.ex != 0.f) {
        const float t0 = plane_t(0, R.xi0x, R.inv_ex), t1 = plane_t(g.nx, R.xi0x, R.inv_ex);
        tmin = fmaxf(tmin, fminf(t0, t1));
        tmax = fminf(tmax, fmaxf(t0, t1));
    } else {
        fx = floorf(R.xi0x);
        miss = miss || !(fx >= 0.f && fx < (float)g.nx);
    }
    if (R.ey != 0.f) {
        const float t0 = plane_t(0, R.xi0y, R.inv_ey), t1 = plane_t(g.ny, R.xi0y, R.inv_ey);
        tmin = fmaxf(tmin, fminf(t0, t1));
        tmax = fminf(tmax, fmaxf(t0, t1));
    } else {
        fy = floorf(R.xi0y);
        miss = miss || !(fy >= 0.f && fy < (float)g.ny);
    }
    if (miss || !(tmax > tmin)) {  // CTA-uniform
        if (MODE == 0 && iv < I.nv) I.sino[ray] = 0.f;
        return;
    }
    float wq = 0.f;  // MODE 1: this row's scaled residual in fixed point
    if (MODE == 1) {
        const float S = group_step(I, view_max, I.kv0, I.nkv);
        wq = iv < I.nv ? sino_s[I.ray0 + ray] * S : 0.f;
        if (__syncthreads_and(wq == 0.f)) return;  // nothing to add (or a bad group)
    }
    const PathXY P = xy_path(R, I, tmin, fx, fy);
    const int nseg = P.nseg;
    // this lane's z: entry layer (unbounded), next crossing, and whether the
    // ray stays inside the z range over the whole (x, y) chord
    const RayZ Z = ray_z(R, row, I.zoff);
    int iz, sgz = 0;
    float tz = INFINITY, fz = 0.f;
    bool zin;
    if (Z.ez != 0.f) {
        sgz = Z.ez > 0.f ? 1 : -1;
        const float t0 = plane_t(0, Z.xi0z, Z.inv_ez), t1 = plane_t(g.nz, Z.xi0z, Z.inv_ez);
        zin = fminf(t0, t1) <= tmin && fmaxf(t0, t1) >= tmax;
        iz = entry_cell(tmin, Z.ez, Z.xi0z, Z.inv_ez, sgz, INT_MIN / 2, INT_MAX / 2);
        fz = (float)(sgz > 0 ? iz + 1 : iz);
        tz = (fz - Z.xi0z) * Z.inv_ez;
    } else {
        const float f = floorf(Z.xi0z);
        zin = f >= 0.f && f < (float)g.nz;
        iz = zin ? (int)f : -1;
    }
    const bool masked = __any_sync(0xffffffffu, !zin);
    float t = tmin, acc = 0.f;
    // TMA: the z window every row of this CTA can reach along the whole path
    Stage G = {0, 1, 4, 0, 3};
    bool staged = false;
    if (TMA) {
        const float za = fmaf(tmin, Z.ez, Z.xi0z), zb = fmaf(tmax, Z.ez, Z.xi0z);
        float lo = fminf(za, zb), hi = fmaxf(za, zb);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            s_zr[0][w] = lo;
            s_zr[1][w] = hi;
        }
        if (threadIdx.x == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_barrier_init();
            s_abort = 0;
        }
        fence_async_smem();
        __syncthreads();
        for (int j = 0; j < PR_THREADS / 32; ++j) {
            lo = fminf(lo, s_zr[0][j]);
            hi = fmaxf(hi, s_zr[1][j]);
        }
        // one voxel of margin each side, z0 rounded down to 4 words (16-byte copies)
        const int zlo = (int)fmaxf(fminf(floorf(lo) - 1.f, (float)g.nz), 0.f) & ~3;
        const int zhi = (int)fminf(fmaxf(floorf(hi) + 1.f, 0.f), (float)(g.nz - 1));
        const int span = (zhi - zlo + 4) & ~3;
        staged = span > 0 && span <= B.tma_zcap;  // CTA-uniform
        G.zlo = zlo;
        G.zspan = max(span, 4);
        G.zhi = zlo + G.zspan - 1;
        if (MODE == 1 && staged) {
            for (int i = threadIdx.x; i < 2 * B.tma_ch * B.tma_zcap; i += PR_THREADS) cols[i] = 0.f;
            __syncthreads();
        }
    }
    int use = 0;  // sub-chunks processed (stage = use & 1, phase = (use >> 1) & 1)
    for (int c0 = 0; c0 < nseg; c0 += SEG_MAX) {
        const int c1 = min(nseg, c0 + SEG_MAX);
        stage_segs<PR_THREADS>(seg, P, R, I, c0, c1);
        if (!TMA || !staged) {
            // a warp whose rows all lie past the detector (nv not a multiple of
            // the CTA's rows) only takes part in the staging
            if (rg * PR_ROWS + w * 32 < I.nv)
                walk_any<MODE, false>(I.multiz, masked, I.vol, I.acc, wq, seg, c0, c0, c1, g.nz, G, t, acc, iz,
                                      fz, tz, sgz, Z.xi0z, Z.inv_ez, (long long)g.nx * g.ny * g.nz, B.status);
            continue;
        }
        // staged: sub-chunks of tma_ch cells, their z windows in shared memory
        const int CH = B.tma_ch, ZC = B.tma_zcap;
        const int nsub = (c1 - c0 + CH - 1) / CH;
        const unsigned bytes = (unsigned)G.zspan * 4u;
        auto issue = [&](int sc, int stg) {  // thread 0: bulk copies of sub-chunk sc into stage stg
            const int s0 = c0 + sc * CH, n = min(CH, c1 - s0);
            mbar_expect_tx(&bar[stg], bytes * (unsigned)n);
            for (int j = 0; j < n; ++j)
                bulk_g2s(cols + (size_t)(stg * CH + j) * ZC, I.vol + seg[s0 + j - c0].cb + G.zlo, bytes, &bar[stg]);
        };
        if (MODE == 0 && threadIdx.x == 0) issue(0, use & 1);
        for (int sc = 0; sc < nsub; ++sc, ++use) {
            const int stg = use & 1;
            Stage Gs = G;
            Gs.s0 = c0 + sc * CH;
            Gs.nslot = min(CH, c1 - Gs.s0);
            const int r1 = Gs.s0 + Gs.nslot;
            float *col = cols + (size_t)stg * CH * ZC;
            if (MODE == 0) {
                if (threadIdx.x == 0 && sc + 1 < nsub) issue(sc + 1, stg ^ 1);
                if (!mbar_wait(&bar[stg], (use >> 1) & 1, B.status)) s_abort = 1;
                Gs.zspan = ZC;  // slots are ZC words apart
                Gs.zlo = G.zlo;
                walk_any<MODE, true>(I.multiz, masked, col, nullptr, wq, seg, c0, Gs.s0, r1, g.nz, Gs, t, acc,
                                     iz, fz, tz, sgz, Z.xi0z, Z.inv_ez);
                __syncthreads();  // this stage may be refilled
                if (s_abort) {
                    // let the copies already in flight land before leaving (bounded)
                    if (threadIdx.x == 0 && sc + 1 < nsub) mbar_wait(&bar[stg ^ 1], ((use + 1) >> 1) & 1, B.status);
                    break;
                }
            } else {
                Gs.zspan = ZC;
                walk_any<MODE, true>(I.multiz, masked, nullptr, reinterpret_cast<int *>(col), wq, seg, c0,
                                     Gs.s0, r1, g.nz, Gs, t, acc, iz, fz, tz, sgz, Z.xi0z, Z.inv_ez);
                fence_async_smem();  // each thread's shared atomics, before the bulk reads
                __syncthreads();
                if (threadIdx.x == 0) {
                    for (int j = 0; j < Gs.nslot; ++j)
                        bulk_s2g_add(I.acc + seg[Gs.s0 + j - c0].cb + G.zlo,
                                     reinterpret_cast<const int *>(col) + (size_t)j * ZC, bytes);
                    bulk_commit();
                    bulk_wait_read1();  // the other stage's adds have read their source
                }
                __syncthreads();
                float *other = cols + (size_t)(stg ^ 1) * CH * ZC;
                for (int i = threadIdx.x; i < CH * ZC; i += PR_THREADS) other[i] = 0.f;
                __syncthreads();
            }
        }
        if (TMA && s_abort) break;
    }
    if (TMA && MODE == 1 && staged && threadIdx.x == 0) bulk_wait_all();
    if (MODE == 0 && iv < I.nv) I.sino[ray] = acc * ray_norm(R, row, I.beam);
}

// a4 / a6 (MODE 0 / 1) with NR rays per thread (2 by default): the CTA covers
// a column of ROWS rows (PR_ROWS as k_path, or 128 / 64 for short detectors)
// with ROWS / NR threads, lane
// l of warp w taking the rows w 32 NR + 32 q + l, q < NR (each load or
// reduction instruction still touches 32 consecutive rows' voxels).  The walk
// keeps one (x, y) path position for all NR rays and pairs their arithmetic
// where it is the same operation (the segment lengths as packed FP32
// subtractions; the projector's sums as packed FMAs, the scatter's length x
// residual products as packed multiplies; each half rounds as the scalar
// operation), so the sinogram and the integer sums are bit-identical to
// k_path's.  Single-crossing geometries only (no instance with multiz), no
// staging: the launchers keep k_path otherwise.
constexpr int PR_NR = 2;  // rays per thread

// MODE 0: acc += length x volume value; MODE 1: the integer sums at the same
// voxels += round(length x wq), as walk_segs1.
template <int MODE, bool MASKZ, int NR>
__device__ __forceinline__ void walk_segs1_xn(const float *__restrict__ vol, int *__restrict__ acci,
                                              const float2 (&wqv)[NR / 2], const Seg *seg, int c0, int r0, int r1,
                                              int nz, float &t, float2 (&acc)[NR / 2], int (&iz)[NR],
                                              float (&fz)[NR], float (&tz)[NR], const int (&sgz)[NR],
                                              const float (&xi0z)[NR], const float (&iez)[NR],
                                              long long nvox, int *status) {
    // segments per unrolled group: 4 loads in flight for the projector; the
    // scatter keeps 2 (fewer registers)
    constexpr int NW = MODE == 0 ? WALK : 2, NP = NR / 2;
    (void)nvox;
    (void)status;
    const unsigned zmax = (unsigned)(nz - 1);
    int zc[NR];
    float fsg[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        zc[q] = (int)min((unsigned)iz[q], zmax);
        fsg[q] = (float)sgz[q];
    }
    for (int r = r0; r < r1; r += NW) {
        float2 l0[NW][NP], l1[NW][NP];
        int a0[NW][NR], a1[NW][NR];
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const Seg S = seg[r + j - c0];  // past the round's end: padding, empty segments
            const float t1 = S.t1;
            float m[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) m[q] = fminf(tz[q], t1);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 d = __fadd2_rn(make_float2(m[2 * p], m[2 * p + 1]), make_float2(-t, -t));
                if (MASKZ) {
                    d.x = (unsigned)iz[2 * p] <= zmax ? d.x : 0.f;
                    d.y = (unsigned)iz[2 * p + 1] <= zmax ? d.y : 0.f;
                }
                l0[j][p] = d;
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) a0[j][q] = S.cb + zc[q];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                if (tz[q] < t1) {
                    iz[q] += sgz[q];
                    fz[q] += fsg[q];
                    tz[q] = (fz[q] - xi0z[q]) * iez[q];
                    zc[q] = (int)min((unsigned)iz[q], zmax);
                }
            }
            // at most one z crossing per cell: the second segment is t1 - m
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 d = __fadd2_rn(make_float2(t1, t1), make_float2(-m[2 * p], -m[2 * p + 1]));
                if (MASKZ) {
                    d.x = (unsigned)iz[2 * p] <= zmax ? d.x : 0.f;
                    d.y = (unsigned)iz[2 * p + 1] <= zmax ? d.y : 0.f;
                }
                l1[j][p] = d;
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) a1[j][q] = S.cb + zc[q];
            t = t1;
        }
        if (MODE == 0) {
            float2 v0[NW][NP], v1[NW][NP];
#pragma unroll
            for (int j = 0; j < NW; ++j)
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    v0[j][p] = make_float2(DGR_INB(a0[j][2 * p], nvox, status) ? __ldg(vol + a0[j][2 * p]) : 0.f,
                                           DGR_INB(a0[j][2 * p + 1], nvox, status) ? __ldg(vol + a0[j][2 * p + 1]) : 0.f);
                    // the second segment's voxel only after a crossing (else its length is 0)
                    v1[j][p] = make_float2(
                        l1[j][p].x != 0.f && DGR_INB(a1[j][2 * p], nvox, status) ? __ldg(vol + a1[j][2 * p]) : 0.f,
                        l1[j][p].y != 0.f && DGR_INB(a1[j][2 * p + 1], nvox, status) ? __ldg(vol + a1[j][2 * p + 1]) : 0.f);
                }
#pragma unroll
            for (int j = 0; j < NW; ++j)
#pragma unroll
                for (int p = 0; p < NP; ++p)
                    acc[p] = __ffma2_rn(l1[j][p], v1[j][p], __ffma2_rn(l0[j][p], v0[j][p], acc[p]));
        } else {
#pragma unroll
            for (int j = 0; j < NW; ++j)
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    // without a crossing the second segment is empty (q1 = 0): one
                    // reduction; integer sums do not depend on how they are split
                    const float2 w0 = __fmul2_rn(l0[j][p], wqv[p]), w1 = __fmul2_rn(l1[j][p], wqv[p]);
                    const int q0a = __float2int_rn(w0.x), q0b = __float2int_rn(w0.y);
                    const int q1a = __float2int_rn(w1.x), q1b = __float2int_rn(w1.y);
                    if (DGR_INB(a0[j][2 * p], nvox, status)) atomicAdd(acci + a0[j][2 * p], q0a);
                    if (DGR_INB(a0[j][2 * p + 1], nvox, status)) atomicAdd(acci + a0[j][2 * p + 1], q0b);
                    if (q1a != 0 && DGR_INB(a1[j][2 * p], nvox, status)) atomicAdd(acci + a1[j][2 * p], q1a);
                    if (q1b != 0 && DGR_INB(a1[j][2 * p + 1], nvox, status)) atomicAdd(acci + a1[j][2 * p + 1], q1b);
                }
        }
    }
}

// (CTAs of fewer rows: as many threads per SM as the PR_ROWS CTAs at 64 registers)
template <int MODE, int NR, int ROWS>
__global__ void __launch_bounds__(ROWS / NR, ROWS == PR_ROWS ? 0 : 8 * PR_ROWS / ROWS) k_path_n(const __grid_constant__ Batch B, RayXY *__restrict__ tab_base,
                                                         const float *__restrict__ sino_s,
                                                         const unsigned *__restrict__ view_max) {
    DEP_ENTER();
    static_assert(NR % 2 == 0 && ROWS % (32 * NR) == 0 && ROWS <= PR_ROWS, "pairs of rays, whole warps");
    constexpr int NT = ROWS / NR, NP = NR / 2;
    __shared__ Seg seg[SEG_MAX + WALK];
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    int ii = 0;
    while (ii + 1 < B.n && B.in[ii + 1].pb0 <= (int)blockIdx.x) ++ii;
    const Inst &I = B.in[ii];
    const dgr_grid &g = I.g;
    const int b = blockIdx.x - I.pb0;
    // the scatter's blocks ordered (row group, view, column): while one group
    // of detector rows is scattered for every view, the integer sums its rays
    // reach (about half of a tall volume's layers) stay in L2 (512^3: 24.6 ->
    // 22.8 ms); the projector keeps (view, row group, column)
    const int iu = b % I.nu;
    const int rg = MODE == 1 ? b / (I.nu * I.nkv) : (b / I.nu) % I.npv;
    const int k = I.kv0 + (MODE == 1 ? (b / I.nu) % I.nkv : b / (I.nu * I.npv));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const RayXY R = T.tab[I.tab0 + k * I.nu + iu];
    int iv[NR];
    RowZ row[NR];
    size_t ray[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        iv[q] = rg * ROWS + w * 32 * NR + 32 * q + lane;
        row[q] = T.rows[I.row0 + min(iv[q], I.nv - 1)];
        ray[q] = ((size_t)k * I.nv + min(iv[q], I.nv - 1)) * I.nu + iu;
    }
    // (x, y) interval of the grid and entry cell: the same for the whole CTA
    float tmin = -INFINITY, tmax = INFINITY;
    bool miss = false;
    float fx = 0.f, fy = 0.f;
    if (R.ex != 0.f) {
        const float t0 = plane_t(0, R.xi0x, R.inv_ex), t1 = plane_t(g.nx, R.xi0x, R.inv_ex);
        tmin = fmaxf(tmin, fminf(t0, t1));
        tmax = fminf(tmax, fmaxf(t0, t1));
    } else {
        fx = floorf(R.xi0x);
        miss = miss || !(fx >= 0.f && fx < (float)g.nx);
    }
    if (R.ey != 0.f) {
        const float t0 = plane_t(0, R.xi0y, R.inv_ey), t1 = plane_t(g.ny, R.xi0y, R.inv_ey);
        tmin = fmaxf(tmin, fminf(t0, t1));
        tmax = fminf(tmax, fmaxf(t0, t1));
    } else {
        fy = floorf(R.xi0y);
        miss = miss || !(fy >= 0.f && fy < (float)g.ny);
    }
    if (miss || !(tmax > tmin)) {  // CTA-uniform
        if (MODE == 0) {
#pragma unroll
            for (int q = 0; q < NR; ++q)
                if (iv[q] < I.nv) I.sino[ray[q]] = 0.f;
        }
        return;
    }
    float2 wqv[NR / 2];  // MODE 1: the rows' scaled residuals in fixed point
#pragma unroll
    for (int p = 0; p < NR / 2; ++p) wqv[p] = make_float2(0.f, 0.f);
    if (MODE == 1) {
        const float S = group_step(I, view_max, I.kv0, I.nkv);
        bool zero = true;
#pragma unroll
        for (int p = 0; p < NR / 2; ++p) {
            wqv[p].x = iv[2 * p] < I.nv ? sino_s[I.ray0 + ray[2 * p]] * S : 0.f;
            wqv[p].y = iv[2 * p + 1] < I.nv ? sino_s[I.ray0 + ray[2 * p + 1]] * S : 0.f;
            zero = zero && wqv[p].x == 0.f && wqv[p].y == 0.f;
        }
        if (__syncthreads_and(zero)) return;  // nothing to add (or a bad group)
    }
    const PathXY P = xy_path(R, I, tmin, fx, fy);
    const int nseg = P.nseg;
    // each ray's z: entry layer (unbounded), next crossing, whether it stays in the z range
    int iz[NR], sgz[NR];
    float tz[NR], fz[NR], xi0z[NR], iez[NR];
    bool out = false;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const RayZ Z = ray_z(R, row[q], I.zoff);
        xi0z[q] = Z.xi0z;
        iez[q] = Z.inv_ez;
        sgz[q] = 0;
        tz[q] = INFINITY;
        fz[q] = 0.f;
        bool zin;
        if (Z.ez != 0.f) {
            sgz[q] = Z.ez > 0.f ? 1 : -1;
            const float t0 = plane_t(0, Z.xi0z, Z.inv_ez), t1 = plane_t(g.nz, Z.xi0z, Z.inv_ez);
            zin = fminf(t0, t1) <= tmin && fmaxf(t0, t1) >= tmax;
            iz[q] = entry_cell(tmin, Z.ez, Z.xi0z, Z.inv_ez, sgz[q], INT_MIN / 2, INT_MAX / 2);
            fz[q] = (float)(sgz[q] > 0 ? iz[q] + 1 : iz[q]);
            tz[q] = (fz[q] - Z.xi0z) * Z.inv_ez;
        } else {
            const float f = floorf(Z.xi0z);
            zin = f >= 0.f && f < (float)g.nz;
            iz[q] = zin ? (int)f : -1;
        }
        out = out || !zin;
    }
    const bool masked = __any_sync(0xffffffffu, out);
    float t = tmin;
    float2 acc[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = make_float2(0.f, 0.f);
    // a warp whose rows all lie past the detector (nv not a multiple of the
    // CTA's rows) only takes part in the staging
    for (int c0 = 0; c0 < nseg; c0 += SEG_MAX) {
        const int c1 = min(nseg, c0 + SEG_MAX);
        stage_segs<NT>(seg, P, R, I, c0, c1);
        if (MODE == 1 && c1 == nseg) {  // no barrier follows the last staging
            const int b1 = blockIdx.x - I.pb0;
            const int rg1 = MODE == 1 ? b1 / (I.nu * I.nkv) : (b1 / I.nu) % I.npv;
            if (rg1 * ROWS + (int)(threadIdx.x >> 5) * 32 * NR >= I.nv) return;
        }
        if (masked)
            walk_segs1_xn<MODE, true, NR>(I.vol, I.acc, wqv, seg, c0, c0, c1, g.nz, t, acc, iz, fz, tz, sgz, xi0z, iez,
                                          (long long)g.nx * g.ny * g.nz, B.status);
        else
            walk_segs1_xn<MODE, false, NR>(I.vol, I.acc, wqv, seg, c0, c0, c1, g.nz, t, acc, iz, fz, tz, sgz, xi0z, iez,
                                           (long long)g.nx * g.ny * g.nz, B.status);
    }
    if (MODE == 0) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (iv[2 * p] < I.nv) I.sino[ray[2 * p]] = acc[p].x * ray_norm(R, row[2 * p], I.beam);
            if (iv[2 * p + 1] < I.nv) I.sino[ray[2 * p + 1]] = acc[p].y * ray_norm(R, row[2 * p + 1], I.beam);
        }
    }
}

// a6, last step of the ray-driven backprojector: after a group of views, the
// integer sums (z fastest) are scaled by the group's fixed-point step and
// added to the FP32 gradient ([nz][ny][nx]; the first group writes it), then
// cleared.  A 32 x 32 (x, z) tile at one y goes through shared memory so both
// sides are coalesced.  blockIdx.x: global tile of the instances in the group.
__global__ void k_bp_fold(const __grid_constant__ Batch B, const unsigned *__restrict__ view_max) {
    DEP_ENTER();
    __shared__ float tile[32][33];
    int ii = 0;
    while (ii + 1 < B.n && B.in[ii + 1].fb0 <= (int)blockIdx.x) ++ii;
    const Inst &I = B.in[ii];
    if (I.nkv <= 0) return;
    const dgr_grid &g = I.g;
    const int ntx = (g.nx + 31) / 32, nty = (g.ny + FOLD_Y - 1) / FOLD_Y, ntz = (g.nz + 31) / 32;
    const int b = blockIdx.x - I.fb0;
    const int bx = b % ntx, by = (b / ntx) % nty, bzt = b / (ntx * nty);
    if (bzt >= ntz) return;
    const float S = group_step(I, view_max, I.kv0, I.nkv);
    const float inv_s = S > 0.f ? 1.f / S : 0.f;  // a power of two: exact
    const int x0 = bx * 32, z0 = bzt * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int y = by * FOLD_Y; y < min(g.ny, (by + 1) * FOLD_Y); ++y) {  // CTA-uniform
        __syncthreads();  // the previous row's readers of the tile are done
        for (int j = ty; j < 32; j += 8) {  // read along z
            const int x = x0 + j, z = z0 + tx;
            if (x < g.nx && z < g.nz) {
                int *p = I.acc + ((size_t)x * g.ny + y) * g.nz + z;
                tile[j][tx] = S > 0.f ? (float)*p * inv_s : NAN;
                *p = 0;
            }
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {  // write along x
            const int z = z0 + j, x = x0 + tx;
            if (x < g.nx && z < g.nz) {
                float *q = I.gvol + ((size_t)z * g.ny + y) * g.nx + x;
                *q = I.kv0 == 0 ? tile[tx][j] : *q + tile[tx][j];
            }
        }
    }
}

// a4 (per-ray projector, for volumes in the C ABI's x-fastest layout when no
// z-fastest copy can be made): one thread per global ray, incremental Siddon
// walk; u-adjacent rays in a warp read neighbouring voxels.
__global__ void __launch_bounds__(128) k_project_ray(const __grid_constant__ Batch B,
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

// x-fastest [nz][ny][nx] -> z-fastest [nx][ny][nz] copy through a 32 x 32
// shared tile (both sides coalesced); blockIdx: (x tile, y, z tile)
__global__ void k_vol_zfast(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny,
                            int nz) {
    __shared__ float tile[32][33];
    const int x0 = blockIdx.x * 32, y = blockIdx.y, z0 = blockIdx.z * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int z = z0 + j, x = x0 + tx;
        if (z < nz && x < nx) tile[j][tx] = src[((size_t)z * ny + y) * nx + x];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int x = x0 + j, z = z0 + tx;
        if (x < nx && z < nz) dst[((size_t)x * ny + y) * nz + z] = tile[tx][j];
    }
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
        if (x < g.nx && z < g.nz) I.gvol[(size_t)z * zs + (size_t)iy * g.nx + x] = out_tile[zz][xx];
    }
}

// residual x |D| per ray, natural layout ([view][v][u]), for the brick
// backprojector, and the largest |residual x |D|| of every view (for its
// fixed-point step).  blockIdx.y: global view; blockIdx.x: 256 rays of it.
__global__ void k_scale_dn(const __grid_constant__ Batch B, RayXY *__restrict__ tab_base,
                           float *__restrict__ out_base, unsigned *__restrict__ view_max) {
    DEP_ENTER();
    __shared__ unsigned s_m;
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    const int vg = blockIdx.y;
    const Inst &I = B.in[inst_of_view(B, vg)];
    const int k = vg - I.view0;
    const int per = I.nu * I.nv;
    if (threadIdx.x == 0) s_m = 0u;
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;  // ray within the view
    unsigned m = 0u;
    if (r < per) {
        const int iu = r % I.nu, iv = r / I.nu;
        const long long ri = (long long)k * per + r;
        const float v = I.sino[ri] * ray_norm(T.tab[I.tab0 + k * I.nu + iu], T.rows[I.row0 + iv], I.beam);
        out_base[I.ray0 + ri] = v;
        const float a = fabsf(v);
        m = a != a ? 0x7fffffffu : __float_as_uint(a);  // NaN: the largest code
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_m, m);
    __syncthreads();
    if (threadIdx.x == 0 && s_m) atomicMax(view_max + vg, s_m);
}

// a6 (brick scatter): a CTA owns a BBX x BBY x BBZ brick of one instance and
// keeps its sums in shared memory.  Views go in groups of VGROUP.  For each
// view the detector columns and rows whose pixels fall in the bounding box of
// the brick's projected corners are the candidates; a work item is one
// (view, column) pair: the warp walks the column's (x, y) path through the
// brick (warp-uniform, the same plane crossings as k_project, hence the same
// chord lengths) carrying SLOTS groups of 32 consecutive rows per lane, and
// adds each segment's length x scaled residual into the brick with a
// shared-memory integer atomic, in fixed point.  Integer sums do not depend on
// the order of the additions, so all items of a group run concurrently and
// the result is still bit-reproducible.  The fixed-point step of a group is a
// power of two chosen from the largest residual of the group's views
// and a bound on the contributions a voxel can receive (VGROUP views x
// col_u x col_v rays per view, each at most the longest chord in t units x
// |residual|), so no sum can overflow; after a group, the integer sums are
// added, in a fixed order, into FP32 sums.  blockIdx.x: global brick.
constexpr int BBX = 8, BBY = 8, BBZ = 88;
constexpr int BBV = BBX * BBY * BBZ;
constexpr int BB_THREADS = 256;
constexpr int SLOTS = 3;

__global__ void __launch_bounds__(BB_THREADS) k_bp_brick(const __grid_constant__ Batch B,
                                                          RayXY *__restrict__ tab_base,
                                                          const float *__restrict__ sino_s,
                                                          const unsigned *__restrict__ view_max) {
    extern __shared__ float accf[];          // [BBY][BBX][BBZ] FP32 sums
    int *acci = reinterpret_cast<int *>(accf + BBV);  // the group's fixed-point sums
    __shared__ int s_rng[VGROUP][4];         // iu0, iu1, iv0, iv1 of each view of the group
    __shared__ int s_cum[VGROUP + 1];        // items before each view
    const Tables T = tables_of(tab_base, B.tot_tab, B.tot_views);
    int ii = 0;
    while (ii + 1 < B.n && B.in[ii + 1].bb0 <= (int)blockIdx.x) ++ii;
    const Inst &I = B.in[ii];
    const dgr_grid &g = I.g;
    const int b = blockIdx.x - I.bb0;
    const int bx = b % I.nbbx, by = (b / I.nbbx) % I.nbby, bz = b / (I.nbbx * I.nbby);
    const int x0 = bx * BBX, y0 = by * BBY, z0 = bz * BBZ;
    const int x1 = min(x0 + BBX, g.nx), y1 = min(y0 + BBY, g.ny), z1 = min(z0 + BBZ, g.nz);
    for (int i = threadIdx.x; i < BBV; i += BB_THREADS) {
        accf[i] = 0.f;
        acci[i] = 0;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const RayXY *__restrict__ tab = T.tab + I.tab0;
    const float2 *__restrict__ view_cs = T.view_cs + I.view0;
    const RowZ *__restrict__ rows = T.rows + I.row0;
    const float *__restrict__ sview0 = sino_s + I.ray0;
    const bool cone = I.beam == DGR_CONE;
    const float h = g.h;
    const float cu = 0.5f * (float)(I.nu - 1), cv = 0.5f * (float)(I.nv - 1);
    const float wx0 = g.ox + x0 * h, wx1 = g.ox + x1 * h, wy0 = g.oy + y0 * h, wy1 = g.oy + y1 * h;
    const float wz0 = g.oz + z0 * h, wz1 = g.oz + z1 * h;
    const int nzb = z1 - z0;
    bool bad = false;  // a non-finite residual: the brick becomes NaN
    for (int kg = 0; kg < I.n_views; kg += VGROUP) {
        const int nvw = min(VGROUP, I.n_views - kg);
        if (threadIdx.x < nvw) {
            const float2 cs = view_cs[kg + threadIdx.x];
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
            s_rng[threadIdx.x][0] = iu0;
            s_rng[threadIdx.x][1] = iu1;
            s_rng[threadIdx.x][2] = iv0;
            s_rng[threadIdx.x][3] = (iv1 >= iv0 && iu1 >= iu0) ? iv1 : iv0 - 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int c = 0;
            for (int j = 0; j < nvw; ++j) {
                s_cum[j] = c;
                c += s_rng[j][3] >= s_rng[j][2] ? s_rng[j][1] - s_rng[j][0] + 1 : 0;
            }
            s_cum[nvw] = c;
        }
        __syncthreads();
        // the group's fixed-point step (0: a non-finite residual)
        const float S = group_step(I, view_max, kg, nvw);
        bad = bad || S == 0.f;
        const int nitems = s_cum[nvw];
        for (int item = w; item < nitems; item += BB_THREADS / 32) {  // warp-uniform
            int j = 0;
            while (j + 1 < nvw && s_cum[j + 1] <= item) ++j;
            const int k = kg + j;
            const int iu = s_rng[j][0] + item - s_cum[j];
            const int iv0 = s_rng[j][2], iv1 = s_rng[j][3];
            const RayXY R = tab[k * I.nu + iu];
            // the brick's (x, y) box along this column's path (uniform)
            float tmin = -INFINITY, tmax = INFINITY;
            bool miss = false;
            float fx = 0.f, fy = 0.f;
            if (R.ex != 0.f) {
                const float ta = plane_t(x0, R.xi0x, R.inv_ex), tb = plane_t(x1, R.xi0x, R.inv_ex);
                tmin = fmaxf(tmin, fminf(ta, tb));
                tmax = fminf(tmax, fmaxf(ta, tb));
            } else {
                fx = floorf(R.xi0x);
                miss = miss || !(fx >= (float)x0 && fx < (float)x1);
            }
            if (R.ey != 0.f) {
                const float ta = plane_t(y0, R.xi0y, R.inv_ey), tb = plane_t(y1, R.xi0y, R.inv_ey);
                tmin = fmaxf(tmin, fminf(ta, tb));
                tmax = fminf(tmax, fmaxf(ta, tb));
            } else {
                fy = floorf(R.xi0y);
                miss = miss || !(fy >= (float)y0 && fy < (float)y1);
            }
            if (miss || !(tmax > tmin)) continue;
            const int sgx = R.ex > 0.f ? 1 : (R.ex < 0.f ? -1 : 0);
            const int sgy = R.ey > 0.f ? 1 : (R.ey < 0.f ? -1 : 0);
            const int ixe = sgx ? entry_cell(tmin, R.ex, R.xi0x, R.inv_ex, sgx, x0, x1 - 1) : (int)fx;
            const int iye = sgy ? entry_cell(tmin, R.ey, R.xi0y, R.inv_ey, sgy, y0, y1 - 1) : (int)fy;
            const int dcx = sgx * BBZ, dcy = sgy * BBX * BBZ;  // cell steps in shared memory
            const float *sv = sview0 + (size_t)k * I.nv * I.nu + iu;
            for (int r0 = iv0; r0 <= iv1; r0 += 32 * SLOTS) {
                // per lane and slot: row, scaled residual x S, z entry layer
                // (unbounded, brick-local), next z crossing
                int iz[SLOTS], sgz[SLOTS], lim[SLOTS];
                float tz[SLOTS], fz[SLOTS], fsg[SLOTS], xz[SLOTS], iez[SLOTS], wq[SLOTS];
#pragma unroll
                for (int s = 0; s < SLOTS; ++s) {
                    const int iv = r0 + 32 * s + lane;
                    const bool act = iv <= iv1;
                    const RowZ row = rows[act ? iv : iv0];
                    const RayZ Z = ray_z(R, row, I.zoff);
                    const float wr = act ? sv[(size_t)iv * I.nu] : 0.f;
                    wq[s] = wr * S;
                    lim[s] = (act && wr != 0.f) ? nzb : 0;  // brick-local zl < lim: add
                    xz[s] = Z.xi0z;
                    iez[s] = Z.inv_ez;
                    tz[s] = INFINITY;
                    fz[s] = 0.f;
                    sgz[s] = 0;
                    fsg[s] = 0.f;
                    if (Z.ez != 0.f) {
                        sgz[s] = Z.ez > 0.f ? 1 : -1;
                        fsg[s] = (float)sgz[s];
                        iz[s] = entry_cell(tmin, Z.ez, Z.xi0z, Z.inv_ez, sgz[s], INT_MIN / 2, INT_MAX / 2);
                        fz[s] = (float)(sgz[s] > 0 ? iz[s] + 1 : iz[s]);
                        tz[s] = (fz[s] - Z.xi0z) * Z.inv_ez;
                    } else {
                        iz[s] = (int)fmaxf(fminf(floorf(Z.xi0z), (float)(INT_MAX / 2)), (float)(INT_MIN / 2));
                    }
                    iz[s] -= z0;
                }
                int ix = ixe, iy = iye;
                float tx = sgx ? plane_t(sgx > 0 ? ix + 1 : ix, R.xi0x, R.inv_ex) : INFINITY;
                float ty = sgy ? plane_t(sgy > 0 ? iy + 1 : iy, R.xi0y, R.inv_ey) : INFINITY;
                int cell = ((iy - y0) * BBX + (ix - x0)) * BBZ;
                float t = tmin;
                for (int it = 0; it < BBX + BBY + 2; ++it) {
                    const float t1 = fminf(tx, ty);
#pragma unroll
                    for (int s = 0; s < SLOTS; ++s) {
                        const float m = fminf(tz[s], t1);
                        const int q0 = __float2int_rn((m - t) * wq[s]);
                        if ((unsigned)iz[s] < (unsigned)lim[s]) atomicAdd(acci + cell + iz[s], q0);
                        if (tz[s] < t1) {  // a z plane inside this cell
                            float ts = tz[s];
                            iz[s] += sgz[s];
                            fz[s] += fsg[s];
                            tz[s] = (fz[s] - xz[s]) * iez[s];
                            const int q1 = __float2int_rn((fminf(tz[s], t1) - ts) * wq[s]);
                            if ((unsigned)iz[s] < (unsigned)lim[s]) atomicAdd(acci + cell + iz[s], q1);
                            // rare: further planes in the same cell (bounded)
                            for (int rep = 0; rep <= nzb && tz[s] < t1; ++rep) {
                                ts = tz[s];
                                iz[s] += sgz[s];
                                fz[s] += fsg[s];
                                tz[s] = (fz[s] - xz[s]) * iez[s];
                                if ((unsigned)iz[s] < (unsigned)lim[s])
                                    atomicAdd(acci + cell + iz[s], __float2int_rn((fminf(tz[s], t1) - ts) * wq[s]));
                            }
                        }
                    }
                    t = t1;
                    if (tx <= ty) {
                        const int ni = ix + sgx;
                        if (ni < x0 || ni >= x1) break;
                        ix = ni;
                        cell += dcx;
                        tx = plane_t(ni + (sgx > 0), R.xi0x, R.inv_ex);
                    } else {
                        const int ni = iy + sgy;
                        if (ni < y0 || ni >= y1) break;
                        iy = ni;
                        cell += dcy;
                        ty = plane_t(ni + (sgy > 0), R.xi0y, R.inv_ey);
                    }
                }
            }
        }
        __syncthreads();
        // the group's integer sums into the FP32 sums (each voxel by one thread)
        const float inv_s = S > 0.f ? 1.f / S : 0.f;  // a power of two: exact
        for (int i = threadIdx.x; i < BBV; i += BB_THREADS) {
            accf[i] += (float)acci[i] * inv_s;
            acci[i] = 0;
        }
        // s_rng and s_cum are rewritten by the next group after its first barrier
        __syncthreads();
    }
    // write the brick (x fastest)
    for (int i = threadIdx.x; i < BBX * BBY * BBZ; i += BB_THREADS) {
        const int xx = i % BBX, yy = (i / BBX) % BBY, zz = i / (BBX * BBY);
        const int x = x0 + xx, y = y0 + yy, z = z0 + zz;
        if (x < x1 && y < y1 && z < z1)
            I.gvol[((size_t)z * g.ny + y) * g.nx + x] = bad ? NAN : accf[(yy * BBX + xx) * BBZ + zz];
    }
}

}  // namespace

size_t ray_table_bytes(long long n_tab, long long n_views, long long n_rows) {
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
// The bound depends on the grid and the geometry's scalars only (every angle
// of the full circle is sampled): cached for the last few (grid, geometry)
// pairs, so an iteration does not redo the 72 x 125 x 8 corner projections.
static void bp_colours_compute(const dgr_grid &g, const dgr_geom &geo, int &cu, int &cv);
void bp_colours(const dgr_grid &g, const dgr_geom &geo, int &cu, int &cv) {
    struct Entry {
        dgr_grid g;
        int beam, nu, nv;
        float pu, pv, dso, dsd;
        int cu, cv;
    };
    static std::mutex mu;
    static Entry cache[32];
    static int next = 0, used = 0;
    auto same = [&](const Entry &e) {
        return memcmp(&e.g, &g, sizeof(dgr_grid)) == 0 && e.beam == geo.beam && e.nu == geo.nu &&
               e.nv == geo.nv && e.pu == geo.pu && e.pv == geo.pv && e.dso == geo.dso && e.dsd == geo.dsd;
    };
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < used; ++i)
            if (same(cache[i])) {
                cu = cache[i].cu;
                cv = cache[i].cv;
                return;
            }
    }
    bp_colours_compute(g, geo, cu, cv);
    std::lock_guard<std::mutex> lock(mu);
    Entry e{};
    e.g = g;
    e.beam = geo.beam; e.nu = geo.nu; e.nv = geo.nv;
    e.pu = geo.pu; e.pv = geo.pv; e.dso = geo.dso; e.dsd = geo.dsd;
    e.cu = cu; e.cv = cv;
    cache[next] = e;
    next = (next + 1) % 32;
    if (used < 32) ++used;
}

static void bp_colours_compute(const dgr_grid &g, const dgr_geom &geo, int &cu, int &cv) {
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

// Whether a ray may cross two z planes inside one (x, y) cell: the z change
// over a cell is at most sqrt(2) |e_z| / |e_xy|, and |e_z| / |e_xy| <=
// v_max / dsd for the cone (|D_xy| >= dsd), 0 for parallel beams.
int multi_z(const dgr_geom &geo) {
    if (geo.beam != DGR_CONE) return 0;
    const double vmax = 0.5 * (geo.nv - 1) * (double)geo.pv;
    return 1.4142135623730951 * vmax / (double)geo.dsd > 0.9 ? 1 : 0;
}

static int g_bp_variant = 0;  // 0: ray scatter, 1: column gather, 2: brick scatter
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
    launch_dep(k_ray_tables, dim3((m + 127) / 128), dim3(128), 0, st, B, tab);
    counted(1);
    return cudaGetLastError();
}

static int g_staged = 0;  // measured slower than the direct walk (see the header)
void set_staged_walk(int on) { g_staged = on ? 1 : 0; }

// The staged (bulk-copy) path walk: every volume z fastest with nz a multiple
// of 4 (16-byte copies), columns of at most 4096 words.  Sets the batch's
// stage geometry; returns the dynamic shared memory (0: unstaged walk).
static int staging(Batch &B, int *status) {
    if (!g_staged || !status) return 0;
    int zc = 4;
    for (int i = 0; i < B.n; ++i) {
        const dgr_grid &g = B.in[i].g;
        if (B.in[i].vsz != 1 || (g.nz & 3) != 0) return 0;
        zc = max(zc, g.nz);
    }
    if (zc > 4096) return 0;
    const int ch = max(4, min(32, 32768 / (2 * zc * 4)));
    B.tma_ch = ch;
    B.tma_zcap = zc;
    B.status = status;
    const int smem = 2 * ch * zc * (int)sizeof(float);  // at most 2 x 4 x 4096 words
    static int attr = 0;  // 0: not tried, 1: set, -1: refused (stay unstaged above 48 KB)
    if (attr == 0) {
        const int most = 2 * 4 * 4096 * (int)sizeof(float);
        const bool ok = cudaFuncSetAttribute(k_path<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most) ==
                            cudaSuccess &&
                        cudaFuncSetAttribute(k_path<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most) ==
                            cudaSuccess;
        if (!ok) cudaGetLastError();  // clear it: the launch below stays within the default
        attr = ok ? 1 : -1;
    }
    if (attr < 0 && smem > 48 * 1024) return 0;
    return smem;
}

static bool multi_crossing(const Batch &B) {
    for (int i = 0; i < B.n; ++i)
        if (B.in[i].multiz) return true;
    return false;
}

// detector rows per CTA of an instance's path walks: the two-ray walk
// (single-crossing geometries, unstaged) takes CTAs of 64 or 128 rows for
// detectors no taller, so short detectors do not leave half or three quarters
// of a 256-row CTA idle; 256 otherwise, and for every instance when full
// (staged walks, or a multi-crossing geometry in the batch: the one-ray walk)
static int inst_rows(const Inst &I, bool full) {
    if (full) return PR_ROWS;
    return I.nv <= 64 ? 64 : (I.nv <= 128 ? 128 : PR_ROWS);
}
constexpr int ROW_CLASSES[3] = {64, 128, PR_ROWS};

// one launch of the walk over the blocks of the instances of one row class
template <int MODE>
static void launch_walk(const Batch &B, int rows, int pb, int smem, bool full, RayXY *tab, const float *sino_s,
                        const unsigned *view_max, cudaStream_t st) {
    if (smem > 0)
        launch_dep(k_path<MODE, true>, dim3(pb), dim3(PR_THREADS), smem, st, B, tab, sino_s, view_max);
    else if (full)
        launch_dep(k_path<MODE, false>, dim3(pb), dim3(PR_THREADS), 0, st, B, tab, sino_s, view_max);
    else if (rows == PR_ROWS)
        launch_dep(k_path_n<MODE, PR_NR, PR_ROWS>, dim3(pb), dim3(PR_ROWS / PR_NR), 0, st, B, tab, sino_s, view_max);
    else if (rows == 128)
        launch_dep(k_path_n<MODE, PR_NR, 128>, dim3(pb), dim3(128 / PR_NR), 0, st, B, tab, sino_s, view_max);
    else
        launch_dep(k_path_n<MODE, PR_NR, 64>, dim3(pb), dim3(64 / PR_NR), 0, st, B, tab, sino_s, view_max);
    counted(1);
}

cudaError_t launch_project(const Batch &B0, const RayXY *tab, int *status, cudaStream_t st,
                           const cudaEvent_t *kev) {
    // row-warp projector when every volume is z fastest, else per-ray
    bool zfast = B0.n > 0;
    for (int i = 0; i < B0.n; ++i) zfast = zfast && B0.in[i].vsz == 1;
    if (!zfast) {
        const long long blocks = (B0.tot_rays + 127) / 128;
        if (blocks == 0) return cudaSuccess;
        if (kev) cudaEventRecord(kev[0], st);
        k_project_ray<<<(unsigned)blocks, 128, 0, st>>>(B0, const_cast<RayXY *>(tab));
        counted(1);
        if (kev) cudaEventRecord(kev[1], st);
        return cudaGetLastError();
    }
    // projector blocks: one detector column x `rows` rows of one view; one
    // launch per row class present (a batch of short and tall detectors)
    static thread_local Batch B;
    B = B0;
    const int smem = staging(B, status);
    const bool full = smem > 0 || multi_crossing(B);
    if (kev) cudaEventRecord(kev[0], st);
    for (const int rows : ROW_CLASSES) {
        int pb = 0;
        for (int i = 0; i < B.n; ++i) {
            Inst &I = B.in[i];
            I.npv = inst_rows(I, full) == rows ? (I.nv + rows - 1) / rows : 0;
            I.pb0 = pb;
            I.kv0 = 0;
            I.nkv = I.n_views;
            pb += I.n_views * I.nu * I.npv;
        }
        if (pb > 0) launch_walk<0>(B, rows, pb, smem, full, const_cast<RayXY *>(tab), nullptr, nullptr, st);
    }
    if (kev) cudaEventRecord(kev[1], st);
    return cudaGetLastError();
}

cudaError_t launch_vol_zfast(const dgr_grid &g, const float *src, float *dst, cudaStream_t st) {
    dim3 grid((g.nx + 31) / 32, g.ny, (g.nz + 31) / 32);
    k_vol_zfast<<<grid, 256, 0, st>>>(src, dst, g.nx, g.ny, g.nz);
    counted(1);
    return cudaGetLastError();
}

// ray-driven backprojector: per group of VGROUP views, the scatter and the fold
// kev: [0] before the first group's scatter, [1] after the last group's
// scatter (with several groups the folds in between fall inside)
static cudaError_t launch_bp_scatter(const Batch &B0, const RayXY *tab, const float *sino_scaled,
                                     const unsigned *view_max, int *acc, int *status, cudaStream_t st,
                                     const cudaEvent_t *kev) {
    static thread_local Batch B;
    B = B0;
    const int smem = staging(B, status);
    const bool full = smem > 0 || multi_crossing(B);
    int ngroups = 0;
    long long ao = 0;
    for (int i = 0; i < B.n; ++i) {
        Inst &I = B.in[i];
        ngroups = max(ngroups, (I.n_views + VGROUP - 1) / VGROUP);
        I.acc = acc + ao;  // z fastest, instances on 64-int boundaries
        ao += ((long long)I.g.nx * I.g.ny * I.g.nz + 63) / 64 * 64;
        I.vsz = 1;
        I.vsy = I.g.nz;
        I.vsx = I.g.ny * I.g.nz;
    }
    bool first = true;
    for (int gi = 0; gi < ngroups; ++gi) {
        int fb = 0;
        for (int i = 0; i < B.n; ++i) {
            Inst &I = B.in[i];
            I.kv0 = gi * VGROUP;
            I.nkv = max(0, min(VGROUP, I.n_views - I.kv0));
            I.fb0 = fb;
            if (I.nkv > 0) fb += ((I.g.nx + 31) / 32) * ((I.g.ny + FOLD_Y - 1) / FOLD_Y) * ((I.g.nz + 31) / 32);
        }
        // the group's scatter: one launch per row class present
        for (const int rows : ROW_CLASSES) {
            int pb = 0;
            for (int i = 0; i < B.n; ++i) {
                Inst &I = B.in[i];
                I.npv = inst_rows(I, full) == rows ? (I.nv + rows - 1) / rows : 0;
                I.pb0 = pb;
                pb += I.nkv * I.nu * I.npv;
            }
            if (pb == 0) continue;
            if (kev && first) cudaEventRecord(kev[0], st);
            first = false;
            launch_walk<1>(B, rows, pb, smem, full, const_cast<RayXY *>(tab), sino_scaled, view_max, st);
            if (kev) cudaEventRecord(kev[1], st);
        }
        if (fb > 0) {
            launch_dep(k_bp_fold, dim3(fb), dim3(256), 0, st, B, view_max);
            counted(1);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_backproject(const Batch &B, const RayXY *tab, float *sino_scaled, int *acc,
                               long long acc_vox, int *status, cudaStream_t st, const cudaEvent_t *kev) {
    long long vox = 0;
    for (int i = 0; i < B.n; ++i) vox += (long long)B.in[i].g.nx * B.in[i].g.ny * B.in[i].g.nz;
    // the ray scatter (0) needs the workspace's integer sums; without them, the brick scatter (2)
    const int variant = (g_bp_variant == 0 && acc_vox < vox) ? 2 : g_bp_variant;
    if (variant == 0 || variant == 2) {
        unsigned *view_max = reinterpret_cast<unsigned *>(sino_scaled + (B.tot_rays + 63) / 64 * 64);
        cudaError_t e = cudaMemsetAsync(view_max, 0, sizeof(unsigned) * B.tot_views, st);
        if (e != cudaSuccess) return e;
        int max_per = 1;
        for (int i = 0; i < B.n; ++i) max_per = max(max_per, B.in[i].nu * B.in[i].nv);
        launch_dep(k_scale_dn, dim3((max_per + 255) / 256, B.tot_views), dim3(256), 0, st, B, const_cast<RayXY *>(tab),
                                                                           sino_scaled, view_max);
        counted(1);
        if (variant == 0) return launch_bp_scatter(B, tab, sino_scaled, view_max, acc, status, st, kev);
        const int smem = 2 * BBV * (int)sizeof(float);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_bp_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            attr = true;
        }
        if (kev) cudaEventRecord(kev[0], st);
        k_bp_brick<<<B.tot_bricks, BB_THREADS, smem, st>>>(B, const_cast<RayXY *>(tab), sino_scaled,
                                                           view_max);
        counted(1);
        if (kev) cudaEventRecord(kev[1], st);
        return cudaGetLastError();
    }
    int max_u = 1, max_v = 1;
    for (int i = 0; i < B.n; ++i) {
        max_u = B.in[i].nu > max_u ? B.in[i].nu : max_u;
        max_v = B.in[i].nv > max_v ? B.in[i].nv : max_v;
    }
    dim3 tgrid((max_u + TR - 1) / TR, (max_v + TR - 1) / TR, B.tot_views);
    k_scale_dn_t<<<tgrid, 256, 0, st>>>(B, const_cast<RayXY *>(tab), sino_scaled);
    if (kev) cudaEventRecord(kev[0], st);
    k_backproject<<<B.tot_blk, 32 * BP_W, 0, st>>>(B, const_cast<RayXY *>(tab), sino_scaled);
    if (kev) cudaEventRecord(kev[1], st);
    counted(2);
    return cudaGetLastError();
}

size_t ray_table_bytes_single(const dgr_geom &geo) {
    return ray_table_bytes((long long)geo.n_views * geo.nu, geo.n_views, geo.nv);
}

cudaError_t launch_project_single(const dgr_grid &g, const dgr_geom &geo, RayXY *tab,
                                  const float *vol, float *sino, cudaStream_t st) {
    static thread_local Batch B;
    memset(&B, 0, sizeof(B));
    B.n = 1;
    Inst &I = B.in[0];
    I.g = g;
    I.g.oz = slab_origin(g);  // a z-slab: an ordinary grid at its first layer
    I.g.z0 = 0;
    I.zoff = -I.g.oz / g.h;
    I.beam = geo.beam; I.n_views = geo.n_views; I.nu = geo.nu; I.nv = geo.nv;
    I.pu = geo.pu; I.pv = geo.pv; I.dso = geo.dso; I.dsd = geo.dsd; I.angles = geo.angles;
    I.vol = const_cast<float *>(vol);
    I.vsx = 1;
    I.vsy = g.nx;
    I.vsz = g.nx * g.ny;
    I.multiz = 1;
    I.sino = sino;
    B.tot_tab = geo.n_views * geo.nu;
    B.tot_views = geo.n_views;
    B.tot_rows = geo.nv;
    B.tot_rays = (long long)geo.n_views * geo.nu * geo.nv;
    cudaError_t e = launch_ray_tables(B, tab, st);
    if (e == cudaSuccess) e = launch_project(B, tab, nullptr, st);
    return e;
}

}  // namespace dgr
