// Fast Volume Reconstruction forward on sm_103a.
//
//   a1  k_prep          per Gaussian: footprint integers (fixed FP32 op
//                       sequence), anchor, delta = u - a, scaled precision A'
//   a2  k_tile_count /  binning: per-tile Gaussian counts, exclusive scan,
//       k_tile_fill /   fill of the (tile, Gaussian) work list, sort of each
//       k_tile_sort     tile's list by Gaussian index (deterministic order)
//   a3  k_voxelize      one CTA per 8x16x32 tile: prep records staged in shared
//                       memory, chunk sums in registers, running sums in
//                       shared memory, one ex2 per in-box pair
//
// The paper (Sec. 4.2, Algorithm 1) materialises a [n, 17, 17, 17]
// contribution tensor and scatter_adds it with global atomics; here nothing
// per pair is stored and every voxel is written once by the CTA owning it.
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

// ---------------------------------------------------------------------------
// footprint integers: the fixed FP32 sequence (every operation rounded on
// its own; no contraction) shared with the CPU oracle by specification only
// ---------------------------------------------------------------------------
struct Foot {
    float R[9];  // rotation of the normalised quaternion (FP32)
    int an[3], lo[3], hi[3];
};

__device__ __forceinline__ void rot_f32_exact(float w, float x, float y, float z, float *R) {
    float n2 = __fmul_rn(w, w);
    n2 = __fadd_rn(n2, __fmul_rn(x, x));
    n2 = __fadd_rn(n2, __fmul_rn(y, y));
    n2 = __fadd_rn(n2, __fmul_rn(z, z));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    w = __fmul_rn(w, inv); x = __fmul_rn(x, inv); y = __fmul_rn(y, inv); z = __fmul_rn(z, inv);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    R[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    R[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    R[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    R[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    R[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    R[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    R[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    R[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    R[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
}

// g.oz is the whole grid's z origin and g.z0 the first layer of the slab g
// describes: the integers are taken in the whole grid's frame, then the z axis
// is shifted to the slab's layers and clipped to them
__device__ __forceinline__ void footprint_f32(const dgr_grid &g, const float *mu, const float *s,
                                              const float4 q, float k, Foot &F) {
    rot_f32_exact(q.x, q.y, q.z, q.w, F.R);
    const int dims[3] = {g.nx, g.ny, g.nz};
    const float org[3] = {g.ox, g.oy, g.oz};
    bool far = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = __fdiv_rn(__fsub_rn(mu[a], org[a]), g.h);
        u = __fsub_rn(u, 0.5f);
        // |u| >= 2^24 voxels: the Gaussian is treated as outside the grid
        if (!(fabsf(u) < 16777216.0f)) { far = true; u = 0.0f; }
        const int an = (int)floorf(u);
        int lo, hi;
        if (k > 0.0f) {
            const float t0 = __fmul_rn(F.R[3 * a + 0], s[0]);
            const float t1 = __fmul_rn(F.R[3 * a + 1], s[1]);
            const float t2 = __fmul_rn(F.R[3 * a + 2], s[2]);
            float var = __fmul_rn(t0, t0);
            var = __fadd_rn(var, __fmul_rn(t1, t1));
            var = __fadd_rn(var, __fmul_rn(t2, t2));
            const float sig = __fdiv_rn(__fsqrt_rn(var), g.h);
            const float kr = __fmul_rn(k, sig);
            // a radius beyond the grid only needs to cover the grid
            const int rad = kr < 65536.0f ? (int)ceilf(kr) : 65536;
            lo = an - rad;
            hi = an + rad + 1;
        } else {
            const int K = (int)(-k);
            const int half = (K - 1) / 2;
            lo = an - half;
            hi = an + half;
        }
        const int sh = a == 2 ? g.z0 : 0;
        lo = max(lo - sh, 0);
        hi = min(hi - sh, dims[a] - 1);
        F.an[a] = an - sh;
        F.lo[a] = lo;
        F.hi[a] = hi;
    }
    if (far) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { F.lo[a] = 1; F.hi[a] = 0; }
    }
}

__device__ __forceinline__ bool finite3(const float *p) {
    return isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]);
}

__global__ void k_footprint(dgr_grid g, int n, const float *__restrict__ mu,
                            const float *__restrict__ s, const float4 *__restrict__ q, float k,
                            int *__restrict__ anchor, int *__restrict__ box) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float m[3] = {mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]};
    float sc[3] = {s[3 * i], s[3 * i + 1], s[3 * i + 2]};
    Foot F;
    footprint_f32(g, m, sc, q[i], k, F);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        anchor[3 * i + a] = F.an[a];
        box[6 * i + a] = F.lo[a];
        box[6 * i + 3 + a] = F.hi[a];
    }
}

// a1: per-Gaussian prep (thread per global Gaussian index).
__global__ void k_prep(const __grid_constant__ Batch B, Prep *__restrict__ prep,
                       uint32_t *__restrict__ itemcnt, int *status) {
    DEP_ENTER();
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= B.tot_g) return;
    const Inst &I = B.in[inst_of_g(B, gi)];
    // the footprint frame: the whole grid's origin and the slab's first layer
    dgr_grid g = I.g;
    g.oz = I.oz_full;
    g.z0 = I.z0;
    const int i = gi - I.g0;
    float m[3] = {I.mu[3 * i], I.mu[3 * i + 1], I.mu[3 * i + 2]};
    float sc[3] = {I.s[3 * i], I.s[3 * i + 1], I.s[3 * i + 2]};
    const float4 qq = reinterpret_cast<const float4 *>(I.q)[i];
    const float r = I.rho[i];
    Prep P;
    bool ok = finite3(m) && finite3(sc) && isfinite(qq.x) && isfinite(qq.y) && isfinite(qq.z) &&
              isfinite(qq.w) && isfinite(r) && sc[0] > 0.f && sc[1] > 0.f && sc[2] > 0.f &&
              (qq.x != 0.f || qq.y != 0.f || qq.z != 0.f || qq.w != 0.f);
    if (!ok) {
        atomicOr(status, DGR_STATUS_NONFINITE);
        P = Prep{};
        P.bx = P.by = P.bz = box_pack(1, 0);  // empty
        prep[gi] = P;
        itemcnt[gi] = 0;
        return;
    }
    Foot F;
    footprint_f32(g, m, sc, qq, I.k, F);
    // delta = u - a, with u in FP64 so the fractional offset is exact to FP32
    // (FP64 divisions and square roots are slow here: one reciprocal of h)
    const double h = (double)g.h, ih = 1.0 / h;
    const double org[3] = {(double)g.ox, (double)g.oy, (double)g.oz};
    float del[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double u = ((double)m[a] - org[a]) * ih - 0.5;
        del[a] = (float)(u - (double)(F.an[a] + (a == 2 ? g.z0 : 0)));
    }
    // column form of the exponent (FP64 per Gaussian): Sigma = R diag(s^2) R^T
    // in voxel units from the normalised quaternion; the z column through
    // (dx, dy) peaks at dz* = Sigma_z,xy (Sigma_xy)^-1 (dx, dy) with the value
    // -1/2 (dx, dy) (Sigma_xy)^-1 (dx, dy)^T, and A_zz = 1 / Var(z | x, y)
    // = sum_k R_zk^2 / s_k^2 (a sum of positive terms).  The xy block is
    // inverted directly (the Schur complement of A would cancel for thin,
    // tilted Gaussians) and split into principal axes.  Scaled by
    // -1/2 log2(e) for ex2.
    const double c = -0.5 * (double)LOG2E;
    double m00, m11, m01, zx, zy, azz;
    bool diag;
    if (sc[0] == sc[1] && sc[1] == sc[2]) {
        // isotropic (the paper's representation): diagonal for any rotation
        const double sv = (double)sc[0] * ih;
        m00 = m11 = azz = 1.0 / (sv * sv);
        m01 = zx = zy = 0.0;
        diag = true;
    } else {
        const double q0 = qq.x, q1 = qq.y, q2 = qq.z, q3 = qq.w;
        const double iq = rsqrt(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        const double w = q0 * iq, x = q1 * iq, y = q2 * iq, z = q3 * iq;
        const double Rd[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                              2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                              2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        double v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double sv = (double)sc[k] * ih;
            v[k] = sv * sv;
        }
        // 1 / v_k from one reciprocal of their product
        const double ip = 1.0 / (v[0] * v[1] * v[2]);
        const double iv[3] = {v[1] * v[2] * ip, v[0] * v[2] * ip, v[0] * v[1] * ip};
        double S[6] = {0, 0, 0, 0, 0, 0};  // 00 11 22 01 02 12
        azz = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            S[0] += Rd[k] * Rd[k] * v[k];
            S[1] += Rd[3 + k] * Rd[3 + k] * v[k];
            S[3] += Rd[k] * Rd[3 + k] * v[k];
            S[4] += Rd[k] * Rd[6 + k] * v[k];
            S[5] += Rd[3 + k] * Rd[6 + k] * v[k];
            azz += Rd[6 + k] * Rd[6 + k] * iv[k];
        }
        const double det = S[0] * S[1] - S[3] * S[3], idet = 1.0 / det;
        m00 = S[1] * idet;
        m11 = S[0] * idet;
        m01 = -S[3] * idet;
        zx = m00 * S[4] + m01 * S[5];
        zy = m01 * S[4] + m11 * S[5];
        diag = S[3] == 0.0 && S[4] == 0.0 && S[5] == 0.0;
    }
    // principal axes of (Sigma_xy)^-1: l1 >= l2 with unit vector n1 (diagonal:
    // the x and y axes, in that order)
    double l1, l2, n1x, n1y;
    if (diag || m01 == 0.0) {
        l1 = m00; l2 = m11; n1x = 1.0; n1y = 0.0;
    } else {
        const double hm = 0.5 * (m00 + m11), dm = 0.5 * (m00 - m11);
        const double r = sqrt(dm * dm + m01 * m01);
        l1 = hm + r;
        // the product of the eigenvalues (det (Sigma_xy)^-1 = 1 / det Sigma_xy) over l1: no cancellation
        l2 = (m00 * m11 - m01 * m01) / l1;
        // eigenvector of l1: (m01, l1 - m00) or (l1 - m11, m01), whichever is longer
        const double ax1 = m01, ay1 = l1 - m00, ax2 = l1 - m11, ay2 = m01;
        const bool first = ax1 * ax1 + ay1 * ay1 >= ax2 * ax2 + ay2 * ay2;
        const double ex = first ? ax1 : ax2, ey = first ? ay1 : ay2;
        const double inv = rsqrt(ex * ex + ey * ey);
        n1x = ex * inv;
        n1y = ey * inv;
    }
    // a Gaussian with off-diagonal terms rules out the separable voxelizer
    if (!diag) status[SEP_FLAG] = 1;
    P.dx = del[0]; P.dy = del[1]; P.dz = del[2]; P.rho = r;
    P.l1 = (float)(c * l1); P.l2 = (float)(c * l2); P.n1x = (float)n1x;
    P.a22 = (float)(c * azz);
    P.zx = diag ? 0.f : (float)zx;
    P.zy = diag ? 0.f : (float)zy;
    P.n1x_d = n1x; P.n1y_d = n1y;
    P.zx_d = diag ? 0.0 : zx; P.zy_d = diag ? 0.0 : zy;
    P.ax = F.an[0]; P.ay = F.an[1]; P.az = F.an[2];
    // an axis that misses the grid empties the whole box (packed as lo 1, hi 0)
    const bool empty = F.lo[0] > F.hi[0] || F.lo[1] > F.hi[1] || F.lo[2] > F.hi[2];
    P.bx = empty ? box_pack(1, 0) : box_pack(F.lo[0], F.hi[0]);
    P.by = empty ? box_pack(1, 0) : box_pack(F.lo[1], F.hi[1]);
    P.bz = empty ? box_pack(1, 0) : box_pack(F.lo[2], F.hi[2]);
    prep[gi] = P;
    // backward work items of at most ~ITEM_VOX voxels (item_count)
    const int ex = F.hi[0] - F.lo[0] + 1, ey = F.hi[1] - F.lo[1] + 1, ez = F.hi[2] - F.lo[2] + 1;
    itemcnt[gi] = empty ? 0u : item_count(ex, ey, ez);
}

// Tile range of a Gaussian (tiles TX x TY x tz); false if its box misses the grid.
__device__ __forceinline__ bool tile_range(const Prep &P, int tz, int &t0x, int &t0y, int &t0z,
                                           int &ntx, int &nty, int &ntz) {
    const int lx = box_lo(P.bx), hx = box_hi(P.bx), ly = box_lo(P.by), hy = box_hi(P.by),
              lz = box_lo(P.bz), hz = box_hi(P.bz);
    if (lx > hx || ly > hy || lz > hz) return false;
    t0x = lx / TX; t0y = ly / TY; t0z = lz / tz;
    ntx = hx / TX - t0x + 1; nty = hy / TY - t0y + 1; ntz = hz / tz - t0z + 1;
    return true;
}

// a2: count Gaussians per tile (one warp per Gaussian, lanes over its tiles).
__global__ void k_tile_count(const __grid_constant__ Batch B, const Prep *__restrict__ prep,
                             uint32_t *__restrict__ tile_cnt) {
    DEP_ENTER();
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < B.tot_g; gi += warps) {
        const Inst &I = B.in[inst_of_g(B, gi)];
        const Prep P = prep[gi];
        int t0x, t0y, t0z, ntx, nty, ntz;
        if (!tile_range(P, B.tz, t0x, t0y, t0z, ntx, nty, ntz)) continue;
        const int tot = ntx * nty * ntz;
        for (int j = lane; j < tot; j += 32) {
            const int jx = j % ntx, jy = (j / ntx) % nty, jz = j / (ntx * nty);
            const int t = I.tile0 + ((t0z + jz) * I.nty + (t0y + jy)) * I.ntx + (t0x + jx);
            atomicAdd(&tile_cnt[t], 1u);
        }
    }
}

// a2: write each Gaussian index into the lists of the tiles it overlaps.
__global__ void k_tile_fill(const __grid_constant__ Batch B, const Prep *__restrict__ prep,
                            const uint32_t *__restrict__ tile_off, uint32_t *__restrict__ tile_fill,
                            uint32_t *__restrict__ list, unsigned long long cap) {
    DEP_ENTER();
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < B.tot_g; gi += warps) {
        const Inst &I = B.in[inst_of_g(B, gi)];
        const Prep P = prep[gi];
        int t0x, t0y, t0z, ntx, nty, ntz;
        if (!tile_range(P, B.tz, t0x, t0y, t0z, ntx, nty, ntz)) continue;
        const int tot = ntx * nty * ntz;
        for (int j = lane; j < tot; j += 32) {
            const int jx = j % ntx, jy = (j / ntx) % nty, jz = j / (ntx * nty);
            const int t = I.tile0 + ((t0z + jz) * I.nty + (t0y + jy)) * I.ntx + (t0x + jx);
            const unsigned long long pos =
                (unsigned long long)tile_off[t] + atomicAdd(&tile_fill[t], 1u);
            if (pos < cap) list[pos] = (uint32_t)gi;
        }
    }
}

// a2: sort each tile's list ascending.  Up to WSORT_MAX entries: a warp in
// registers (below); up to SORT_SMEM entries: bitonic sort in shared memory
// (padded there with +inf).  Longer lists: sort chunks
// of SORT_SMEM in shared memory the same way, then merge runs pairwise
// (width doubling) through a scratch list of the same layout, each output
// position finding its source by a co-rank (merge-path) binary search.
constexpr int SORT_THREADS = 256;
constexpr int SORT_SMEM = 4096;

__device__ void bitonic_smem(uint32_t *a, int m2) {
    for (int k = 2; k <= m2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const uint32_t x = a[i], y = a[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) { a[i] = y; a[l] = x; }
                }
            }
            __syncthreads();
        }
}

// sorts seg[0, m) (m <= SORT_SMEM) through shared memory
__device__ void sort_chunk(uint32_t *seg, int m, uint32_t *sm) {
    int m2 = 1;
    while (m2 < m) m2 <<= 1;
    for (int i = threadIdx.x; i < m2; i += blockDim.x) sm[i] = i < m ? seg[i] : 0xffffffffu;
    __syncthreads();
    bitonic_smem(sm, m2);
    for (int i = threadIdx.x; i < m; i += blockDim.x) seg[i] = sm[i];
    __syncthreads();
}

// elements taken from run A among the first k outputs of the stable merge of
// sorted runs A and B (ties from A first); at most log2(alen) + 1 steps
__device__ __forceinline__ int corank(int k, const uint32_t *A, int alen, const uint32_t *Bv, int blen) {
    int lo = max(0, k - blen), hi = min(k, alen);
    while (lo < hi) {
        const int i = (lo + hi) >> 1, j = k - i;
        if (j > 0 && i < alen && Bv[j - 1] > A[i]) lo = i + 1; else hi = i;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Work units of the voxelizer: units 0 .. tiles - 1 are the tiles (their whole
// list, or its first segment), then one unit per further segment of a split
// tile
// ---------------------------------------------------------------------------
// a2 (once the tile lists are complete), for tile t: per instance with P list
// entries in all, the segment length is L = max(SPLIT_LMIN, 3P / (2
// SPLIT_BUDGET)) rounded up to whole chunks; a tile with more than 2L entries
// takes r = min(SPLIT_SMAX, ceil(len / L)) segments and r partial slots.  As
// len / L > 2, r < 1.5 len / L, so an instance's slots stay below 1.5 P / L
// <= SPLIT_BUDGET: every request fits, and whether and how a tile splits
// depends only on its own instance's lists (a batch splits exactly as its
// instances alone).  Slots and extra units are handed out by atomic counters
// (zeroed before): where a segment's partial sits does not change a bit of
// the result.
__device__ __forceinline__ void plan_tile(const Batch &B, int t, const uint32_t *__restrict__ tile_off,
                                          unsigned long long cap, const VoxSplit &S) {
    const int i = inst_of_tile(B, t);
    const Inst &I = B.in[i];
    const auto off = [&](int j) {
        const unsigned long long o = tile_off[j];
        return o > cap ? cap : o;
    };
    const unsigned long long tot = off(I.tile0 + I.ntx * I.nty * I.ntz) - off(I.tile0);
    unsigned long long L = (3ull * tot + 2ull * SPLIT_BUDGET - 1) / (2ull * SPLIT_BUDGET);
    if (L < (unsigned long long)SPLIT_LMIN) L = SPLIT_LMIN;
    L = (L + VOX_CHUNK - 1) / VOX_CHUNK * VOX_CHUNK;
    const unsigned long long b = off(t), e = off(t + 1), len = e > b ? e - b : 0;
    const int r = len > 2ull * L ? (int)min((unsigned long long)SPLIT_SMAX, (len + L - 1) / L) : 1;
    S.nseg[t] = r;
    S.done[t] = 0;
    if (r > 1) {
        S.slot[t] = i * SPLIT_BUDGET + atomicAdd(S.ctr + 1 + i, r);
        const int x = atomicAdd(S.ctr, r - 1);
        for (int sg = 1; sg < r; ++sg) S.extra[x + sg - 1] = t | (sg << 24);
    } else {
        S.slot[t] = -1;
    }
}

// plan_tile for every tile (when the lists are not sorted; k_tile_sort_warp
// does it otherwise)
__global__ void k_split_plan(const __grid_constant__ Batch B, const uint32_t *__restrict__ tile_off,
                             unsigned long long cap, const VoxSplit S) {
    DEP_ENTER();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < B.tot_tiles) plan_tile(B, t, tile_off, cap, S);
}

// Lists of at most WSORT_MAX entries are sorted by one warp in registers
// (k_tile_sort_warp); k_tile_sort takes the longer ones.
constexpr int WSORT_MAX = 256;

// bitonic sort of the 32 E values of a warp, ascending in i = lane E + r:
// partners in other lanes through shuffles, in the same lane by register
__device__ __forceinline__ uint32_t umin_(uint32_t a, uint32_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t umax_(uint32_t a, uint32_t b) { return a < b ? b : a; }
template <int E>
__device__ __forceinline__ void warp_bitonic(uint32_t (&v)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
                const bool lower = (lane & lj) == 0;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const bool up = ((lane * E + r) & k) == 0;
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, v[r], lj);
                    v[r] = lower == up ? umin_(v[r], o) : umax_(v[r], o);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int q = r ^ j;
                    if (q > r) {
                        const bool up = ((lane * E + r) & k) == 0;
                        const uint32_t a = v[r], b = v[q];
                        v[r] = up ? umin_(a, b) : umax_(a, b);
                        v[q] = up ? umax_(a, b) : umin_(a, b);
                    }
                }
            }
        }
    }
}
template <int E>
__device__ __forceinline__ void warp_sort_list(uint32_t *seg, int m, int lane) {
    uint32_t v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        v[r] = i < m ? seg[i] : 0xffffffffu;
    }
    warp_bitonic<E>(v, lane);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int i = lane * E + r;
        if (i < m) seg[i] = v[r];
    }
}

// a2: a warp per tile sorts lists of 2 .. WSORT_MAX entries
__global__ void __launch_bounds__(256) k_tile_sort_warp(const __grid_constant__ Batch B,
                                                        const uint32_t *__restrict__ tile_off,
                                                        uint32_t *__restrict__ list, unsigned long long cap,
                                                        const VoxSplit S) {
    DEP_ENTER();
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int ntiles = B.tot_tiles;
    if (t >= ntiles) return;
    if (lane == 0) plan_tile(B, t, tile_off, cap, S);  // the voxelizer's work units
    unsigned long long b = tile_off[t], e = tile_off[t + 1];
    if (e > cap) e = cap;
    if (b >= e) return;
    const int m = (int)(e - b);
    if (m < 2 || m > WSORT_MAX) return;
    uint32_t *seg = list + b;
    if (m <= 32) warp_sort_list<1>(seg, m, lane);
    else if (m <= 64) warp_sort_list<2>(seg, m, lane);
    else if (m <= 128) warp_sort_list<4>(seg, m, lane);
    else warp_sort_list<8>(seg, m, lane);
}

__global__ void k_tile_sort(int ntiles, const uint32_t *__restrict__ tile_off,
                            uint32_t *__restrict__ list, uint32_t *__restrict__ scratch,
                            unsigned long long cap) {
    DEP_ENTER();
    __shared__ uint32_t sm[SORT_SMEM];
    const int t = blockIdx.x;
    unsigned long long b = tile_off[t], e = tile_off[t + 1];
    if (e > cap) e = cap;
    if (b >= e) return;
    const int m = (int)(e - b);
    if (m <= WSORT_MAX) return;  // k_tile_sort_warp
    uint32_t *seg = list + b;
    if (m <= SORT_SMEM) {
        sort_chunk(seg, m, sm);
        return;
    }
    for (int c0 = 0; c0 < m; c0 += SORT_SMEM) sort_chunk(seg + c0, min(SORT_SMEM, m - c0), sm);
    uint32_t *src = seg, *dst = scratch + b;
    for (int w = SORT_SMEM; w < m; w <<= 1) {
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int s0 = (k / (2 * w)) * (2 * w);
            const int alen = min(w, m - s0);
            const int b0 = s0 + alen;
            const int blen = max(0, min(w, m - b0));
            const int kk = k - s0;
            const int i = corank(kk, src + s0, alen, src + b0, blen), j = kk - i;
            dst[k] = (i < alen && (j >= blen || src[s0 + i] <= src[b0 + j])) ? src[s0 + i]
                                                                             : src[b0 + j];
        }
        __syncthreads();
        uint32_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != seg) {
        for (int k = threadIdx.x; k < m; k += blockDim.x) seg[k] = src[k];
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


// Layer masks of a z group of TZG partly inside a box: row lo * TZG + hi adds
// 0 to the exponent of the layers lo..hi of the group and -1e30 (ex2 -> 0) to
// the others, so the range test costs one packed FP32 add per pair on the FMA
// pipe instead of integer compares and selects per layer.  Adding 0 leaves
// the exponent's bits as they are (-0 becomes +0; ex2 of either is 1).
struct ZMask {
    float4 v[TZG * TZG][TZG / 4];
};
constexpr ZMask make_zmask() {
    ZMask t{};
    for (int lo = 0; lo < TZG; ++lo)
        for (int hi = 0; hi < TZG; ++hi)
            for (int k4 = 0; k4 < TZG / 4; ++k4) {
                float e[4] = {};
                for (int c = 0; c < 4; ++c) {
                    const int k = 4 * k4 + c;
                    e[c] = (lo <= k && k <= hi) ? 0.f : -1e30f;
                }
                t.v[lo * TZG + hi][k4] = float4{e[0], e[1], e[2], e[3]};
            }
    return t;
}
__constant__ ZMask c_zmask = make_zmask();

// Per (tile, Gaussian) record of a staged chunk, built once per CTA by one
// thread, so that a warp's visit of the Gaussian costs only the per-lane set-up
// of its column's quadratic:
//   r0 = (c1', c2', tau, rho): the principal coordinates n1 . d, n2 . d of the
//        tile's centre column, scaled by s1 = sqrt(-l1) and s2 = sqrt(-l2) (the
//        column's peak value is then -(c1'^2 + c2'^2)), and the offset tau of
//        the tile's middle layer from that column's peak, in FP64 (then
//        rounded): lanes add only offsets of at most 3.5 (x) and 7.5 (y)
//        voxels, so the exponent keeps its precision however far the tile lies
//        from the Gaussian's centre
//   r1 = (s1 n1x, s1 n1y, a22, -zx), r2 = (-s2 n1y, s2 n1x, -zy, 0)
//   lane masks: per warp, bit l set when lane l's (x, y) column lies in the box
//   zinfo: bits 0-3 the z groups of TZG layers the box reaches, bits 4-7 those
//          it covers whole; bits 8 + 6 g .. 13 + 6 g: for a partly covered
//          group g, the row (lo * TZG + hi) of the layer-mask table
struct VisitChunk {
    float4 r0[VOX_CHUNK], r1[VOX_CHUNK], r2[VOX_CHUNK];
    unsigned lanes[VOX_THREADS / 32][VOX_CHUNK];
    int zinfo[VOX_CHUNK];
};

// list range [b, e) of segment seg of nseg: whole chunks, the last one short
// (possibly empty)
__device__ __forceinline__ void segment_range(unsigned long long &b, unsigned long long &e, int nseg, int seg) {
    const unsigned long long len = e - b;
    unsigned long long L = (len + nseg - 1) / nseg;
    L = (L + VOX_CHUNK - 1) / VOX_CHUNK * VOX_CHUNK;
    const unsigned long long sb = min(e, b + (unsigned long long)seg * L);
    e = min(e, sb + L);
    b = sb;
}

// End of a segment of a split tile: its sums val(k), k < TZ, go to its
// partial slot; the CTA that finishes the tile's last segment (whichever it
// is) reads every slot of the tile and leaves in out[k][thread] the sum over
// the segments in segment order, Kahan-compensated -- the same bits whatever
// the order in which the segments ran.  Returns true for that CTA (it writes
// the tile), false for the others.  CTA-uniform; flag: a shared int.
template <int TZ, class Get>
__device__ __forceinline__ bool fold_segments(const VoxSplit &S, int tg, int seg, int nseg, Get val,
                                              float (*out)[VOX_THREADS], int *flag) {
    const int slot = S.slot[tg];
    float *mine = S.part + (size_t)(slot + seg) * VOX_SLOT + threadIdx.x;
#pragma unroll
    for (int k = 0; k < TZ; ++k) mine[k * VOX_THREADS] = val(k);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *flag = atomicAdd(S.done + tg, 1) == nseg - 1;
    __syncthreads();
    if (!*flag) return false;
    __threadfence();
    const float *first = S.part + (size_t)slot * VOX_SLOT + threadIdx.x;
#pragma unroll 1
    for (int k = 0; k < TZ; ++k) {
        float sum = 0.f, c = 0.f;
        for (int s = 0; s < nseg; ++s) {
            const float y = __ldcg(first + (size_t)s * VOX_SLOT + k * VOX_THREADS) - c;
            const float t = sum + y;
            c = (t - sum) - y;
            sum = t;
        }
        out[k][threadIdx.x] = sum;
    }
    return true;
}

// a3: persistent CTAs take tiles from a global queue (tiles of every instance
// back to back).  Warp w covers y in [ty0 + 4w, ty0 + 4w + 4), lane
// (lx, ly) = (lane & 7, lane >> 3), and the column z in [tz0, tz0 + TZ).
// Per chunk of VOX_CHUNK Gaussians of the tile's list: the staging threads
// build the visit records; each warp visits (ballot over the chunk) only the
// Gaussians whose box covers one of its columns, in list order; per visit a
// lane sets up its column's peak (value qmin from its principal coordinates,
// offset t0 of the tile's middle layer from the peak) and evaluates
// q = qmin + a22 t^2, t = t0 + k - (TZ - 1)/2, on the z groups of TZG layers
// the box reaches (a partly covered group adds 0 or -1e30 from the
// layer-mask table to the exponent: ex2 of the latter is 0).
template <int TZ>
__global__ void __launch_bounds__(VOX_THREADS) k_voxelize(
    const __grid_constant__ Batch B, const Prep *__restrict__ prep,
    const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ list,
    unsigned long long cap, int *__restrict__ queue, const int *__restrict__ sep_off, const VoxSplit S) {
    DEP_ENTER();
    static_assert(TZ / TZG <= 4, "z groups are tracked in 4-bit masks");
    constexpr int NG = TZ / TZG;
    __shared__ VisitChunk vc;
    // the running per-voxel sums and their Kahan compensations: one column per
    // thread (touched by that thread only), kept out of registers so that more
    // CTAs fit on an SM
    __shared__ float s_acc[TZ][VOX_THREADS], s_cmp[TZ][VOX_THREADS];
    __shared__ int s_tile, s_last;
    if (sep_off && *sep_off == 0) return;  // every Gaussian separable: k_voxelize_sep runs
    const int n_units = B.tot_tiles + S.ctr[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the lane's column relative to the tile's centre column
    const float lxc = (float)(lane & 7) - 0.5f * (TX - 1), lyc = (float)(4 * w + (lane >> 3)) - 0.5f * (TY - 1);
    for (;;) {
        __syncthreads();  // everyone is done with s_tile and the records
        if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
        __syncthreads();
        const int u = s_tile;  // work unit: a tile or a segment of its list
        if (u >= n_units) return;
        int tg = u, seg = 0;
        if (u >= B.tot_tiles) {
            const int xu = S.extra[u - B.tot_tiles];
            tg = xu & 0xffffff;
            seg = xu >> 24;
        }
        const Inst &I = B.in[inst_of_tile(B, tg)];
        const dgr_grid &g = I.g;
        const int t = tg - I.tile0;
        const int tx = t % I.ntx, ty = (t / I.ntx) % I.nty, tz = t / (I.ntx * I.nty);
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * TZ;
        const int x = x0 + (lane & 7);
        const int y = y0 + 4 * w + (lane >> 3);
        unsigned long long b = tile_off[tg], e = tile_off[tg + 1];
        if (e > cap) e = cap;
        if (b > e) b = e;
        const int nseg = S.nseg[tg];
        if (nseg > 1) segment_range(b, e, nseg, seg);
        // the chunk's plain sums, z pairs in packed FP32 (each half rounds
        // exactly as the scalar FMA); a z outside a box contributes
        // exp2(-inf) = 0
        float2 cs[TZ / 2];
#pragma unroll
        for (int k = 0; k < TZ / 2; ++k) cs[k] = make_float2(0.f, 0.f);
        for (unsigned long long c0 = b; c0 < e; c0 += VOX_CHUNK) {
            const int nc = (int)min((unsigned long long)VOX_CHUNK, e - c0);
            if (c0 != b) __syncthreads();
            if (threadIdx.x < nc) {
                const int j = threadIdx.x;
                uint32_t gj = list[c0 + j];
                if (!DGR_INB(gj, B.tot_g, B.status)) gj = 0;  // (bounds-checked build) a bad list entry
                const float4 *pp = reinterpret_cast<const float4 *>(prep + gj);
                const float4 p0 = pp[0], p1 = pp[1], p2 = pp[2], p3 = pp[3];
                const double2 n1 = reinterpret_cast<const double2 *>(pp + 4)[0],
                              zz = reinterpret_cast<const double2 *>(pp + 4)[1];
                const int ax = __float_as_int(p2.z), ay = __float_as_int(p2.w), az = __float_as_int(p3.x);
                const int bx = __float_as_int(p3.y), by = __float_as_int(p3.z), bz = __float_as_int(p3.w);
                const int xl = max(box_lo(bx) - x0, 0), xh = min(box_hi(bx) - x0, TX - 1);
                const int yl = box_lo(by) - y0, yh = box_hi(by) - y0;
                const int zl = max(box_lo(bz) - z0, 0), zh = min(box_hi(bz) - z0, TZ - 1);
                const unsigned xm = xl <= xh ? (0xffu >> (TX - 1 - xh)) & (0xffu << xl) : 0u;
#pragma unroll
                for (int ww = 0; ww < VOX_THREADS / 32; ++ww) {
                    unsigned m = 0u;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (4 * ww + r >= yl && 4 * ww + r <= yh) m |= xm << (8 * r);
                    vc.lanes[ww][j] = m;
                }
                int act = 0, full = 0, rows = 0;
#pragma unroll
                for (int g8 = 0; g8 < NG; ++g8) {
                    const int lo = zl - g8 * TZG, hi = zh - g8 * TZG;
                    if (hi >= 0 && lo < TZG && zl <= zh) {
                        act |= 1 << g8;
                        if (lo <= 0 && hi >= TZG - 1) full |= 1 << g8;
                        rows |= (max(lo, 0) * TZG + min(hi, TZG - 1)) << (6 * g8);
                    }
                }
                vc.zinfo[j] = act | (full << 4) | (rows << 8);
                // the tile's centre column and middle layer relative to the
                // Gaussian's centre, in FP64
                const double Xc = (double)(x0 - ax) + 0.5 * (TX - 1) - (double)p0.x;
                const double Yc = (double)(y0 - ay) + 0.5 * (TY - 1) - (double)p0.y;
                const double Zc = (double)(z0 - az) + 0.5 * (TZ - 1) - (double)p0.z;
                const double c1 = n1.x * Xc + n1.y * Yc, c2 = n1.x * Yc - n1.y * Xc;
                const double tau = Zc - (zz.x * Xc + zz.y * Yc);
                // principal coordinates scaled by sqrt(-l1), sqrt(-l2): the peak
                // value is then -(c1'^2 + c2'^2)
                const double s1 = sqrtf(fmaxf(-p1.x, 0.f)), s2 = sqrtf(fmaxf(-p1.y, 0.f));
                vc.r0[j] = make_float4((float)(s1 * c1), (float)(s2 * c2), (float)tau, p0.w);
                vc.r1[j] = make_float4((float)(s1 * n1.x), (float)(s1 * n1.y), p1.z, -p2.x);
                vc.r2[j] = make_float4((float)(-s2 * n1.y), (float)(s2 * n1.x), -p2.y, 0.f);
            }
            __syncthreads();
            // this warp's visits, in list order: the chunk's two halves of 32
#pragma unroll 1
            for (int h = 0; h < VOX_CHUNK; h += 32) {
                unsigned vis = __ballot_sync(0xffffffffu, lane + h < nc && vc.lanes[w][lane + h] != 0u);
                while (vis) {
                    const int j = h + __ffs(vis) - 1;
                    vis &= vis - 1;
                    const bool in = (vc.lanes[w][j] >> lane) & 1u;
                    const float4 r0 = vc.r0[j], r1 = vc.r1[j], r2 = vc.r2[j];
                    const int zi = vc.zinfo[j];
                    // the column's principal coordinates, its peak value (<= 0,
                    // already scaled) and the offset of the tile's middle layer
                    // from the peak
                    const float c1 = fmaf(r1.x, lxc, fmaf(r1.y, lyc, r0.x));
                    const float c2 = fmaf(r2.x, lxc, fmaf(r2.y, lyc, r0.y));
                    float qm = -fmaf(c1, c1, c2 * c2);
                    qm = in ? qm : -INFINITY;
                    const float t0 = fmaf(r1.w, lxc, fmaf(r2.z, lyc, r0.z));
                    const float2 a22v = make_float2(r1.z, r1.z), qmv = make_float2(qm, qm),
                                 rv = make_float2(r0.w, r0.w);
                    // (t, t + 1) at layers (0, 1); each pair's offsets are added to
                    // it directly, so the pairs do not wait on one another
                    const float2 tb = __fadd2_rn(make_float2(t0, t0),
                                                 make_float2(-0.5f * (TZ - 1), 1.f - 0.5f * (TZ - 1)));
#pragma unroll
                    for (int g8 = 0; g8 < NG; ++g8) {
                        if (!(zi & (1 << g8))) continue;  // warp-uniform
                        if (zi & (16 << g8)) {  // whole group in the box (warp-uniform)
#pragma unroll
                            for (int kk = 0; kk < TZG; kk += 2) {
                                const int k = g8 * TZG + kk;
                                const float2 t = k == 0 ? tb : __fadd2_rn(tb, make_float2((float)k, (float)k));
                                const float2 q = __ffma2_rn(__fmul2_rn(a22v, t), t, qmv);
                                cs[k / 2] = __ffma2_rn(rv, make_float2(ex2_approx(q.x), ex2_approx(q.y)), cs[k / 2]);
                            }
                        } else {
                            const int row = (zi >> (8 + 6 * g8)) & 63;
                            const float4 zm0 = c_zmask.v[row][0], zm1 = c_zmask.v[row][1];
                            const float zmv[TZG] = {zm0.x, zm0.y, zm0.z, zm0.w, zm1.x, zm1.y, zm1.z, zm1.w};
#pragma unroll
                            for (int kk = 0; kk < TZG; kk += 2) {
                                const int k = g8 * TZG + kk;
                                const float2 t = k == 0 ? tb : __fadd2_rn(tb, make_float2((float)k, (float)k));
                                float2 q = __ffma2_rn(__fmul2_rn(a22v, t), t, qmv);
                                q = __fadd2_rn(q, make_float2(zmv[kk], zmv[kk + 1]));
                                cs[k / 2] = __ffma2_rn(rv, make_float2(ex2_approx(q.x), ex2_approx(q.y)), cs[k / 2]);
                            }
                        }
                    }
                }
            }
            // Kahan: each chunk sum joins the running sum with compensation, so
            // a voxel inside thousands of boxes keeps its FP32 sum within a few
            // ulps of the exact sum.  The first chunk's sum is the running sum
            // as it stands (Kahan from zero gives the same bits); a tile of one
            // chunk keeps it in registers.
            const bool more = c0 + VOX_CHUNK < e;
            if (c0 == b) {
                if (more) {
#pragma unroll
                    for (int k = 0; k < TZ; ++k) {
                        s_acc[k][threadIdx.x] = (k & 1) ? cs[k / 2].y : cs[k / 2].x;
                        s_cmp[k][threadIdx.x] = 0.f;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < TZ; ++k) {
                    const float a = s_acc[k][threadIdx.x];
                    const float yv = ((k & 1) ? cs[k / 2].y : cs[k / 2].x) - s_cmp[k][threadIdx.x];
                    const float tsum = a + yv;
                    s_cmp[k][threadIdx.x] = (tsum - a) - yv;
                    s_acc[k][threadIdx.x] = tsum;
                }
            }
            if (more) {
#pragma unroll
                for (int k = 0; k < TZ / 2; ++k) cs[k] = make_float2(0.f, 0.f);
            }
        }
        if (e - b > (unsigned long long)VOX_CHUNK) {
#pragma unroll
            for (int k = 0; k < TZ / 2; ++k) cs[k] = make_float2(s_acc[2 * k][threadIdx.x], s_acc[2 * k + 1][threadIdx.x]);
        }
        const auto acc = [&](int k) { return (k & 1) ? cs[k / 2].y : cs[k / 2].x; };
        // a segment of a split tile: its partial sums; the tile's last one adds
        // them up (through the thread's own column of s_acc, free once the
        // sums are in registers)
        if (nseg > 1) {
            if (!fold_segments<TZ>(S, tg, seg, nseg, acc, s_acc, &s_last)) continue;
#pragma unroll
            for (int k = 0; k < TZ / 2; ++k) cs[k] = make_float2(s_acc[2 * k][threadIdx.x], s_acc[2 * k + 1][threadIdx.x]);
        }
        if (x < g.nx && y < g.ny) {
            // element strides: x fastest (the C ABI's layout) or z fastest
            // (the step's internal layout, read by the row-warp projector)
            float *col = I.vol + (size_t)x * I.vsx + (size_t)y * I.vsy;
            if (I.vsz == 1 && (g.nz & 3) == 0 && z0 + TZ <= g.nz &&
                (reinterpret_cast<uintptr_t>(I.vol) & 15) == 0) {
#pragma unroll
                for (int k = 0; k < TZ; k += 4)
                    *reinterpret_cast<float4 *>(col + z0 + k) =
                        make_float4(acc(k), acc(k + 1), acc(k + 2), acc(k + 3));
            } else {
                const size_t zs = (size_t)I.vsz;
#pragma unroll
                for (int k = 0; k < TZ; ++k)
                    if (z0 + k < g.nz) col[(size_t)(z0 + k) * zs] = acc(k);
            }
        }
    }
}

// FVR for separable Gaussians (the paper's isotropic representation, or
// axis-aligned ones): with A diagonal (m00 = a00, m11 = a11, no column shift),
// rho exp2(a00 dx^2 + a11 dy^2 + a22 dz^2)
// = EXY(x, y) EZ(z).  Same tiles, work lists, warps and skips as k_voxelize
// (a warp owns an 8 x 4 (x, y) patch, each lane a z column of the tile), but
// per chunk of Gaussians the z factors EZ (zero outside each box) are built
// once in shared memory, each lane evaluates one exponential per (Gaussian,
// column), and every (Gaussian, voxel) pair costs one FMA on a value read as
// part of a 16-byte shared load.  Chunk sums join the running sums with Kahan
// compensation.  Runs only when every Gaussian of the call is separable
// (k_prep's flag), tile depth 32.
constexpr int SEP_TZ = 32;

__global__ void __launch_bounds__(VOX_THREADS) k_voxelize_sep(
    const __grid_constant__ Batch B, const Prep *__restrict__ prep,
    const uint32_t *__restrict__ tile_off, const uint32_t *__restrict__ list,
    unsigned long long cap, int *__restrict__ queue, const int *__restrict__ sep_off, const VoxSplit S) {
    DEP_ENTER();
    __shared__ float4 sp[VOX_CHUNK * 4];
    __shared__ __align__(16) float ez[VOX_CHUNK][SEP_TZ];
    // running sums and Kahan compensations, one column per thread (as in k_voxelize)
    __shared__ float s_acc[SEP_TZ][VOX_THREADS], s_cmp[SEP_TZ][VOX_THREADS];
    __shared__ int s_tile, s_last;
    if (*sep_off != 0) return;  // a non-separable Gaussian: the general kernel runs
    const int n_units = B.tot_tiles + S.ctr[0];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
        __syncthreads();
        const int u = s_tile;  // work unit: a tile or a segment of its list
        if (u >= n_units) return;
        int tg = u, seg = 0;
        if (u >= B.tot_tiles) {
            const int xu = S.extra[u - B.tot_tiles];
            tg = xu & 0xffffff;
            seg = xu >> 24;
        }
        const Inst &I = B.in[inst_of_tile(B, tg)];
        const dgr_grid &g = I.g;
        const int tl = tg - I.tile0;
        const int tx = tl % I.ntx, ty = (tl / I.ntx) % I.nty, tz = tl / (I.ntx * I.nty);
        const int x0 = tx * TX, y0 = ty * TY, z0 = tz * SEP_TZ;
        const int x = x0 + (lane & 7);
        const int wy0 = y0 + 4 * w;
        const int y = wy0 + (lane >> 3);
#pragma unroll
        for (int k = 0; k < SEP_TZ; ++k) s_acc[k][threadIdx.x] = s_cmp[k][threadIdx.x] = 0.f;
        unsigned long long b = tile_off[tg], e = tile_off[tg + 1];
        if (e > cap) e = cap;
        if (b > e) b = e;
        const int nseg = S.nseg[tg];
        if (nseg > 1) segment_range(b, e, nseg, seg);
        for (unsigned long long c0 = b; c0 < e; c0 += VOX_CHUNK) {
            const int nc = (int)min((unsigned long long)VOX_CHUNK, e - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < nc * 4; i += VOX_THREADS) {
                const uint32_t gi = list[c0 + (i >> 2)];
                sp[i] = reinterpret_cast<const float4 *>(prep + gi)[i & 3];
            }
            __syncthreads();
            // z factors of the chunk, zero outside each box
            for (int f = threadIdx.x; f < nc * SEP_TZ; f += VOX_THREADS) {
                const int j = f / SEP_TZ, k = f % SEP_TZ, z = z0 + k;
                const float4 p0 = sp[4 * j], p1 = sp[4 * j + 1], p3 = sp[4 * j + 3];
                const int bz = __float_as_int(p3.w), az = __float_as_int(p3.x);
                const float dz = (float)(z - az) - p0.z;
                ez[j][k] = (z >= box_lo(bz) && z <= box_hi(bz)) ? ex2_approx(p1.z * dz * dz) : 0.f;
            }
            __syncthreads();
            float2 cs[SEP_TZ / 2];  // z pairs in packed FP32 (each half as the scalar FMA)
#pragma unroll
            for (int k = 0; k < SEP_TZ / 2; ++k) cs[k] = make_float2(0.f, 0.f);
            for (int j = 0; j < nc; ++j) {
                const float4 p3 = sp[4 * j + 3];
                const int bx = __float_as_int(p3.y), by = __float_as_int(p3.z), bz = __float_as_int(p3.w);
                const int lx = box_lo(bx), hx = box_hi(bx), ly = box_lo(by), hy = box_hi(by);
                const int zlo = max(box_lo(bz) - z0, 0), zhi = min(box_hi(bz) - z0, SEP_TZ - 1);
                // warp-uniform skip: the warp's 8 x 4 patch or the z range misses the box
                if (hx < x0 || lx > x0 + 7 || hy < wy0 || ly > wy0 + 3 || zlo > zhi) continue;
                const float4 p0 = sp[4 * j], p1 = sp[4 * j + 1], p2 = sp[4 * j + 2];
                const int ax = __float_as_int(p2.z), ay = __float_as_int(p2.w);
                const float dx = (float)(x - ax) - p0.x;
                const float dy = (float)(y - ay) - p0.y;
                const bool in = x >= lx && x <= hx && y >= ly && y <= hy;
                const float a = in ? p0.w * ex2_approx(fmaf(p1.x * dx, dx, p1.y * dy * dy)) : 0.f;
                const float4 *e4 = reinterpret_cast<const float4 *>(ez[j]);
#pragma unroll
                for (int g8 = 0; g8 < SEP_TZ / 8; ++g8) {
                    if (zhi < g8 * 8 || zlo >= (g8 + 1) * 8) continue;  // warp-uniform
                    const float4 u = e4[2 * g8], v = e4[2 * g8 + 1];
                    const float2 av = make_float2(a, a);
                    cs[4 * g8 + 0] = __ffma2_rn(av, make_float2(u.x, u.y), cs[4 * g8 + 0]);
                    cs[4 * g8 + 1] = __ffma2_rn(av, make_float2(u.z, u.w), cs[4 * g8 + 1]);
                    cs[4 * g8 + 2] = __ffma2_rn(av, make_float2(v.x, v.y), cs[4 * g8 + 2]);
                    cs[4 * g8 + 3] = __ffma2_rn(av, make_float2(v.z, v.w), cs[4 * g8 + 3]);
                }
            }
#pragma unroll
            for (int k = 0; k < SEP_TZ; ++k) {  // Kahan: chunk sum into the running sum
                const float a = s_acc[k][threadIdx.x];
                const float yv = ((k & 1) ? cs[k / 2].y : cs[k / 2].x) - s_cmp[k][threadIdx.x];
                const float tsum = a + yv;
                s_cmp[k][threadIdx.x] = (tsum - a) - yv;
                s_acc[k][threadIdx.x] = tsum;
            }
        }
        const auto acc = [&](int k) { return s_acc[k][threadIdx.x]; };
        if (nseg > 1 && !fold_segments<SEP_TZ>(S, tg, seg, nseg, acc, s_acc, &s_last)) continue;
        if (x < g.nx && y < g.ny) {
            float *col = I.vol + (size_t)x * I.vsx + (size_t)y * I.vsy;
            if (I.vsz == 1 && (g.nz & 3) == 0 && z0 + SEP_TZ <= g.nz &&
                (reinterpret_cast<uintptr_t>(I.vol) & 15) == 0) {
#pragma unroll
                for (int k = 0; k < SEP_TZ; k += 4)
                    *reinterpret_cast<float4 *>(col + z0 + k) = make_float4(acc(k), acc(k + 1), acc(k + 2), acc(k + 3));
            } else {
                const size_t zs = (size_t)I.vsz;
#pragma unroll
                for (int k = 0; k < SEP_TZ; ++k)
                    if (z0 + k < g.nz) col[(size_t)(z0 + k) * zs] = acc(k);
            }
        }
    }
}

}  // namespace

static int g_tile_depth = 32;
static int g_separable = 1;
void set_separable(int on) { g_separable = on ? 1 : 0; }
int tile_depth() { return g_tile_depth; }
void set_tile_depth(int tz) { g_tile_depth = tz; }

int tile_dims(const dgr_grid &g, int &ntx, int &nty, int &ntz) {
    const int tz = g_tile_depth;
    ntx = (g.nx + TX - 1) / TX;
    nty = (g.ny + TY - 1) / TY;
    ntz = (g.nz + tz - 1) / tz;
    return ntx * nty * ntz;
}

cudaError_t launch_footprint(const dgr_grid &g, int n, const float *mu, const float *s,
                             const float *q, float k, int *anchor, int *box, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_footprint<<<(n + 127) / 128, 128, 0, st>>>(g, n, mu, s, reinterpret_cast<const float4 *>(q),
                                                 k, anchor, box);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_prep(const Batch &B, Prep *prep, uint32_t *itemcnt, int *status, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(status + SEP_FLAG, 0, sizeof(int), st);
    if (e != cudaSuccess || B.tot_g == 0) return e;
    launch_dep(k_prep, dim3((B.tot_g + 127) / 128), dim3(128), 0, st, B, prep, itemcnt, status);
    counted(1);
    return cudaGetLastError();
}

static int warp_grid(int n) {
    int blocks = (n + 7) / 8;  // 8 warps per 256-thread block
    return blocks < 1 ? 1 : (blocks > 148 * 16 ? 148 * 16 : blocks);
}

cudaError_t launch_count_pairs(const Batch &B, const Prep *prep, dgr_ws *ws, unsigned long long cap,
                               cudaStream_t st) {
    uint32_t *tile_cnt = ws_ptr<uint32_t>(ws, ws->tile_cnt);
    uint32_t *tile_off = ws_ptr<uint32_t>(ws, ws->tile_off);
    int *status = ws_ptr<int>(ws, ws->status);
    cudaError_t err = cudaMemsetAsync(tile_cnt, 0, sizeof(uint32_t) * B.tot_tiles, st);
    if (err != cudaSuccess) return err;
    if (B.tot_g > 0) {
        launch_dep(k_tile_count, dim3(warp_grid(B.tot_g)), dim3(256), 0, st, B, prep, tile_cnt);
        counted(1);
    }
    return scan_u32(tile_cnt, tile_off, B.tot_tiles, cap, status, DGR_STATUS_PAIR_OVERFLOW,
                    ws_ptr<unsigned long long>(ws, ws->scan_tmp), st);
}

template <int TZ>
static cudaError_t launch_vox_tz(const Batch &B, const Prep *prep, const uint32_t *tile_off,
                                 const uint32_t *list, unsigned long long cap, int *queue,
                                 const int *sep_flag, const VoxSplit &S, cudaStream_t st) {
    // work units: the tiles plus at most SPLIT_BUDGET extra segments per instance
    const int units = B.tot_tiles + B.n * SPLIT_BUDGET;
    const int grid = max(1, min(units, wave_ctas((const void *)k_voxelize<TZ>, VOX_THREADS, 0)));
    // depth 32: the separable kernel as well; exactly one of the two does the work
    const bool sep = TZ == SEP_TZ && g_separable;
    launch_dep(k_voxelize<TZ>, dim3(grid), dim3(VOX_THREADS), 0, st, B, prep, tile_off, list, cap, queue, sep ? sep_flag : nullptr, S);
    counted(1);
    if (sep) {
        const int grid2 = max(1, min(units, wave_ctas((const void *)k_voxelize_sep, VOX_THREADS, 0)));
        launch_dep(k_voxelize_sep, dim3(grid2), dim3(VOX_THREADS), 0, st, B, prep, tile_off, list, cap, queue, sep_flag, S);
        counted(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_voxelize(const Batch &B, const Prep *prep, dgr_ws *ws, int deterministic,
                            cudaStream_t st, const cudaEvent_t *kev) {
    uint32_t *tile_off = ws_ptr<uint32_t>(ws, ws->tile_off);
    uint32_t *tile_fill = ws_ptr<uint32_t>(ws, ws->tile_fill);
    uint32_t *list = ws_ptr<uint32_t>(ws, ws->list);
    int *queue = ws_ptr<int>(ws, ws->status) + VOX_QUEUE;  // unit queue head
    const unsigned long long cap = (unsigned long long)ws->plan.max_pairs;
    cudaError_t err = launch_count_pairs(B, prep, ws, cap, st);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(tile_fill, 0, sizeof(uint32_t) * B.tot_tiles, st);
    // the queue head and the split counters
    if (err == cudaSuccess) err = cudaMemsetAsync(queue, 0, sizeof(int) * (VOX_SLOTCTR + MAX_INST - VOX_QUEUE), st);
    if (err != cudaSuccess) return err;
    if (B.tot_g > 0) {
        launch_dep(k_tile_fill, dim3(warp_grid(B.tot_g)), dim3(256), 0, st, B, prep, tile_off, tile_fill, list, cap);
        counted(1);
    }
    const VoxSplit S = vox_split_of(ws_ptr<int>(ws, ws->vsplit), ws_ptr<float>(ws, ws->vpart),
                                    ws_ptr<int>(ws, ws->status), B.tot_tiles);
    if (deterministic) {
        launch_dep(k_tile_sort_warp, dim3((B.tot_tiles + 7) / 8), dim3(256), 0, st, B, tile_off, list, cap, S);
        launch_dep(k_tile_sort, dim3(B.tot_tiles), dim3(SORT_THREADS), 0, st, B.tot_tiles, tile_off, list,
                                                          ws_ptr<uint32_t>(ws, ws->list_tmp), cap);
        counted(2);
    } else {
        launch_dep(k_split_plan, dim3((B.tot_tiles + 255) / 256), dim3(256), 0, st, B, tile_off, cap, S);
        counted(1);
    }
    // persistent: enough CTAs to fill every SM, each pulling units from the queue
    const int *sep_flag = ws_ptr<int>(ws, ws->status) + SEP_FLAG;
    if (kev && (err = cudaEventRecord(kev[0], st)) != cudaSuccess) return err;
    switch (B.tz) {
        case 8: err = launch_vox_tz<8>(B, prep, tile_off, list, cap, queue, sep_flag, S, st); break;
        case 16: err = launch_vox_tz<16>(B, prep, tile_off, list, cap, queue, sep_flag, S, st); break;
        default: err = launch_vox_tz<32>(B, prep, tile_off, list, cap, queue, sep_flag, S, st);
    }
    if (err == cudaSuccess && kev) err = cudaEventRecord(kev[1], st);
    return err;
}

}  // namespace dgr
