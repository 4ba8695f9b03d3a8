// Adjoint of Fast Volume Reconstruction (a7) on sm_103a.
//
// Gaussian-driven gather: the volume gradient G_V is read at each pair, so no
// per-voxel scatter and no atomics are needed.  Each Gaussian's box is cut into
// z-chunks of at most ~ITEM_VOX voxels (work items, so one huge Gaussian is
// spread over many warps).  A warp walks its item: lanes over the (x, y) patch,
// an inner loop over z with the quadratic form updated in closed form, and
// accumulates the 10 moments
//     M0 = sum G e,  M1 = sum G e d,  M2 = sum G e d d^T      (d = v - u)
// that determine the whole gradient.  Per-item moments are reduced across the
// warp with shuffles and summed per Gaussian in item order (deterministic).
// The per-Gaussian epilogue chains
//     dL/drho = M0,  dL/du = rho A M1,  dL/dA = -1/2 rho M2
// through u = (mu - o)/h - 1/2 and A = h^2 R(q/|q|) diag(s^-2) R^T.
#include <math.h>

#include <type_traits>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Transposing butterfly over the 32 lanes for NMOM = 10 partial sums per
// lane.  Level xor 16: lists of 10 split 5 / 5; xor 8: 5 split 3 / 2; xor 4:
// 3 (the 2-lists padded with a zero) split 2 / 1; xor 2: 2 split 1 / 1; xor
// 1: both lanes add their single values.  Per shuffle, the lane whose mask
// bit is clear keeps the low part and sends the high one, its partner the
// reverse.  m[0] then holds, for lane pair p = lane / 2, the full sum of
// moment kMomOfPair[p] (-1: a padding zero).
static_assert(NMOM == 10, "the butterfly's splits are laid out for 10 moments");
__constant__ int kMomOfPair[16] = {0, 1, 2, -1, 3, 4, -1, -1, 5, 6, 7, -1, 8, 9, -1, -1};
__device__ __forceinline__ void mom_reduce(float *v, int lane) {
    const unsigned FULL = 0xffffffffu;
    {   // 10 -> 5
        const bool hi = lane & 16;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float send = hi ? v[i] : v[5 + i], keep = hi ? v[5 + i] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 16);
        }
    }
    {   // 5 -> 3 (low: 0..2) or 2 (high: 3..4, padded to 3)
        const bool hi = lane & 8;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float h = i < 2 ? v[3 + i] : 0.f;
            const float send = hi ? v[i] : h, keep = hi ? h : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, 8);
        }
    }
    {   // 3 -> 2 (low: 0..1) or 1 (high: 2)
        const bool hi = lane & 4;
        const float s0 = hi ? v[0] : v[2], k0 = hi ? v[2] : v[0];
        const float s1 = hi ? v[1] : 0.f, k1 = hi ? 0.f : v[1];
        v[0] = k0 + __shfl_xor_sync(FULL, s0, 4);
        v[1] = k1 + __shfl_xor_sync(FULL, s1, 4);
    }
    {   // 2 -> 1
        const bool hi = lane & 2;
        const float send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(FULL, send, 2);
    }
    v[0] += __shfl_xor_sync(FULL, v[0], 1);
}

// items per run taken from the queue: consecutive items mostly belong to
// the same Gaussian, so a run costs one owner search
constexpr int ITEM_RUN = 8;

__global__ void __launch_bounds__(256, 4) k_bwd_items(
    const __grid_constant__ Batch B, const Prep *__restrict__ prep,
    const uint32_t *__restrict__ item_off, unsigned long long cap, float *__restrict__ part,
    int *__restrict__ queue) {
    DEP_ENTER();
    const int n = B.tot_g;
    const int lane = threadIdx.x & 31;
    unsigned long long total = item_off[n];
    if (total > cap) total = cap;
    // warps take runs of ITEM_RUN consecutive items from a global queue (load
    // balance for uneven items); one owner search per run, then the owner
    // only moves forward
    for (;;) {
        int run = 0;
        if (lane == 0) run = atomicAdd(queue, 1);
        run = __shfl_sync(0xffffffffu, run, 0);
        const long long it0 = (long long)run * ITEM_RUN;
        if (it0 >= (long long)total) break;
        const long long it1 = min((long long)total, it0 + ITEM_RUN);
        int gi = -1;
        for (long long it = it0; it < it1; ++it) {
            if (gi < 0) {
                // Gaussian owning item `it`: the last gi with item_off[gi] <= it, by a
                // 32-ary search (each round every lane probes one pivot)
                int lo = 0, hi = n;  // item_off[lo] <= it < item_off[hi]
                while (hi - lo > 1) {
                    const int step = (hi - lo + 31) >> 5;
                    const int probe = lo + lane * step;
                    const bool le = probe < hi && (unsigned long long)item_off[probe] <= (unsigned long long)it;
                    const unsigned m = __ballot_sync(0xffffffffu, le);  // lane 0 always set
                    const int k = 31 - __clz(m);
                    lo += k * step;
                    hi = min(hi, lo + step);
                }
                gi = lo;
            } else {
                // it < total <= item_off[n]: stops at gi <= n - 1 (skips Gaussians without items)
                while ((unsigned long long)item_off[gi + 1] <= (unsigned long long)it) ++gi;
            }
            const int c = (int)(it - item_off[gi]);
            const Inst &I = B.in[inst_of_g(B, gi)];
            const dgr_grid &g = I.g;
            const float *__restrict__ gv = I.gvol;
            const long long nvox = (long long)g.nx * g.ny * g.nz;
            (void)nvox;
            const Prep P = prep[gi];
            const float n1y = (float)P.n1y_d;
            const int lx = box_lo(P.bx), hx = box_hi(P.bx), ly = box_lo(P.by), hy = box_hi(P.by),
                      lz = box_lo(P.bz), hz = box_hi(P.bz);
            const int ex = hx - lx + 1, ey = hy - ly + 1;
            int yb, ye, zb, ze;
            item_range(c, ex, ey, ly, hy, lz, hz, yb, ye, zb, ze);
            float m[NMOM];
#pragma unroll
            for (int k = 0; k < NMOM; ++k) m[k] = 0.f;
            const int exy = ex * (ye - yb + 1);
            const float dz0 = (float)(zb - P.az) - P.dz;
            const float inv_ex = 1.0f / (float)ex;
            for (int j = lane; j < exy; j += 32) {
                // j = row * ex + col, by a float reciprocal and one correction
                int row = (int)((float)j * inv_ex);
                row -= row * ex > j;
                row += (row + 1) * ex <= j;
                const int yy = yb + row, xx = lx + (j - row * ex);
                const float dx = (float)(xx - P.ax) - P.dx;
                const float dy = (float)(yy - P.ay) - P.dy;
                // column form: q = qm + a22 t^2, t = dz - dz* (the column's peak),
                // qm from the column's principal coordinates
                const float c1 = fmaf(P.n1x, dx, n1y * dy), c2 = fmaf(-n1y, dx, P.n1x * dy);
                const float qm = fmaf(P.l1 * c1, c1, P.l2 * c2 * c2);
                const float dzs = fmaf(P.zx, dx, P.zy * dy);
                const float t0 = dz0 - dzs;
                const float *col = gv + ((size_t)zb * g.ny + yy) * g.nx + xx;
                const size_t zs = (size_t)g.nx * g.ny;
                // the column's sums over z of ge, ge t, ge t^2 (ge = G_V e), in two
                // packed FP32 lanes (even and odd layers of each group of four)
                const float2 a22v = make_float2(P.a22, P.a22), qmv = make_float2(qm, qm),
                             t0v = make_float2(t0, t0);
                float2 s0v = make_float2(0.f, 0.f), s1v = s0v, s2v = s0v;
                int z = zb;
                // U layers at a time (8, then 4): loads first, then the arithmetic
                auto layers = [&](auto U_) {
                    constexpr int U = decltype(U_)::value;
                    float gz[U];
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        gz[u] = DGR_INB(col + u * zs - gv, nvox, B.status) ? __ldg(col + u * zs) : 0.f;
                    col += U * zs;
#pragma unroll
                    for (int u = 0; u < U; u += 2) {
                        const float2 t = __fadd2_rn(t0v, make_float2((float)(z + u - zb), (float)(z + u + 1 - zb)));
                        const float2 q = __ffma2_rn(__fmul2_rn(a22v, t), t, qmv);
                        const float2 ge = __fmul2_rn(make_float2(gz[u], gz[u + 1]),
                                                     make_float2(ex2_approx(q.x), ex2_approx(q.y)));
                        s0v = __fadd2_rn(s0v, ge);
                        const float2 gt = __fmul2_rn(ge, t);
                        s1v = __fadd2_rn(s1v, gt);
                        s2v = __ffma2_rn(gt, t, s2v);
                    }
                    z += U;
                };
                while (z + 7 <= ze) layers(std::integral_constant<int, 8>());
                if (z + 3 <= ze) layers(std::integral_constant<int, 4>());
                for (; z <= ze; ++z) {
                    const float t = t0 + (float)(z - zb);
                    const float e = ex2_approx(fmaf(P.a22 * t, t, qm));
                    const float ge = (DGR_INB(col - gv, nvox, B.status) ? __ldg(col) : 0.f) * e;
                    col += zs;
                    s0v.x += ge;
                    const float gt = ge * t;
                    s1v.x += gt;
                    s2v.x = fmaf(gt, t, s2v.x);
                }
                // back to moments in dz = t + dz*
                const float s0 = s0v.x + s0v.y, s1t = s1v.x + s1v.y, s2t = s2v.x + s2v.y;
                const float s1 = fmaf(dzs, s0, s1t);
                const float s2 = fmaf(dzs, fmaf(dzs, s0, 2.f * s1t), s2t);
                m[0] += s0;
                m[1] = fmaf(dx, s0, m[1]);
                m[2] = fmaf(dy, s0, m[2]);
                m[3] += s1;
                m[4] = fmaf(dx * dx, s0, m[4]);  // xx
                m[5] = fmaf(dy * dy, s0, m[5]);  // yy
                m[6] += s2;                      // zz
                m[7] = fmaf(dx * dy, s0, m[7]);  // xy
                m[8] = fmaf(dx, s1, m[8]);       // xz
                m[9] = fmaf(dy, s1, m[9]);       // yz
            }
            // the 10 sums over the warp by a transposing butterfly: at each
            // level the pair of lanes splits its list of partial sums, each
            // keeping one half and adding the partner's copy of it (12
            // shuffles instead of 10 x 5); the even lanes of 10 lane pairs end
            // with one moment each (mom_of_pair)
            mom_reduce(m, lane);
            const int k = kMomOfPair[lane >> 1];
            if ((lane & 1) == 0 && k >= 0) part[(size_t)it * NMOM + k] = m[0];
        }
    }
}

// the chain rule of one Gaussian from its summed moments M (empty: no
// voxel of its box was reached, every gradient is zero)
__device__ void bwd_finish(const Inst &I, int i, bool empty, const float *M) {
    const dgr_grid &g = I.g;
    const float *__restrict__ s = I.s;
    const float4 *__restrict__ q = reinterpret_cast<const float4 *>(I.q);
    const float *__restrict__ rho = I.rho;
    float *__restrict__ g_mu = I.g_mu;
    float *__restrict__ g_s = I.g_s;
    float *__restrict__ g_q = I.g_q;
    float *__restrict__ g_rho = I.g_rho;
    if (empty) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { g_mu[3 * i + a] = 0.f; g_s[3 * i + a] = 0.f; }
#pragma unroll
        for (int a = 0; a < 4; ++a) g_q[4 * i + a] = 0.f;
        g_rho[i] = 0.f;
        return;
    }
    // rotation of the normalised quaternion
    const float4 qq = q[i];
    const float qnorm = sqrtf(qq.x * qq.x + qq.y * qq.y + qq.z * qq.z + qq.w * qq.w);
    const float iq = 1.0f / qnorm;
    const float w = qq.x * iq, x = qq.y * iq, y = qq.z * iq, z = qq.w * iq;
    float R[9];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    const float h = g.h, h2 = h * h;
    const float sx = s[3 * i], sy = s[3 * i + 1], sz = s[3 * i + 2];
    const float D[3] = {1.f / (sx * sx), 1.f / (sy * sy), 1.f / (sz * sz)};
    // A = h^2 R D R^T
    float A[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2)
            A[3 * a + b2] = h2 * (R[3 * a] * R[3 * b2] * D[0] + R[3 * a + 1] * R[3 * b2 + 1] * D[1] +
                                  R[3 * a + 2] * R[3 * b2 + 2] * D[2]);
    const float r = rho[i];
    g_rho[i] = M[0];
    const float M1[3] = {M[1], M[2], M[3]};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        g_mu[3 * i + a] = r * (A[3 * a] * M1[0] + A[3 * a + 1] * M1[1] + A[3 * a + 2] * M1[2]) / h;
    // dL/dA = -1/2 rho M2 (symmetric)
    const float c = -0.5f * r;
    const float GA[9] = {c * M[4], c * M[7], c * M[8],
                         c * M[7], c * M[5], c * M[9],
                         c * M[8], c * M[9], c * M[6]};
    // GR = GA R  (3x3)
    float GR[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            GR[3 * a + k] = GA[3 * a] * R[k] + GA[3 * a + 1] * R[3 + k] + GA[3 * a + 2] * R[6 + k];
    // dL/ds_k = h^2 (R^T GA R)_kk (-2 / s_k^3)
    const float sv[3] = {sx, sy, sz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float rgr = R[k] * GR[k] + R[3 + k] * GR[3 + k] + R[6 + k] * GR[6 + k];
        g_s[3 * i + k] = h2 * rgr * (-2.f / (sv[k] * sv[k] * sv[k]));
    }
    // dL/dR = 2 h^2 GA R D
    float gR[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) gR[3 * a + k] = 2.f * h2 * GR[3 * a + k] * D[k];
    const float gw = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    const float gx = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] +
                            z * gR[6] + w * gR[7] - 2.f * x * gR[8]);
    const float gy = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] -
                            w * gR[6] + z * gR[7] - 2.f * y * gR[8]);
    const float gz = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] +
                            y * gR[5] + x * gR[6] + y * gR[7]);
    const float dot = w * gw + x * gx + y * gy + z * gz;
    g_q[4 * i + 0] = (gw - w * dot) * iq;
    g_q[4 * i + 1] = (gx - x * dot) * iq;
    g_q[4 * i + 2] = (gy - y * dot) * iq;
    g_q[4 * i + 3] = (gz - z * dot) * iq;
}

__global__ void k_bwd_final(const __grid_constant__ Batch B,
                            const uint32_t *__restrict__ item_off, unsigned long long cap,
                            const float *__restrict__ part, uint32_t *__restrict__ big,
                            int *__restrict__ big_count) {
    DEP_ENTER();
    // four lanes per Gaussian: lane c of the quad sums items b + c, b + c + 4,
    // ... (compensated FP32), two fixed butterfly steps combine the quad, lane
    // 0 of it finishes the chain rule
    const int gi = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 2), c4 = threadIdx.x & 3;
    if (gi >= B.tot_g) return;  // quad-uniform (quads never straddle a warp)
    const Inst &I = B.in[inst_of_g(B, gi)];
    const int i = gi - I.g0;
    unsigned long long b = item_off[gi], e = item_off[gi + 1];
    if (e > cap) e = cap;
    // a Gaussian with many items goes to k_bwd_big (a CTA each)
    if (e > b + BIG_ITEMS) {
        if (c4 == 0) big[atomicAdd(big_count, 1)] = (uint32_t)gi;
        return;
    }
    // item partials in compensated FP32 (Kahan: the sum s and the running
    // error c, exact sum ~ s - c; at most BIG_ITEMS items, BIG_ITEMS / 4 per
    // lane), the quad's lanes combined by an error-free two-sum.  A fixed order
    // throughout: bit-reproducible.
    float Ms[NMOM], Mc[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) Ms[k] = Mc[k] = 0.f;
    for (unsigned long long it = b + c4; it < e; it += 4) {
        const float *src = part + it * NMOM;
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            const float y = src[k] - Mc[k];
            const float t = Ms[k] + y;
            Mc[k] = (t - Ms[k]) - y;
            Ms[k] = t;
        }
    }
    // the quad's lanes are consecutive: xor 1 then xor 2 stays inside it
    const unsigned qmask = 0xFu << (threadIdx.x & 28);
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            const float a = Ms[k], bb = __shfl_xor_sync(qmask, Ms[k], o);
            const float cb = __shfl_xor_sync(qmask, Mc[k], o);
            const float t = a + bb, bp = t - a;
            const float err = (a - (t - bp)) + (bb - bp);  // a + bb = t + err exactly
            Ms[k] = t;
            Mc[k] = (Mc[k] + cb) - err;
        }
    }
    if (c4 != 0) return;
    float M[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) M[k] = Ms[k] - Mc[k];
    bwd_finish(I, i, b >= e, M);
}

// Gaussians with more than BIG_ITEMS items: a CTA each (CTAs stride over the
// list k_bwd_final built); every thread sums items b + t, b + t + 256, ... with
// Kahan-compensated FP32 sums, the CTA combines them in FP64 in a fixed order
__global__ void __launch_bounds__(256) k_bwd_big(const __grid_constant__ Batch B,
                                                 const uint32_t *__restrict__ item_off, unsigned long long cap,
                                                 const float *__restrict__ part,
                                                 const uint32_t *__restrict__ big,
                                                 const int *__restrict__ big_count) {
    DEP_ENTER();
    __shared__ double sred[256 / 32][NMOM];
    const int nbig = *big_count;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = blockIdx.x; j < nbig; j += gridDim.x) {  // CTA-uniform
        const int gi = (int)big[j];
        const Inst &I = B.in[inst_of_g(B, gi)];
        unsigned long long b = item_off[gi], e = item_off[gi + 1];
        if (e > cap) e = cap;
        float sm[NMOM], cm[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) sm[k] = cm[k] = 0.f;
        for (unsigned long long it = b + threadIdx.x; it < e; it += 256) {
            const float *src = part + it * NMOM;
#pragma unroll
            for (int k = 0; k < NMOM; ++k) {
                const float y = src[k] - cm[k];
                const float t = sm[k] + y;
                cm[k] = (t - sm[k]) - y;
                sm[k] = t;
            }
        }
        double d[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            d[k] = (double)sm[k] - (double)cm[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d[k] += __shfl_xor_sync(0xffffffffu, d[k], o);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NMOM; ++k) sred[w][k] = d[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            float M[NMOM];
#pragma unroll
            for (int k = 0; k < NMOM; ++k) {
                double t = 0.0;
                for (int u = 0; u < 256 / 32; ++u) t += sred[u][k];
                M[k] = (float)t;
            }
            bwd_finish(I, gi - I.g0, false, M);
        }
        __syncthreads();  // sred is rewritten by the next Gaussian
    }
}

}  // namespace

cudaError_t launch_voxelize_backward(const Batch &B, const Prep *prep, dgr_ws *ws, cudaStream_t st,
                                     const cudaEvent_t *kev) {
    if (B.tot_g == 0) return cudaSuccess;
    uint32_t *itemcnt = ws_ptr<uint32_t>(ws, ws->itemcnt);
    uint32_t *item_off = ws_ptr<uint32_t>(ws, ws->item_off);
    float *part = ws_ptr<float>(ws, ws->partials);
    int *status = ws_ptr<int>(ws, ws->status);
    const unsigned long long cap = (unsigned long long)ws->plan.max_items;
    cudaError_t err = scan_u32(itemcnt, item_off, B.tot_g, cap, status, DGR_STATUS_ITEM_OVERFLOW,
                               ws_ptr<unsigned long long>(ws, ws->scan_tmp), st);
    if (err != cudaSuccess) return err;
    // the item counts are consumed by the scan: their array holds the list of
    // Gaussians with many items, its length in the status word BIG_COUNT
    uint32_t *big = itemcnt;
    int *big_count = status + BIG_COUNT;
    static_assert(ITEM_QUEUE == BIG_COUNT + 1, "one memset zeroes both words");
    err = cudaMemsetAsync(big_count, 0, 2 * sizeof(int), st);
    if (err != cudaSuccess) return err;
    // one wave of resident CTAs; warps take runs of items from the queue
    if (kev && (err = cudaEventRecord(kev[0], st)) != cudaSuccess) return err;
    launch_dep(k_bwd_items, dim3(wave_ctas((const void *)k_bwd_items, 256, 0)), dim3(256), 0, st, B, prep, item_off, cap, part,
                                                                              status + ITEM_QUEUE);
    if (kev && (err = cudaEventRecord(kev[1], st)) != cudaSuccess) return err;
    launch_dep(k_bwd_final, dim3((unsigned)(((long long)B.tot_g * 4 + 127) / 128)), dim3(128), 0, st, B, item_off, cap, part, big,
                                                                                    big_count);
    launch_dep(k_bwd_big, dim3(148 * 2), dim3(256), 0, st, B, item_off, cap, part, big, big_count);
    counted(3);
    return cudaGetLastError();
}

}  // namespace dgr
