// The paper's full objective (Sec. 4.3; App. D.1):
//     L = w_l1 L1(P_hat, P) + w_ssim (1 - SSIM(P_hat, P)) + w_tv TV(V)
// with weights 0.6 / 0.2 / 1 in the paper.  SSIM is taken on every projection
// image (view) with the windowed statistics of Wang et al. 2004: an 11 x 11
// Gaussian window (sigma 1.5, zero outside the image), C1 = (0.01 L)^2,
// C2 = (0.03 L)^2, averaged over all pixels of all views.  TV is the
// anisotropic total variation of the volume, sum over axes of |forward
// differences| divided by the number of voxels.
//
//   k_ssim_stats  per 32 x 16 pixel tile of a view: windowed means, variances
//                 and covariance through a shared-memory tile with a 5-pixel
//                 halo (separable window), the SSIM map's sum, and the three
//                 maps A = dS/dmu_x - 2 mu_x dS/dsxx - mu_y dS/dsxy,
//                 B = dS/dsxx, C = dS/dsxy of the gradient
//   k_ssim_grad   d(1 - SSIM)/dP_hat = -[(w*A) + 2 P_hat (w*B) + P (w*C)] / N,
//                 scaled by w_ssim, for the residual of the backprojector
//   k_tv          TV partial sums and w_tv dTV/dV added to the volume gradient
//                 (shared-memory tile of the volume with a one-voxel halo)
//   k_loss_final  per instance, fixed order: the weighted sum of the terms
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr int SW = 11, SR = 5;        // window taps, radius
constexpr int STX = 32, STY = 16;     // SSIM output tile (u, v)
constexpr int SHX = STX + 2 * SR, SHY = STY + 2 * SR;
constexpr int S_THREADS = 256;

__device__ __forceinline__ int inst_of_st(const Batch &B, int t) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].st0 <= t) ++i;
    return i;
}
__device__ __forceinline__ int inst_of_tv(const Batch &B, int t) {
    int i = 0;
    while (i + 1 < B.n && B.in[i + 1].tv0 <= t) ++i;
    return i;
}

// block sum in a fixed order (warp shuffles, then warp 0 over the warp sums)
__device__ __forceinline__ float block_sum(float s) {
    __shared__ float wsum[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    return t;
}

struct SsimTile {
    const Inst *I;
    int k, u0, v0;
};

__device__ __forceinline__ SsimTile ssim_tile(const Batch &B, int bid) {
    SsimTile T;
    const Inst &I = B.in[inst_of_st(B, bid)];
    const int b = bid - I.st0;
    const int ntu = (I.nu + STX - 1) / STX, ntv = (I.nv + STY - 1) / STY;
    T.I = &I;
    T.u0 = (b % ntu) * STX;
    T.v0 = ((b / ntu) % ntv) * STY;
    T.k = b / (ntu * ntv);
    return T;
}

// windowed sums of NM maps of a tile: in[m][SHY][SHX] (halo included) ->
// out[m][STY][STX] through the separable window
template <int NM>
__device__ __forceinline__ void blur_tile(const float (*in)[SHY][SHX], float (*hs)[SHY][STX],
                                          const float *w, float out[][2], int py[2], int px) {
    for (int e = threadIdx.x; e < NM * SHY * STX; e += S_THREADS) {
        const int m = e / (SHY * STX), r = (e / STX) % SHY, c = e % STX;
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < SW; ++t) s = fmaf(w[t], in[m][r][c + t], s);
        hs[m][r][c] = s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < SW; ++t) s = fmaf(w[t], hs[m][py[j] + t][px], s);
            out[m][j] = s;
        }
}

__global__ void __launch_bounds__(S_THREADS) k_ssim_stats(const __grid_constant__ Batch B,
                                                          float *__restrict__ maps,
                                                          float *__restrict__ spart) {
    DEP_ENTER();
    __shared__ float in[5][SHY][SHX];
    __shared__ float hs[5][SHY][STX];
    const SsimTile T = ssim_tile(B, blockIdx.x);
    const Inst &I = *T.I;
    const size_t plane = (size_t)I.nv * I.nu;
    const float *x = I.sino + (size_t)T.k * plane;  // prediction
    const float *y = I.meas + (size_t)T.k * plane;  // measurement
    for (int e = threadIdx.x; e < SHY * SHX; e += S_THREADS) {
        const int r = e / SHX, c = e % SHX;
        const int v = T.v0 + r - SR, u = T.u0 + c - SR;
        float a = 0.f, b = 0.f;
        if (v >= 0 && v < I.nv && u >= 0 && u < I.nu) {
            a = x[(size_t)v * I.nu + u];
            b = y[(size_t)v * I.nu + u];
        }
        in[0][r][c] = a;
        in[1][r][c] = b;
        in[2][r][c] = a * a;
        in[3][r][c] = b * b;
        in[4][r][c] = a * b;
    }
    __syncthreads();
    const int px = threadIdx.x % STX;
    int py[2] = {(int)(threadIdx.x / STX), (int)(threadIdx.x / STX) + S_THREADS / STX};
    float st[5][2];
    blur_tile<5>(in, hs, B.ssim_w, st, py, px);
    const size_t tot = (size_t)B.tot_rays;
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int u = T.u0 + px, v = T.v0 + py[j];
        if (u >= I.nu || v >= I.nv) continue;
        const float mx = st[0][j], my = st[1][j];
        const float sxx = st[2][j] - mx * mx, syy = st[3][j] - my * my, sxy = st[4][j] - mx * my;
        const float n1 = 2.f * mx * my + I.ssim_c1, n2 = 2.f * sxy + I.ssim_c2;
        const float d1 = mx * mx + my * my + I.ssim_c1, d2 = sxx + syy + I.ssim_c2;
        const float dd = d1 * d2;
        const float S = n1 * n2 / dd;
        const float dmx = 2.f * my * n2 / dd - 2.f * mx * S / d1;
        const float dsxx = -S / d2;
        const float dsxy = 2.f * n1 / dd;
        const size_t o = (size_t)I.ray0 + (size_t)T.k * plane + (size_t)v * I.nu + u;
        maps[o] = dmx - 2.f * mx * dsxx - my * dsxy;  // A
        maps[tot + o] = dsxx;                          // B
        maps[2 * tot + o] = dsxy;                      // C
        s += S;
    }
    const float t = block_sum(s);
    if (threadIdx.x == 0) spart[blockIdx.x] = t;
}

__global__ void __launch_bounds__(S_THREADS) k_ssim_grad(const __grid_constant__ Batch B,
                                                         const float *__restrict__ maps,
                                                         float *__restrict__ gout) {
    DEP_ENTER();
    __shared__ float in[3][SHY][SHX];
    __shared__ float hs[3][SHY][STX];
    const SsimTile T = ssim_tile(B, blockIdx.x);
    const Inst &I = *T.I;
    const size_t plane = (size_t)I.nv * I.nu;
    const size_t base = (size_t)I.ray0 + (size_t)T.k * plane;
    const size_t tot = (size_t)B.tot_rays;
    for (int e = threadIdx.x; e < SHY * SHX; e += S_THREADS) {
        const int r = e / SHX, c = e % SHX;
        const int v = T.v0 + r - SR, u = T.u0 + c - SR;
        float a = 0.f, b = 0.f, cc = 0.f;
        if (v >= 0 && v < I.nv && u >= 0 && u < I.nu) {
            const size_t o = base + (size_t)v * I.nu + u;
            a = maps[o];
            b = maps[tot + o];
            cc = maps[2 * tot + o];
        }
        in[0][r][c] = a;
        in[1][r][c] = b;
        in[2][r][c] = cc;
    }
    __syncthreads();
    const int px = threadIdx.x % STX;
    int py[2] = {(int)(threadIdx.x / STX), (int)(threadIdx.x / STX) + S_THREADS / STX};
    float wb[3][2];
    blur_tile<3>(in, hs, B.ssim_w, wb, py, px);
    // d(1 - mean S)/dx = -(...)/N, N every pixel of every view of the instance
    const float scale = -I.w_ssim / (float)((double)I.n_views * plane);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int u = T.u0 + px, v = T.v0 + py[j];
        if (u >= I.nu || v >= I.nv) continue;
        const size_t o = base + (size_t)v * I.nu + u;
        const float xv = I.sino[o - I.ray0], yv = I.meas[o - I.ray0];
        gout[o] = scale * (wb[0][j] + 2.f * xv * wb[1][j] + yv * wb[2][j]);
    }
}

// TV: tile of 32 (x) x TVY (y) x TVZ (z) voxels; the volume with a one-voxel
// halo in x, y and z goes through shared memory once (rows y-1 .. y+TVY), so
// each voxel is read about (TVY + 2) / TVY times
constexpr int TVX = 32, TVY = 8, TVZ = 16;
__global__ void __launch_bounds__(256) k_tv(const __grid_constant__ Batch B, float *__restrict__ tpart,
                                            int accumulate) {
    DEP_ENTER();
    __shared__ float s[TVY + 2][TVZ + 2][TVX + 3];
    const Inst &I = B.in[inst_of_tv(B, blockIdx.x)];
    const dgr_grid &g = I.g;
    const int ntx = (g.nx + TVX - 1) / TVX, nty = (g.ny + TVY - 1) / TVY;
    const int b = blockIdx.x - I.tv0;
    const int x0 = (b % ntx) * TVX, y0 = ((b / ntx) % nty) * TVY, z0 = (b / (ntx * nty)) * TVZ;
    const bool zfast = I.vsz == 1;
    // load V[x0-1 .. x0+32][y0-1 .. y0+TVY][z0-1 .. z0+TVZ] (zero outside)
    const int nl = (TVY + 2) * (TVZ + 2) * (TVX + 2);
    for (int e = threadIdx.x; e < nl; e += 256) {
        int dy, zz, xx;
        if (zfast) {  // consecutive threads along z
            zz = e % (TVZ + 2); xx = (e / (TVZ + 2)) % (TVX + 2); dy = e / ((TVZ + 2) * (TVX + 2));
        } else {      // consecutive threads along x
            xx = e % (TVX + 2); zz = (e / (TVX + 2)) % (TVZ + 2); dy = e / ((TVZ + 2) * (TVX + 2));
        }
        const int x = x0 + xx - 1, yy = y0 + dy - 1, z = z0 + zz - 1;
        float v = 0.f;
        if (x >= 0 && x < g.nx && yy >= 0 && yy < g.ny && z >= 0 && z < g.nz)
            v = I.vol[(size_t)x * I.vsx + (size_t)yy * I.vsy + (size_t)z * I.vsz];
        s[dy][zz][xx] = v;
    }
    __syncthreads();
    const float w = I.w_tv / (float)((double)g.nx * g.ny * g.nz);
    const int xx = threadIdx.x & 31, r8 = threadIdx.x >> 5;  // 32 x 8
    const int x = x0 + xx;
    float acc = 0.f;
    for (int e = r8; e < TVY * TVZ; e += 8) {
        const int yy = e / TVZ, zz = e % TVZ;
        const int y = y0 + yy, z = z0 + zz;
        if (x >= g.nx || y >= g.ny || z >= g.nz) continue;
        const float c = s[yy + 1][zz + 1][xx + 1];
        float grad = 0.f;
        // forward differences (the term) and the two differences each voxel is in
        if (x + 1 < g.nx) { const float d = s[yy + 1][zz + 1][xx + 2] - c; acc += fabsf(d); grad -= (d > 0.f) - (d < 0.f); }
        if (x > 0) { const float d = c - s[yy + 1][zz + 1][xx]; grad += (d > 0.f) - (d < 0.f); }
        if (y + 1 < g.ny) { const float d = s[yy + 2][zz + 1][xx + 1] - c; acc += fabsf(d); grad -= (d > 0.f) - (d < 0.f); }
        if (y > 0) { const float d = c - s[yy][zz + 1][xx + 1]; grad += (d > 0.f) - (d < 0.f); }
        if (z + 1 < g.nz) { const float d = s[yy + 1][zz + 2][xx + 1] - c; acc += fabsf(d); grad -= (d > 0.f) - (d < 0.f); }
        if (z > 0) { const float d = c - s[yy + 1][zz][xx + 1]; grad += (d > 0.f) - (d < 0.f); }
        float *o = I.gvol + ((size_t)z * g.ny + y) * g.nx + x;
        *o = accumulate ? fmaf(w, grad, *o) : w * grad;
    }
    const float t = block_sum(acc);
    if (threadIdx.x == 0) tpart[blockIdx.x] = t;
}

// one warp per instance: fixed-order FP64 sums of the partials
__global__ void k_loss_final(const __grid_constant__ Batch B, const float *__restrict__ l1part,
                             int l1_blocks, const float *__restrict__ spart,
                             const float *__restrict__ tpart) {
    DEP_ENTER();
    const Inst &I = B.in[blockIdx.x];
    const double m = (double)I.n_views * I.nu * I.nv;
    double l1 = 0.0, ss = 0.0, tv = 0.0;
    for (int i = threadIdx.x; i < l1_blocks; i += 32) l1 += (double)l1part[blockIdx.x * l1_blocks + i];
    if (I.w_ssim != 0.f)
        for (int i = I.st0 + threadIdx.x; i < I.st0 + I.nst; i += 32) ss += (double)spart[i];
    if (I.w_tv != 0.f)
        for (int i = I.tv0 + threadIdx.x; i < I.tv0 + I.ntv; i += 32) tv += (double)tpart[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        tv += __shfl_xor_sync(0xffffffffu, tv, o);
    }
    if (threadIdx.x == 0) {
        // the L1 partials are sums of |d| (the mean is taken here)
        double L = 0.0;
        if (I.w_l1 != 0.f) L += (double)I.w_l1 * (l1 / m);
        if (I.w_ssim != 0.f) L += (double)I.w_ssim * (1.0 - ss / m);
        if (I.w_tv != 0.f) L += (double)I.w_tv * (tv / ((double)I.g.nx * I.g.ny * I.g.nz));
        *I.loss = (float)L;
    }
}

}  // namespace

// the window of the SSIM statistics, from its definition (host, FP64)
void ssim_window(float *w) {
    double g[SW], z = 0.0;
    for (int i = 0; i < SW; ++i) {
        const double d = i - SR;
        g[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
        z += g[i];
    }
    for (int i = 0; i < SW; ++i) w[i] = (float)(g[i] / z);
}

// tile counts of the SSIM and TV passes; fills st0/nst and tv0/ntv
void loss_tiles(Batch &B) {
    int st = 0, tv = 0;
    for (int i = 0; i < B.n; ++i) {
        Inst &I = B.in[i];
        I.st0 = st;
        I.nst = I.w_ssim != 0.f ? I.n_views * ((I.nu + STX - 1) / STX) * ((I.nv + STY - 1) / STY) : 0;
        st += I.nst;
        I.tv0 = tv;
        I.ntv = I.w_tv != 0.f
                    ? ((I.g.nx + TVX - 1) / TVX) * ((I.g.ny + TVY - 1) / TVY) * ((I.g.nz + TVZ - 1) / TVZ)
                    : 0;
        tv += I.ntv;
    }
    B.tot_st = st;
    B.tot_tv = tv;
    ssim_window(B.ssim_w);
}

size_t ssim_tiles_cap(long long max_views, int max_nu, int max_nv, int ninst) {
    return (size_t)max_views * ((max_nu + STX - 1) / STX) * ((max_nv + STY - 1) / STY) + ninst;
}
size_t tv_tiles_cap(long long max_vox, int ninst) {
    // a tile holds up to 32 x 8 x 16 voxels; thin grids (fewer than 8 voxels
    // in x times y times z per tile) need more tiles than this and are refused
    return (size_t)(max_vox / 8) + (size_t)4096 * ninst;
}

cudaError_t launch_ssim(const Batch &B, float *maps, float *spart, float *gout, cudaStream_t st) {
    if (B.tot_st == 0) return cudaSuccess;
    launch_dep(k_ssim_stats, dim3(B.tot_st), dim3(S_THREADS), 0, st, B, maps, spart);
    launch_dep(k_ssim_grad, dim3(B.tot_st), dim3(S_THREADS), 0, st, B, maps, gout);
    counted(2);
    return cudaGetLastError();
}

cudaError_t launch_tv(const Batch &B, float *tpart, int accumulate, cudaStream_t st) {
    if (B.tot_tv == 0) return cudaSuccess;
    launch_dep(k_tv, dim3(B.tot_tv), dim3(256), 0, st, B, tpart, accumulate);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_loss_final(const Batch &B, const float *l1part, int l1_blocks, const float *spart,
                              const float *tpart, cudaStream_t st) {
    launch_dep(k_loss_final, dim3(B.n), dim3(32), 0, st, B, l1part, l1_blocks, spart, tpart);
    counted(1);
    return cudaGetLastError();
}

}  // namespace dgr
