// L1 data term (a5), optimiser-variable transforms and fused Adam (a8).
//
// Objective: the L1 term of the paper's loss (Sec. 4.3, Eq. 13; the SSIM and TV
// terms are in loss.cu, the weighted total in k_loss_final); Adam with the
// learning rate decaying 3e-4 -> 3e-5 over the run (Sec. 5.1).  The decay law,
// the Adam constants and the parameterisation are not stated in the paper; the
// choices (exponential decay; betas 0.9/0.999, eps 1e-8; mu in [-1,1]^3 box
// coordinates, log s, raw q, inverse-softplus rho) are this library's.
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr int L1_THREADS = 256;

// per-instance loss partials: grid (L1_BLOCKS, instance), grid-stride over the
// instance's rays; resid = w sign(pred - meas) / m (+ gadd, the other terms'
// gradient with respect to pred) written over pred
__device__ __forceinline__ float l1_block(const float *pred, const float *meas, long long m,
                                          float *resid, int blk, int nblk, float w,
                                          const float *gadd) {
    __shared__ float ws[L1_THREADS / 32];
    const float wm = (float)((double)w / (double)m);
    float s = 0.f;
#pragma unroll 4
    for (long long i = (long long)blk * L1_THREADS + threadIdx.x; i < m;
         i += (long long)nblk * L1_THREADS) {
        const float d = pred[i] - meas[i];
        s += fabsf(d);
        float r = d > 0.f ? wm : (d < 0.f ? -wm : 0.f);
        if (gadd) r += gadd[i];
        resid[i] = r;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int w = 0; w < L1_THREADS / 32; ++w) t += ws[w];
    return t;
}

__global__ void __launch_bounds__(L1_THREADS) k_l1(const __grid_constant__ Batch B,
                                                   float *__restrict__ part,
                                                   const float *__restrict__ gadd) {
    DEP_ENTER();
    const Inst &I = B.in[blockIdx.y];
    const long long m = (long long)I.n_views * I.nu * I.nv;
    const float t = l1_block(I.sino, I.meas, m, I.sino, blockIdx.x, gridDim.x, I.w_l1,
                             (gadd && I.w_ssim != 0.f) ? gadd + I.ray0 : nullptr);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = t;
}

__global__ void k_l1_single(const float *__restrict__ pred, const float *__restrict__ meas,
                            long long m, float w, float *resid, float *__restrict__ part) {
    const float t = l1_block(pred, meas, m, resid, blockIdx.x, gridDim.x, w, nullptr);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// one warp per instance, fixed order: lane-strided FP64 sums, then a shuffle
// tree; loss = w x (sum / m)
__device__ __forceinline__ void l1_final(const float *part, int nb, long long m, float w, float *loss) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += (double)part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *loss = (float)((double)w * (s / (double)m));
}

__global__ void k_l1_final_single(const float *__restrict__ part, long long m, float w, float *loss) {
    l1_final(part, L1_BLOCKS, m, w, loss);
}

struct Affine {
    float c[3], half[3];
};

__host__ __device__ inline Affine grid_affine(const dgr_grid &g) {
    Affine A;
    const float ext[3] = {g.nx * g.h, g.ny * g.h, g.nz * g.h};
    const float org[3] = {g.ox, g.oy, g.oz};
    for (int a = 0; a < 3; ++a) {
        A.half[a] = 0.5f * ext[a];
        A.c[a] = org[a] + A.half[a];
    }
    return A;
}

__device__ __forceinline__ float softplus(float t) {
    return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t));
}
__device__ __forceinline__ float sigmoid(float t) { return 1.f / (1.f + expf(-t)); }

__global__ void k_params_init(dgr_grid g, dgr_params p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = p.n;
    if (i == 0) *p.step = 0;
    if (i >= n) return;
    const Affine A = grid_affine(g);
    float *th = p.theta;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        th[3 * i + a] = (p.mu[3 * i + a] - A.c[a]) / A.half[a];
        th[3 * n + 3 * i + a] = logf(p.s[3 * i + a]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) th[6 * n + 4 * i + a] = p.q[4 * i + a];
    const float r = fmaxf(p.rho[i], 1e-6f);
    th[10 * n + i] = r + logf(-expm1f(-r));  // inverse softplus
    for (int j = 0; j < 11; ++j) {
        const int o = (j < 3) ? 3 * i + j : (j < 6) ? 3 * n + 3 * i + (j - 3)
                      : (j < 10) ? 6 * n + 4 * i + (j - 6) : 10 * n + i;
        p.m[o] = 0.f;
        p.v[o] = 0.f;
    }
}

// Adam on the optimiser variables of every instance (thread per global
// Gaussian); gradients w.r.t. (mu, s, q, rho) are read from Inst::g_*.
__global__ void k_adam(const __grid_constant__ Batch B) {
    DEP_ENTER();
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= B.tot_g) return;
    const Inst &I = B.in[inst_of_g(B, gi)];
    const int i = gi - I.g0;
    const int n = I.n;
    const int t = *I.step + 1;
    const float lr0 = I.lr0, lr1 = I.lr1, b1 = I.b1, b2 = I.b2, eps = I.eps;
    const int n_iters = I.n_iters;
    const float lr = n_iters > 1 ? lr0 * powf(lr1 / lr0, (float)(t - 1) / (float)(n_iters - 1)) : lr0;
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    const Affine A = grid_affine(I.g);
    float *th = I.theta;
    float *pm = I.m, *pv = I.v;
    auto upd = [&](int o, float gr) {
        const float m = b1 * pm[o] + (1.f - b1) * gr;
        const float v = b2 * pv[o] + (1.f - b2) * gr * gr;
        pm[o] = m;
        pv[o] = v;
        const float nt = th[o] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        th[o] = nt;
        return nt;
    };
    if (I.gacc) {  // densification statistic: |dL/dmu| in world units
        const float gx = I.g_mu[3 * i], gy = I.g_mu[3 * i + 1], gz = I.g_mu[3 * i + 2];
        I.gacc[i] += sqrtf(gx * gx + gy * gy + gz * gz);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float tm = upd(3 * i + a, I.g_mu[3 * i + a] * A.half[a]);
        I.mu_w[3 * i + a] = A.c[a] + A.half[a] * tm;
        const float sc = I.s_w[3 * i + a];
        const float ts = upd(3 * n + 3 * i + a, I.g_s[3 * i + a] * sc);
        I.s_w[3 * i + a] = expf(ts);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) I.q_w[4 * i + a] = upd(6 * n + 4 * i + a, I.g_q[4 * i + a]);
    const int orho = 10 * n + i;
    const float tr = th[orho];
    const float trn = upd(orho, I.g_rho[i] * sigmoid(tr));
    I.rho_w[i] = softplus(trn);
}

__global__ void k_step_inc(const __grid_constant__ Batch B) {
    DEP_ENTER();
    if (threadIdx.x < B.n) *B.in[threadIdx.x].step += 1;
}

}  // namespace

cudaError_t launch_l1(const Batch &B, float *part, const float *gadd, cudaStream_t st) {
    launch_dep(k_l1, dim3(L1_BLOCKS, B.n), dim3(L1_THREADS), 0, st, B, part, gadd);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_l1_single(const float *pred, const float *meas, long long m, float w, float *resid,
                             float *loss, float *part, cudaStream_t st) {
    k_l1_single<<<L1_BLOCKS, L1_THREADS, 0, st>>>(pred, meas, m, w, resid, part);
    k_l1_final_single<<<1, 32, 0, st>>>(part, m, w, loss);
    counted(2);
    return cudaGetLastError();
}

cudaError_t launch_params_init(const dgr_problem &P, const dgr_params &p, cudaStream_t st) {
    const int n = p.n;
    k_params_init<<<(n + 127) / 128 + (n == 0), 128, 0, st>>>(P.grid, p);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_adam(const Batch &B, cudaStream_t st) {
    if (B.tot_g > 0) {
        launch_dep(k_adam, dim3((B.tot_g + 127) / 128), dim3(128), 0, st, B);
        counted(1);
    }
    launch_dep(k_step_inc, dim3(1), dim3(32), 0, st, B);
    counted(1);
    return cudaGetLastError();
}

}  // namespace dgr
