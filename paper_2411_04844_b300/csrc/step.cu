// L1 data term (a5), optimiser-variable transforms and fused Adam (a8).
//
// Objective: the L1 term of the paper's loss (Sec. 4.3, Eq. 13); Adam with the
// learning rate decaying 3e-4 -> 3e-5 over the run (Sec. 5.1).  The decay law,
// the Adam constants and the parameterisation are not stated in the paper; the
// choices (exponential decay; betas 0.9/0.999, eps 1e-8; mu in [-1,1]^3 box
// coordinates, log s, raw q, inverse-softplus rho) are this library's.
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr int L1_THREADS = 256;

// loss partials: fixed grid, grid-stride; resid = sign(pred - meas) / m
__global__ void __launch_bounds__(L1_THREADS) k_l1(const float *__restrict__ pred,
                                                   const float *__restrict__ meas, long long m,
                                                   float *resid, float *__restrict__ part) {
    __shared__ float ws[L1_THREADS / 32];
    const float invm = (float)(1.0 / (double)m);
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * L1_THREADS + threadIdx.x; i < m;
         i += (long long)gridDim.x * L1_THREADS) {
        const float d = pred[i] - meas[i];
        s += fabsf(d);
        resid[i] = d > 0.f ? invm : (d < 0.f ? -invm : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < L1_THREADS / 32; ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_l1_final(const float *__restrict__ part, int nb, long long m, float *loss) {
    // one warp, fixed order: lane-strided FP64 sums, then a shuffle tree
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += (double)part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *loss = (float)(s / (double)m);
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

// grads: [g_mu 3n | g_s 3n | g_q 4n | g_rho n] w.r.t. (mu, s, q, rho)
__global__ void k_adam(dgr_grid g, dgr_params p, const float *__restrict__ grads, float lr0,
                       float lr1, int n_iters, float b1, float b2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = p.n;
    if (i >= n) return;
    const int t = *p.step + 1;
    const float lr = n_iters > 1 ? lr0 * powf(lr1 / lr0, (float)(t - 1) / (float)(n_iters - 1)) : lr0;
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    const Affine A = grid_affine(g);
    float *th = p.theta;
    auto upd = [&](int o, float gr) {
        const float m = b1 * p.m[o] + (1.f - b1) * gr;
        const float v = b2 * p.v[o] + (1.f - b2) * gr * gr;
        p.m[o] = m;
        p.v[o] = v;
        const float nt = th[o] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        th[o] = nt;
        return nt;
    };
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float tm = upd(3 * i + a, grads[3 * i + a] * A.half[a]);
        p.mu[3 * i + a] = A.c[a] + A.half[a] * tm;
        const int os = 3 * n + 3 * i + a;
        const float sc = p.s[3 * i + a];
        const float ts = upd(os, grads[os] * sc);
        p.s[3 * i + a] = expf(ts);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int o = 6 * n + 4 * i + a;
        p.q[4 * i + a] = upd(o, grads[o]);
    }
    const int orho = 10 * n + i;
    const float tr = th[orho];
    const float trn = upd(orho, grads[orho] * sigmoid(tr));
    p.rho[i] = softplus(trn);
}

__global__ void k_step_inc(int *step) { *step += 1; }

}  // namespace

cudaError_t launch_l1(const float *pred, const float *meas, long long m, float *resid, float *loss,
                      float *part, cudaStream_t st) {
    k_l1<<<L1_BLOCKS, L1_THREADS, 0, st>>>(pred, meas, m, resid, part);
    k_l1_final<<<1, 32, 0, st>>>(part, L1_BLOCKS, m, loss);
    counted(2);
    return cudaGetLastError();
}

cudaError_t launch_params_init(const dgr_problem &P, const dgr_params &p, cudaStream_t st) {
    const int n = p.n;
    k_params_init<<<(n + 127) / 128 + (n == 0), 128, 0, st>>>(P.grid, p);
    counted(1);
    return cudaGetLastError();
}

cudaError_t launch_adam(const dgr_problem &P, const dgr_params &p, const float *grads,
                        cudaStream_t st) {
    const int n = p.n;
    if (n > 0) {
        k_adam<<<(n + 127) / 128, 128, 0, st>>>(P.grid, p, grads, P.lr0, P.lr1, P.n_iters, P.beta1,
                                                P.beta2, P.eps);
        counted(1);
    }
    k_step_inc<<<1, 1, 0, st>>>(p.step);
    counted(1);
    return cudaGetLastError();
}

}  // namespace dgr
