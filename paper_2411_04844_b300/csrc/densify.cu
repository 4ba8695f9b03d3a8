// Adaptive density control (paper App. F, Algorithm 2) on the GPU.
//
// Every `iters` iterations the optimiser's per-Gaussian accumulated
// |dL/dmu| (dgr_params.grad_accum, added by the Adam kernel) gives the mean
// gradient avg; sigma is the largest axis scale.
//   clone  (avg >= tau, sigma <= theta): the n_clone with the largest avg,
//          n_clone <= n_max - n; the original and its copy share the intensity
//   split  (avg >= tau, sigma > theta): the n_split with the largest avg,
//          n_split <= n_max - n - n_clone; each becomes two children drawn from
//          its own density, mu + R(q) diag(s) z (z given), scales s / 2^(1/3)
//   prune  the remaining originals with avg <= tau or sigma > 3 size h
// Output order: surviving originals, clones, children (two per split) -- the
// same order as the oracle.  Selections are exact integer decisions on the
// FP32 avg bits, ties by lower index.
//
//   k_dens_flags   avg bits and candidate flags per Gaussian
//   k_dens_select  one CTA: the k-th largest candidate key by bisection over
//                  the 32 key bits, then ties in index order by a block scan;
//                  clone first, split with the room that is left
//   k_dens_mark    keep / prune flags
//   scan_u32 x 3   output offsets of survivors, clones, split pairs
//   k_dens_write   the new state (theta, m, v: survivors keep theirs, new
//                  entries start from zero moments)
#include <math.h>

#include "dgr_internal.cuh"

namespace dgr {
namespace {

constexpr unsigned F_CC = 1u, F_CS = 2u, F_CLONE = 4u, F_SPLIT = 8u, F_KEEP = 16u;
constexpr int SEL_THREADS = 1024;

struct DensArgs {
    dgr_grid g;
    int n, n_max, iters;
    float tau, theta, prune_sigma;
    const float *mu, *s, *q, *rho, *theta_in, *m_in, *v_in, *acc;
    const int *step_in;
    const float *normals;  // [n][2][3]
    float *mu_o, *s_o, *q_o, *rho_o, *theta_o, *m_o, *v_o, *acc_o;
    int *step_o;
    unsigned *key, *flag, *off_keep, *off_clone, *off_split;
    int *counts;           // [0] n_clone, [1] n_split, [2] n_out
};

__global__ void k_dens_flags(const __grid_constant__ DensArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const float avg = A.acc[i] / (float)A.iters;
    const float sig = fmaxf(A.s[3 * i], fmaxf(A.s[3 * i + 1], A.s[3 * i + 2]));
    unsigned f = 0u;
    if (avg >= A.tau) f |= sig <= A.theta ? F_CC : F_CS;
    A.flag[i] = f;
    A.key[i] = __float_as_uint(fmaxf(avg, 0.f));  // non-negative: bits order like values
}

__device__ unsigned block_count(unsigned v) {
    __shared__ unsigned part[SEL_THREADS / 32];
    __shared__ unsigned total;
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned t = part[threadIdx.x];
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0) total = t;
    }
    __syncthreads();
    const unsigned r = total;
    __syncthreads();
    return r;
}

// marks with `sel` the k candidates (flag & cand) of largest key, ties by index
__device__ void select_top(const DensArgs &A, unsigned cand, unsigned sel, unsigned k) {
    const int n = A.n;
    unsigned cnt = 0;
    for (int i = threadIdx.x; i < n; i += SEL_THREADS) cnt += (A.flag[i] & cand) ? 1u : 0u;
    const unsigned total = block_count(cnt);
    if (k == 0) return;
    if (k >= total) {
        for (int i = threadIdx.x; i < n; i += SEL_THREADS)
            if (A.flag[i] & cand) A.flag[i] |= sel;
        __syncthreads();
        return;
    }
    // largest T with #(key >= T) >= k, bit by bit from the top
    unsigned T = 0u;
    for (int b = 31; b >= 0; --b) {
        const unsigned t = T | (1u << b);
        unsigned c = 0;
        for (int i = threadIdx.x; i < n; i += SEL_THREADS) c += ((A.flag[i] & cand) && A.key[i] >= t) ? 1u : 0u;
        if (block_count(c) >= k) T = t;
    }
    unsigned c = 0;
    for (int i = threadIdx.x; i < n; i += SEL_THREADS) c += ((A.flag[i] & cand) && A.key[i] > T) ? 1u : 0u;
    const unsigned above = block_count(c);
    const unsigned ties = k - above;  // equal keys taken in index order
    __shared__ unsigned wpre[SEL_THREADS / 32];
    unsigned taken = 0;
    for (int base = 0; base < n; base += SEL_THREADS) {
        const int i = base + threadIdx.x;
        const bool cd = i < n && (A.flag[i] & cand);
        const bool eq = cd && A.key[i] == T;
        // exclusive rank of this equal key among the equal keys of the chunk
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) wpre[w] = __popc(bal);
        __syncthreads();
        unsigned before = 0, chunk = 0;
        for (int j = 0; j < SEL_THREADS / 32; ++j) {
            if (j < (int)w) before += wpre[j];
            chunk += wpre[j];
        }
        before += __popc(bal & ((1u << lane) - 1u));
        if (cd && (A.key[i] > T || (eq && taken + before < ties))) A.flag[i] |= sel;
        taken += chunk;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SEL_THREADS) k_dens_select(const __grid_constant__ DensArgs A) {
    unsigned cc = 0, cs = 0;
    for (int i = threadIdx.x; i < A.n; i += SEL_THREADS) {
        cc += (A.flag[i] & F_CC) ? 1u : 0u;
        cs += (A.flag[i] & F_CS) ? 1u : 0u;
    }
    const unsigned ncc = block_count(cc), ncs = block_count(cs);
    const long long room1 = (long long)A.n_max - A.n;
    const unsigned n_clone = (unsigned)max(0ll, min(room1, (long long)ncc));
    select_top(A, F_CC, F_CLONE, n_clone);
    const long long room2 = room1 - n_clone;
    const unsigned n_split = (unsigned)max(0ll, min(room2, (long long)ncs));
    select_top(A, F_CS, F_SPLIT, n_split);
    if (threadIdx.x == 0) {
        A.counts[0] = (int)n_clone;
        A.counts[1] = (int)n_split;
    }
}

__global__ void k_dens_mark(const __grid_constant__ DensArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.n) return;
    const unsigned f = A.flag[i];
    const float avg = __uint_as_float(A.key[i]);
    const float sig = fmaxf(A.s[3 * i], fmaxf(A.s[3 * i + 1], A.s[3 * i + 2]));
    const bool prune = avg <= A.tau || sig > A.prune_sigma;
    const bool keep = !(f & F_SPLIT) && !prune;
    A.flag[i] = keep ? (f | F_KEEP) : f;
    // 0/1 inputs of the three offset scans
    A.off_keep[i] = keep ? 1u : 0u;
    A.off_clone[i] = (f & F_CLONE) ? 1u : 0u;
    A.off_split[i] = (f & F_SPLIT) ? 1u : 0u;
}

__device__ __forceinline__ float softplus_inv(float r) {
    r = fmaxf(r, 1e-6f);
    return r + logf(-expm1f(-r));
}

__device__ void write_new(const DensArgs &A, int o, int n_out, const float *mu, const float *s,
                          const float *q, float rho) {
    // theta of a new entry: ((mu - c)/half, log s, q, softplus^-1 rho); zero moments
    const dgr_grid &g = A.g;
    const float ext[3] = {g.nx * g.h, g.ny * g.h, g.nz * g.h};
    const float org[3] = {g.ox, g.oy, g.oz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float half = 0.5f * ext[a], c = org[a] + half;
        A.mu_o[3 * o + a] = mu[a];
        A.s_o[3 * o + a] = s[a];
        A.theta_o[3 * o + a] = (mu[a] - c) / half;
        A.theta_o[3 * n_out + 3 * o + a] = logf(s[a]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        A.q_o[4 * o + a] = q[a];
        A.theta_o[6 * n_out + 4 * o + a] = q[a];
    }
    A.rho_o[o] = rho;
    A.theta_o[10 * n_out + o] = softplus_inv(rho);
    for (int j = 0; j < 11; ++j) {
        const int k = (j < 3) ? 3 * o + j : (j < 6) ? 3 * n_out + 3 * o + (j - 3)
                      : (j < 10) ? 6 * n_out + 4 * o + (j - 6) : 10 * n_out + o;
        A.m_o[k] = 0.f;
        A.v_o[k] = 0.f;
    }
    if (A.acc_o) A.acc_o[o] = 0.f;
}

__global__ void k_dens_write(const __grid_constant__ DensArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = A.n;
    const int n_keep = (int)A.off_keep[n], n_clone = A.counts[0], n_split = A.counts[1];
    const int n_out = n_keep + n_clone + 2 * n_split;
    if (i == 0) {
        A.counts[2] = n_out;
        *A.step_o = *A.step_in;
    }
    if (i >= n) return;
    const unsigned f = A.flag[i];
    const float *mu = A.mu + 3 * i, *s = A.s + 3 * i, *q = A.q + 4 * i;
    const float rho = (f & F_CLONE) ? 0.5f * A.rho[i] : A.rho[i];
    if (f & F_KEEP) {  // survivor: state copied (a cloned one's intensity halved)
        const int o = (int)A.off_keep[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A.mu_o[3 * o + a] = mu[a];
            A.s_o[3 * o + a] = s[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) A.q_o[4 * o + a] = q[a];
        A.rho_o[o] = rho;
        for (int j = 0; j < 11; ++j) {
            const int ki = (j < 3) ? 3 * i + j : (j < 6) ? 3 * n + 3 * i + (j - 3)
                           : (j < 10) ? 6 * n + 4 * i + (j - 6) : 10 * n + i;
            const int ko = (j < 3) ? 3 * o + j : (j < 6) ? 3 * n_out + 3 * o + (j - 3)
                           : (j < 10) ? 6 * n_out + 4 * o + (j - 6) : 10 * n_out + o;
            A.theta_o[ko] = (j == 10 && (f & F_CLONE)) ? softplus_inv(rho) : A.theta_in[ki];
            A.m_o[ko] = A.m_in[ki];
            A.v_o[ko] = A.v_in[ki];
        }
        if (A.acc_o) A.acc_o[o] = 0.f;
    }
    if (f & F_CLONE) write_new(A, n_keep + (int)A.off_clone[i], n_out, mu, s, q, rho);
    if (f & F_SPLIT) {
        // R(q / |q|) by the standard formula
        const float qq = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] * qq, x = q[1] * qq, y = q[2] * qq, z = q[3] * qq;
        const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                               {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                               {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
        const float c = 0.79370052598409973737f;  // 2^(-1/3): two children keep the volume
        const float sc[3] = {s[0] * c, s[1] * c, s[2] * c};
        for (int ch = 0; ch < 2; ++ch) {
            const float *zz = A.normals + 6 * i + 3 * ch;
            float m2[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                m2[a] = mu[a] + R[a][0] * s[0] * zz[0] + R[a][1] * s[1] * zz[1] + R[a][2] * s[2] * zz[2];
            write_new(A, n_keep + n_clone + 2 * (int)A.off_split[i] + ch, n_out, m2, sc, q, A.rho[i]);
        }
    }
}

}  // namespace

cudaError_t launch_densify(const dgr_grid &g, const dgr_densify_cfg &cfg, int iters, const dgr_params &in,
                           const float *normals, const dgr_params &out, dgr_ws *ws, int *counts_dev,
                           cudaStream_t st) {
    DensArgs A;
    memset(&A, 0, sizeof(A));
    A.g = g;
    A.n = in.n;
    A.n_max = cfg.n_max;
    A.iters = iters;
    A.tau = cfg.tau;
    const double diag = sqrt((double)g.nx * g.nx + (double)g.ny * g.ny + (double)g.nz * g.nz) * g.h;
    A.theta = (float)(cfg.theta_frac * diag);
    A.prune_sigma = 3.f * cfg.size * g.h;
    A.mu = in.mu; A.s = in.s; A.q = in.q; A.rho = in.rho;
    A.theta_in = in.theta; A.m_in = in.m; A.v_in = in.v; A.acc = in.grad_accum; A.step_in = in.step;
    A.normals = normals;
    A.mu_o = out.mu; A.s_o = out.s; A.q_o = out.q; A.rho_o = out.rho;
    A.theta_o = out.theta; A.m_o = out.m; A.v_o = out.v; A.acc_o = out.grad_accum; A.step_o = out.step;
    const int n = in.n;
    unsigned *base = ws_ptr<unsigned>(ws, ws->dens);
    const size_t stride = (size_t)ws->plan.max_n + 1;
    A.key = base;
    A.flag = base + stride;
    A.off_keep = base + 2 * stride;
    A.off_clone = base + 3 * stride;
    A.off_split = base + 4 * stride;
    A.counts = counts_dev;
    const int blocks = (n + 255) / 256 + (n == 0);
    k_dens_flags<<<blocks, 256, 0, st>>>(A);
    k_dens_select<<<1, SEL_THREADS, 0, st>>>(A);
    k_dens_mark<<<blocks, 256, 0, st>>>(A);
    counted(3);
    int *status = ws_ptr<int>(ws, ws->status);
    unsigned long long *tmp = ws_ptr<unsigned long long>(ws, ws->scan_tmp);
    cudaError_t e = cudaGetLastError();
    // in-place exclusive scans (off_*[n] = totals)
    if (e == cudaSuccess) e = scan_u32(A.off_keep, A.off_keep, n, ~0ull, status, 0, tmp, st);
    if (e == cudaSuccess) e = scan_u32(A.off_clone, A.off_clone, n, ~0ull, status, 0, tmp, st);
    if (e == cudaSuccess) e = scan_u32(A.off_split, A.off_split, n, ~0ull, status, 0, tmp, st);
    if (e != cudaSuccess) return e;
    k_dens_write<<<blocks, 256, 0, st>>>(A);
    counted(1);
    return cudaGetLastError();
}

}  // namespace dgr
