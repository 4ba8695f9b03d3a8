// dgr_pipe_rate: how many operations of one arithmetic pipe an SM completes
// per clock, measured on the running GPU.  The voxelizer is bound by the
// special-function unit's exp2 (one per in-box pair, Eq. 4) and its adjoint by
// the FP32 FMA pipe; their roofline peaks are these measured rates x SMs x the
// SM clock sampled during the run.  The paper has no counterpart.
//
// Each thread runs 8 independent dependency chains (enough warps and chains
// in flight that the pipe, not latency, limits), unrolled 4 times per
// iteration.  Cycles come from clock64() (the SM's own clock), so the rate is
// per clock whatever the clock frequency: per SM, operations of its CTAs
// divided by (latest end - earliest start).
#include "dgr_internal.cuh"

namespace {

constexpr int RATE_THREADS = 256;
constexpr int CHAINS = 8;
constexpr int UNROLL = 4;

__device__ __forceinline__ float ex2_neg(float x) {
    float y;
    asm volatile("{\n\t.reg .f32 t;\n\tneg.f32 t, %1;\n\tex2.approx.ftz.f32 %0, t;\n\t}"
                 : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// KIND 0: y <- exp2(-y) (stays in [0.5, 1]); 1: y <- y * a + b (FFMA);
// 2: the FFMA on packed float2 pairs (two FMAs per instruction)
template <int KIND>
__global__ void __launch_bounds__(RATE_THREADS) k_pipe_rate(int iters, unsigned long long *rec,
                                                            float *sink) {
    float y[CHAINS];
    float2 y2[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) {
        y[i] = 0.5f + 1e-4f * (float)(threadIdx.x + 7 * i);
        y2[i] = make_float2(y[i], 1.f - y[i]);
    }
    const float a = 0.9990234375f, b = 0.0009765625f;
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int i = 0; i < CHAINS; ++i) {
                if (KIND == 0) y[i] = ex2_neg(y[i]);
                else if (KIND == 1) y[i] = fmaf(y[i], a, b);
                else y2[i] = __ffma2_rn(y2[i], a2, b2);
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) s += KIND == 2 ? y2[i].x + y2[i].y : y[i];
    sink[(size_t)blockIdx.x * RATE_THREADS + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        const unsigned long long per_op = KIND == 2 ? 2ull : 1ull;  // FMAs per instruction
        rec[4 * blockIdx.x + 0] = smid();
        rec[4 * blockIdx.x + 1] = (unsigned long long)t0;
        rec[4 * blockIdx.x + 2] = (unsigned long long)t1;
        rec[4 * blockIdx.x + 3] =
            (unsigned long long)RATE_THREADS * iters * UNROLL * CHAINS * per_op;
    }
}

// L2 bandwidth: passes over a buffer small enough to stay in L2 after the
// first pass.  KIND 0 reads float4s (grid-stride, coalesced) and keeps a sum;
// KIND 1 adds 1 to every 32-bit word with a reduction (red.global.add, the
// backprojector's integer scatter), a warp's 32 lanes on 32 consecutive words
// (4 sectors per instruction, as the scatter's lanes on neighbouring z).
template <int KIND>
__global__ void __launch_bounds__(256) k_l2_rate(long long n16, int passes, float4 *buf, float *sink) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
            if (KIND == 0) {
                const float4 v = __ldcg(buf + i);
                acc += (v.x + v.y) + (v.z + v.w);
            } else {
                // word j = 4 (i - lane) + 32 c + lane: the warp's 4 x 32 words, 32 at a time
                const int lane = threadIdx.x & 31;
                int *w = reinterpret_cast<int *>(buf + (i - lane)) + lane;
                atomicAdd(w, 1); atomicAdd(w + 32, 1); atomicAdd(w + 64, 1); atomicAdd(w + 96, 1);
            }
        }
    }
    if (KIND == 0) sink[(long long)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" int dgr_l2_rate(int kind, long long bytes, int passes, int n_blocks, void *buf, float *sink,
                           cudaStream_t stream) {
    // kind 1: whole warps of 32 float4 (512 bytes), so every lane's 4 words stay in the buffer
    if (kind < 0 || kind > 1 || bytes < 16 || (bytes & 15) || (kind == 1 && (bytes & 511)) ||
        passes < 1 || n_blocks < 1 || n_blocks > (1 << 16) || !buf || !sink || ((uintptr_t)buf & 15))
        return DGR_ERR_ARG;
    const long long n16 = bytes / 16;
    if (kind == 0)
        k_l2_rate<0><<<n_blocks, 256, 0, stream>>>(n16, passes, static_cast<float4 *>(buf), sink);
    else
        k_l2_rate<1><<<n_blocks, 256, 0, stream>>>(n16, passes, static_cast<float4 *>(buf), sink);
    dgr::counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

extern "C" int dgr_pipe_rate(int kind, int iters, int n_blocks, unsigned long long *rec,
                             float *sink, cudaStream_t stream) {
    if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 20) || n_blocks < 1 ||
        n_blocks > (1 << 16) || !rec || !sink)
        return DGR_ERR_ARG;
    switch (kind) {
        case 0: k_pipe_rate<0><<<n_blocks, RATE_THREADS, 0, stream>>>(iters, rec, sink); break;
        case 1: k_pipe_rate<1><<<n_blocks, RATE_THREADS, 0, stream>>>(iters, rec, sink); break;
        default: k_pipe_rate<2><<<n_blocks, RATE_THREADS, 0, stream>>>(iters, rec, sink);
    }
    dgr::counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}
