// Exclusive prefix sum of uint32 counts (work-list offsets of the voxelizer's
// binning and of the backward work items).  Three launches: per-block sums,
// one-block scan of the block sums (64-bit, so an overflow is detected), and a
// per-block scan that adds the block offset; one launch when the input fits
// one block.  Deterministic (no atomics).
#include "dgr_internal.cuh"

namespace dgr {
namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 4;
constexpr int SCAN_BLOCK = SCAN_THREADS * SCAN_PER_THREAD;  // elements per block

template <class T>
__device__ T block_exclusive_scan(T v, T *warp_tot, T *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        T w = lane < nw ? warp_tot[lane] : T(0);
        T t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t - w;  // exclusive warp offsets
        if (lane == nw - 1) *total = t;
    }
    __syncthreads();
    return warp_tot[wid] + x - v;
}

__global__ void k_block_sums(const uint32_t *in, int len, unsigned long long *bsum) {
    DEP_ENTER();
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long tot;
    const long long base = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x * SCAN_PER_THREAD;
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i)
        if (base + i < len) s += in[base + i];
    block_exclusive_scan<unsigned long long>(s, wt, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_block_sums(unsigned long long *bsum, int nb, uint32_t *out, int len,
                                  unsigned long long cap, int *status, int flag) {
    DEP_ENTER();
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long tot;
    // nb <= SCAN_BLOCK: each thread owns SCAN_PER_THREAD consecutive sums
    const int base = threadIdx.x * SCAN_PER_THREAD;
    unsigned long long v[SCAN_PER_THREAD], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        v[i] = base + i < nb ? bsum[base + i] : 0ull;
        s += v[i];
    }
    unsigned long long off = block_exclusive_scan<unsigned long long>(s, wt, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        if (base + i < nb) bsum[base + i] = off;
        off += v[i];
    }
    if (threadIdx.x == 0) {
        unsigned long long t = tot;
        if (t > cap) atomicOr(status, flag);
        out[len] = t > 0xffffffffull ? 0xffffffffu : (uint32_t)t;
    }
}

__global__ void k_block_scan(const uint32_t *in, int len, const unsigned long long *boff,
                             uint32_t *out) {
    DEP_ENTER();
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long tot;
    const long long base = (long long)blockIdx.x * SCAN_BLOCK + threadIdx.x * SCAN_PER_THREAD;
    uint32_t v[SCAN_PER_THREAD];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        v[i] = base + i < len ? in[base + i] : 0u;
        s += v[i];
    }
    unsigned long long off = block_exclusive_scan<unsigned long long>(s, wt, &tot) + boff[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        if (base + i < len) out[base + i] = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
        off += v[i];
    }
}
// len <= SCAN_BLOCK: the whole scan, the total and the capacity check in
// one block
__global__ void k_scan_single(const uint32_t *in, int len, uint32_t *out, unsigned long long cap,
                              int *status, int flag) {
    DEP_ENTER();
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long tot;
    const int base = threadIdx.x * SCAN_PER_THREAD;
    uint32_t v[SCAN_PER_THREAD];
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        v[i] = base + i < len ? in[base + i] : 0u;
        s += v[i];
    }
    unsigned long long off = block_exclusive_scan<unsigned long long>(s, wt, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_PER_THREAD; ++i) {
        if (base + i < len) out[base + i] = off > 0xffffffffull ? 0xffffffffu : (uint32_t)off;
        off += v[i];
    }
    if (threadIdx.x == 0) {
        const unsigned long long t = tot;
        if (t > cap) atomicOr(status, flag);
        out[len] = t > 0xffffffffull ? 0xffffffffu : (uint32_t)t;
    }
}
}  // namespace

size_t scan_tmp_elems(int len) { return (size_t)(len + SCAN_BLOCK - 1) / SCAN_BLOCK + 1; }

cudaError_t scan_u32(const uint32_t *in, uint32_t *out, int len, unsigned long long cap,
                     int *status, int flag, unsigned long long *tmp, cudaStream_t st) {
    const int nb = (len + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb > SCAN_BLOCK) return cudaErrorInvalidValue;  // len > 16.7M elements
    if (nb == 0) {
        // empty input: total 0
        return cudaMemsetAsync(out, 0, sizeof(uint32_t), st);
    }
    if (nb == 1) {
        launch_dep(k_scan_single, dim3(1), dim3(SCAN_THREADS), 0, st, in, len, out, cap, status, flag);
        counted(1);
        return cudaGetLastError();
    }
    launch_dep(k_block_sums, dim3(nb), dim3(SCAN_THREADS), 0, st, in, len, tmp);
    launch_dep(k_scan_block_sums, dim3(1), dim3(SCAN_THREADS), 0, st, tmp, nb, out, len, cap, status, flag);
    launch_dep(k_block_scan, dim3(nb), dim3(SCAN_THREADS), 0, st, in, len, tmp, out);
    counted(3);
    return cudaGetLastError();
}

}  // namespace dgr
