// Warm-start network: a small 3D convolutional encoder-decoder that maps a
// coarse backprojection (n^3, one channel) to per-voxel (density, log-scale)
// proposals used to seed the Gaussians.  (A learned initialisation is not part
// of the paper; it sits on top of the method.)
//
//   a1 = relu(conv3(x, 1->16) + b1)                  n^3       (CUDA cores)
//   a2 = relu(conv3(pool(a1), 16->32) + b2)          (n/2)^3   (tensor cores)
//   a3 = relu(conv3(pool(a2), 32->64) + b3)          (n/4)^3   (tensor cores)
//   a4 = relu(conv3(up(a3), 64->32) + b4 + a2)       (n/2)^3   (tensor cores)
//   a5 = relu(conv3(up(a4), 32->16) + b5 + a1)       n^3       (tensor cores)
//   y  = conv1(a5, 16->2) + b6                       n^3 x 2   (CUDA cores)
// pool: 2^3 average; up: 2^3 nearest.  Activations are BF16, channels-last
// ([z][y][x][c]); every convolution accumulates in FP32.
//
// The tensor-core convolutions are implicit GEMMs (BF16 operands, FP32
// accumulators):
//   forward      C[p][co] = sum_{tap,ci} X[p + tap][ci] W[tap][ci][co]
//   data grad    C[p][ci] = sum_{tap,co} G[p - tap][co] W[tap][ci][co]
//   weight grad  C[tap*Ci + ci][co] = sum_p X[p + tap][ci] G[p][co]
//                (split over voxel ranges; partials summed in a fixed order)
// By default all three run on tcgen05 over TMA-loaded halo blocks with
// several taps per MMA (k_conv_dz: the three z taps of one (dy, dx);
// k_wgrad_dz: z offsets on M, y offsets on N; k_wgrad_halo for the 16 -> 32
// layer); dgr_set_conv_engine selects the earlier designs for comparison:
// halo blocks with one MMA per tap (k_conv_halo, k_wgrad_halo), gathered
// 128-row tcgen05 tiles for forward and data gradient (k_conv_umma) or
// mma.sync m16n8k16 (k_conv_gemm, also the weight gradient of engines 0, 1).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "async_ops.cuh"
#include "dgr_internal.cuh"

namespace dgr {
namespace {

using bf16 = __nv_bfloat16;

constexpr int GM = 64;       // GEMM tile rows per CTA
constexpr int GK = 32;       // GEMM K step
constexpr int KPAD = GK + 8; // shared-memory row pitch (bf16), 80 bytes
constexpr int GEMM_THREADS = 128;
constexpr int WG_SPLIT = 4096;  // voxels per weight-gradient split

enum { MODE_FWD = 0, MODE_DGRAD = 1, MODE_WGRAD = 2 };

struct ConvArgs {
    int n;            // grid side of the convolution (cubic, voxels)
    int ci, co;       // input / output channels
    const bf16 *x;    // FWD/WGRAD: input activations [n^3][ci]; DGRAD: output grads [n^3][co]
    const bf16 *w;    // [27][ci][co]
    const float *bias;  // FWD: [co]
    const bf16 *skip;   // FWD: optional residual [n^3][co]
    const bf16 *g;    // WGRAD: output grads [n^3][co]
    bf16 *y;          // FWD: output [n^3][co]
    float *out;       // DGRAD: [n^3][ci] FP32; WGRAD: partials [splits][27*ci][co]
    const bf16 *wt;   // tcgen05 FWD / DGRAD: the weights as B, K-major [N][K]
    const bf16 *wdz;  // k_conv_dz FWD / DGRAD: the weights as its B (k_wpack_dz)
    int *status;      // device status word (bounded waits)
    int up_adj;       // k_conv_dz DGRAD: write the 2^3 child sums at half resolution (see k_conv_dz)
};

__device__ __forceinline__ void tap_offset(int tap, int &dx, int &dy, int &dz) {
    dz = tap / 9 - 1;
    dy = (tap / 3) % 3 - 1;
    dx = tap % 3 - 1;
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                        const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r0), "=r"(r1)
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One CTA: GM rows x BN columns of C, K in steps of GK.  Warp w owns rows
// [16 w, 16 w + 16) and all BN columns.
template <int MODE, int BN>
__global__ void __launch_bounds__(GEMM_THREADS) k_conv_gemm(const ConvArgs a) {
    __shared__ __align__(16) bf16 As[GM][KPAD];
    __shared__ __align__(16) bf16 Bs[BN][KPAD];
    const int n = a.n, n3 = n * n * n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // GEMM dimensions
    int M, K, kb, ke;
    const int m0 = blockIdx.x * GM;
    if (MODE == MODE_FWD) { M = n3; K = 27 * a.ci; kb = 0; ke = K; }
    else if (MODE == MODE_DGRAD) { M = n3; K = 27 * a.co; kb = 0; ke = K; }
    else { M = 27 * a.ci; K = n3; kb = blockIdx.y * WG_SPLIT; ke = min(K, kb + WG_SPLIT); }
    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += GK) {
        __syncthreads();
        // gather A (GM x GK)
        for (int e = threadIdx.x; e < GM * GK; e += GEMM_THREADS) {
            const int r = e / GK, c = e % GK;
            const int m = m0 + r, k = k0 + c;
            bf16 v = __float2bfloat16(0.f);
            if (m < M && k < ke) {
                if (MODE == MODE_FWD || MODE == MODE_DGRAD) {
                    const int C = MODE == MODE_FWD ? a.ci : a.co;
                    const int tap = k / C, ch = k % C;
                    int dx, dy, dz;
                    tap_offset(tap, dx, dy, dz);
                    if (MODE == MODE_DGRAD) { dx = -dx; dy = -dy; dz = -dz; }
                    const int px = m % n, py = (m / n) % n, pz = m / (n * n);
                    const int qx = px + dx, qy = py + dy, qz = pz + dz;
                    if (qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n)
                        v = a.x[((size_t)(qz * n + qy) * n + qx) * C + ch];
                } else {
                    const int tap = m / a.ci, ch = m % a.ci;
                    int dx, dy, dz;
                    tap_offset(tap, dx, dy, dz);
                    const int px = k % n, py = (k / n) % n, pz = k / (n * n);
                    const int qx = px + dx, qy = py + dy, qz = pz + dz;
                    if (qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n)
                        v = a.x[((size_t)(qz * n + qy) * n + qx) * a.ci + ch];
                }
            }
            As[r][c] = v;
        }
        // gather B (stored [BN][GK], k contiguous)
        for (int e = threadIdx.x; e < BN * GK; e += GEMM_THREADS) {
            const int nn = e / GK, c = e % GK;
            const int k = k0 + c;
            bf16 v = __float2bfloat16(0.f);
            if (k < ke) {
                if (MODE == MODE_FWD) {
                    const int tap = k / a.ci, ch = k % a.ci;
                    if (nn < a.co) v = a.w[((size_t)tap * a.ci + ch) * a.co + nn];
                } else if (MODE == MODE_DGRAD) {
                    const int tap = k / a.co, ch = k % a.co;
                    if (nn < a.ci) v = a.w[((size_t)tap * a.ci + nn) * a.co + ch];
                } else {
                    if (nn < a.co) v = a.g[(size_t)k * a.co + nn];
                }
            }
            Bs[nn][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk += 16) {
            uint32_t af[4];
            {
                const int q = lane >> 3, rr = lane & 7;
                const bf16 *p = &As[16 * w + rr + (q & 1) * 8][kk + (q >> 1) * 8];
                ldsm_x4(af[0], af[1], af[2], af[3], p);
            }
#pragma unroll
            for (int j = 0; j < BN / 8; ++j) {
                uint32_t bfr[2];
                const int q = (lane >> 3) & 1, rr = lane & 7;
                const bf16 *p = &Bs[8 * j + rr][kk + q * 8];
                ldsm_x2(bfr[0], bfr[1], p);
                mma_bf16(acc[j], af, bfr);
            }
        }
    }
    // epilogue
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = m0 + 16 * w + g + 8 * h;
#pragma unroll
            for (int c2 = 0; c2 < 2; ++c2) {
                const int col = 8 * j + 2 * t4 + c2;
                const float v = acc[j][2 * h + c2];
                if (m >= M) continue;
                if (MODE == MODE_FWD) {
                    if (col >= a.co) continue;
                    float z = v + a.bias[col];
                    if (a.skip) z += __bfloat162float(a.skip[(size_t)m * a.co + col]);
                    a.y[(size_t)m * a.co + col] = __float2bfloat16(fmaxf(z, 0.f));
                } else if (MODE == MODE_DGRAD) {
                    if (col >= a.ci) continue;
                    a.out[(size_t)m * a.ci + col] = v;
                } else {
                    if (col >= a.co) continue;
                    a.out[((size_t)blockIdx.y * M + m) * a.co + col] = v;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same forward and data-gradient GEMMs on the fifth-generation tensor
// cores (tcgen05).  A CTA of four warps owns UM = 128 rows (voxels) and all
// BN columns; the FP32 accumulator D[128][BN] lives in tensor memory (row i in
// lane i).  K runs in stages of UK = 64 through two shared-memory buffers:
// every thread gathers its own row of A (eight 16-byte chunks; a chunk is 8
// channels of one tap, since C is a multiple of 8) and a share of B from the
// packed K-major weights, then one thread issues UK / 16 MMAs of
// 128 x BN x 16 and commits them to the buffer's mbarrier, which frees the
// buffer for the stage after next.  Operands use the no-swizzle K-major
// layout: core matrix (8 rows x 16 bytes) (g, c) of a row group g and K chunk
// c at byte (g UK / 8 + c) 128, so K-adjacent core matrices are 128 bytes
// apart and M-adjacent ones UK / 8 x 128.
// ---------------------------------------------------------------------------
constexpr int UM = 128, UK = 64;

__host__ __device__ constexpr int umma_cols(int bn) { return bn <= 32 ? 32 : bn; }
__host__ __device__ constexpr size_t umma_smem(int bn) {
    return 1024 + 2 * (size_t)UM * UK * 2 + 2 * (size_t)bn * UK * 2 + 64;
}

// 16 consecutive accumulator columns c0 .. c0 + 15 of output row `row`:
// forward relu(v + bias (+ skip)) to BF16, data gradient FP32 as is
template <int MODE>
__device__ __forceinline__ void store_row16(const ConvArgs &a, size_t row, int c0, float *v) {
    if (MODE == MODE_FWD) {
        if (a.skip) {
            const uint4 *sp = reinterpret_cast<const uint4 *>(a.skip + row * a.co + c0);
            const uint4 s0 = sp[0], s1 = sp[1];
            const uint32_t su[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                __nv_bfloat162 h;
                memcpy(&h, &su[i], 4);
                const float2 f = __bfloat1622float2(h);
                v[2 * i] += f.x;
                v[2 * i + 1] += f.y;
            }
        }
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(v[2 * i] + a.bias[c0 + 2 * i], 0.f),
                                                           fmaxf(v[2 * i + 1] + a.bias[c0 + 2 * i + 1], 0.f));
            memcpy(&pk[i], &h, 4);
        }
        uint4 *yp = reinterpret_cast<uint4 *>(a.y + row * a.co + c0);
        yp[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        yp[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    } else {
        float4 *op = reinterpret_cast<float4 *>(a.out + row * a.ci + c0);
#pragma unroll
        for (int i = 0; i < 4; ++i) op[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
}

// forward output of 16 channels: relu(v + bias + residual) as BF16 (the
// residual, 16 BF16, passed in two uint4; zero without one)
__device__ __forceinline__ void store_fwd16(bf16 *y, float *v, const float *bias, uint4 s0, uint4 s1) {
    const uint32_t su[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    uint32_t pk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        __nv_bfloat162 h;
        memcpy(&h, &su[i], 4);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 o = __floats2bfloat162_rn(fmaxf(v[2 * i] + f.x + bias[2 * i], 0.f),
                                                       fmaxf(v[2 * i + 1] + f.y + bias[2 * i + 1], 0.f));
        memcpy(&pk[i], &o, 4);
    }
    uint4 *yp = reinterpret_cast<uint4 *>(y);
    yp[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    yp[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

template <int MODE, int BN>
__global__ void __launch_bounds__(128) k_conv_umma(const ConvArgs a) {
    static_assert(MODE == MODE_FWD || MODE == MODE_DGRAD, "forward and data gradient only");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 64, "M = 128 needs N a multiple of 16");
    constexpr unsigned NCOL = umma_cols(BN);
    constexpr int ABYTES = UM * UK * 2, BBYTES = BN * UK * 2;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char *As = sm, *Bs = sm + 2 * ABYTES;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm + 2 * ABYTES + 2 * BBYTES);
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);

    const int n = a.n, n3 = n * n * n;
    const int C = MODE == MODE_FWD ? a.ci : a.co;
    const int K = 27 * C;
    const int w = threadIdx.x >> 5;
    if (w == 0) {
        tmem_alloc(tslot, NCOL);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    // this thread's row of A: voxel m
    const int r = threadIdx.x, m = blockIdx.x * UM + r;
    const bool mv = m < n3;
    const int px = m % n, py = (m / n) % n, pz = m / (n * n);
    const int nk = (K + UK - 1) / UK;
    constexpr unsigned IDESC = idesc_bf16_f32(UM, BN);
    int issued = -1;  // last stage whose MMAs were committed
    bool ok = true;
    for (int ks = 0; ks < nk; ++ks) {
        const int s = ks & 1;
        // the MMAs of stage ks - 2 read this buffer
        if (ks >= 2 && !mbar_wait(&bar[s], ((ks >> 1) - 1) & 1, a.status)) ok = false;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        unsigned char *A = As + s * ABYTES, *Bm = Bs + s * BBYTES;
        const int k0 = ks * UK;
#pragma unroll
        for (int c = 0; c < UK / 8; ++c) {
            const int k = k0 + 8 * c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (mv && k < K) {
                const int tap = k / C, ch = k - tap * C;
                int dx, dy, dz;
                tap_offset(tap, dx, dy, dz);
                if (MODE == MODE_DGRAD) { dx = -dx; dy = -dy; dz = -dz; }
                const int qx = px + dx, qy = py + dy, qz = pz + dz;
                if (qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n)
                    v = *reinterpret_cast<const uint4 *>(a.x + ((size_t)(qz * n + qy) * n + qx) * C + ch);
            }
            *reinterpret_cast<uint4 *>(A + ((r >> 3) * (UK / 8) + c) * 128 + (r & 7) * 16) = v;
        }
        for (int e = threadIdx.x; e < BN * (UK / 8); e += 128) {
            const int nn = e % BN, c = e / BN, k = k0 + 8 * c;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (k < K) v = *reinterpret_cast<const uint4 *>(a.wt + (size_t)nn * K + k);
            *reinterpret_cast<uint4 *>(Bm + ((nn >> 3) * (UK / 8) + c) * 128 + (nn & 7) * 16) = v;
        }
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const unsigned ab = smem_u32(A), bb = smem_u32(Bm);
#pragma unroll
            for (int kk = 0; kk < UK / 16; ++kk)
                umma_bf16(tmem, smem_desc(ab + kk * 256, 128, (UK / 8) * 128),
                          smem_desc(bb + kk * 256, 128, (UK / 8) * 128), IDESC, (ks | kk) != 0);
            umma_commit(&bar[s]);
        }
        issued = ks;
    }
    // the last commit arrives once every MMA of the tile has completed
    if (issued >= 0 && !mbar_wait(&bar[issued & 1], (issued >> 1) & 1, a.status)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (ok && issued == nk - 1) {
        const int row = blockIdx.x * UM + 32 * w + (threadIdx.x & 31);
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((unsigned)(32 * w) << 16) + (unsigned)c0, v);
            if (row >= n3) continue;
            store_row16<MODE>(a, (size_t)row, c0, v);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOL);
    }
}

// ---------------------------------------------------------------------------
// Halo-tile form of the same convolutions on tcgen05: no im2col at all.  A
// CTA loads the input block of an output tile of 8 (x) x 16 (y) x ZT (z)
// voxels plus a one-voxel halo (10 x 18 x (ZT + 2) voxels, C channels) into
// shared memory once, and every tap's A operand is a descriptor into that
// block: with 16-byte channel chunks stored x-contiguous, eight consecutive x
// voxels of one (y, z) line are a core matrix (rows 16 bytes apart) starting
// at any x, the 16 lines of the tile are M-adjacent core matrices (one line,
// 160 bytes, apart) and the next channel chunk is K-adjacent (one chunk plane
// apart).  Shifting by a tap (dx, dy, dz) moves the start address only.  The
// whole packed weight matrix B [N][27 C] sits in shared memory for the CTA's
// lifetime; per output slice z one FP32 accumulator of 128 x N in tensor
// memory; per tile 27 ZT C / 16 MMAs from one thread, then one commit.
// The CTA walks tiles (persistent); the halo block is rewritten only after
// the tile's commit has arrived.
// ---------------------------------------------------------------------------
// Threads of the halo-tile kernels: eight warps load; warp w reads tensor
// memory lanes 32 (w % 4) .. + 31 (its lane quarter) and takes every other
// 16-column chunk of the epilogue with its partner warp w ^ 4.
constexpr int HALO_THREADS = 256;

// the input block of a tile: voxels x0-1 .. x0+8, y0-1 .. y0+16, z0-1 ..
// z0+HZ-2 of x [n^3][C] (zero outside) as 16-byte channel chunks at
// chunk plane c, offset ((zz 18 + yy) 10 + xx) 16, by asynchronous copies
// (all of a thread's copies in flight at once; the caller commits and waits)
template <int C, int HZ>
__device__ __forceinline__ void load_halo(const bf16 *__restrict__ x, int n, int x0, int y0, int z0,
                                          unsigned char *Hs, unsigned plane) {
    constexpr int CH = C / 8, TOT = 10 * 18 * HZ * CH;
    for (int e = threadIdx.x; e < TOT; e += HALO_THREADS) {
        const int c = e % CH, v = e / CH;
        const int xx = v % 10, yy = (v / 10) % 18, zz = v / 180;
        const int qx = x0 + xx - 1, qy = y0 + yy - 1, qz = z0 + zz - 1;
        const bool in = qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n;
        const bf16 *src = in ? x + ((size_t)(qz * n + qy) * n + qx) * C + 8 * c : x;
        cp_async16(Hs + c * plane + ((zz * 18 + yy) * 10 + xx) * 16, src, in ? 16u : 0u);
    }
}

// the input block of an 8 x 16 x ZT tile with its one-voxel halo, C channels
template <int C, int ZT>
struct HaloBlock {
    static constexpr int HX = 10, HY = 18, HZ = ZT + 2;
    static constexpr int CH = C / 8;  // 16-byte chunks per voxel
    // chunk-plane pitch in 16-byte slots, padded to (8 / CH) mod 8 so the CH
    // chunks of the 8 / CH voxels that 8 lanes store together fall in
    // different 16-byte bank slots
    static constexpr unsigned BASE16 = (unsigned)HX * HY * HZ;
    static constexpr unsigned PLANE = 16u * (BASE16 + (8u + (unsigned)(8 / CH) - BASE16 % 8u) % 8u);
    static constexpr unsigned HBYTES = PLANE * CH;
    static_assert(PLANE % 16 == 0 && (PLANE >> 4) < 16384, "descriptor field");
};

// forward / data gradient: the block plus the packed weights B [N][27 C]
template <int C, int N, int ZT>
struct Halo : HaloBlock<C, ZT> {
    using HaloBlock<C, ZT>::CH;
    using HaloBlock<C, ZT>::HBYTES;
    static constexpr unsigned BLEAD = (unsigned)N * 16;  // K-chunk pitch of B
    static constexpr unsigned BBYTES = (unsigned)27 * CH * BLEAD;
};

// single-buffered kernel: B, one block, one accumulator set
template <int C, int N, int ZT>
struct Halo1 : Halo<C, N, ZT> {
    static constexpr unsigned NCOL = ZT * N <= 32 ? 32 : (ZT * N <= 64 ? 64 : (ZT * N <= 128 ? 128 : 256));
    static constexpr size_t SMEM = 1024 + (size_t)Halo<C, N, ZT>::BBYTES + Halo<C, N, ZT>::HBYTES + 64;
    static_assert(ZT * N <= 256, "accumulators exceed the tensor-memory allocation");
};

template <int MODE, int C, int N, int ZT>
__global__ void __launch_bounds__(HALO_THREADS) k_conv_halo(const ConvArgs a) {
    static_assert(MODE == MODE_FWD || MODE == MODE_DGRAD, "forward and data gradient only");
    static_assert(N % 16 == 0 && N >= 16 && N <= 64 && C % 16 == 0, "tile shapes");
    using H = Halo1<C, N, ZT>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char *Bs = sm, *Hs = sm + H::BBYTES;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(Hs + H::HBYTES);
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 1);

    const int n = a.n;
    const int w = threadIdx.x >> 5;
    if (w == 0) {
        tmem_alloc(tslot, H::NCOL);
        tmem_relinquish();
    }
    // one MMA issuer per output slice (lane 0 of warp zs), one arrival each
    if (threadIdx.x == 0) {
        mbar_init(bar, ZT);
        fence_barrier_init();
    }
    // B: the packed weights [N][27 C] (K-major rows) as core matrices
    // (n group g, K chunk kc) at kc BLEAD + g 128
    for (int e = threadIdx.x; e < N * 27 * H::CH; e += HALO_THREADS) {
        const int nn = e % N, kc = e / N;
        const uint4 v = *reinterpret_cast<const uint4 *>(a.wt + (size_t)nn * 27 * C + 8 * kc);
        *reinterpret_cast<uint4 *>(Bs + kc * H::BLEAD + (nn >> 3) * 128 + (nn & 7) * 16) = v;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const unsigned hs = smem_u32(Hs), bs = smem_u32(Bs);
    constexpr unsigned IDESC = idesc_bf16_f32(128, N);

    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + ZT - 1) / ZT;
    const int ntiles = ntx * nty * ntz;
    bool ok = true;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int x0 = (tile % ntx) * 8, y0 = ((tile / ntx) % nty) * 16, z0 = (tile / (ntx * nty)) * ZT;
        load_halo<C, H::HZ>(a.x, n, x0, y0, z0, Hs, H::PLANE);
        cp_async_commit();
        cp_async_wait<0>();
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && w < ZT) {
            const int zs = w;
            tc_fence_after();
            // descriptors built once; a tap or chunk moves the start address
            // field only (offsets in 16-byte units, no carry: shared
            // addresses stay below 2^18)
            const uint64_t ad0 = smem_desc(hs, H::PLANE, H::HX * 16) + (uint64_t)(zs * H::HY * H::HX),
                           bd0 = smem_desc(bs, H::BLEAD, 128);
            for (int tap = 0; tap < 27; ++tap) {
                int dx, dy, dz;
                tap_offset(tap, dx, dy, dz);
                if (MODE == MODE_DGRAD) { dx = -dx; dy = -dy; dz = -dz; }
                const uint64_t at = ad0 + (uint64_t)(((1 + dz) * H::HY + 1 + dy) * H::HX + 1 + dx);
                const uint64_t bt = bd0 + (uint64_t)(tap * H::CH * (H::BLEAD / 16));
#pragma unroll
                for (int cp = 0; cp < H::CH; cp += 2)
                    umma_bf16(tmem + (unsigned)(zs * N), at + (uint64_t)(cp * (H::PLANE / 16)),
                              bt + (uint64_t)(cp * (H::BLEAD / 16)), IDESC, (tap | cp) != 0);
            }
            umma_commit(bar);
        }
        if (!mbar_wait(bar, it & 1, a.status)) ok = false;
        if (!__syncthreads_and(ok)) { ok = false; break; }
        tc_fence_after();
        // epilogue: thread of row m = 32 (w % 4) + lane holds voxel (x0 + m % 8,
        // y0 + m / 8); warps w and w ^ 4 share the 16-column chunks
        const int q = w & 3, m = 32 * q + (threadIdx.x & 31);
        const int x = x0 + (m & 7), y = y0 + (m >> 3);
        for (int j = w >> 2; j < ZT * (N / 16); j += 2) {
            const int zs = j / (N / 16), c0 = 16 * (j % (N / 16));
            const int z = z0 + zs;
            float v[16];
            tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(zs * N + c0), v);
            if (x < n && y < n && z < n) store_row16<MODE>(a, ((size_t)z * n + y) * n + x, c0, v);
        }
        // every thread's tensor-memory reads are complete (tmem_ld16 waits)
        // before the next tile's first MMA overwrites the accumulators
        tc_fence_before();
    }
    // after a wait gave up: let the MMAs in flight finish (bounded) before
    // the tensor memory is freed
    if (!ok && threadIdx.x == 0) mbar_wait(bar, it & 1, a.status);
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, H::NCOL);
    }
}

// Double-buffered form: two input blocks and two accumulator sets, so the
// MMAs of tile i run while the accumulators of tile i - 1 are drained and
// the block of tile i + 1 is in flight.  Per iteration i: wait for tile i's
// copies; one thread issues tile i's MMAs into accumulator set i & 1 and
// commits them to barrier i & 1; all wait for tile i - 1's commit (its block
// and accumulators are then free), start the copies of tile i + 1 into that
// block, and write tile i - 1's output.
template <int C, int N, int ZT>
struct Halo2 {
    using H = Halo<C, N, ZT>;
    static constexpr unsigned HB = (H::HBYTES + 1023u) & ~1023u;  // one input block
    static constexpr int COLS = 2 * ZT * N;
    static constexpr unsigned NCOL = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
    static constexpr size_t SMEM = 1024 + (size_t)H::BBYTES + 2 * (size_t)HB + 64;
    static_assert(COLS <= 512, "accumulators exceed tensor memory");
};

template <int MODE, int C, int N, int ZT>
__global__ void __launch_bounds__(HALO_THREADS) k_conv_halo2(const ConvArgs a) {
    static_assert(MODE == MODE_FWD || MODE == MODE_DGRAD, "forward and data gradient only");
    static_assert(N % 16 == 0 && N >= 16 && N <= 64 && C % 16 == 0, "tile shapes");
    using H = Halo<C, N, ZT>;
    using H2 = Halo2<C, N, ZT>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char *Bs = sm, *Hs = sm + H::BBYTES;  // blocks at Hs and Hs + HB
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(Hs + 2 * H2::HB);  // [2]
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);

    const int n = a.n;
    const int w = threadIdx.x >> 5;
    if (w == 0) {
        tmem_alloc(tslot, H2::NCOL);
        tmem_relinquish();
    }
    // one MMA issuer per output slice (lane 0 of warp zs): each commit is one
    // arrival, the barrier completes when all ZT slices' MMAs have
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], ZT);
        mbar_init(&bar[1], ZT);
        fence_barrier_init();
    }
    for (int e = threadIdx.x; e < N * 27 * H::CH; e += HALO_THREADS) {
        const int nn = e % N, kc = e / N;
        const uint4 v = *reinterpret_cast<const uint4 *>(a.wt + (size_t)nn * 27 * C + 8 * kc);
        *reinterpret_cast<uint4 *>(Bs + kc * H::BLEAD + (nn >> 3) * 128 + (nn & 7) * 16) = v;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const unsigned hs0 = smem_u32(Hs), bs = smem_u32(Bs);
    constexpr unsigned IDESC = idesc_bf16_f32(128, N);

    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + ZT - 1) / ZT;
    const int ntiles = ntx * nty * ntz;
    const int cnt = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    auto origin = [&](int i, int &x0, int &y0, int &z0) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (tile % ntx) * 8;
        y0 = ((tile / ntx) % nty) * 16;
        z0 = (tile / (ntx * nty)) * ZT;
    };
    auto load = [&](int i) {
        int x0, y0, z0;
        origin(i, x0, y0, z0);
        load_halo<C, H::HZ>(a.x, n, x0, y0, z0, Hs + (i & 1) * H2::HB, H::PLANE);
        cp_async_commit();
    };
    // output of tile i from accumulator set i & 1: thread of row m = 32 (w % 4)
    // + lane holds voxel (x0 + m % 8, y0 + m / 8); warps w, w ^ 4 share chunks
    auto drain = [&](int i) {
        int x0, y0, z0;
        origin(i, x0, y0, z0);
        const int q = w & 3, m = 32 * q + (threadIdx.x & 31);
        const int x = x0 + (m & 7), y = y0 + (m >> 3);
        const unsigned acc = tmem + (unsigned)((i & 1) * ZT * N);
        for (int j = w >> 2; j < ZT * (N / 16); j += 2) {
            const int zs = j / (N / 16), c0 = 16 * (j % (N / 16));
            const int z = z0 + zs;
            float v[16];
            tmem_ld16(acc + ((unsigned)(32 * q) << 16) + (unsigned)(zs * N + c0), v);
            if (x < n && y < n && z < n) store_row16<MODE>(a, ((size_t)z * n + y) * n + x, c0, v);
        }
    };
    bool ok = true;
    int issued = -1;
    if (cnt > 0) load(0);
    for (int i = 0; i < cnt; ++i) {
        const int b = i & 1;
        cp_async_wait<0>();  // tile i's block has landed
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && w < ZT) {
            const int zs = w;
            tc_fence_after();
            const uint64_t ad0 = smem_desc(hs0 + b * H2::HB, H::PLANE, H::HX * 16) +
                                 (uint64_t)(zs * H::HY * H::HX),
                           bd0 = smem_desc(bs, H::BLEAD, 128);
            const unsigned acc = tmem + (unsigned)(b * ZT * N + zs * N);
            for (int tap = 0; tap < 27; ++tap) {
                int dx, dy, dz;
                tap_offset(tap, dx, dy, dz);
                if (MODE == MODE_DGRAD) { dx = -dx; dy = -dy; dz = -dz; }
                const uint64_t at = ad0 + (uint64_t)(((1 + dz) * H::HY + 1 + dy) * H::HX + 1 + dx);
                const uint64_t bt = bd0 + (uint64_t)(tap * H::CH * (H::BLEAD / 16));
#pragma unroll
                for (int cp = 0; cp < H::CH; cp += 2)
                    umma_bf16(acc, at + (uint64_t)(cp * (H::PLANE / 16)), bt + (uint64_t)(cp * (H::BLEAD / 16)),
                              IDESC, (tap | cp) != 0);
            }
            umma_commit(&bar[b]);
        }
        issued = i;
        // tile i - 1: its block and accumulators are free once its commit arrived
        if (i >= 1 && !mbar_wait(&bar[b ^ 1], ((i - 1) >> 1) & 1, a.status)) ok = false;
        if (__syncthreads_or(!ok)) { ok = false; break; }
        if (i + 1 < cnt) load(i + 1);
        if (i >= 1) {
            tc_fence_after();
            drain(i - 1);
        }
        tc_fence_before();
    }
    // the last tile
    if (ok && issued >= 0) {
        if (!mbar_wait(&bar[issued & 1], (issued >> 1) & 1, a.status)) ok = false;
        if (__syncthreads_and(ok)) {
            tc_fence_after();
            drain(issued);
        } else {
            ok = false;
        }
    }
    cp_async_wait<0>();
    // after a wait gave up: let the MMAs in flight finish (bounded) before
    // the tensor memory is freed
    if (!ok && issued >= 0 && threadIdx.x == 0) mbar_wait(&bar[issued & 1], (issued >> 1) & 1, a.status);
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, H2::NCOL);
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05 over the same halo blocks.  Per tap,
//   dW_tap[ci][co] = sum_p X[p + tap][ci] G[p][co]
// is a GEMM with K = voxels whose operands are both channel-contiguous
// (MN-major): A = G of an output tile (M = 128 rows: the CO channels, the
// rest padding planes of zeros whose rows are discarded), B = the shifted
// input window (N = CI).  A core matrix is 8 voxels (K) x 16 bytes (8
// channels); K-adjacent core matrices are the next line of the tile (128
// bytes in the G block, 160 in the halo block), MN-adjacent ones the next
// channel plane.  A CTA owns a group of TPG taps (TPG x CI accumulator
// columns in tensor memory) and a range of tiles, accumulates over all of
// them and writes its partial [split][tap][ci][co]; the partials are summed
// in a fixed order.  Without swizzling the descriptor's stride field holds
// the MN-direction core-matrix pitch and the leading field the K-direction
// pitch for MN-major operands too (checked against the mma.sync weight
// gradient; the exchanged assignment gives wrong sums).
// ---------------------------------------------------------------------------
template <int CI, int CO, int ZT>
struct WgHalo {
    using H = HaloBlock<CI, ZT>;  // the X block of the forward kernels
    static constexpr unsigned GPLANE = 8u * 16 * ZT * 16;  // bytes of one G channel plane
    static constexpr unsigned GREAL = (CO / 8) * GPLANE;    // the CO / 8 planes that are loaded
    // one buffer: G planes, then the X block; two buffers (double buffering)
    static constexpr unsigned BUF = (GREAL + H::HBYTES + 1023u) & ~1023u;
    // rows CO .. 127 of A read planes CO / 8 .. 15 past a buffer's G planes:
    // whatever lies there (rows discarded), but inside the allocation
    static constexpr unsigned REACH = BUF + 16 * GPLANE;
    static constexpr unsigned DATA = 2 * BUF > REACH ? 2 * BUF : REACH;
    static constexpr size_t SMEM = 1024 + (size_t)DATA + 64;
};

template <int CI, int CO, int TPG, int ZT>
__global__ void __launch_bounds__(HALO_THREADS) k_wgrad_halo(const ConvArgs a, int splits) {
    static_assert(CI % 16 == 0 && CI <= 64 && CO % 8 == 0 && CO <= 128, "channels");
    using W = WgHalo<CI, CO, ZT>;
    using H = typename W::H;
    constexpr int NCOLS = TPG * CI;
    constexpr unsigned NCOL = NCOLS <= 32 ? 32 : (NCOLS <= 64 ? 64 : (NCOLS <= 128 ? 128 : (NCOLS <= 256 ? 256 : 512)));
    static_assert(NCOLS <= 512, "accumulators exceed tensor memory");
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm + W::DATA);  // [2]
    unsigned *tslot = reinterpret_cast<unsigned *>(bar + 2);

    const int n = a.n;
    const int w = threadIdx.x >> 5;
    const int grp = blockIdx.x % ((27 + TPG - 1) / TPG), split = blockIdx.x / ((27 + TPG - 1) / TPG);
    const int tap0 = grp * TPG, ntap = min(TPG, 27 - tap0);
    if (w == 0) {
        tmem_alloc(tslot, NCOL);
        tmem_relinquish();
    }
    // MMA issuers: lane 0 of warps 0 .. NI - 1, warp w taking taps w, w + NI, ..;
    // each commit is one arrival
    const int NI = min(HALO_THREADS / 32, ntap);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], NI);
        mbar_init(&bar[1], NI);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;
    const unsigned base = smem_u32(sm);
    constexpr unsigned IDESC = idesc_bf16_f32(128, CI) | (1u << 15) | (1u << 16);  // A, B MN-major

    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + ZT - 1) / ZT;
    const long long ntiles = (long long)ntx * nty * ntz;
    const long long tb = ntiles * split / splits, te = ntiles * (split + 1) / splits;
    const int cnt = (int)(te - tb);
    // asynchronous copies of tile tb + i into buffer i & 1: the X block with
    // its halo, and G of the tile (no halo; zero outside the grid, where it
    // adds nothing)
    auto load = [&](int i) {
        const long long tile = tb + i;
        const int x0 = (int)(tile % ntx) * 8, y0 = (int)((tile / ntx) % nty) * 16,
                  z0 = (int)(tile / ((long long)ntx * nty)) * ZT;
        unsigned char *G = sm + (i & 1) * W::BUF;
        load_halo<CI, H::HZ>(a.x, n, x0, y0, z0, G + W::GREAL, H::PLANE);
        for (int e = threadIdx.x; e < 8 * 16 * ZT * (CO / 8); e += HALO_THREADS) {
            const int c = e % (CO / 8), v = e / (CO / 8);
            const int qx = x0 + v % 8, qy = y0 + (v / 8) % 16, qz = z0 + v / 128;
            const bool in = qx < n && qy < n && qz < n;
            const bf16 *src = in ? a.g + ((size_t)(qz * n + qy) * n + qx) * CO + 8 * c : a.g;
            cp_async16(G + c * W::GPLANE + v * 16, src, in ? 16u : 0u);
        }
        cp_async_commit();
    };
    bool ok = true;
    int i = 0;
    if (cnt > 0) load(0);
    for (; i < cnt; ++i) {
        const int b = i & 1;
        if (i + 1 < cnt) {
            // buffer b ^ 1 was read by the MMAs of tile i - 1
            if (i >= 1 && !mbar_wait(&bar[b ^ 1], ((i - 1) >> 1) & 1, a.status)) ok = false;
            if (__syncthreads_or(!ok)) break;
            load(i + 1);
            cp_async_wait<1>();  // tile i's copies have landed
        } else {
            cp_async_wait<0>();
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if ((threadIdx.x & 31) == 0 && w < NI) {
            tc_fence_after();
            const unsigned gs = base + b * W::BUF, hs = gs + W::GREAL;
            // descriptors built once; taps, slices and line pairs move the
            // start address field only (16-byte units, no carry)
            const uint64_t ad0 = smem_desc(gs, 128, W::GPLANE), bd0 = smem_desc(hs, H::HX * 16, H::PLANE);
            for (int j = w; j < ntap; j += NI) {
                int dx, dy, dz;
                tap_offset(tap0 + j, dx, dy, dz);
                const uint64_t bt = bd0 + (uint64_t)(((1 + dz) * H::HY + 1 + dy) * H::HX + 1 + dx);
#pragma unroll
                for (int zs = 0; zs < ZT; ++zs)
#pragma unroll
                    for (int l = 0; l < 16; l += 2)  // K = 16 voxels: lines l and l + 1
                        umma_bf16(tmem + (unsigned)(j * CI), ad0 + (uint64_t)((zs * 16 + l) * 8),
                                  bt + (uint64_t)((zs * H::HY + l) * H::HX), IDESC, (i | zs | l) != 0);
            }
            umma_commit(&bar[b]);
        }
    }
    cp_async_wait<0>();
    // the last commit arrives once every MMA of the CTA has completed
    const int last = i - 1;
    if (last >= 0 && !mbar_wait(&bar[last & 1], (last >> 1) & 1, a.status)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    // partial of this split: rows m < CO of the accumulators (row m = lane m)
    if (ok) {
        const int q = w & 3, m = 32 * q + (threadIdx.x & 31);
        float *out = a.out + (size_t)split * 27 * CI * CO;
        // warps w and w ^ 4 share the 16-column chunks (tap j, channels c0 ..)
        for (int k = w >> 2; k < ntap * (CI / 16); k += 2) {
            const int j = k / (CI / 16), c0 = 16 * (k % (CI / 16));
            float v[16];
            tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(j * CI + c0), v);
            if (m >= CO) continue;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                // a CTA with no tiles holds no accumulator: its partial is zero
                out[((size_t)(tap0 + j) * CI + c0 + u) * CO + m] = cnt > 0 ? v[u] : 0.f;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOL);
    }
}

// ---------------------------------------------------------------------------
// Forward and data gradient on tcgen05 with the three z taps of one (dy, dx)
// in one MMA.  Output slice zo of a tile takes input slice zo + 1 + dz (halo
// coordinates) through the weights of input offset dz, so one input slice zi
// feeds the output slices zi - 2, zi - 1 and zi through the offsets dz = +1, 0
// and -1: with B holding those three weight matrices side by side (N = 3 NO)
// and the accumulators of consecutive output slices in consecutive
// tensor-memory columns, one MMA of N = 3 NO per (input slice, dy, dx, K
// chunk pair) covers all three.  Per tile that is (ZT + 2) x 9 x C / 16 MMAs
// instead of 27 ZT C / 16 with N = NO: the A tile (128 voxels x 16 channels,
// read from shared memory by the tensor core for every MMA) is read about
// 3 ZT / (ZT + 2) times less often.  Input slices at the ends feed only the
// output slices inside the tile (narrower N, no wasted products).
//
// The MMAs of one thread do not overlap one another on the tensor core (for
// these narrow MMAs each costs about its operand reads + math + accumulate),
// so ISS threads issue them: thread k the input slices zi = k (mod ISS), into
// its own accumulator set (no two threads write the same columns); the
// epilogue adds the sets.  Every MMA accumulates: the epilogue zeroes a set
// after draining it (and once at the start).
//
// The input block of a tile (10 x 18 x (ZT + 2) voxels with the one-voxel
// halo, zero outside the grid) arrives by TMA, one 4D box per 8-channel chunk
// plane: elements [z][y][x][8 channels] in a plane, so eight consecutive x
// voxels of a line are a K-major core matrix (rows 16 bytes apart), lines are
// M-adjacent (160 bytes) and chunk planes K-adjacent.  Units of CH / KS chunk
// planes of one tile cycle through S stages.  Warp roles: warp 0 lane 0
// issues the copies, lane 0 of warps 1 .. ISS the MMAs (two accumulator
// buffers, so tile i's MMAs run while tile i - 1 is drained), warps 4-7 drain
// the accumulators (warp w reads tensor-memory lanes 32 (w % 4) ..) into the
// output.  Every wait is bounded; a role that gives up stops, and the copies
// and MMAs it issued are waited for (bounded) before the tensor memory is
// freed.
// ---------------------------------------------------------------------------
template <int C, int NO, int ZT, int KS, int S, int ISS>
struct DzCfg {
    static constexpr int HX = 10, HY = 18, HZ = ZT + 2, CH = C / 8, CHS = CH / KS;
    static constexpr unsigned PLANE = 16u * HX * HY * HZ;  // one chunk plane of the input block
    static constexpr unsigned STAGE = PLANE * CHS;         // one unit: CHS chunk planes of a tile
    static constexpr int N3 = 3 * NO;
    static constexpr unsigned BLEAD = (unsigned)N3 * 16;  // K-chunk pitch of B
    static constexpr unsigned BBYTES = 9u * CH * BLEAD;    // = 27 C NO bf16
    static constexpr unsigned SOFF = (BBYTES + 1023u) & ~1023u;
    static constexpr unsigned BAROFF = SOFF + (unsigned)S * STAGE;
    static constexpr int SET = ZT * NO;               // columns of one accumulator set
    static constexpr int COLS = 2 * ISS * SET;        // two buffers of ISS sets
    static constexpr unsigned NCOL = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
    static constexpr size_t SMEM = 1024 + (size_t)BAROFF + 512;  // + barriers, tensor-memory slot, biases
    static_assert(PLANE % 128 == 0, "TMA destinations are 128-byte aligned");
    static_assert(CH % KS == 0 && CHS % 2 == 0, "units of whole K chunk pairs");
    static_assert(NO % 16 == 0 && N3 <= 256 && COLS <= 512, "MMA and tensor-memory shapes");
    static_assert(ISS >= 1 && ISS <= 3 && SMEM <= 232448, "issuers, shared memory");
};

constexpr int DZ_THREADS = 256;

template <int MODE, int C, int NO, int ZT, int KS, int S, int ISS>
__global__ void __launch_bounds__(DZ_THREADS, 1) k_conv_dz(const __grid_constant__ CUtensorMap tmap,
                                                           const ConvArgs a) {
    static_assert(MODE == MODE_FWD || MODE == MODE_DGRAD, "forward and data gradient only");
    using D = DzCfg<C, NO, ZT, KS, S, ISS>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char *Bs = sm, *St = sm + D::SOFF;
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sm + D::BAROFF);
    unsigned long long *empty = full + S, *accf = full + 2 * S, *acce = full + 2 * S + 2;
    unsigned *tslot = reinterpret_cast<unsigned *>(full + 2 * S + 4);

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 0) {
        tmem_alloc(tslot, D::NCOL);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);     // the producer's expect_tx arrival (+ the copies' bytes)
            mbar_init(&empty[s], ISS);  // one commit per issuer
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], ISS);  // each issuer's commit after a tile's last MMA
            mbar_init(&acce[b], 4);    // one arrival per draining warp (zeroed, free)
        }
        fence_barrier_init();
    }
    // B: the weights of the three z offsets of each (dy, dx) side by side,
    // core matrix (n group g, K chunk t9 CH + kc) at (t9 CH + kc) BLEAD + g 128
    for (int e = threadIdx.x; e < 9 * D::CH * D::N3; e += DZ_THREADS) {
        const int tk = e / D::N3, r = e % D::N3;
        const uint4 v = reinterpret_cast<const uint4 *>(a.wdz)[e];
        *reinterpret_cast<uint4 *>(Bs + tk * D::BLEAD + (r >> 3) * 128 + (r & 7) * 16) = v;
    }
    float *sbias = reinterpret_cast<float *>(tslot + 1);  // NO biases (forward)
    if (MODE == MODE_FWD)
        for (int c = threadIdx.x; c < NO; c += DZ_THREADS) sbias[c] = a.bias[c];
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    const int n = a.n;
    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + ZT - 1) / ZT;
    const int ntiles = ntx * nty * ntz;
    const int cnt = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int units = cnt * KS;
    auto origin = [&](int i, int &x0, int &y0, int &z0) {
        const int tile = (int)blockIdx.x + i * (int)gridDim.x;
        x0 = (tile % ntx) * 8;
        y0 = ((tile / ntx) % nty) * 16;
        z0 = (tile / (ntx * nty)) * ZT;
    };

    if (w == 0 && lane == 0) {
        // producer: unit u = (tile i, channel group ks) into stage u % S
        int u = 0;
        for (; u < units; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(&empty[s], ((u / S) - 1) & 1, a.status)) break;
            const int i = u / KS, ks = u % KS;
            int x0, y0, z0;
            origin(i, x0, y0, z0);
            mbar_expect_tx(&full[s], D::STAGE);
#pragma unroll
            for (int c = 0; c < D::CHS; ++c)
                tma_load_4d(St + s * D::STAGE + c * D::PLANE, &tmap, 8 * (ks * D::CHS + c), x0 - 1, y0 - 1,
                            z0 - 1, &full[s]);
        }
        // the copies of the last units land before the CTA can exit (already
        // waited for by the MMA issuers unless they gave up)
        for (int v = u - S > 0 ? u - S : 0; v < u; ++v) mbar_wait(&full[v % S], (v / S) & 1, a.status);
    } else if (w >= 1 && w <= ISS && lane == 0) {
        // MMA issuer k = w - 1: input slices zi = k (mod ISS) into set k
        const int k = w - 1;
        const uint64_t bd0 = smem_desc(smem_u32(Bs), D::BLEAD, 128);
        int u = 0;
        for (; u < units; ++u) {
            const int s = u % S, i = u / KS, ks = u % KS, b = i & 1;
            if (!mbar_wait(&full[s], (u / S) & 1, a.status)) break;
            // accumulator buffer b is drained and zeroed (tile i - 2, or the start)
            if (ks == 0 && !mbar_wait(&acce[b], (i >> 1) & 1, a.status)) break;
            tc_fence_after();
            const uint64_t ad0 = smem_desc(smem_u32(St + s * D::STAGE), D::PLANE, D::HX * 16);
            const unsigned acc = tmem + (unsigned)((b * ISS + k) * D::SET);
            for (int zi = k; zi < D::HZ; zi += ISS) {
                // blocks blo .. bhi of B (dz = +1, 0, -1) feed output slices zi - 2 + blk inside the tile
                const int blo = zi < 2 ? 2 - zi : 0, bhi = zi > ZT - 1 ? ZT + 1 - zi : 2, nb = bhi - blo + 1;
                const unsigned idesc = idesc_bf16_f32(128, nb * NO);
                const unsigned col = acc + (unsigned)((zi - 2 + blo) * NO);
                for (int t9 = 0; t9 < 9; ++t9) {
                    const uint64_t at = ad0 + (uint64_t)((zi * D::HY + t9 / 3) * D::HX + t9 % 3);
                    const uint64_t bt = bd0 + (uint64_t)((t9 * D::CH + ks * D::CHS) * (D::BLEAD / 16) + blo * NO);
#pragma unroll
                    for (int cp = 0; cp < D::CHS; cp += 2)
                        umma_bf16(col, at + (uint64_t)(cp * (D::PLANE / 16)),
                                  bt + (uint64_t)(cp * (D::BLEAD / 16)), idesc, 1);
                }
            }
            umma_commit(&empty[s]);
            if (ks == KS - 1) umma_commit(&accf[b]);
        }
        // every MMA issued has completed before the tensor memory is freed
        if (u > 0) mbar_wait(&empty[(u - 1) % S], ((u - 1) / S) & 1, a.status);
    } else if (w >= 4) {
        // epilogue: thread of row m = 32 (w % 4) + lane holds voxel (x0 + m % 8, y0 + m / 8)
        const int q = w & 3, m = 32 * q + lane;
        const unsigned lrow = (unsigned)(32 * q) << 16;
        // zero both buffers, then hand them to the issuers
        for (int c0 = 0; c0 < 2 * ISS * D::SET; c0 += 16) tmem_zero16(tmem + lrow + (unsigned)c0);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&acce[0]);
            mbar_arrive(&acce[1]);
        }
        for (int i = 0; i < cnt; ++i) {
            const int b = i & 1;
            int x0, y0, z0;
            origin(i, x0, y0, z0);
            const int x = x0 + (m & 7), y = y0 + (m >> 3);
            // the residual rows of this thread's voxel, all slices at once
            // (independent loads in flight while the MMAs finish)
            uint4 sk[MODE == MODE_FWD ? ZT * NO / 8 : 1];
            if (MODE == MODE_FWD) {
#pragma unroll
                for (int zo = 0; zo < ZT; ++zo)
#pragma unroll
                    for (int c8 = 0; c8 < NO / 8; ++c8) {
                        const bool in = a.skip && x < n && y < n && z0 + zo < n;
                        sk[zo * (NO / 8) + c8] =
                            in ? reinterpret_cast<const uint4 *>(a.skip + (((size_t)(z0 + zo) * n + y) * n + x) * NO)[c8]
                               : make_uint4(0u, 0u, 0u, 0u);
                    }
            }
            const bool got = mbar_wait(&accf[b], (i >> 1) & 1, a.status);
            if (!__all_sync(0xffffffffu, got)) break;
            tc_fence_after();
            const unsigned acc = tmem + lrow + (unsigned)(b * ISS * D::SET);
            if (MODE == MODE_DGRAD && a.up_adj) {
                // the adjoint of the next layer's 2^3 nearest upsampling: the sum
                // over the 8 children (x pairs: lanes ^ 1; y pairs: lanes ^ 8;
                // z pairs: slices 2 zp, 2 zp + 1) written at half resolution by
                // the lane of the even child (n is even: every in-grid parent
                // has its 8 children in the grid)
                const int hn = n / 2, px = x >> 1, py = y >> 1;
#pragma unroll 1
                for (int zp = 0; zp < ZT / 2; ++zp) {
                    const int pz = (z0 >> 1) + zp;
#pragma unroll 1
                    for (int c0 = 0; c0 < NO; c0 += 16) {
                        float v[16];
                        tmem_ld16(acc + (unsigned)(2 * zp * NO + c0), v);
#pragma unroll
                        for (int k = 0; k < 2 * ISS; ++k) {
                            if (k == 0) continue;
                            float v2[16];
                            tmem_ld16(acc + (unsigned)((k % ISS) * D::SET + (2 * zp + k / ISS) * NO + c0), v2);
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[j] += v2[j];
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 1);
                            v[j] += __shfl_xor_sync(0xffffffffu, v[j], 8);
                        }
                        if ((lane & 9) == 0 && px < hn && py < hn && pz < hn) {
                            float4 *op = reinterpret_cast<float4 *>(a.out + (((size_t)pz * hn + py) * hn + px) * NO + c0);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                op[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        }
                    }
                }
            } else
#pragma unroll
            for (int zo = 0; zo < ZT; ++zo) {
                const int z = z0 + zo;
#pragma unroll
                for (int c0 = 0; c0 < NO; c0 += 16) {
                    float v[16];
                    tmem_ld16(acc + (unsigned)(zo * NO + c0), v);
#pragma unroll
                    for (int k = 1; k < ISS; ++k) {
                        float v2[16];
                        tmem_ld16(acc + (unsigned)(k * D::SET + zo * NO + c0), v2);
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] += v2[j];
                    }
                    if (x < n && y < n && z < n) {
                        const size_t row = ((size_t)z * n + y) * n + x;
                        if (MODE == MODE_FWD)
                            store_fwd16(a.y + row * NO + c0, v, sbias + c0, sk[zo * (NO / 8) + c0 / 8],
                                        sk[zo * (NO / 8) + c0 / 8 + 1]);
                        else
                            store_row16<MODE>(a, row, c0, v);
                    }
                }
            }
            for (int c0 = 0; c0 < ISS * D::SET; c0 += 16) tmem_zero16(acc + (unsigned)c0);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
        }
    }
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, D::NCOL);
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on tcgen05 with the input channels and z offsets on M and
// the y offsets and output channels on N.  For one x offset dx,
//   D[(dz, ci)][(j, co)] = sum_p X[p + (dx, 0, dz)][ci] G[p + (0, j - 1, 0)][co]
//                        = dW[tap (dz, 1 - j, dx)][ci][co]
// (substituting q = p + (0, j - 1, 0); the terms the substitution moves out
// of the tiles multiply a zero: X or G outside the grid).  A = the input
// block, MN-major: a core matrix is 8 consecutive x voxels (K, 16 bytes
// apart) x 8 channels; with the block stored as [chunk][z][y][x] planes of
// 16 lines, the 16 M-adjacent core matrices of 4 chunks x 4 z offsets are one
// plane (2,560 bytes) apart, so rows (chunk, dz + 1) cover four z offsets of
// 32 channels (the fourth discarded: a quarter of the rows wasted instead of
// seven eighths with the output channels on M); K-adjacent core matrices are
// the next line.  B = the output gradient with a one-line y halo stored as
// [z][y][chunk][x]: N-adjacent core matrices (8 channels) one chunk apart run
// on into the next line, so N = 3 COG covers the three y offsets of a group
// of COG output channels.  Per (tile of 8 x 16 x 2 voxels, dx, M half, z
// slice, line pair) one MMA of 128 x 3 COG x 16.  A CTA owns a group of
// COG output channels and a range of tiles (a split); its accumulators stay
// in tensor memory over all of them and it writes its partial
// [split][tap][ci][co] at the end (summed over splits in a fixed order).
// Copies: the input block by TMA (one 4D box per 8-channel chunk: 10 x 16 x 4
// voxels) from warp 0 lane 0, the output-gradient block by cp.async from
// warps 4-5 (zero outside the grid).  The MMAs of one thread do not overlap
// one another, so three threads issue them (lane 0 of warps 1-3), one per dx,
// each into its own accumulators.  S stages.
// ---------------------------------------------------------------------------
template <int CI, int CO, int COG, int S>
struct WzCfg {
    static constexpr int ZT = 2, HX = 10, LINES = 16, CH = CI / 8, MH = CI / 32;
    static constexpr unsigned XP = 16u * HX * LINES;          // one (chunk, z) plane of the input block
    static constexpr unsigned XBYTES = (unsigned)CH * 4 * XP;  // chunks x 4 z slices
    static constexpr unsigned LS = (unsigned)(COG / 8) * 128;  // output-gradient line pitch
    static constexpr unsigned GBYTES = (unsigned)ZT * 18 * LS;
    static constexpr unsigned STAGE = XBYTES + GBYTES;
    static constexpr int NG = CO / COG, NB = 3 * COG, COLS = 3 * MH * NB;
    static constexpr unsigned NCOL = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
    static constexpr unsigned BAROFF = (unsigned)S * STAGE;
    static constexpr size_t SMEM = 1024 + (size_t)BAROFF + 256;
    static_assert(CI % 32 == 0 && CO % COG == 0 && COG % 16 == 0 && NB <= 256 && COLS <= 512, "shapes");
    // the discarded rows of the last chunk read one plane past the input block
    static_assert(STAGE % 128 == 0 && GBYTES >= XP, "layout");
    static_assert(SMEM <= 232448, "shared memory");
};

constexpr int WZ_THREADS = 256;

template <int CI, int CO, int COG, int S>
__global__ void __launch_bounds__(WZ_THREADS, 1) k_wgrad_dz(const __grid_constant__ CUtensorMap tmap,
                                                            const ConvArgs a, int splits) {
    using W = WzCfg<CI, CO, COG, S>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sm + W::BAROFF);
    unsigned long long *empty = full + S, *done = full + 2 * S;
    unsigned *tslot = reinterpret_cast<unsigned *>(full + 2 * S + 1);

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = (int)blockIdx.x % W::NG, split = (int)blockIdx.x / W::NG, co0 = grp * COG;
    if (w == 0) {
        tmem_alloc(tslot, W::NCOL);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1 + 64);  // the TMA's expect_tx arrival + one per cp.async thread
            mbar_init(&empty[s], 3);      // one commit per issuer
        }
        mbar_init(done, 3);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    const int n = a.n;
    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + W::ZT - 1) / W::ZT;
    const long long ntiles = (long long)ntx * nty * ntz;
    const long long tb = ntiles * split / splits, te = ntiles * (split + 1) / splits;
    const int cnt = (int)(te - tb);
    auto origin = [&](int i, int &x0, int &y0, int &z0) {
        const long long tile = tb + i;
        x0 = (int)(tile % ntx) * 8;
        y0 = (int)((tile / ntx) % nty) * 16;
        z0 = (int)(tile / ((long long)ntx * nty)) * W::ZT;
    };

    if (w == 0 && lane == 0) {
        // input block of unit u by TMA: chunk c at (4 c) planes
        int u = 0;
        for (; u < cnt; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(&empty[s], ((u / S) - 1) & 1, a.status)) break;
            int x0, y0, z0;
            origin(u, x0, y0, z0);
            unsigned char *X = sm + s * W::STAGE;
            mbar_expect_tx(&full[s], W::XBYTES);
#pragma unroll
            for (int c = 0; c < W::CH; ++c) tma_load_4d(X + c * 4 * W::XP, &tmap, 8 * c, x0 - 1, y0, z0 - 1, &full[s]);
        }
        for (int v = u - S > 0 ? u - S : 0; v < u; ++v) mbar_wait(&full[v % S], (v / S) & 1, a.status);
    } else if (w == 4 || w == 5) {
        // output-gradient block of unit u (lines y0 - 1 .. y0 + 16, the group's channels)
        const int t = threadIdx.x - 128;
        constexpr int CC = COG / 8, TOT = W::ZT * 18 * CC * 8;
        for (int u = 0; u < cnt; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(&empty[s], ((u / S) - 1) & 1, a.status)) break;
            int x0, y0, z0;
            origin(u, x0, y0, z0);
            unsigned char *G = sm + s * W::STAGE + W::XBYTES;
            for (int e = t; e < TOT; e += 64) {
                const int xv = e % 8, cc = (e / 8) % CC, ly = (e / (8 * CC)) % 18, zs = e / (8 * CC * 18);
                const int qx = x0 + xv, qy = y0 + ly - 1, qz = z0 + zs;
                const bool in = qx < n && qy >= 0 && qy < n && qz < n;
                const bf16 *src = in ? a.g + ((size_t)(qz * n + qy) * n + qx) * CO + co0 + 8 * cc : a.g;
                cp_async16(G + ((zs * 18 + ly) * CC + cc) * 128 + xv * 16, src, in ? 16u : 0u);
            }
            cp_async_mbar_arrive(&full[s]);
        }
        cp_async_wait<0>();
    } else if (w >= 1 && w <= 3 && lane == 0) {
        // MMA issuer of x offset dxi = w - 1 (its accumulators: MH halves)
        const int dxi = w - 1;
        constexpr unsigned IDESC = idesc_bf16_f32(128, W::NB) | (1u << 15) | (1u << 16);  // A, B MN-major
        for (int u = 0; u < cnt; ++u) {
            const int s = u % S;
            if (!mbar_wait(&full[s], (u / S) & 1, a.status)) break;
            fence_async_smem();  // the cp.async writes, for the tensor core's reads
            tc_fence_after();
            const unsigned xs = smem_u32(sm + s * W::STAGE), gs = xs + W::XBYTES;
#pragma unroll 1
            for (int zs = 0; zs < W::ZT; ++zs)
#pragma unroll 2
                for (int lp = 0; lp < 8; ++lp) {
                    const uint64_t bd = smem_desc(gs + (unsigned)(zs * 18 + 2 * lp) * W::LS, W::LS, 128);
#pragma unroll
                    for (int h = 0; h < W::MH; ++h) {
                        const uint64_t ad = smem_desc(
                            xs + (unsigned)(h * 16 + zs) * W::XP + (unsigned)(2 * lp * 160 + dxi * 16), 160, W::XP);
                        umma_bf16(tmem + (unsigned)((dxi * W::MH + h) * W::NB), ad, bd, IDESC, (u | zs | lp) != 0);
                    }
                }
            umma_commit(&empty[s]);
        }
        // arrives once every MMA this thread issued has completed
        umma_commit(done);
    }
    if (w >= 4) {
        const bool got = mbar_wait(done, 0, a.status);
        __syncwarp();
        tc_fence_after();
        // row m = (chunk c, dz + 1) of an M half, channel ci = 8 c + m % 8
        const int q = w & 3, m = 32 * q + lane, mg = m >> 3, dzp = mg & 3;
        float *out = a.out + (size_t)split * 27 * CI * CO;
        for (int dxi = 0; dxi < 3; ++dxi)
            for (int h = 0; h < W::MH; ++h) {
                const int ci = 8 * (h * 4 + (mg >> 2)) + (m & 7);
                for (int j = 0; j < 3; ++j)
#pragma unroll 1
                    for (int c16 = 0; c16 < COG; c16 += 16) {
                        float v[16];
                        tmem_ld16(tmem + ((unsigned)(32 * q) << 16) +
                                      (unsigned)((dxi * W::MH + h) * W::NB + j * COG + c16),
                                  v);
                        if (dzp == 3 || !got) continue;
                        const int tap = dzp * 9 + (2 - j) * 3 + dxi;
                        float *o = out + ((size_t)tap * CI + ci) * CO + co0 + c16;
#pragma unroll
                        for (int k = 0; k < 16; ++k) o[k] = cnt > 0 ? v[k] : 0.f;  // no tiles: no accumulator
                    }
            }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, W::NCOL);
    }
}

// Weight gradient for few input channels (16): the roles of k_wgrad_dz's
// operands swapped.  A = the output-gradient block (MN-major, [z][y][chunk][x]
// with a one-line y halo): M-adjacent core matrices one chunk apart run on
// into the next line, so the 128 rows are (j, co) for four y offsets j (the
// fourth discarded) of 32 output channels; B = the input block (MN-major,
// [chunk][z][y][x] planes): N = (chunk, dz + 1) x 8 channels = 4 CI columns
// (the fourth z offset discarded).  D[(j, co)][(dz, ci)] = dW[tap (dz, 1 - j,
// dx)][ci][co] for one dx, with the same substitution as k_wgrad_dz.  Rows
// wasted: a quarter, against three quarters with the output channels alone
// on M.  Copies, issuers (one per dx) and stages as in k_wgrad_dz.
template <int CI, int CO, int S>
struct WtCfg {
    static constexpr int ZT = 2, HX = 10, LINES = 16, CH = CI / 8;
    static constexpr unsigned XP = 16u * HX * LINES;          // one (chunk, z) plane of the input block
    static constexpr unsigned XBYTES = (unsigned)CH * 4 * XP;  // chunks x 4 z slices
    static constexpr unsigned LS = (unsigned)(CO / 8) * 128;   // output-gradient line pitch
    // 18 lines per slice; the discarded fourth y offset reads up to two lines
    // past the last slice: padding
    static constexpr unsigned GBYTES = (unsigned)(ZT * 18 + 2) * LS;
    static constexpr unsigned STAGE = XBYTES + GBYTES;
    static constexpr int NB = 4 * CI, COLS = 3 * NB;
    static constexpr unsigned NCOL = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
    static constexpr unsigned BAROFF = (unsigned)S * STAGE;
    static constexpr size_t SMEM = 1024 + (size_t)BAROFF + 256;
    static_assert(CO * 4 == 128 && NB % 16 == 0 && NB <= 256 && COLS <= 512, "shapes");
    // the discarded z offset of the last chunk reads one plane past the input block
    static_assert(STAGE % 128 == 0 && GBYTES >= XP, "layout");
    static_assert(SMEM <= 232448, "shared memory");
};

template <int CI, int CO, int S>
__global__ void __launch_bounds__(WZ_THREADS, 1) k_wgrad_dzt(const __grid_constant__ CUtensorMap tmap,
                                                             const ConvArgs a, int splits) {
    using W = WtCfg<CI, CO, S>;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(sm + W::BAROFF);
    unsigned long long *empty = full + S, *done = full + 2 * S;
    unsigned *tslot = reinterpret_cast<unsigned *>(full + 2 * S + 1);

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = (int)blockIdx.x;
    if (w == 0) {
        tmem_alloc(tslot, W::NCOL);
        tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1 + 64);  // the TMA's expect_tx arrival + one per cp.async thread
            mbar_init(&empty[s], 3);      // one commit per issuer
        }
        mbar_init(done, 3);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    const int n = a.n;
    const int ntx = (n + 7) / 8, nty = (n + 15) / 16, ntz = (n + W::ZT - 1) / W::ZT;
    const long long ntiles = (long long)ntx * nty * ntz;
    const long long tb = ntiles * split / splits, te = ntiles * (split + 1) / splits;
    const int cnt = (int)(te - tb);
    auto origin = [&](int i, int &x0, int &y0, int &z0) {
        const long long tile = tb + i;
        x0 = (int)(tile % ntx) * 8;
        y0 = (int)((tile / ntx) % nty) * 16;
        z0 = (int)(tile / ((long long)ntx * nty)) * W::ZT;
    };

    if (w == 0 && lane == 0) {
        int u = 0;
        for (; u < cnt; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(&empty[s], ((u / S) - 1) & 1, a.status)) break;
            int x0, y0, z0;
            origin(u, x0, y0, z0);
            unsigned char *X = sm + s * W::STAGE;
            mbar_expect_tx(&full[s], W::XBYTES);
#pragma unroll
            for (int c = 0; c < W::CH; ++c) tma_load_4d(X + c * 4 * W::XP, &tmap, 8 * c, x0 - 1, y0, z0 - 1, &full[s]);
        }
        for (int v = u - S > 0 ? u - S : 0; v < u; ++v) mbar_wait(&full[v % S], (v / S) & 1, a.status);
    } else if (w == 4 || w == 5) {
        const int t = threadIdx.x - 128;
        constexpr int CC = CO / 8, TOT = W::ZT * 18 * CC * 8;
        for (int u = 0; u < cnt; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(&empty[s], ((u / S) - 1) & 1, a.status)) break;
            int x0, y0, z0;
            origin(u, x0, y0, z0);
            unsigned char *G = sm + s * W::STAGE + W::XBYTES;
            for (int e = t; e < TOT; e += 64) {
                const int xv = e % 8, cc = (e / 8) % CC, ly = (e / (8 * CC)) % 18, zs = e / (8 * CC * 18);
                const int qx = x0 + xv, qy = y0 + ly - 1, qz = z0 + zs;
                const bool in = qx < n && qy >= 0 && qy < n && qz < n;
                const bf16 *src = in ? a.g + ((size_t)(qz * n + qy) * n + qx) * CO + 8 * cc : a.g;
                cp_async16(G + ((zs * 18 + ly) * CC + cc) * 128 + xv * 16, src, in ? 16u : 0u);
            }
            cp_async_mbar_arrive(&full[s]);
        }
        cp_async_wait<0>();
    } else if (w >= 1 && w <= 3 && lane == 0) {
        const int dxi = w - 1;
        constexpr unsigned IDESC = idesc_bf16_f32(128, W::NB) | (1u << 15) | (1u << 16);  // A, B MN-major
        for (int u = 0; u < cnt; ++u) {
            const int s = u % S;
            if (!mbar_wait(&full[s], (u / S) & 1, a.status)) break;
            fence_async_smem();  // the cp.async writes, for the tensor core's reads
            tc_fence_after();
            const unsigned xs = smem_u32(sm + s * W::STAGE), gs = xs + W::XBYTES;
#pragma unroll 1
            for (int zs = 0; zs < W::ZT; ++zs)
#pragma unroll 2
                for (int lp = 0; lp < 8; ++lp) {
                    const uint64_t ad = smem_desc(gs + (unsigned)(zs * 18 + 2 * lp) * W::LS, W::LS, 128);
                    const uint64_t bd =
                        smem_desc(xs + (unsigned)zs * W::XP + (unsigned)(2 * lp * 160 + dxi * 16), 160, W::XP);
                    umma_bf16(tmem + (unsigned)(dxi * W::NB), ad, bd, IDESC, (u | zs | lp) != 0);
                }
            umma_commit(&empty[s]);
        }
        umma_commit(done);
    }
    if (w >= 4) {
        const bool got = mbar_wait(done, 0, a.status);
        __syncwarp();
        tc_fence_after();
        // row m = (j, co): j = m / CO (the warp's lane quarter), co = m % CO
        const int q = w & 3, m = 32 * q + lane, j = m / CO, co = m % CO;
        float *out = a.out + (size_t)split * 27 * CI * CO;
        for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll 1
            for (int n0 = 0; n0 < W::NB; n0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((unsigned)(32 * q) << 16) + (unsigned)(dxi * W::NB + n0), v);
                if (j == 3 || !got) continue;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    // column n0 + k = ((chunk c) 4 + dz + 1) 8 + channel
                    const int g = (n0 + k) >> 3, c = g >> 2, dzp = g & 3, ci = 8 * c + ((n0 + k) & 7);
                    if (dzp == 3) continue;
                    const int tap = dzp * 9 + (2 - j) * 3 + dxi;
                    out[((size_t)tap * CI + ci) * CO + co] = cnt > 0 ? v[k] : 0.f;
                }
            }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, W::NCOL);
    }
}

// the weights [27][ci][co] as k_conv_dz's B: wt[((t9 CH + kc) 3 NO + r) 8 + k]
// for (dy, dx) = t9, chunk kc of the C input channels, row r = blk NO + o
// (input offset dz = 1 - blk) and the k-th channel of the chunk:
//   forward        W[tap (dz, dy, dx)][ci 8 kc + k][co o]
//   data gradient  W[tap (-dz, -dy, -dx)][ci o][co 8 kc + k]  (input offset = -tap)
// grid.y: 0 forward, 1 data gradient
__global__ void k_wpack_dz(int ci, int co, const bf16 *__restrict__ w, bf16 *__restrict__ wf,
                           bf16 *__restrict__ wd) {
    const int mode = blockIdx.y;
    const int C = mode == 0 ? ci : co, NO = mode == 0 ? co : ci, CH = C / 8;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 27 * C * NO) return;
    const int k = i % 8, r = (i / 8) % (3 * NO), tk = i / (24 * NO);
    const int kc = tk % CH, t9 = tk / CH;
    const int dz = 1 - r / NO, o = r % NO, dy = t9 / 3 - 1, dx = t9 % 3 - 1, c = 8 * kc + k;
    if (mode == 0) {
        const int tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
        wf[i] = w[((size_t)tap * ci + c) * co + o];
    } else {
        const int tap = (1 - dz) * 9 + (1 - dy) * 3 + (1 - dx);
        wd[i] = w[((size_t)tap * ci + o) * co + c];
    }
}

// the weights [27][ci][co] as the B operand of the tcgen05 GEMMs, K-major:
//   forward       wt[co][tap ci + ch] = w[tap][ch][co]
//   data gradient wt[ci][tap co + ch] = w[tap][ci][ch]
__global__ void k_wpack(int mode, int ci, int co, const bf16 *__restrict__ w, bf16 *__restrict__ wt) {
    const int C = mode == MODE_FWD ? ci : co, N = mode == MODE_FWD ? co : ci, K = 27 * C;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * K) return;
    const int nn = i / K, k = i % K, tap = k / C, ch = k % C;
    wt[i] = mode == MODE_FWD ? w[((size_t)tap * ci + ch) * co + nn] : w[((size_t)tap * ci + nn) * co + ch];
}

// ---------------------------------------------------------------------------
// CUDA-core layers and elementwise kernels
// ---------------------------------------------------------------------------
// 8 / 16 consecutive BF16 values (16-byte aligned) to and from FP32
__device__ __forceinline__ void load8_bf16(const bf16 *p, float *v) {
    const uint4 u = *reinterpret_cast<const uint4 *>(p);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h;
        memcpy(&h, &w[i], 4);
        const float2 f = __bfloat1622float2(h);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}
__device__ __forceinline__ void store8_bf16(bf16 *p, const float *v) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        memcpy(&w[i], &h, 4);
    }
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ void load16_bf16(const bf16 *p, float *v) {
    load8_bf16(p, v);
    load8_bf16(p + 8, v + 8);
}
__device__ __forceinline__ void store16_bf16(bf16 *p, const float *v) {
    store8_bf16(p, v);
    store8_bf16(p + 8, v + 8);
}

// first layer: 1 -> 16 channels, input FP32.  A thread computes 4
// consecutive x voxels; the block's weights and biases sit in shared memory
// (read as float4 broadcasts).  Per (dz, dy) the six inputs x0 - 1 .. x0 + 4
// of the row are loaded once and feed the three dx taps: 6 loads + 12
// float4 weight reads per 192 FMAs.
constexpr int C1_VX = 4;
__global__ void __launch_bounds__(128) k_conv1_fwd(int n, const float *__restrict__ x, const float *__restrict__ w,
                                                   const float *__restrict__ b, bf16 *__restrict__ y) {
    __shared__ __align__(16) float wsm[27 * 16 + 16];
    for (int e = threadIdx.x; e < 27 * 16 + 16; e += blockDim.x) wsm[e] = e < 27 * 16 ? w[e] : b[e - 27 * 16];
    __syncthreads();
    const int nxg = (n + C1_VX - 1) / C1_VX;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nxg * n * n) return;
    const int px0 = (int)(t % nxg) * C1_VX, py = (int)((t / nxg) % n), pz = (int)(t / ((long long)nxg * n));
    float acc[C1_VX][16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const float bc = wsm[27 * 16 + c];
#pragma unroll
        for (int i = 0; i < C1_VX; ++i) acc[i][c] = bc;
    }
#pragma unroll
    for (int r = 0; r < 9; ++r) {  // (dz, dy) = (r / 3 - 1, r % 3 - 1)
        const int qy = py + r % 3 - 1, qz = pz + r / 3 - 1;
        const bool rowok = qy >= 0 && qy < n && qz >= 0 && qz < n;
        const float *row = x + ((size_t)(rowok ? qz : 0) * n + (rowok ? qy : 0)) * n;
        float xv[C1_VX + 2];
#pragma unroll
        for (int i = 0; i < C1_VX + 2; ++i) {
            const int qx = px0 + i - 1;
            xv[i] = (rowok && qx >= 0 && qx < n) ? row[qx] : 0.f;
        }
#pragma unroll
        for (int dxi = 0; dxi < 3; ++dxi) {
            const float4 *wt = reinterpret_cast<const float4 *>(wsm + (r * 3 + dxi) * 16);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 wk = wt[k];
#pragma unroll
                for (int i = 0; i < C1_VX; ++i) {
                    const float v = xv[i + dxi];
                    acc[i][4 * k] = fmaf(v, wk.x, acc[i][4 * k]);
                    acc[i][4 * k + 1] = fmaf(v, wk.y, acc[i][4 * k + 1]);
                    acc[i][4 * k + 2] = fmaf(v, wk.z, acc[i][4 * k + 2]);
                    acc[i][4 * k + 3] = fmaf(v, wk.w, acc[i][4 * k + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < C1_VX; ++i) {
        if (px0 + i >= n) break;
        float o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = fmaxf(acc[i][c], 0.f);
        store16_bf16(y + (((size_t)pz * n + py) * n + px0 + i) * 16, o);
    }
}

// weight gradient of the first layer: a block walks 8^3 voxel tiles (tile
// b, b + gridDim.x, ...) with the input block (10^3, zero outside) and the
// tile's gz [512][16] in shared memory, double-buffered (the next tile's
// copies run during this tile's sums).  Thread i < 144 owns the three taps
// (dz, dy, dx = -1, 0, 1) of row r = i % 9 and the voxels v = i / 9 (mod 16)
// of each tile, for all 16 channels: per voxel three inputs and four float4
// gz reads (broadcasts: the lanes of a warp share at most three voxels) feed
// 48 FMAs.  Threads 144 .. 159 sum gz per channel (the bias gradient).  At
// the end the 16 voxel groups are summed in a fixed order: one partial
// [27 x 16 + 16] per block (tap-major, then channel), summed over blocks
// afterwards.
constexpr int C1_THREADS = 160;
constexpr size_t C1_SMEM = sizeof(float) * 2 * (1000 + 512 * 16);  // dynamic: two (input, gz) buffers
__global__ void __launch_bounds__(C1_THREADS) k_conv1_wgrad(int n, const float *__restrict__ x,
                                                            const float *__restrict__ gz,
                                                            float *__restrict__ part) {
    extern __shared__ __align__(16) float c1sm[];
    float(*xs)[1000] = reinterpret_cast<float(*)[1000]>(c1sm);               // [2][1000]
    float(*gs)[512 * 16] = reinterpret_cast<float(*)[512 * 16]>(c1sm + 2000);  // [2][8192], 16-byte aligned
    const int nt = (n + 7) / 8, ntiles = nt * nt * nt;
    const int i = threadIdx.x;
    const int r = i % 9, g = i / 9;  // for i < 144; i >= 144: bias channel i - 144
    const int dz = r / 3 - 1, dy = r % 3 - 1;
    float acc[3][16];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[d][c] = 0.f;
    auto load = [&](int t, int buf) {
        const int x0 = (t % nt) * 8, y0 = ((t / nt) % nt) * 8, z0 = (t / (nt * nt)) * 8;
        for (int e = i; e < 1000; e += C1_THREADS) {
            const int qx = x0 + e % 10 - 1, qy = y0 + (e / 10) % 10 - 1, qz = z0 + e / 100 - 1;
            const bool in = qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n;
            cp_async4(&xs[buf][e], in ? x + ((size_t)qz * n + qy) * n + qx : x, in ? 4u : 0u);
        }
        for (int e = i; e < 512 * 4; e += C1_THREADS) {  // 16-byte pieces of gz (zero outside)
            const int v = e >> 2, q = e & 3;
            const int px = x0 + (v & 7), py = y0 + ((v >> 3) & 7), pz = z0 + (v >> 6);
            const bool in = px < n && py < n && pz < n;
            cp_async16(&gs[buf][4 * e], in ? gz + (((size_t)pz * n + py) * n + px) * 16 + 4 * q : gz, in ? 16u : 0u);
        }
        cp_async_commit();
    };
    int buf = 0;
    if ((int)blockIdx.x < ntiles) load(blockIdx.x, 0);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
        if (t + (int)gridDim.x < ntiles) {
            load(t + gridDim.x, buf ^ 1);
            cp_async_wait<1>();  // this tile's copies have landed
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (i < 144) {
            const float *xb = xs[buf];
#pragma unroll 2
            for (int v = g; v < 512; v += 16) {
                const int vx = v & 7, vy = (v >> 3) & 7, vz = v >> 6;
                const float *xr = xb + ((vz + 1 + dz) * 10 + vy + 1 + dy) * 10 + vx;  // dx = -1 at xr[0]
                const float x0v = xr[0], x1v = xr[1], x2v = xr[2];
                const float4 *gp = reinterpret_cast<const float4 *>(gs[buf] + v * 16);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 gk = gp[k];
                    const float gv[4] = {gk.x, gk.y, gk.z, gk.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        acc[0][4 * k + e] = fmaf(x0v, gv[e], acc[0][4 * k + e]);
                        acc[1][4 * k + e] = fmaf(x1v, gv[e], acc[1][4 * k + e]);
                        acc[2][4 * k + e] = fmaf(x2v, gv[e], acc[2][4 * k + e]);
                    }
                }
            }
        } else {
            const int c = i - 144;
#pragma unroll 8
            for (int v = 0; v < 512; ++v) acc[0][0] += gs[buf][v * 16 + c];
        }
        __syncthreads();  // buffer buf is refilled two tiles on
    }
    // per (tap, group) sums through shared memory, then the 16 groups in order
    float *red = gs[0];  // 432 x 16 floats fit in the 8,192 of a gz buffer
    if (i < 144) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int c = 0; c < 16; ++c) red[((r * 3 + d) * 16 + g) * 16 + c] = acc[d][c];
    }
    __syncthreads();
    float *out = part + (size_t)blockIdx.x * (27 * 16 + 16);
    for (int o = i; o < 432; o += C1_THREADS) {
        const int tp = o / 16, c = o % 16;
        float s = 0.f;
        for (int k = 0; k < 16; ++k) s += red[(tp * 16 + k) * 16 + c];
        out[o] = s;
    }
    if (i >= 144) out[432 + i - 144] = acc[0][0];  // the bias threads' sums
}

// head: 1x1 conv 16 -> 2, FP32 output [n^3][2]
__global__ void k_head_fwd(int n3, const bf16 *__restrict__ a, const float *__restrict__ w,
                           const float *__restrict__ b, float *__restrict__ y) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n3) return;
    float v[16];
    load16_bf16(a + (size_t)p * 16, v);
    float o0 = b[0], o1 = b[1];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        o0 = fmaf(v[c], w[c * 2 + 0], o0);
        o1 = fmaf(v[c], w[c * 2 + 1], o1);
    }
    reinterpret_cast<float2 *>(y)[p] = make_float2(o0, o1);
}

// head backward with the ReLU of the layer below: gz = (a > 0) gy W^T (BF16
// and FP32 [n^3][16]); partial dW, db per block
__global__ void k_head_bwd(int n3, const bf16 *__restrict__ a, const float *__restrict__ w,
                           const float *__restrict__ gy, bf16 *__restrict__ gz_bf, float *__restrict__ gz_f,
                           float *__restrict__ part) {
    __shared__ float s[34 * 8];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;  // 8 warps
    float loc[34];
#pragma unroll
    for (int i = 0; i < 34; ++i) loc[i] = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += gridDim.x * blockDim.x) {
        const float2 g = reinterpret_cast<const float2 *>(gy)[p];
        float v[16], gz[16];
        load16_bf16(a + (size_t)p * 16, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            gz[c] = v[c] > 0.f ? g.x * w[c * 2] + g.y * w[c * 2 + 1] : 0.f;
            loc[c * 2] = fmaf(v[c], g.x, loc[c * 2]);
            loc[c * 2 + 1] = fmaf(v[c], g.y, loc[c * 2 + 1]);
        }
        loc[32] += g.x;
        loc[33] += g.y;
        store16_bf16(gz_bf + (size_t)p * 16, gz);
        float4 *fp = reinterpret_cast<float4 *>(gz_f + (size_t)p * 16);
#pragma unroll
        for (int i = 0; i < 4; ++i) fp[i] = make_float4(gz[4 * i], gz[4 * i + 1], gz[4 * i + 2], gz[4 * i + 3]);
    }
#pragma unroll
    for (int i = 0; i < 34; ++i) {
        float v = loc[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s[i * 8 + wi] = v;
    }
    __syncthreads();
    if (threadIdx.x < 34) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += s[threadIdx.x * 8 + k];
        part[(size_t)blockIdx.x * 34 + threadIdx.x] = t;
    }
}

// 2^3 average pool, channels-last: [(2m)^3][c] -> [m^3][c]; a thread per 8 channels
__global__ void k_pool(int m, int c, const bf16 *__restrict__ in, bf16 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c8 = c / 8;
    const long long tot = (long long)m * m * m * c8;
    if (i >= tot) return;
    const int ch = (int)(i % c8) * 8;
    const long long p = i / c8;
    const int x = (int)(p % m), y = (int)((p / m) % m), z = (int)(p / ((long long)m * m));
    const int n = 2 * m;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int qx = 2 * x + (d & 1), qy = 2 * y + ((d >> 1) & 1), qz = 2 * z + (d >> 2);
        float v[8];
        load8_bf16(in + ((size_t)(qz * n + qy) * n + qx) * c + ch, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += v[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] *= 0.125f;
    store8_bf16(out + (size_t)p * c + ch, s);
}

// 2^3 nearest upsample: [m^3][c] -> [(2m)^3][c]; a thread per 8 channels
__global__ void k_up(int m, int c, const bf16 *__restrict__ in, bf16 *__restrict__ out) {
    const int n = 2 * m, c8 = c / 8;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)n * n * n * c8;
    if (i >= tot) return;
    const int ch8 = (int)(i % c8);
    const long long p = i / c8;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((long long)n * n));
    reinterpret_cast<uint4 *>(out)[i] =
        reinterpret_cast<const uint4 *>(in)[((size_t)((z / 2) * m + y / 2) * m + x / 2) * c8 + ch8];
}

// gradient through relu(z) = a (a > 0) of the pre-activation, in BF16 for the
// next tensor-core GEMM, from the FP32 sum of its incoming gradients:
//   gz = (a > 0) * (g1 + up^T(g2) + pool^T(g3) + g4)  (terms optional)
// g2: FP32 at twice the resolution (nearest-upsample adjoint: sum of the 8
// children); g3: FP32 at half the resolution (average-pool adjoint: 1/8).
// A thread per 4 channels.
__global__ void k_relu_grad(int n, int c, const bf16 *__restrict__ a, const float *__restrict__ g1,
                            const float *__restrict__ g2, const float *__restrict__ g3,
                            const float *__restrict__ g4, bf16 *__restrict__ gz_bf,
                            float *__restrict__ gz_f) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // a float4 of channels
    const int c4 = c / 4;
    const long long tot = (long long)n * n * n * c4;
    if (i >= tot) return;
    const int ch = (int)(i % c4) * 4;
    const long long p = i / c4;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((long long)n * n));
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    auto add = [&](float4 v, float k) {
        s.x = fmaf(k, v.x, s.x);
        s.y = fmaf(k, v.y, s.y);
        s.z = fmaf(k, v.z, s.z);
        s.w = fmaf(k, v.w, s.w);
    };
    if (g1) add(reinterpret_cast<const float4 *>(g1)[i], 1.f);
    if (g4) add(reinterpret_cast<const float4 *>(g4)[i], 1.f);
    if (g2) {
        const int N2 = 2 * n;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int qx = 2 * x + (d & 1), qy = 2 * y + ((d >> 1) & 1), qz = 2 * z + (d >> 2);
            add(*reinterpret_cast<const float4 *>(g2 + ((size_t)(qz * N2 + qy) * N2 + qx) * c + ch), 1.f);
        }
    }
    if (g3) {
        const int h = n / 2;
        add(*reinterpret_cast<const float4 *>(g3 + ((size_t)((z / 2) * h + y / 2) * h + x / 2) * c + ch), 0.125f);
    }
    const uint2 av = reinterpret_cast<const uint2 *>(a)[i];
    __nv_bfloat162 a01, a23;
    memcpy(&a01, &av.x, 4);
    memcpy(&a23, &av.y, 4);
    const float2 f01 = __bfloat1622float2(a01), f23 = __bfloat1622float2(a23);
    const float4 gz = make_float4(f01.x > 0.f ? s.x : 0.f, f01.y > 0.f ? s.y : 0.f, f23.x > 0.f ? s.z : 0.f,
                                  f23.y > 0.f ? s.w : 0.f);
    if (gz_bf) {
        const __nv_bfloat162 b01 = __floats2bfloat162_rn(gz.x, gz.y), b23 = __floats2bfloat162_rn(gz.z, gz.w);
        uint2 o;
        memcpy(&o.x, &b01, 4);
        memcpy(&o.y, &b23, 4);
        reinterpret_cast<uint2 *>(gz_bf)[i] = o;
    }
    if (gz_f) reinterpret_cast<float4 *>(gz_f)[i] = gz;
}

// out[i] = sum over k of part[k][i] (splits, blocks), in a fixed order: a
// block of 32 x 8 threads owns 32 consecutive i; warp j sums k = j, j + 8,
// ..., then the eight warp sums are added in order
__global__ void __launch_bounds__(256) k_reduce_parts(int splits, int len, const float *__restrict__ part,
                                                      float *__restrict__ out) {
    __shared__ float sm[8][32];
    const int i = blockIdx.x * 32 + threadIdx.x, j = threadIdx.y;
    float s = 0.f;
    if (i < len)
        for (int k = j; k < splits; k += 8) s += part[(size_t)k * len + i];
    sm[j][threadIdx.x] = s;
    __syncthreads();
    if (j == 0 && i < len) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += sm[k][threadIdx.x];
        out[i] = t;
    }
}

// bias gradient: sum of gz [P][c] over P (block partials, fixed order)
// per-block partial sums over the voxels of gz [P][c] (c a multiple of 4, at
// most 64; 256 threads): a thread reads float4s of one channel group (the
// grid stride is a multiple of c / 4), then the block sums its threads per
// channel in a fixed order; part[block][c]
__global__ void __launch_bounds__(256) k_bias_part(long long P, int c, const float *__restrict__ gz,
                                                   float *__restrict__ part) {
    __shared__ float4 s[256];
    const int c4 = c / 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long tot = P * c4;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < tot; e += (long long)gridDim.x * 256) {
        const float4 v = reinterpret_cast<const float4 *>(gz)[e];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < c4) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = threadIdx.x; k < 256; k += c4) {
            t.x += s[k].x;
            t.y += s[k].y;
            t.z += s[k].z;
            t.w += s[k].w;
        }
        reinterpret_cast<float4 *>(part + (size_t)blockIdx.x * c)[threadIdx.x] = t;
    }
}

__global__ void k_to_bf16(long long n, const float *__restrict__ in, bf16 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(in[i]);
}

// loss: mean over voxels of sum_c wt_c (y_c - t_c)^2; gy = d loss / d y
__global__ void k_mse(long long n3, const float *__restrict__ y, const float *__restrict__ t,
                      float w0, float w1, float *__restrict__ gy, float *__restrict__ part) {
    __shared__ float s[256];
    float acc = 0.f;
    const float inv = 1.0f / (float)n3;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n3;
         p += (long long)gridDim.x * blockDim.x) {
        const float d0 = y[2 * p] - t[2 * p], d1 = y[2 * p + 1] - t[2 * p + 1];
        acc += w0 * d0 * d0 + w1 * d1 * d1;
        gy[2 * p] = 2.f * w0 * d0 * inv;
        gy[2 * p + 1] = 2.f * w1 * d1 * inv;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0] * inv;
}

__global__ void k_adam_flat(long long n, float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}


// ---------------------------------------------------------------------------
// FDK-style input and Gaussian seeding
// ---------------------------------------------------------------------------
// cosine weight and ramp filter along detector rows (Ram-Lak kernel in the
// spatial domain: h(0) = 1/(4 p^2), h(odd k) = -1/(pi k p)^2, h(even) = 0,
// times the pitch): one thread per output pixel, direct convolution.
__global__ void k_fdk_filter(dgr_geom geo, float scale, const float *__restrict__ in, float *__restrict__ out) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)geo.n_views * geo.nv * geo.nu;
    if (r >= tot) return;
    const int iu = (int)(r % geo.nu);
    const long long row = r / geo.nu;
    const int iv = (int)(row % geo.nv);
    const float cu = 0.5f * (float)(geo.nu - 1), cv = 0.5f * (float)(geo.nv - 1);
    const float pu = geo.pu, pi = 3.14159265358979f;
    const float *src = in + row * geo.nu;
    const float v = ((float)iv - cv) * geo.pv;
    float acc = 0.f;
    for (int j = 0; j < geo.nu; ++j) {
        const int k = iu - j;
        float hk;
        if (k == 0) hk = 1.0f / (4.0f * pu * pu);
        else if (k & 1) hk = -1.0f / (pi * pi * (float)k * (float)k * pu * pu);
        else continue;
        float wgt = 1.f;
        if (geo.beam == DGR_CONE) {
            const float u = ((float)j - cu) * pu;
            wgt = geo.dsd * rsqrtf(geo.dsd * geo.dsd + u * u + v * v);
        }
        acc = fmaf(hk * pu, wgt * src[j], acc);
    }
    out[r] = scale * acc;
}

// proposals for seeding: density = max(src[c * i], 0); log-scale = the second
// channel (c = 2, the network's output) or a constant (c = 1, an FDK volume)
__global__ void k_proposals(long long n, const float *__restrict__ src, int c, float log_default,
                            float *__restrict__ density, float *__restrict__ log_scale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    density[i] = fmaxf(src[c * i], 0.f);
    log_scale[i] = c == 2 ? src[2 * i + 1] : log_default;
}

// per-Gaussian weight rho * mean_a log(s_a / h) (the intensity-weighted
// log-scale, voxelized to build training targets)
__global__ void k_logscale_weight(int n, const float *__restrict__ s, const float *__restrict__ rho,
                                  float inv_h, float *__restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float l = (logf(s[3 * i] * inv_h) + logf(s[3 * i + 1] * inv_h) + logf(s[3 * i + 2] * inv_h)) *
                    (1.f / 3.f);
    w[i] = rho[i] * l;
}

// training targets [n][2]: the fitted density and, where it exceeds
// min_density, the density-weighted mean log-scale clamped to [lo, hi]
// (log_default elsewhere)
__global__ void k_fit_targets(long long n, const float *__restrict__ dens, const float *__restrict__ wsum,
                              float min_density, float lo, float hi, float log_default,
                              float *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float d = dens[i];
    const float l = d > min_density ? wsum[i] / fmaxf(d, min_density) : log_default;
    out[2 * i] = d;
    out[2 * i + 1] = fminf(fmaxf(l, lo), hi);
}

// per-block sums of a non-negative field (FP64) for the sampling CDF
__global__ void k_cdf_blocks(long long n, const float *__restrict__ d, double *__restrict__ bsum) {
    __shared__ double s[256];
    const long long b0 = (long long)blockIdx.x * 4096;
    double acc = 0.0;
    for (long long i = b0 + threadIdx.x; i < min(n, b0 + 4096); i += blockDim.x) acc += fmax((double)d[i], 0.0);
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

// exclusive scan of the block sums (one thread, nb <= a few thousand)
__global__ void k_cdf_scan(int nb, double *__restrict__ bsum) {
    double run = 0.0;
    for (int i = 0; i < nb; ++i) {
        const double v = bsum[i];
        bsum[i] = run;
        run += v;
    }
    bsum[nb] = run;
}

// sample voxel k with probability d_k / sum(d): u in [0, 1) per sample;
// finds the block by binary search over block offsets, then walks the block.
// Writes mu (voxel centre + jitter in [-h/2, h/2)), isotropic s from
// exp(log-scale) in voxels (clamped to [0.3, 8]) x h, identity q, rho = d_k.
__global__ void k_seed(int n_side, float h, float ox, float oy, float oz, const float *__restrict__ d,
                       const float *__restrict__ logs, const double *__restrict__ boff, int nb,
                       int ns, const float *__restrict__ u, const float *__restrict__ jit,
                       float *__restrict__ mu, float *__restrict__ sc, float *__restrict__ q,
                       float *__restrict__ rho, int *__restrict__ vidx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const long long n3 = (long long)n_side * n_side * n_side;
    const double target = (double)u[i] * boff[nb];
    int lo = 0, hi = nb;  // boff[lo] <= target < boff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (boff[mid] <= target) lo = mid; else hi = mid;
    }
    double run = boff[lo];
    long long k = (long long)lo * 4096;
    const long long kend = min(n3, k + 4096);
    long long pick = kend - 1;
    for (; k < kend; ++k) {
        run += fmax((double)d[k], 0.0);
        if (run > target) { pick = k; break; }
    }
    const int x = (int)(pick % n_side), y = (int)((pick / n_side) % n_side),
              z = (int)(pick / ((long long)n_side * n_side));
    mu[3 * i + 0] = ox + ((float)x + 0.5f + jit[3 * i + 0]) * h;
    mu[3 * i + 1] = oy + ((float)y + 0.5f + jit[3 * i + 1]) * h;
    mu[3 * i + 2] = oz + ((float)z + 0.5f + jit[3 * i + 2]) * h;
    const float sv = fminf(fmaxf(expf(logs[pick]), 0.3f), 8.0f) * h;
    sc[3 * i] = sc[3 * i + 1] = sc[3 * i + 2] = sv;
    q[4 * i] = 1.f; q[4 * i + 1] = q[4 * i + 2] = q[4 * i + 3] = 0.f;
    rho[i] = fmaxf(d[pick], 1e-4f);
    vidx[i] = (int)pick;
}

// fixed-point refinement of the seeds' intensities: the voxelized field of
// the seeds should match the proposed density at the seed voxels
__global__ void k_seed_rescale(int ns, const int *__restrict__ vidx, const float *__restrict__ d,
                               const float *__restrict__ vol, float *__restrict__ rho) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const float target = fmaxf(d[vidx[i]], 0.f), cur = vol[vidx[i]];
    const float f = cur > 1e-6f ? target / cur : 1.f;
    rho[i] = fmaxf(rho[i] * fminf(fmaxf(f, 0.25f), 4.0f), 1e-5f);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side: parameter layout, workspace layout, forward / backward
// ---------------------------------------------------------------------------
namespace net {

struct Layer {
    int ci, co, taps;
};
constexpr Layer L[6] = {{1, 16, 27}, {16, 32, 27}, {32, 64, 27}, {64, 32, 27}, {32, 16, 27}, {16, 2, 1}};
constexpr int C1_BLOCKS = 1024;  // most blocks (partials) of the first layer's weight gradient
constexpr int BIAS_BLOCKS = 592;  // blocks (partials) of a bias gradient: 4 per SM of a 148-SM device
constexpr int HEAD_BLOCKS = 592;  // blocks (partials) of the head's backward

inline size_t w_off(int l) {
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)L[i].taps * L[i].ci * L[i].co + L[i].co;
    return o;
}
inline size_t b_off(int l) { return w_off(l) + (size_t)L[l].taps * L[l].ci * L[l].co; }
inline size_t n_params() { return w_off(6); }

struct WS {
    size_t a1, p1, a2, p2, a3, u2, a4, u1, a5;  // BF16 activations
    size_t wbf;                                  // BF16 copy of every parameter
    size_t gz5b, gz5f, gu1f, gz4b, gz4f, gu2f, gz3b, gz3f, gp2f, gz2b, gz2f, gp1f, gz1f;
    size_t part, bpart, lpart;
    size_t part_n;  // floats of the weight-gradient partial buffer
    size_t wpk;     // tcgen05 B operands: per layer 1..4, forward then data gradient
    size_t wdz;     // the same for k_conv_dz (three z offsets side by side), same offsets
    size_t status;  // device status word
    size_t total;
};

// offset (elements) of layer l's packed weights for mode (0 forward, 1 data gradient)
inline size_t wpk_off(int l, int mode) {
    size_t o = 0;
    for (int i = 1; i < l; ++i) o += 2 * (size_t)27 * L[i].ci * L[i].co;
    return o + (mode ? (size_t)27 * L[l].ci * L[l].co : 0);
}

inline WS layout(int n) {
    WS w;
    size_t o = 0;
    auto take = [&](size_t b) {
        const size_t at = o;
        o = align_up(o + b);
        return at;
    };
    const size_t n3 = (size_t)n * n * n, h3 = n3 / 8, q3 = n3 / 64;
    w.a1 = take(2 * n3 * 16);
    w.p1 = take(2 * h3 * 16);
    w.a2 = take(2 * h3 * 32);
    w.p2 = take(2 * q3 * 32);
    w.a3 = take(2 * q3 * 64);
    w.u2 = take(2 * h3 * 64);
    w.a4 = take(2 * h3 * 32);
    w.u1 = take(2 * n3 * 32);
    w.a5 = take(2 * n3 * 16);
    w.wbf = take(2 * n_params());
    w.gz5b = take(2 * n3 * 16);
    w.gz5f = take(4 * n3 * 16);
    w.gu1f = take(4 * n3 * 32);
    w.gz4b = take(2 * h3 * 32);
    w.gz4f = take(4 * h3 * 32);
    w.gu2f = take(4 * h3 * 64);
    w.gz3b = take(2 * q3 * 64);
    w.gz3f = take(4 * q3 * 64);
    w.gp2f = take(4 * q3 * 32);
    w.gz2b = take(2 * h3 * 32);
    w.gz2f = take(4 * h3 * 32);
    w.gp1f = take(4 * h3 * 16);
    w.gz1f = take(4 * n3 * 16);
    // weight-gradient partials: the largest of the tensor-core layers' split
    // partials, the first layer's block partials and the head's
    size_t pmax = 0;
    const size_t side3[5] = {n3, h3, q3, h3, n3};
    for (int l = 1; l <= 4; ++l) {
        const size_t splits = (side3[l] + WG_SPLIT - 1) / WG_SPLIT;
        const size_t v = splits * 27 * L[l].ci * L[l].co;
        pmax = v > pmax ? v : pmax;
    }
    const size_t c1 = (size_t)C1_BLOCKS * (27 * 16 + 16);
    pmax = c1 > pmax ? c1 : pmax;
    pmax = (size_t)HEAD_BLOCKS * 34 > pmax ? (size_t)HEAD_BLOCKS * 34 : pmax;
    w.part = take(4 * pmax);
    w.part_n = pmax;
    w.bpart = take(4 * (size_t)BIAS_BLOCKS * 64);
    w.lpart = take(4 * 1024);
    w.wpk = take(2 * wpk_off(5, 0));
    w.wdz = take(2 * wpk_off(5, 0));
    w.status = take(4);
    w.total = o;
    return w;
}

}  // namespace net

template <int MODE, int BN>
static void gemm(const ConvArgs &a, int grid_x, int grid_y, cudaStream_t st) {
    k_conv_gemm<MODE, BN><<<dim3(grid_x, grid_y), GEMM_THREADS, 0, st>>>(a);
    counted(1);
}

template <int MODE>
static void gemm_bn(int bn, const ConvArgs &a, int gx, int gy, cudaStream_t st) {
    if (bn <= 16) gemm<MODE, 16>(a, gx, gy, st);
    else if (bn <= 32) gemm<MODE, 32>(a, gx, gy, st);
    else gemm<MODE, 64>(a, gx, gy, st);
}

// convolution engine: 2 tcgen05 halo tiles (all three GEMMs), 1 tcgen05
// gathered tiles (forward, data gradient), 0 mma.sync
std::atomic<int> g_conv_engine{2};

template <int MODE, int BN>
static bool umma(const ConvArgs &a, long long rows, cudaStream_t st) {
    static int attr = 0;  // 1 set, -1 refused
    if (attr == 0) {
        attr = cudaFuncSetAttribute(k_conv_umma<MODE, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)umma_smem(BN)) == cudaSuccess ? 1 : -1;
        if (attr < 0) (void)cudaGetLastError();
    }
    if (attr < 0) return false;
    k_conv_umma<MODE, BN><<<(unsigned)((rows + UM - 1) / UM), 128, umma_smem(BN), st>>>(a);
    counted(1);
    return true;
}

// persistent halo-tile launch: as many CTAs as fit on the device at once
template <int MODE, int C, int N, int ZT>
static bool halo(const ConvArgs &a, cudaStream_t st) {
    using HH = Halo1<C, N, ZT>;
    static int per_sm = 0;  // resident CTAs per SM; -1 refused
    static int sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                  cudaFuncSetAttribute(k_conv_halo<MODE, C, N, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)HH::SMEM) == cudaSuccess &&
                  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_halo<MODE, C, N, ZT>, HALO_THREADS,
                                                                HH::SMEM) == cudaSuccess;
        if (!ok || per_sm < 1) {
            per_sm = -1;
            (void)cudaGetLastError();
        }
    }
    if (per_sm < 0) return false;
    const int n = a.n;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + ZT - 1) / ZT);
    const long long cap = (long long)sms * per_sm;
    k_conv_halo<MODE, C, N, ZT><<<(unsigned)(tiles < cap ? tiles : cap), HALO_THREADS, HH::SMEM, st>>>(a);
    counted(1);
    return true;
}

// persistent double-buffered halo-tile launch
template <int MODE, int C, int N, int ZT>
static bool halo2(const ConvArgs &a, cudaStream_t st) {
    using HH = Halo2<C, N, ZT>;
    static int per_sm = 0;  // resident CTAs per SM; -1 refused
    static int sms = 0;
    if (per_sm == 0) {
        int dev = 0;
        bool ok = cudaGetDevice(&dev) == cudaSuccess &&
                  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                  cudaFuncSetAttribute(k_conv_halo2<MODE, C, N, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)HH::SMEM) == cudaSuccess &&
                  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_halo2<MODE, C, N, ZT>,
                                                                HALO_THREADS, HH::SMEM) == cudaSuccess;
        if (!ok || per_sm < 1) {
            per_sm = -1;
            (void)cudaGetLastError();
        }
    }
    if (per_sm < 0) return false;
    // tensor memory: at most 512 columns per SM between the resident CTAs
    const int fit = (int)(512 / HH::NCOL);
    const int per = per_sm < fit ? per_sm : fit;
    const int n = a.n;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + ZT - 1) / ZT);
    const long long cap = (long long)sms * per;
    k_conv_halo2<MODE, C, N, ZT><<<(unsigned)(tiles < cap ? tiles : cap), HALO_THREADS, HH::SMEM, st>>>(a);
    counted(1);
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

// tensor map of BF16 activations [n][n][n][c] (channels fastest) read in
// boxes of 8 channels x bx x by x bz voxels, zero outside the grid
static bool act_tmap(CUtensorMap *tm, const bf16 *x, int n, int c, int bx, int by, int bz) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || (uintptr_t)x % 16 != 0 || c % 8 != 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)n * c * 2, (cuuint64_t)n * n * c * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(x), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// persistent k_conv_dz launch, one CTA per SM
template <int MODE, int C, int NO, int ZT, int KS, int S, int ISS>
static bool dz(const ConvArgs &a, cudaStream_t st) {
    using D = DzCfg<C, NO, ZT, KS, S, ISS>;
    static int sms = 0, attr = 0;  // attr: 1 set, -1 refused
    if (attr == 0) {
        int dev = 0;
        attr = (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaFuncSetAttribute(k_conv_dz<MODE, C, NO, ZT, KS, S, ISS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)D::SMEM) == cudaSuccess)
                   ? 1
                   : -1;
        if (attr < 0) (void)cudaGetLastError();
    }
    if (attr < 0) return false;
    CUtensorMap tm;
    if (!act_tmap(&tm, a.x, a.n, C, D::HX, D::HY, D::HZ)) return false;
    const int n = a.n;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + ZT - 1) / ZT);
    k_conv_dz<MODE, C, NO, ZT, KS, S, ISS><<<(unsigned)(tiles < sms ? tiles : sms), DZ_THREADS, D::SMEM, st>>>(tm, a);
    counted(1);
    return true;
}

template <int MODE>
static bool dz_cn(int C, int N, const ConvArgs &a, cudaStream_t st) {
    if (C == 16 && N == 32) return dz<MODE, 16, 32, 4, 1, 4, 2>(a, st);
    if (C == 32 && N == 64) return dz<MODE, 32, 64, 2, 2, 4, 2>(a, st);
    if (C == 64 && N == 32) return dz<MODE, 64, 32, 4, 4, 3, 2>(a, st);
    if (C == 32 && N == 16) return dz<MODE, 32, 16, 8, 2, 3, 2>(a, st);
    return false;
}

template <int MODE>
static bool halo_cn(int C, int N, const ConvArgs &a, cudaStream_t st) {
    if (C == 16 && N == 32) return halo2<MODE, 16, 32, 4>(a, st);
    if (C == 32 && N == 64) return halo2<MODE, 32, 64, 2>(a, st);
    if (C == 64 && N == 32) return halo<MODE, 64, 32, 2>(a, st);  // two blocks do not fit next to B
    if (C == 32 && N == 16) return halo2<MODE, 32, 16, 4>(a, st);
    return false;
}

// weight gradient on tcgen05: partials [splits][27 ci][co] into a.out;
// returns the number of splits, 0 if not launched
template <int CI, int CO, int TPG>
static int wgrad_halo(const ConvArgs &a, int max_splits, cudaStream_t st) {
    constexpr int ZT = 2;
    using WW = WgHalo<CI, CO, ZT>;
    static int sms = 0, attr = 0;
    if (attr == 0) {
        int dev = 0;
        attr = (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaFuncSetAttribute(k_wgrad_halo<CI, CO, TPG, ZT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WW::SMEM) == cudaSuccess)
                   ? 1
                   : -1;
        if (attr < 0) (void)cudaGetLastError();
    }
    if (attr < 0) return 0;
    const int n = a.n, ng = (27 + TPG - 1) / TPG;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + ZT - 1) / ZT);
    long long s = (long long)sms / ng;  // one CTA per SM (up to 512 tensor-memory columns each)
    if (s > max_splits) s = max_splits;
    if (s > tiles) s = tiles;
    if (s < 1) s = 1;
    k_wgrad_halo<CI, CO, TPG, ZT><<<(unsigned)(s * ng), HALO_THREADS, WW::SMEM, st>>>(a, (int)s);
    counted(1);
    return (int)s;
}

// weight gradient by k_wgrad_dz: partials [splits][27 ci][co] into a.out;
// returns the number of splits, 0 if not launched
template <int CI, int CO, int COG, int S>
static int wgrad_dz(const ConvArgs &a, int max_splits, cudaStream_t st) {
    using W = WzCfg<CI, CO, COG, S>;
    static int sms = 0, attr = 0;
    if (attr == 0) {
        int dev = 0;
        attr = (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaFuncSetAttribute(k_wgrad_dz<CI, CO, COG, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)W::SMEM) == cudaSuccess)
                   ? 1
                   : -1;
        if (attr < 0) (void)cudaGetLastError();
    }
    if (attr < 0) return 0;
    CUtensorMap tm;
    if (!act_tmap(&tm, a.x, a.n, CI, W::HX, W::LINES, W::ZT + 2)) return 0;
    const int n = a.n;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + W::ZT - 1) / W::ZT);
    long long s = (long long)sms / W::NG;  // one CTA per SM
    if (s > max_splits) s = max_splits;
    if (s > tiles) s = tiles;
    if (s < 1) s = 1;
    k_wgrad_dz<CI, CO, COG, S><<<(unsigned)(s * W::NG), WZ_THREADS, W::SMEM, st>>>(tm, a, (int)s);
    counted(1);
    return (int)s;
}

template <int CI, int CO, int S>
static int wgrad_dzt(const ConvArgs &a, int max_splits, cudaStream_t st) {
    using W = WtCfg<CI, CO, S>;
    static int sms = 0, attr = 0;
    if (attr == 0) {
        int dev = 0;
        attr = (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                cudaFuncSetAttribute(k_wgrad_dzt<CI, CO, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)W::SMEM) == cudaSuccess)
                   ? 1
                   : -1;
        if (attr < 0) (void)cudaGetLastError();
    }
    if (attr < 0) return 0;
    CUtensorMap tm;
    if (!act_tmap(&tm, a.x, a.n, CI, W::HX, W::LINES, W::ZT + 2)) return 0;
    const int n = a.n;
    const long long tiles = (long long)((n + 7) / 8) * ((n + 15) / 16) * ((n + W::ZT - 1) / W::ZT);
    long long s = sms;  // one CTA per SM
    if (s > max_splits) s = max_splits;
    if (s > tiles) s = tiles;
    if (s < 1) s = 1;
    k_wgrad_dzt<CI, CO, S><<<(unsigned)s, WZ_THREADS, W::SMEM, st>>>(tm, a, (int)s);
    counted(1);
    return (int)s;
}

static int wgrad_dz_cn(const ConvArgs &a, int max_splits, cudaStream_t st) {
    if (a.ci == 32 && a.co == 16) return wgrad_dz<32, 16, 16, 4>(a, max_splits, st);
    if (a.ci == 64 && a.co == 32) return wgrad_dz<64, 32, 16, 2>(a, max_splits, st);
    if (a.ci == 32 && a.co == 64) return wgrad_dz<32, 64, 32, 3>(a, max_splits, st);
    if (a.ci == 16 && a.co == 32) return wgrad_dzt<16, 32, 4>(a, max_splits, st);
    return 0;
}

static int wgrad_halo_cn(const ConvArgs &a, int max_splits, cudaStream_t st) {
    if (a.ci == 16 && a.co == 32) return wgrad_halo<16, 32, 27>(a, max_splits, st);
    if (a.ci == 32 && a.co == 64) return wgrad_halo<32, 64, 14>(a, max_splits, st);
    if (a.ci == 64 && a.co == 32) return wgrad_halo<64, 32, 7>(a, max_splits, st);
    if (a.ci == 32 && a.co == 16) return wgrad_halo<32, 16, 14>(a, max_splits, st);
    return 0;
}

// forward / data-gradient convolution: tcgen05 when selected and the shapes
// fit it (halo tiles: the four layer shapes; gathered tiles: N in {16, 32,
// 64}, C a multiple of 8; 16-byte aligned operands), else mma.sync
template <int MODE>
// Returns whether the output went out in the form a.up_adj asks for (only
// k_conv_dz sums a data gradient over the children of an upsampling; the
// other engines write every voxel).
static bool conv_gemm(ConvArgs a, long long rows, cudaStream_t st) {
    const int N = MODE == MODE_FWD ? a.co : a.ci, C = MODE == MODE_FWD ? a.ci : a.co;
    const bool aligned = ((uintptr_t)a.x | (uintptr_t)a.wt | (uintptr_t)a.wdz | (uintptr_t)a.skip |
                          (uintptr_t)(MODE == MODE_FWD ? (void *)a.y : (void *)a.out)) % 16 == 0;
    const int engine = g_conv_engine.load();
    if (MODE == MODE_FWD || a.n % 2 != 0) a.up_adj = 0;
    if (engine == 2 && a.wdz && aligned && dz_cn<MODE>(C, N, a, st)) return true;
    const bool want = a.up_adj != 0;
    a.up_adj = 0;
    if (engine == 3 && a.wt && aligned && halo_cn<MODE>(C, N, a, st)) return !want;
    if (engine >= 1 && a.wt && C % 8 == 0 && aligned && (N == 16 || N == 32 || N == 64)) {
        bool done = N == 16 ? umma<MODE, 16>(a, rows, st)
                            : N == 32 ? umma<MODE, 32>(a, rows, st) : umma<MODE, 64>(a, rows, st);
        if (done) return !want;
    }
    gemm_bn<MODE>(N, a, (int)((rows + GM - 1) / GM), 1, st);
    return !want;
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

static void reduce_parts(int splits, int len, const float *part, float *out, cudaStream_t st) {
    k_reduce_parts<<<nblk(len, 32), dim3(32, 8), 0, st>>>(splits, len, part, out);
}

}  // namespace dgr

using namespace dgr;

static bool net_side_ok(int n) { return n >= 4 && n % 4 == 0 && n <= 256; }

extern "C" {

long long dgr_net_param_count(void) { return (long long)net::n_params(); }

int dgr_net_ws_bytes(int n, size_t *bytes) {
    if (!net_side_ok(n) || !bytes) return DGR_ERR_ARG;
    *bytes = net::layout(n).total;
    return DGR_OK;
}

int dgr_net_forward(int n, const float *params, const float *input, float *output, void *ws,
                    size_t ws_bytes, cudaStream_t st) {
    if (!net_side_ok(n) || !params || !input || !output || !ws) return DGR_ERR_ARG;
    const net::WS W = net::layout(n);
    if (ws_bytes < W.total) return DGR_ERR_WS_TOO_SMALL;
    char *base = static_cast<char *>(ws);
    auto B = [&](size_t off) { return reinterpret_cast<bf16 *>(base + off); };
    const int h = n / 2, q = n / 4;
    const long long n3 = (long long)n * n * n, h3 = n3 / 8, q3 = n3 / 64;
    bf16 *wbf = B(W.wbf);
    const long long np = (long long)net::n_params();
    k_to_bf16<<<nblk(np, 256), 256, 0, st>>>(np, params, wbf);
    int *status = reinterpret_cast<int *>(base + W.status);
    cudaMemsetAsync(status, 0, sizeof(int), st);
    bf16 *wpk = B(W.wpk), *wdz = B(W.wdz);
    for (int l = 1; l <= 4; ++l) {
        for (int mode = 0; mode < 2; ++mode)
            k_wpack<<<nblk(27 * net::L[l].ci * net::L[l].co, 256), 256, 0, st>>>(
                mode, net::L[l].ci, net::L[l].co, wbf + net::w_off(l), wpk + net::wpk_off(l, mode));
        k_wpack_dz<<<dim3(nblk(27 * net::L[l].ci * net::L[l].co, 256), 2), 256, 0, st>>>(
            net::L[l].ci, net::L[l].co, wbf + net::w_off(l), wdz + net::wpk_off(l, 0), wdz + net::wpk_off(l, 1));
    }
    counted(12);
    k_conv1_fwd<<<nblk((long long)((n + C1_VX - 1) / C1_VX) * n * n, 128), 128, 0, st>>>(n, input, params + net::w_off(0),
                                                params + net::b_off(0), B(W.a1));
    k_pool<<<nblk(h3 * 2, 256), 256, 0, st>>>(h, 16, B(W.a1), B(W.p1));
    counted(3);
    auto conv = [&](int l, int side, const bf16 *x, const bf16 *skip, bf16 *y) {
        ConvArgs a{};
        a.n = side; a.ci = net::L[l].ci; a.co = net::L[l].co;
        a.x = x; a.w = wbf + net::w_off(l); a.bias = params + net::b_off(l); a.skip = skip; a.y = y;
        a.wt = wpk + net::wpk_off(l, 0); a.wdz = wdz + net::wpk_off(l, 0); a.status = status;
        conv_gemm<MODE_FWD>(a, (long long)side * side * side, st);
    };
    conv(1, h, B(W.p1), nullptr, B(W.a2));
    k_pool<<<nblk(q3 * 4, 256), 256, 0, st>>>(q, 32, B(W.a2), B(W.p2));
    conv(2, q, B(W.p2), nullptr, B(W.a3));
    k_up<<<nblk(h3 * 8, 256), 256, 0, st>>>(q, 64, B(W.a3), B(W.u2));
    conv(3, h, B(W.u2), B(W.a2), B(W.a4));
    k_up<<<nblk(n3 * 4, 256), 256, 0, st>>>(h, 32, B(W.a4), B(W.u1));
    conv(4, n, B(W.u1), B(W.a1), B(W.a5));
    k_head_fwd<<<nblk(n3, 256), 256, 0, st>>>((int)n3, B(W.a5), params + net::w_off(5),
                                               params + net::b_off(5), output);
    counted(4);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_net_backward(int n, const float *params, const float *input, const float *grad_output,
                     float *grad_params, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (!net_side_ok(n) || !params || !input || !grad_output || !grad_params || !ws)
        return DGR_ERR_ARG;
    const net::WS W = net::layout(n);
    if (ws_bytes < W.total) return DGR_ERR_WS_TOO_SMALL;
    char *base = static_cast<char *>(ws);
    auto B = [&](size_t off) { return reinterpret_cast<bf16 *>(base + off); };
    auto F = [&](size_t off) { return reinterpret_cast<float *>(base + off); };
    const int h = n / 2, q = n / 4;
    const long long n3 = (long long)n * n * n, h3 = n3 / 8, q3 = n3 / 64;
    const bf16 *wbf = B(W.wbf);
    float *part = F(W.part), *bpart = F(W.bpart);
    // head: dW6, db6 and the pre-activation gradient of layer 5, (a5 > 0) dL/da5
    k_head_bwd<<<net::HEAD_BLOCKS, 256, 0, st>>>((int)n3, B(W.a5), params + net::w_off(5), grad_output,
                                                B(W.gz5b), F(W.gz5f), part);
    reduce_parts(net::HEAD_BLOCKS, 34, part, grad_params + net::w_off(5), st);
    counted(2);
    // the packed weights and the status word come from the forward pass on this workspace
    const bf16 *wpk = B(W.wpk), *wdz = B(W.wdz);
    int *status = reinterpret_cast<int *>(base + W.status);
    // weight and bias gradients of tensor-core layer l (input x at side^3)
    auto wgrad = [&](int l, int side, const bf16 *x, const bf16 *gz_b, const float *gz_f) {
        const int ci = net::L[l].ci, co = net::L[l].co;
        const long long s3 = (long long)side * side * side;
        ConvArgs a{};
        a.n = side; a.ci = ci; a.co = co; a.x = x; a.g = gz_b; a.out = part;
        const int max_splits = (int)nblk(s3, WG_SPLIT);  // mma.sync: splits of WG_SPLIT voxels
        // tcgen05: as many splits as the partial buffer holds (the launch
        // takes at most one per SM and tile)
        const long long cap = (long long)(W.part_n / ((size_t)27 * ci * co));
        const int tc_splits = (int)(cap < 4096 ? cap : 4096);
        const int engine = g_conv_engine.load();
        const bool aligned = ((uintptr_t)a.x | (uintptr_t)a.g) % 16 == 0;
        int splits = 0;
        if (engine >= 2 && aligned) {
            a.status = status;
            if (engine == 2) splits = wgrad_dz_cn(a, tc_splits, st);
            if (splits == 0) splits = wgrad_halo_cn(a, engine == 2 ? tc_splits : max_splits, st);
        }
        if (splits == 0) {
            splits = max_splits;
            gemm_bn<MODE_WGRAD>(co, a, (int)nblk(27 * ci, GM), splits, st);
        }
        reduce_parts(splits, 27 * ci * co, part, grad_params + net::w_off(l), st);
        k_bias_part<<<net::BIAS_BLOCKS, 256, 0, st>>>(s3, co, gz_f, bpart);
        reduce_parts(net::BIAS_BLOCKS, co, bpart, grad_params + net::b_off(l), st);
        counted(3);
    };
    // data gradient of layer l into gx; with up_adj, asks for it summed over
    // the 2^3 children of the upsampling that fed layer l (half resolution);
    // returns whether it came in that form (else every voxel, full resolution)
    auto dgrad = [&](int l, int side, const bf16 *gz_b, float *gx, bool up_adj) {
        ConvArgs d{};
        d.n = side; d.ci = net::L[l].ci; d.co = net::L[l].co; d.x = gz_b; d.w = wbf + net::w_off(l);
        d.out = gx; d.wt = wpk + net::wpk_off(l, 1); d.wdz = wdz + net::wpk_off(l, 1); d.status = status;
        d.up_adj = up_adj ? 1 : 0;
        return conv_gemm<MODE_DGRAD>(d, (long long)side * side * side, st) && up_adj;
    };
    // layer 5: a5 = relu(conv(u1) + b5 + a1); its pre-activation gradient came with the head's
    wgrad(4, n, B(W.u1), B(W.gz5b), F(W.gz5f));
    const bool up4 = dgrad(4, n, B(W.gz5b), F(W.gu1f), true);
    // layer 4: a4 = relu(conv(up(a3)) + b4 + a2); its gradient is up^T(gu1)
    k_relu_grad<<<nblk(h3 * 8, 256), 256, 0, st>>>(h, 32, B(W.a4), up4 ? F(W.gu1f) : nullptr,
                                                   up4 ? nullptr : F(W.gu1f), nullptr, nullptr, B(W.gz4b),
                                                   F(W.gz4f));
    counted(1);
    wgrad(3, h, B(W.u2), B(W.gz4b), F(W.gz4f));
    const bool up3 = dgrad(3, h, B(W.gz4b), F(W.gu2f), true);
    // layer 3: a3 = relu(conv(pool(a2)) + b3); gradient up^T(gu2)
    k_relu_grad<<<nblk(q3 * 16, 256), 256, 0, st>>>(q, 64, B(W.a3), up3 ? F(W.gu2f) : nullptr,
                                                   up3 ? nullptr : F(W.gu2f), nullptr, nullptr, B(W.gz3b),
                                                   F(W.gz3f));
    counted(1);
    wgrad(2, q, B(W.p2), B(W.gz3b), F(W.gz3f));
    dgrad(2, q, B(W.gz3b), F(W.gp2f), false);
    // layer 2: a2 = relu(conv(pool(a1)) + b2); gradient: skip of layer 4 + pool^T(gp2)
    k_relu_grad<<<nblk(h3 * 8, 256), 256, 0, st>>>(h, 32, B(W.a2), F(W.gz4f), nullptr, F(W.gp2f),
                                                   nullptr, B(W.gz2b), F(W.gz2f));
    counted(1);
    wgrad(1, h, B(W.p1), B(W.gz2b), F(W.gz2f));
    dgrad(1, h, B(W.gz2b), F(W.gp1f), false);
    // layer 1: a1 = relu(conv(x) + b1); gradient: skip of layer 5 + pool^T(gp1)
    k_relu_grad<<<nblk(n3 * 4, 256), 256, 0, st>>>(n, 16, B(W.a1), F(W.gz5f), nullptr, F(W.gp1f),
                                                   nullptr, nullptr, F(W.gz1f));
    // three resident blocks per SM, each walking many tiles (its copies
    // double-buffered); blocks = partials
    static int c1_sms = 0;
    if (c1_sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&c1_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            c1_sms = 148;
    }
    const unsigned c1t = (unsigned)(((n + 7) / 8) * ((n + 7) / 8) * ((n + 7) / 8));
    unsigned c1b = (unsigned)(3 * c1_sms);
    if (c1b > (unsigned)net::C1_BLOCKS) c1b = (unsigned)net::C1_BLOCKS;
    if (c1b > c1t) c1b = c1t;
    static const bool c1_attr =
        cudaFuncSetAttribute(k_conv1_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C1_SMEM) == cudaSuccess;
    if (!c1_attr) return DGR_ERR_CUDA;
    k_conv1_wgrad<<<c1b, C1_THREADS, C1_SMEM, st>>>(n, input, F(W.gz1f), part);
    reduce_parts((int)c1b, 27 * 16 + 16, part, grad_params + net::w_off(0), st);
    counted(3);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

// loss = mean over voxels of w0 (y0 - t0)^2 + w1 (y1 - t1)^2 and its gradient
int dgr_net_loss(int n, const float *output, const float *target, float w_density, float w_scale,
                 float *grad_output, float *loss, void *ws, size_t ws_bytes, cudaStream_t st) {
    if (!net_side_ok(n) || !output || !target || !grad_output || !loss || !ws) return DGR_ERR_ARG;
    const net::WS W = net::layout(n);
    if (ws_bytes < W.total) return DGR_ERR_WS_TOO_SMALL;
    float *lp = reinterpret_cast<float *>(static_cast<char *>(ws) + W.lpart);
    const long long n3 = (long long)n * n * n;
    k_mse<<<256, 256, 0, st>>>(n3, output, target, w_density, w_scale, grad_output, lp);
    reduce_parts(256, 1, lp, loss, st);
    counted(2);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_set_conv_engine(int engine) {
    if (engine < 0 || engine > 3) return DGR_ERR_ARG;
    g_conv_engine.store(engine);
    return DGR_OK;
}

int dgr_net_status(int n, const void *ws, size_t ws_bytes, int *status) {
    if (!net_side_ok(n) || !ws || !status) return DGR_ERR_ARG;
    const net::WS W = net::layout(n);
    if (ws_bytes < W.total) return DGR_ERR_WS_TOO_SMALL;
    return cudaMemcpy(status, static_cast<const char *>(ws) + W.status, sizeof(int), cudaMemcpyDeviceToHost) ==
                   cudaSuccess
               ? DGR_OK
               : DGR_ERR_CUDA;
}

int dgr_adam_flat(long long n, float *params, const float *grads, float *m, float *v, int t,
                  float lr, float beta1, float beta2, float eps, cudaStream_t st) {
    if (n < 0 || t < 1 || !(lr > 0.f) || (n > 0 && (!params || !grads || !m || !v))) return DGR_ERR_ARG;
    if (n == 0) return DGR_OK;
    const float bc1 = 1.f - powf(beta1, (float)t), bc2 = 1.f - powf(beta2, (float)t);
    k_adam_flat<<<nblk(n, 256), 256, 0, st>>>(n, params, grads, m, v, lr, beta1, beta2, eps, bc1, bc2);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_fdk_filter(const dgr_geom *geom, float scale, const float *sino, float *out, cudaStream_t st) {
    if (!geom || !sino || !out || geom->n_views <= 0 || geom->nu <= 0 || geom->nv <= 0 || !isfinite(scale))
        return DGR_ERR_ARG;
    if (geom->beam != DGR_PARALLEL && geom->beam != DGR_CONE) return DGR_ERR_ARG;
    const long long tot = (long long)geom->n_views * geom->nv * geom->nu;
    k_fdk_filter<<<nblk(tot, 128), 128, 0, st>>>(*geom, scale, sino, out);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_proposals(long long n_vox, const float *src, int channels, float log_scale_default,
                  float *density, float *log_scale, cudaStream_t st) {
    if (n_vox < 0 || (channels != 1 && channels != 2) || !isfinite(log_scale_default) ||
        (n_vox > 0 && (!src || !density || !log_scale)))
        return DGR_ERR_ARG;
    if (n_vox == 0) return DGR_OK;
    k_proposals<<<nblk(n_vox, 256), 256, 0, st>>>(n_vox, src, channels, log_scale_default, density, log_scale);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_logscale_weight(int n, const float *s, const float *rho, float h, float *w, cudaStream_t st) {
    if (n < 0 || !(h > 0.f) || (n > 0 && (!s || !rho || !w))) return DGR_ERR_ARG;
    if (n == 0) return DGR_OK;
    k_logscale_weight<<<nblk(n, 256), 256, 0, st>>>(n, s, rho, 1.f / h, w);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_fit_targets(long long n_vox, const float *density, const float *wsum, float min_density,
                    float log_lo, float log_hi, float log_default, float *out, cudaStream_t st) {
    if (n_vox < 0 || !(min_density > 0.f) || !(log_lo <= log_hi) || !isfinite(log_default) ||
        (n_vox > 0 && (!density || !wsum || !out)))
        return DGR_ERR_ARG;
    if (n_vox == 0) return DGR_OK;
    k_fit_targets<<<nblk(n_vox, 256), 256, 0, st>>>(n_vox, density, wsum, min_density, log_lo, log_hi,
                                                    log_default, out);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

// scratch: doubles of (n^3 / 4096 + 2)
int dgr_seed_bytes(int n_side, size_t *bytes) {
    if (n_side <= 0 || !bytes) return DGR_ERR_ARG;
    const long long n3 = (long long)n_side * n_side * n_side;
    *bytes = 8 * (size_t)((n3 + 4095) / 4096 + 2);
    return DGR_OK;
}

int dgr_seed(const dgr_grid *grid, const float *density, const float *log_scale, int ns,
             const float *u, const float *jitter, float *mu, float *s, float *q, float *rho,
             int *voxel, void *scratch, size_t scratch_bytes, cudaStream_t st) {
    if (!grid || grid->nx <= 0 || grid->nx != grid->ny || grid->nx != grid->nz || grid->z0 != 0 || ns < 0)
        return DGR_ERR_ARG;
    if (ns > 0 && (!density || !log_scale || !u || !jitter || !mu || !s || !q || !rho || !voxel || !scratch))
        return DGR_ERR_ARG;
    const long long n3 = (long long)grid->nx * grid->nx * grid->nx;
    const int nb = (int)((n3 + 4095) / 4096);
    if (scratch_bytes < 8 * (size_t)(nb + 2)) return DGR_ERR_WS_TOO_SMALL;
    if (ns == 0) return DGR_OK;
    double *boff = static_cast<double *>(scratch);
    k_cdf_blocks<<<nb, 256, 0, st>>>(n3, density, boff);
    k_cdf_scan<<<1, 1, 0, st>>>(nb, boff);
    k_seed<<<nblk(ns, 128), 128, 0, st>>>(grid->nx, grid->h, grid->ox, grid->oy, grid->oz, density,
                                           log_scale, boff, nb, ns, u, jitter, mu, s, q, rho, voxel);
    counted(3);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_seed_rescale(int ns, const int *voxel, const float *density, const float *vol, float *rho,
                     cudaStream_t st) {
    if (ns < 0 || (ns > 0 && (!voxel || !density || !vol || !rho))) return DGR_ERR_ARG;
    if (ns == 0) return DGR_OK;
    k_seed_rescale<<<nblk(ns, 128), 128, 0, st>>>(ns, voxel, density, vol, rho);
    counted(1);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

}  // extern "C"
