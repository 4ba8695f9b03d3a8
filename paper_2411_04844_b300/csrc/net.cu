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
// By default all three run on tcgen05 over halo blocks (k_conv_halo,
// k_wgrad_halo); dgr_set_conv_engine selects gathered 128-row tcgen05 tiles
// for forward and data gradient (k_conv_umma) or mma.sync m16n8k16
// (k_conv_gemm, also the weight gradient of the other two engines).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

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
    int *status;      // device status word (bounded waits)
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
// first layer: 1 -> 16 channels, input FP32
__global__ void k_conv1_fwd(int n, const float *__restrict__ x, const float *__restrict__ w,
                            const float *__restrict__ b, bf16 *__restrict__ y) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int n3 = n * n * n;
    if (p >= n3) return;
    const int px = p % n, py = (p / n) % n, pz = p / (n * n);
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = b[c];
    for (int tap = 0; tap < 27; ++tap) {
        int dx, dy, dz;
        tap_offset(tap, dx, dy, dz);
        const int qx = px + dx, qy = py + dy, qz = pz + dz;
        if (qx < 0 || qx >= n || qy < 0 || qy >= n || qz < 0 || qz >= n) continue;
        const float v = x[(qz * n + qy) * n + qx];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = fmaf(v, w[tap * 16 + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) y[(size_t)p * 16 + c] = __float2bfloat16(fmaxf(acc[c], 0.f));
}

// weight gradient of the first layer: a block walks 8^3 voxel tiles (tile
// b, b + gridDim.x, ...) with the input block (10^3, zero outside) and the
// tile's gz [512][16] in shared memory; thread i < 432 owns (tap, c) = (i / 16,
// i % 16), threads 432 .. 447 the bias sums; one partial per block, summed
// in a fixed order afterwards
constexpr int C1_THREADS = 448;
__global__ void __launch_bounds__(C1_THREADS) k_conv1_wgrad(int n, const float *__restrict__ x,
                                                            const float *__restrict__ gz,
                                                            float *__restrict__ part) {
    __shared__ float xs[10 * 10 * 10];
    __shared__ __align__(16) float gs[512 * 16];
    const int nt = (n + 7) / 8, ntiles = nt * nt * nt;
    const int i = threadIdx.x;
    int tap = 0, c = 0, dx = 0, dy = 0, dz = 0;
    if (i < 432) {
        tap = i / 16;
        c = i % 16;
        tap_offset(tap, dx, dy, dz);
    } else {
        c = i - 432;
    }
    float acc = 0.f;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int x0 = (t % nt) * 8, y0 = ((t / nt) % nt) * 8, z0 = (t / (nt * nt)) * 8;
        __syncthreads();
        for (int e = i; e < 1000; e += C1_THREADS) {
            const int qx = x0 + e % 10 - 1, qy = y0 + (e / 10) % 10 - 1, qz = z0 + e / 100 - 1;
            xs[e] = (qx >= 0 && qx < n && qy >= 0 && qy < n && qz >= 0 && qz < n) ? x[((size_t)qz * n + qy) * n + qx]
                                                                                   : 0.f;
        }
        for (int e = i; e < 512 * 4; e += C1_THREADS) {  // float4 of gz (zero outside)
            const int v = e >> 2, q = e & 3;
            const int px = x0 + (v & 7), py = y0 + ((v >> 3) & 7), pz = z0 + (v >> 6);
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (px < n && py < n && pz < n)
                g = reinterpret_cast<const float4 *>(gz + (((size_t)pz * n + py) * n + px) * 16)[q];
            reinterpret_cast<float4 *>(gs)[e] = g;
        }
        __syncthreads();
        if (i < 432) {
            for (int v = 0; v < 512; ++v) {
                const int vx = v & 7, vy = (v >> 3) & 7, vz = v >> 6;
                acc = fmaf(xs[((vz + 1 + dz) * 10 + vy + 1 + dy) * 10 + vx + 1 + dx], gs[v * 16 + c], acc);
            }
        } else {
            for (int v = 0; v < 512; ++v) acc += gs[v * 16 + c];
        }
    }
    part[(size_t)blockIdx.x * (27 * 16 + 16) + i] = acc;
}

// head: 1x1 conv 16 -> 2, FP32 output [n^3][2]
__global__ void k_head_fwd(int n3, const bf16 *__restrict__ a, const float *__restrict__ w,
                           const float *__restrict__ b, float *__restrict__ y) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n3) return;
    float o0 = b[0], o1 = b[1];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const float v = __bfloat162float(a[(size_t)p * 16 + c]);
        o0 = fmaf(v, w[c * 2 + 0], o0);
        o1 = fmaf(v, w[c * 2 + 1], o1);
    }
    y[(size_t)p * 2] = o0;
    y[(size_t)p * 2 + 1] = o1;
}

// head backward: da = gy W^T (FP32 [n^3][16]); partial dW, db per block
__global__ void k_head_bwd(int n3, const bf16 *__restrict__ a, const float *__restrict__ w,
                           const float *__restrict__ gy, float *__restrict__ da,
                           float *__restrict__ part) {
    __shared__ float s[34 * 8];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;  // 8 warps
    float loc[34];
#pragma unroll
    for (int i = 0; i < 34; ++i) loc[i] = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n3; p += gridDim.x * blockDim.x) {
        const float g0 = gy[(size_t)p * 2], g1 = gy[(size_t)p * 2 + 1];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float v = __bfloat162float(a[(size_t)p * 16 + c]);
            da[(size_t)p * 16 + c] = g0 * w[c * 2] + g1 * w[c * 2 + 1];
            loc[c * 2] = fmaf(v, g0, loc[c * 2]);
            loc[c * 2 + 1] = fmaf(v, g1, loc[c * 2 + 1]);
        }
        loc[32] += g0;
        loc[33] += g1;
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

// 2^3 average pool, channels-last: [(2m)^3][c] -> [m^3][c]
__global__ void k_pool(int m, int c, const bf16 *__restrict__ in, bf16 *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)m * m * m * c;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long p = i / c;
    const int x = (int)(p % m), y = (int)((p / m) % m), z = (int)(p / ((long long)m * m));
    const int n = 2 * m;
    float s = 0.f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int qx = 2 * x + (d & 1), qy = 2 * y + ((d >> 1) & 1), qz = 2 * z + (d >> 2);
        s += __bfloat162float(in[((size_t)(qz * n + qy) * n + qx) * c + ch]);
    }
    out[i] = __float2bfloat16(0.125f * s);
}

// 2^3 nearest upsample: [m^3][c] -> [(2m)^3][c]
__global__ void k_up(int m, int c, const bf16 *__restrict__ in, bf16 *__restrict__ out) {
    const int n = 2 * m;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)n * n * n * c;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long p = i / c;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((long long)n * n));
    out[i] = in[((size_t)((z / 2) * m + y / 2) * m + x / 2) * c + ch];
}

// gradient through relu(z) = a (a > 0) of the pre-activation, in BF16 for the
// next tensor-core GEMM, from the FP32 sum of its incoming gradients:
//   gz = (a > 0) * (g1 + up^T(g2) + pool^T(g3) + g4)  (terms optional)
// g2: FP32 at twice the resolution (nearest-upsample adjoint: sum of the 8
// children); g3: FP32 at half the resolution (average-pool adjoint: 1/8).
__global__ void k_relu_grad(int n, int c, const bf16 *__restrict__ a, const float *__restrict__ g1,
                            const float *__restrict__ g2, const float *__restrict__ g3,
                            const float *__restrict__ g4, bf16 *__restrict__ gz_bf,
                            float *__restrict__ gz_f) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)n * n * n * c;
    if (i >= tot) return;
    const int ch = (int)(i % c);
    const long long p = i / c;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((long long)n * n));
    float s = 0.f;
    if (g1) s += g1[i];
    if (g4) s += g4[i];
    if (g2) {
        const int N2 = 2 * n;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int qx = 2 * x + (d & 1), qy = 2 * y + ((d >> 1) & 1), qz = 2 * z + (d >> 2);
            s += g2[((size_t)(qz * N2 + qy) * N2 + qx) * c + ch];
        }
    }
    if (g3) {
        const int h = n / 2;
        s += 0.125f * g3[((size_t)((z / 2) * h + y / 2) * h + x / 2) * c + ch];
    }
    const float gz = __bfloat162float(a[i]) > 0.f ? s : 0.f;
    if (gz_bf) gz_bf[i] = __float2bfloat16(gz);
    if (gz_f) gz_f[i] = gz;
}

// sum over splits (fixed order) and, for biases, over the output positions
__global__ void k_reduce_parts(int splits, int len, const float *__restrict__ part,
                               float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * len + i];
    out[i] = s;
}

// bias gradient: sum of gz [P][c] over P (block partials, fixed order)
__global__ void k_bias_part(long long P, int c, const float *__restrict__ gz, float *__restrict__ part) {
    __shared__ float s[256];
    const int ch = blockIdx.y;
    float acc = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x)
        acc += gz[p * c + ch];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * gridDim.y + ch] = s[0];
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
    size_t ga5f, gz5b, gz5f, gu1f, gz4b, gz4f, gu2f, gz3b, gz3f, gp2f, gz2b, gz2f, gp1f, gz1f;
    size_t part, bpart, lpart;
    size_t wpk;     // tcgen05 B operands: per layer 1..4, forward then data gradient
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
    w.ga5f = take(4 * n3 * 16);
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
    pmax = (size_t)256 * 34 > pmax ? (size_t)256 * 34 : pmax;
    w.part = take(4 * pmax);
    w.bpart = take(4 * 64 * 64);
    w.lpart = take(4 * 1024);
    w.wpk = take(2 * wpk_off(5, 0));
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
static void conv_gemm(const ConvArgs &a, long long rows, cudaStream_t st) {
    const int N = MODE == MODE_FWD ? a.co : a.ci, C = MODE == MODE_FWD ? a.ci : a.co;
    const bool aligned = ((uintptr_t)a.x | (uintptr_t)a.wt | (uintptr_t)a.skip |
                          (uintptr_t)(MODE == MODE_FWD ? (void *)a.y : (void *)a.out)) % 16 == 0;
    const int engine = g_conv_engine.load();
    if (engine == 2 && a.wt && aligned && halo_cn<MODE>(C, N, a, st)) return;
    if (engine >= 1 && a.wt && C % 8 == 0 && aligned && (N == 16 || N == 32 || N == 64)) {
        bool done = N == 16 ? umma<MODE, 16>(a, rows, st)
                            : N == 32 ? umma<MODE, 32>(a, rows, st) : umma<MODE, 64>(a, rows, st);
        if (done) return;
    }
    gemm_bn<MODE>(N, a, (int)((rows + GM - 1) / GM), 1, st);
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

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
    bf16 *wpk = B(W.wpk);
    for (int l = 1; l <= 4; ++l)
        for (int mode = 0; mode < 2; ++mode)
            k_wpack<<<nblk(27 * net::L[l].ci * net::L[l].co, 256), 256, 0, st>>>(
                mode, net::L[l].ci, net::L[l].co, wbf + net::w_off(l), wpk + net::wpk_off(l, mode));
    counted(8);
    k_conv1_fwd<<<nblk(n3, 128), 128, 0, st>>>(n, input, params + net::w_off(0),
                                                params + net::b_off(0), B(W.a1));
    k_pool<<<nblk(h3 * 16, 256), 256, 0, st>>>(h, 16, B(W.a1), B(W.p1));
    counted(3);
    auto conv = [&](int l, int side, const bf16 *x, const bf16 *skip, bf16 *y) {
        ConvArgs a{};
        a.n = side; a.ci = net::L[l].ci; a.co = net::L[l].co;
        a.x = x; a.w = wbf + net::w_off(l); a.bias = params + net::b_off(l); a.skip = skip; a.y = y;
        a.wt = wpk + net::wpk_off(l, 0); a.status = status;
        conv_gemm<MODE_FWD>(a, (long long)side * side * side, st);
    };
    conv(1, h, B(W.p1), nullptr, B(W.a2));
    k_pool<<<nblk(q3 * 32, 256), 256, 0, st>>>(q, 32, B(W.a2), B(W.p2));
    conv(2, q, B(W.p2), nullptr, B(W.a3));
    k_up<<<nblk(h3 * 64, 256), 256, 0, st>>>(q, 64, B(W.a3), B(W.u2));
    conv(3, h, B(W.u2), B(W.a2), B(W.a4));
    k_up<<<nblk(n3 * 32, 256), 256, 0, st>>>(h, 32, B(W.a4), B(W.u1));
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
    // head: dL/da5, dW6, db6
    k_head_bwd<<<256, 256, 0, st>>>((int)n3, B(W.a5), params + net::w_off(5), grad_output,
                                    F(W.ga5f), part);
    k_reduce_parts<<<1, 64, 0, st>>>(256, 34, part, grad_params + net::w_off(5));
    counted(2);
    // the packed weights and the status word come from the forward pass on this workspace
    const bf16 *wpk = B(W.wpk);
    int *status = reinterpret_cast<int *>(base + W.status);
    // weight and bias gradients of tensor-core layer l (input x at side^3)
    auto wgrad = [&](int l, int side, const bf16 *x, const bf16 *gz_b, const float *gz_f) {
        const int ci = net::L[l].ci, co = net::L[l].co;
        const long long s3 = (long long)side * side * side;
        ConvArgs a{};
        a.n = side; a.ci = ci; a.co = co; a.x = x; a.g = gz_b; a.out = part;
        const int max_splits = (int)nblk(s3, WG_SPLIT);  // the partial buffer's capacity
        const int engine = g_conv_engine.load();
        const bool aligned = ((uintptr_t)a.x | (uintptr_t)a.g) % 16 == 0;
        int splits = 0;
        if (engine == 2 && aligned) {
            a.status = status;
            splits = wgrad_halo_cn(a, max_splits, st);
        }
        if (splits == 0) {
            splits = max_splits;
            gemm_bn<MODE_WGRAD>(co, a, (int)nblk(27 * ci, GM), splits, st);
        }
        k_reduce_parts<<<nblk(27 * ci * co, 256), 256, 0, st>>>(splits, 27 * ci * co, part,
                                                                grad_params + net::w_off(l));
        k_bias_part<<<dim3(64, co), 256, 0, st>>>(s3, co, gz_f, bpart);
        k_reduce_parts<<<1, 64, 0, st>>>(64, co, bpart, grad_params + net::b_off(l));
        counted(3);
    };
    auto dgrad = [&](int l, int side, const bf16 *gz_b, float *gx) {
        ConvArgs d{};
        d.n = side; d.ci = net::L[l].ci; d.co = net::L[l].co; d.x = gz_b; d.w = wbf + net::w_off(l);
        d.out = gx; d.wt = wpk + net::wpk_off(l, 1); d.status = status;
        conv_gemm<MODE_DGRAD>(d, (long long)side * side * side, st);
    };
    // layer 5: a5 = relu(conv(u1) + b5 + a1)
    k_relu_grad<<<nblk(n3 * 16, 256), 256, 0, st>>>(n, 16, B(W.a5), F(W.ga5f), nullptr, nullptr,
                                                   nullptr, B(W.gz5b), F(W.gz5f));
    counted(1);
    wgrad(4, n, B(W.u1), B(W.gz5b), F(W.gz5f));
    dgrad(4, n, B(W.gz5b), F(W.gu1f));
    // layer 4: a4 = relu(conv(up(a3)) + b4 + a2); its gradient is up^T(gu1)
    k_relu_grad<<<nblk(h3 * 32, 256), 256, 0, st>>>(h, 32, B(W.a4), nullptr, F(W.gu1f), nullptr,
                                                   nullptr, B(W.gz4b), F(W.gz4f));
    counted(1);
    wgrad(3, h, B(W.u2), B(W.gz4b), F(W.gz4f));
    dgrad(3, h, B(W.gz4b), F(W.gu2f));
    // layer 3: a3 = relu(conv(pool(a2)) + b3); gradient up^T(gu2)
    k_relu_grad<<<nblk(q3 * 64, 256), 256, 0, st>>>(q, 64, B(W.a3), nullptr, F(W.gu2f), nullptr,
                                                   nullptr, B(W.gz3b), F(W.gz3f));
    counted(1);
    wgrad(2, q, B(W.p2), B(W.gz3b), F(W.gz3f));
    dgrad(2, q, B(W.gz3b), F(W.gp2f));
    // layer 2: a2 = relu(conv(pool(a1)) + b2); gradient: skip of layer 4 + pool^T(gp2)
    k_relu_grad<<<nblk(h3 * 32, 256), 256, 0, st>>>(h, 32, B(W.a2), F(W.gz4f), nullptr, F(W.gp2f),
                                                   nullptr, B(W.gz2b), F(W.gz2f));
    counted(1);
    wgrad(1, h, B(W.p1), B(W.gz2b), F(W.gz2f));
    dgrad(1, h, B(W.gz2b), F(W.gp1f));
    // layer 1: a1 = relu(conv(x) + b1); gradient: skip of layer 5 + pool^T(gp1)
    k_relu_grad<<<nblk(n3 * 16, 256), 256, 0, st>>>(n, 16, B(W.a1), F(W.gz5f), nullptr, F(W.gp1f),
                                                   nullptr, nullptr, F(W.gz1f));
    const unsigned c1t = (unsigned)(((n + 7) / 8) * ((n + 7) / 8) * ((n + 7) / 8));
    const unsigned c1b = c1t < (unsigned)net::C1_BLOCKS ? c1t : (unsigned)net::C1_BLOCKS;  // blocks = partials
    k_conv1_wgrad<<<c1b, C1_THREADS, 0, st>>>(n, input, F(W.gz1f), part);
    k_reduce_parts<<<nblk(27 * 16 + 16, 256), 256, 0, st>>>((int)c1b, 27 * 16 + 16, part,
                                                            grad_params + net::w_off(0));
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
    k_reduce_parts<<<1, 32, 0, st>>>(256, 1, lp, loss);
    counted(2);
    return cudaGetLastError() == cudaSuccess ? DGR_OK : DGR_ERR_CUDA;
}

int dgr_set_conv_engine(int engine) {
    if (engine < 0 || engine > 2) return DGR_ERR_ARG;
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
