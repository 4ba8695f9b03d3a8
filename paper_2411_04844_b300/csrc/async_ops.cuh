// Asynchronous-proxy helpers for sm_103a, as inline PTX: mbarriers, bulk
// copies (the Tensor Memory Accelerator's 1D form), and the fifth-generation
// tensor core (tcgen05: MMA issued by one thread, operands in shared memory
// through matrix descriptors, accumulator in tensor memory).  Every wait is
// bounded: it gives up after a fixed number of polls and flags the status
// word instead of spinning forever.
#pragma once
#include <stdint.h>

#include "dgr.h"

namespace dgr {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------------------
// mbarriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// a bounded wait for the phase of the given parity to complete: gives up (and
// flags the status word) after `polls` unsuccessful polls instead of spinning
// forever (every kernel of the library waits with the default limit).  An
// unsuccessful try_wait suspends the thread for about 3 us on the B300, so the
// default gives up after about 0.8 s; the copies and MMAs waited for complete
// in microseconds.
constexpr int MBAR_POLLS = 1 << 18;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *status,
                                          int polls = MBAR_POLLS) {
    for (int it = 0; it < polls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(status, DGR_STATUS_TIMEOUT);
    return false;
}

// ---------------------------------------------------------------------------
// bulk copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g_add(int *dst, const int *src, unsigned bytes) {
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u32 [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}
// 4D tiled tensor copy global -> shared through a tensor map (the tensor map
// a __grid_constant__ kernel parameter; coordinates innermost first, elements
// outside the tensor read as zero), completing on an mbarrier with its bytes.
// The innermost coordinate times the element size must be a multiple of 16
// bytes and the destination 128-byte aligned.
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// 16-byte asynchronous copy global -> shared through L2 (cp.async); with
// src_bytes = 0 nothing is read and the 16 bytes are zero-filled
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// 4-byte form (through L1); src_bytes = 0 zero-fills
__device__ __forceinline__ void cp_async4(void *dst, const void *src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// the mbarrier receives one arrival (counted in its expected count) once every
// cp.async this thread issued so far has completed
__device__ __forceinline__ void cp_async_mbar_arrive(unsigned long long *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// generic-proxy shared-memory writes become visible to the asynchronous proxy
// (bulk copies, tensor-core operand reads)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---------------------------------------------------------------------------
// tcgen05
// ---------------------------------------------------------------------------
// Tensor memory: allocated in columns (a power of two >= 32) by one whole
// warp, which writes the base address to shared memory; freed by the same
// warp before the CTA exits.
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, the byte
// distance between core matrices adjacent in K (leading) and in M or N
// (stride), the fixed version field 1 (bits 46-47), base offset 0, layout 0.
// A core matrix is 8 rows x 16 bytes stored as 128 contiguous bytes: 8 M/N
// rows of 8 K elements (K-major) or 8 K rows of 8 M/N elements (MN-major);
// the leading / stride assignment is the same for both.
__device__ __forceinline__ uint64_t smem_desc(unsigned saddr, unsigned lead_bytes, unsigned stride_bytes) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lead_bytes >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((stride_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulation,
// dense: D format bits 4-5 = 1 (F32), A format bits 7-9 = 1 (BF16), B format
// bits 10-12 = 1, N >> 3 at bits 17-22, M >> 4 at bits 24-28; A and B K-major
// (OR in bit 15 / bit 16 for an MN-major A / B).
__host__ __device__ constexpr unsigned idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}
// D[tmem] (+)= A[smem] B[smem]^T, one thread issues
__device__ __forceinline__ void umma_bf16(unsigned d_tmem, uint64_t a_desc, uint64_t b_desc, unsigned idesc,
                                          int accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier receives one arrival once every MMA this thread issued so far
// has completed (its shared-memory operands may then be overwritten and the
// accumulator read)
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 16 consecutive FP32 columns of one tensor-memory lane per thread: warp w
// (of a warpgroup) reads lanes 32 w .. 32 w + 31, thread t lane 32 w + t.
// The wait is tied to the registers so no use moves above it.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of one tensor-memory lane per thread written
// with zeros (lanes as for tmem_ld16); waits until the stores are done
__device__ __forceinline__ void tmem_zero16(unsigned taddr) {
    const unsigned z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
            taddr),
        "r"(z)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

}  // namespace dgr
