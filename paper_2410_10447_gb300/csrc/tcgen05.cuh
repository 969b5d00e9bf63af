// Fifth-generation tensor-core primitives for sm_103a, as inline PTX:
// tensor-memory (TMEM) allocation, register <-> TMEM moves, the
// single-thread-issued tcgen05.mma with its shared-memory operand
// descriptor and instruction descriptor, completion through an mbarrier,
// and the proxy / thread-sync fences that order them.
//
// Encodings follow the PTX ISA description of tcgen05 (shared-memory matrix
// descriptor: start address >> 4 in bits 0-13, leading-dimension byte
// offset >> 4 in 16-29, stride-dimension byte offset >> 4 in 32-45, the
// descriptor version 1 in 46-47, base offset in 49-51, swizzle mode in
// 61-63; instruction descriptor: D format in 4-5, A/B formats in 7-9 and
// 10-12, A/B major-ness in 15/16, N >> 3 in 17-22, M >> 4 in 24-28).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace adgb {
namespace tc05 {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ TMEM
// One whole warp executes alloc / dealloc (.sync.aligned).  ncols is a power
// of two >= 32; the allocated base address (lane 0, first column) is written
// to shared memory at `slot`.  alloc waits while the SM's 512 columns are
// held by other CTAs.
__device__ __forceinline__ void alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(ncols) : "memory");
}
__device__ __forceinline__ void relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM address: lane in bits 31-16, column in 15-0.  A warp may only touch
// the 32 lanes of its quadrant (warp index mod 4).
__device__ __forceinline__ uint32_t lane_addr(uint32_t taddr, int quadrant, int col) {
    return taddr + ((uint32_t)(quadrant * 32) << 16) + (uint32_t)col;
}

// 32 lanes x 16 consecutive 32-bit columns, one row per thread of the warp.
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t v[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
          "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
          "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Load 32 lanes x 16 columns and wait for the load in the same statement,
// so that no use of the destination registers can be scheduled before the
// wait.
__device__ __forceinline__ void ld16_wait(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------ descriptors
// K-major operand in the 128-byte swizzled canonical layout: 8-row atoms of
// 8 x 128 bytes (1024-byte aligned), the 16-byte chunk c of row r stored at
// chunk c ^ r; atoms stacked along M/N every `sbo` bytes.  The leading
// offset is unused for this layout when the MMA's K extent (32 bytes for
// TF32, K = 8) lies inside one 128-byte row; it is set to 1 (16 bytes).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4)
         | ((uint64_t)1 << 16)
         | ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32)
         | ((uint64_t)1 << 46)
         | ((uint64_t)2 << 61);
}

// K-major operand without swizzling: 8-row x 16-byte core matrices of 128
// contiguous bytes, `lbo` bytes apart along K and `sbo` bytes apart along
// M/N.
__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4)
         | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16)
         | ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32)
         | ((uint64_t)1 << 46);
}

// kind::tf32, D in FP32, A and B K-major, dense, no negation.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[tmem] . B[smem]^T, issued by one thread for the CTA.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                            uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
        ::"r"(d_tmem), "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[smem] . B[smem]^T, issued by one thread for the CTA.
__device__ __forceinline__ void mma_tf32_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                            uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when every MMA this thread issued so far has
// completed (its operand reads included).
__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(mbar)) : "memory");
}

// ------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One potentially blocking probe: the hardware suspends the thread until the
// phase with the given parity completes or a system-dependent time limit
// passes.
__device__ __forceinline__ bool mbar_try(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity to complete; false after
// `limit` probes.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; i++)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// Generic-proxy shared-memory writes made visible to the tensor core.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace tc05
}  // namespace adgb
