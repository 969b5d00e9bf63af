// Warp-level sum of an 8-wide per-thread vector, every lane receiving the
// totals: the reduce-and-broadcast operation of Sec. 3 (one call here where
// the paper's kernel makes seven one-value calls), in the two forms the
// paper compares (Sec. 4.2): FP32 warp shuffles, and tensor-core matrix
// products with an all-ones operand.
//
// The tensor-core form is this library's own design for sm_103a, not the
// paper's WMMA code: operands are split into several lower-precision terms
// whose products with exact 0/1 operands are exact, accumulation is FP32,
// and the per-lane data is staged through shared memory so that the
// reduction axis (the 32 lanes) becomes the MMA's K axis.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "adgb.h"
#include "tcgen05.cuh"

namespace adgb {

__device__ __forceinline__ float shfl_xor(float v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// Reduce-scatter by recursive halving (4+2+1 exchanges), then two
// butterfly steps finish the component the lane holds, then an all-gather
// (8 indexed shuffles).  17 shuffles for 8 values.  Lane bits (4,3,2) name
// the component each lane finishes with.
__device__ __forceinline__ void warp_sum8_shfl(float v[8]) {
    const int lane = threadIdx.x & 31;
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float send = up ? v[k] : v[k + 4];
            float keep = up ? v[k + 4] : v[k];
            v[k] = keep + shfl_xor(send, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            float send = up ? v[k] : v[k + 2];
            float keep = up ? v[k + 2] : v[k];
            v[k] = keep + shfl_xor(send, 8);
        }
    }
    {
        const bool up = lane & 4;
        float send = up ? v[0] : v[1];
        float keep = up ? v[1] : v[0];
        v[0] = keep + shfl_xor(send, 4);
    }
    float t = v[0] + shfl_xor(v[0], 2);
    t = t + shfl_xor(t, 1);
    // component c lives in lanes with bits (4,3,2) = (c>>2, c>>1, c) & 1
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int src = ((c >> 2) & 1) << 4 | ((c >> 1) & 1) << 3 | (c & 1) << 2;
        v[c] = __shfl_sync(0xffffffffu, t, src);
    }
}

// ---------------------------------------------------------------- MMA helpers
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32_16x8x8(float d[4], uint32_t a0, uint32_t a1,
                                                uint32_t a2, uint32_t a3, uint32_t b0,
                                                uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16_16x8x16(float d[4], uint32_t a0, uint32_t a1,
                                                 uint32_t a2, uint32_t a3, uint32_t b0,
                                                 uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Round-to-nearest-even float -> bf16 bits, and back.
__device__ __forceinline__ uint32_t bf16_bits(float x) {
    uint32_t r;
    asm("{ .reg .b16 h; cvt.rn.bf16.f32 h, %1; cvt.u32.u16 %0, h; }" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float bf16_val(uint32_t b) { return __uint_as_float(b << 16); }

// Split x into three bf16 terms hi + mid + lo (about 24 significant bits).
__device__ __forceinline__ void split_bf16x3(float x, uint32_t &h, uint32_t &m, uint32_t &l) {
    h = bf16_bits(x);
    float r1 = x - bf16_val(h);
    m = bf16_bits(r1);
    float r2 = r1 - bf16_val(m);
    l = bf16_bits(r2);
}

// Tensor-core sum over the 32 lanes with TF32 operands split in two terms
// (hi = tf32(x), lo = tf32(x - hi): 22 significant bits).  stage: this
// warp's 32 x 8 floats of shared memory.
//
// D (16x8) = A (16 x K) * ones (K x 8), K = the 32 source lanes in four
// k8 chunks.  Row m < 8 of A holds the hi term of component m, row m + 8
// its lo term, so D[g][*] + D[g+8][*] is the total of component g, which
// the m16n8k8 accumulator layout hands to the four lanes of quad g.
__device__ __forceinline__ void warp_sum8_mma_tf32x2(float v[8], float *stage) {
    const int lane = threadIdx.x & 31;
    float4 *row = reinterpret_cast<float4 *>(stage + lane * 8);
    row[0] = make_float4(v[0], v[1], v[2], v[3]);
    row[1] = make_float4(v[4], v[5], v[6], v[7]);
    __syncwarp();
    const int g = lane >> 2, t = lane & 3;
    const uint32_t one = to_tf32(1.0f);
    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float x0 = stage[(8 * q + t) * 8 + g];
        float x1 = stage[(8 * q + t + 4) * 8 + g];
        uint32_t h0 = to_tf32(x0), h1 = to_tf32(x1);
        uint32_t l0 = to_tf32(x0 - __uint_as_float(h0));
        uint32_t l1 = to_tf32(x1 - __uint_as_float(h1));
        // a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4)
        mma_tf32_16x8x8(d, h0, l0, h1, l1, one, one);
    }
    __syncwarp();
    const float mine = d[0] + d[2];
#pragma unroll
    for (int c = 0; c < 8; c++) v[c] = __shfl_sync(0xffffffffu, mine, 4 * c);
}

// Same with bf16 operands split in three terms (about FP32 precision).
// m16n8k16: rows m < 8 of A carry hi, rows m + 8 carry mid in the first
// pass; the second pass carries lo in rows m < 8.  Two k16 chunks cover the
// 32 lanes.  stage rows are 12 floats apart (bank-conflict-free reads).
__device__ __forceinline__ void warp_sum8_mma_bf16x3(float v[8], float *stage) {
    const int lane = threadIdx.x & 31;
    float4 *row = reinterpret_cast<float4 *>(stage + lane * 12);
    row[0] = make_float4(v[0], v[1], v[2], v[3]);
    row[1] = make_float4(v[4], v[5], v[6], v[7]);
    __syncwarp();
    const int g = lane >> 2, t = lane & 3;
    const uint32_t one2 = 0x3f803f80u;  // (1.0, 1.0) in bf16
    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int k0 = 16 * q + 2 * t;
        float x0 = stage[(k0 + 0) * 12 + g], x1 = stage[(k0 + 1) * 12 + g];
        float x8 = stage[(k0 + 8) * 12 + g], x9 = stage[(k0 + 9) * 12 + g];
        uint32_t h0, m0, l0, h1, m1, l1, h8, m8, l8, h9, m9, l9;
        split_bf16x3(x0, h0, m0, l0);
        split_bf16x3(x1, h1, m1, l1);
        split_bf16x3(x8, h8, m8, l8);
        split_bf16x3(x9, h9, m9, l9);
        // registers: {A[g][2t], A[g][2t+1]}, {A[g+8][..]}, {A[g][2t+8], A[g][2t+9]}, {A[g+8][..]}
        mma_bf16_16x8x16(d, h0 | (h1 << 16), m0 | (m1 << 16), h8 | (h9 << 16),
                         m8 | (m9 << 16), one2, one2);
        mma_bf16_16x8x16(d, l0 | (l1 << 16), 0u, l8 | (l9 << 16), 0u, one2, one2);
    }
    __syncwarp();
    const float mine = d[0] + d[2];
#pragma unroll
    for (int c = 0; c < 8; c++) v[c] = __shfl_sync(0xffffffffu, mine, 4 * c);
}

template <int VAR>
__device__ __forceinline__ void warp_sum8(float v[8], float *stage) {
    static_assert(VAR == ADGB_REDUCE_SHFL || VAR == ADGB_REDUCE_MMA_TF32X2 ||
                  VAR == ADGB_REDUCE_MMA_BF16X3, "warp_sum8: register / mma.sync variants only");
    if constexpr (VAR == ADGB_REDUCE_SHFL) {
        warp_sum8_shfl(v);
    } else if constexpr (VAR == ADGB_REDUCE_MMA_TF32X2) {
        warp_sum8_mma_tf32x2(v, stage);
    } else {
        warp_sum8_mma_bf16x3(v, stage);
    }
}

// ------------------------------------------------------- tcgen05 warp form
// Per-warp state of the fifth-generation tensor-core reduction.  Each warp
// owns a 2 KB shared-memory B operand (two 128-byte-swizzled 8-row atoms:
// rows 0-7 the TF32 hi terms of the 8 values, rows 8-15 the lo terms; K =
// the 32 lanes), an mbarrier, and 16 TMEM columns for its D = ones . B^T
// (M = 128, N = 16); the all-ones A operand (128 x 8 TF32, 4 KB of shared
// memory) is shared by the block's warps.  Every row of D holds the column
// sums, and each warp reads them from its own lane quadrant.
struct Tc05Warp {
    unsigned char *b;     // generic address of this warp's B operand
    uint64_t *mbar;       // completion barrier of this warp's MMAs
    uint32_t b_s;         // shared-window address of the B operand
    uint32_t d_col;       // TMEM address of D (lane 0, first column)
    uint32_t d_lane;      // TMEM address of D in this warp's lane quadrant
    uint64_t a_desc;      // descriptor of the shared all-ones A operand
    uint32_t taddr, ncols;
    uint32_t phase;       // completed reductions (mbarrier phase)
    int ok;               // 0 once a completion wait gave up (results NaN)
};

constexpr int TC05_WAIT_LIMIT = 1 << 16;   // mbarrier probes, each suspending up to a time limit

// Tensor-core completion waits that gave up in this translation unit's
// kernels on the current device (monotonic, one count a warp; the host reads
// it after a call and reports ADGB_EDEVICE when it grew).
static __device__ unsigned int g_tc_gave_up;

// The tcgen05 reduction in two halves, so that independent work can run
// while the MMAs are in flight: tc05_issue stages the warp's partials (TF32
// hi and lo terms) and has one lane issue the MMAs and commit them to the
// warp's mbarrier; tc05_finish waits (bounded) and loads the totals from
// TMEM.  v is not changed by tc05_issue.
__device__ __forceinline__ void tc05_issue(const float v[8], Tc05Warp &t) {
    const int lane = threadIdx.x & 31, cq = lane >> 2;
    if (!t.ok) return;
    unsigned char *mine = t.b + (lane & 3) * 4;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const uint32_t hi = to_tf32(v[c]);
        const uint32_t lo = to_tf32(v[c] - __uint_as_float(hi));
        *reinterpret_cast<uint32_t *>(mine + c * 128 + ((cq ^ c) << 4)) = hi;
        *reinterpret_cast<uint32_t *>(mine + 1024 + c * 128 + ((cq ^ c) << 4)) = lo;
    }
    tc05::fence_proxy_async_smem();
    tc05::fence_before();
    __syncwarp();
    if (lane == 0) {
        tc05::fence_after();
        constexpr uint32_t idesc = tc05::idesc_tf32(128, 16);
#pragma unroll
        for (int s = 0; s < 4; s++)   // K = 32 lanes in four K = 8 slices
            tc05::mma_tf32_ss(t.d_col, t.a_desc, tc05::desc_sw128(t.b_s + 32u * s, 1024), idesc,
                              s > 0);
        tc05::commit(t.mbar);
    }
}

__device__ __forceinline__ void tc05_finish(float v[8], Tc05Warp &t) {
    if (!t.ok) {
#pragma unroll
        for (int c = 0; c < 8; c++) v[c] = __int_as_float(0x7fc00000);
        return;
    }
    const bool done = __all_sync(0xffffffffu, tc05::mbar_wait(t.mbar, t.phase & 1, TC05_WAIT_LIMIT));
    t.phase++;
    if (!done) {
        t.ok = 0;
        if ((threadIdx.x & 31) == 0) atomicAdd(&g_tc_gave_up, 1u);
#pragma unroll
        for (int c = 0; c < 8; c++) v[c] = __int_as_float(0x7fc00000);
        return;
    }
    tc05::fence_after();
    float d[16];
    tc05::ld16_wait(t.d_lane, d);
#pragma unroll
    for (int c = 0; c < 8; c++) v[c] = d[c] + d[8 + c];
    tc05::fence_before();   // these TMEM reads precede the warp's next MMA
}

__device__ __forceinline__ void warp_sum8_tc05(float v[8], Tc05Warp &t) {
    tc05_issue(v, t);
    tc05_finish(v, t);
}

}  // namespace adgb
