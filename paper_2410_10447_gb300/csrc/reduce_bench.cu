// Block reduce-and-broadcast of one four-element vector per thread: the test
// kernel of Sec. 5.2.  Variants:
//  - the per-component shuffle + shared-memory atomic reduction profiled in
//    Sec. 3 (warp shuffles, one atomic add per warp, three barriers, called
//    once per component);
//  - this library's FP32 shuffle form (reduce-scatter inside each warp, one
//    barrier, every warp finishes the cross-warp sum itself);
//  - the tensor-core forms (warp_sum8 with TF32x2 / BF16x3 operands) at
//    both levels, also with a single barrier;
//  - the paper's own matrix form (Sec. 4.2) in FP16: V <- A.P + V over
//    64-vector chunks, then W <- Q.V, with FP16 operands and accumulators,
//    one warp issuing the products and two barriers;
//  - a block-wide fifth-generation tensor-core form: every thread's split
//    TF32 vector goes into one shared-memory operand, a single thread issues
//    tcgen05.mma with an all-ones TMEM operand, and each thread reads the
//    totals from its own TMEM row (one barrier and one mbarrier wait).
// `reps` repeats the reduction inside the kernel so that its cost, not the
// loads and stores around it, dominates the measured time; with tiny = 0
// every repetition reduces the same input.
#include "adgb_internal.cuh"
#include "reduce.cuh"
#include "tcgen05.cuh"

#include <cuda_fp16.h>

namespace adgb {

__device__ __forceinline__ float warp_allsum_5(float v) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Sec. 3: shuffle tree, lane 0 adds into a shared accumulator, all read it.
__device__ __forceinline__ float reduce_fs(float v, float *acc) {
    if (threadIdx.x == 0) *acc = 0.f;
    __syncthreads();
    v = warp_allsum_5(v);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, v);
    __syncthreads();
    v = *acc;
    __syncthreads();
    return v;
}

template <int VAR>
__device__ __forceinline__ float4 block_sum4(float4 x, float *red, float *stage) {
    float v[8] = {x.x, x.y, x.z, x.w, 0.f, 0.f, 0.f, 0.f};
    warp_sum8<VAR>(v, stage);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    if (lane == 0) reinterpret_cast<float4 *>(red)[w] = make_float4(v[0], v[1], v[2], v[3]);
    __syncthreads();
    float4 p = lane < W ? reinterpret_cast<float4 *>(red)[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float u[8] = {p.x, p.y, p.z, p.w, 0.f, 0.f, 0.f, 0.f};
    warp_sum8<VAR>(u, stage);
    return make_float4(u[0], u[1], u[2], u[3]);
}

template <int VAR>
__global__ void __launch_bounds__(1024) reduce4_kernel(const float4 *in, float4 *out, int reps,
                                                       float tiny) {
    extern __shared__ __align__(16) float rsm[];
    float *red0 = rsm;                  // [2][32][4] (double-buffered across reps)
    float *stage = rsm + 256 + (threadIdx.x >> 5) * 32 * 12;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float4 x0 = in[idx];
    float4 x = x0, tot = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = 0; r < reps; r++) {
        if constexpr (VAR == ADGB_REDUCE4_PAPER_FS) {
            tot.x = reduce_fs(x.x, red0);
            tot.y = reduce_fs(x.y, red0);
            tot.z = reduce_fs(x.z, red0);
            tot.w = reduce_fs(x.w, red0);
        } else {
            tot = block_sum4<VAR>(x, red0 + (r & 1) * 128, stage);
        }
        x.x = x0.x + tot.x * tiny;
        x.y = x0.y + tot.y * tiny;
        x.z = x0.z + tot.z * tiny;
        x.w = x0.w + tot.w * tiny;
    }
    out[idx] = tot;
}

// ---------------------------------------------------------------------------
// Sec. 4.2 in FP16.  Thread t stores (x, y, z, e) of its vector as four
// halves at A[4t..4t+3], so every 64 threads fill one 16x16 column-major
// matrix A (column j = vectors 4j..4j+3).  Warp 0 forms V <- A.P + V over
// the chunks (P all ones, only its first 8 columns are needed because all
// columns of V are equal) and W <- Q.V (Q = 4x4 blocks of I4), both with
// FP16 accumulators; W's first column holds the four totals.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma_f16acc_16x8x16(uint32_t d[2], uint32_t a0, uint32_t a1,
                                                   uint32_t a2, uint32_t a3, uint32_t b0,
                                                   uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f16.f16.f16.f16 "
        "{%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%0,%1};\n"
        : "+r"(d[0]), "+r"(d[1])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_h2(__half lo, __half hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

__device__ __forceinline__ uint32_t q_pair(int r, int s) {  // (Q[r][s], Q[r][s+1])
    const __half one = __ushort_as_half(0x3C00), zero = __ushort_as_half(0);
    return pack_h2((r & 3) == (s & 3) ? one : zero, (r & 3) == ((s + 1) & 3) ? one : zero);
}

__global__ void __launch_bounds__(1024) reduce4_half_kernel(const float4 *in, float4 *out,
                                                            int reps, float tiny) {
    extern __shared__ __align__(16) unsigned char hsm[];
    const int chunks = (blockDim.x + 63) >> 6;
    __half *A = reinterpret_cast<__half *>(hsm);     // [chunks][16][16] column-major
    __half *res = A + chunks * 256;                  // W[0..3][0]
    const int tid = threadIdx.x, lane = tid & 31, g = lane >> 2, t = lane & 3;
    for (int i = blockDim.x * 4 + tid; i < chunks * 256; i += blockDim.x) A[i] = __float2half(0.f);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + tid;
    const float4 x0 = in[idx];
    float4 x = x0, tot = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = 0; r < reps; r++) {
        uint2 h;
        h.x = pack_h2(__float2half_rn(x.x), __float2half_rn(x.y));
        h.y = pack_h2(__float2half_rn(x.z), __float2half_rn(x.w));
        reinterpret_cast<uint2 *>(A)[tid] = h;
        __syncthreads();
        if (tid < 32) {
            const uint32_t ones = 0x3C003C00u;
            uint32_t v[2] = {0u, 0u};
            for (int q = 0; q < chunks; q++) {
                const __half *Aq = A + q * 256;
                auto at = [&](int row, int col) { return Aq[col * 16 + row]; };
                const uint32_t a0 = pack_h2(at(g, 2 * t), at(g, 2 * t + 1));
                const uint32_t a1 = pack_h2(at(g + 8, 2 * t), at(g + 8, 2 * t + 1));
                const uint32_t a2 = pack_h2(at(g, 2 * t + 8), at(g, 2 * t + 9));
                const uint32_t a3 = pack_h2(at(g + 8, 2 * t + 8), at(g + 8, 2 * t + 9));
                mma_f16acc_16x8x16(v, a0, a1, a2, a3, ones, ones);
            }
            // B operand of Q.V: rows 2t, 2t+1 (and +8) of V, any column; row
            // k of V sits in lanes 4k..4k+3 (k < 8: v[0], else v[1]).
            const uint32_t r0 = __shfl_sync(0xffffffffu, v[0], 8 * t);
            const uint32_t r1 = __shfl_sync(0xffffffffu, v[0], 8 * t + 4);
            const uint32_t r8 = __shfl_sync(0xffffffffu, v[1], 8 * t);
            const uint32_t r9 = __shfl_sync(0xffffffffu, v[1], 8 * t + 4);
            const uint32_t b0 = (r0 & 0xFFFFu) | (r1 << 16);
            const uint32_t b1 = (r8 & 0xFFFFu) | (r9 << 16);
            uint32_t w[2] = {0u, 0u};
            mma_f16acc_16x8x16(w, q_pair(g, 2 * t), q_pair(g + 8, 2 * t), q_pair(g, 2 * t + 8),
                               q_pair(g + 8, 2 * t + 8), b0, b1);
            if (t == 0 && g < 4) res[g] = __ushort_as_half((unsigned short)(w[0] & 0xFFFFu));
        }
        __syncthreads();
        tot = make_float4(__half2float(res[0]), __half2float(res[1]), __half2float(res[2]),
                          __half2float(res[3]));
        x.x = x0.x + tot.x * tiny;
        x.y = x0.y + tot.y * tiny;
        x.z = x0.z + tot.z * tiny;
        x.w = x0.w + tot.w * tiny;
    }
    out[idx] = tot;
}

// ---------------------------------------------------------------------------
// Block-wide reduction on the fifth-generation tensor cores.
//
// D[128 x N] = A[128 x K] . B[N x K]^T with A all ones (in TMEM) and B the
// block's data: K runs over threads, so every row of D holds column sums of
// B, and row m of D sits in TMEM lane m.  Each warp reads the rows of its
// own lane quadrant, so every thread receives the totals without a second
// stage or a broadcast.  Each thread contributes 8 rows' worth of one K
// column: its four components as TF32 hi and lo terms (hi = x rounded to
// TF32, lo = (x - hi) rounded to TF32); products with 1.0 are exact and D
// accumulates in FP32.  The block's threads are split into NG groups (one
// group = an 8-row atom along N), warp w filling K columns 32(w / NG) ..
// +31 of group w % NG, so N = 8 NG and K = blockDim / NG.
//
// B uses the 128-byte swizzled K-major layout: a warp's 32 threads x 8 rows
// fill exactly one 1024-byte atom, row r of thread (lane) at chunk
// (lane / 4) ^ r, which makes each of the 8 per-thread stores free of bank
// conflicts.  MMA s covers K columns 8s .. 8s+7: atom column s / 4 and a
// 32-byte offset (s % 4) inside the atom rows.
//
// A completion wait that gives up (it never should) turns the outputs into
// NaN; the TMEM is still released.
// ---------------------------------------------------------------------------
constexpr int TC_WAIT_LIMIT = 1 << 16;   // probes, each suspending up to a time limit
constexpr int TC_SELFTEST_LIMIT = 64;     // the wait self-test gives up after 64 probes

template <int NG>
struct TcShape {
    static constexpr int N = 8 * NG;
    static constexpr int NCOLS = N + 8 <= 32 ? 32 : (N + 8 <= 64 ? 64 : 128);
};

__host__ __device__ constexpr int tc_smem_bytes(int threads) { return 16 + 1024 + 32 * threads; }

// wait_limit: mbarrier probes before a wait gives up; no_mma (the wait
// self-test): nothing is issued or committed, so every wait gives up.
template <int NG>
__global__ void __launch_bounds__(1024) reduce4_tc05_kernel(const float4 *in, float4 *out,
                                                            int reps, float tiny, int wait_limit,
                                                            int no_mma) {
    constexpr int N = TcShape<NG>::N, NCOLS = TcShape<NG>::NCOLS;
    extern __shared__ __align__(16) unsigned char tsm[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tsm);
    uint32_t *slot = reinterpret_cast<uint32_t *>(tsm + 8);
    const uint32_t base_s = tc05::smem_u32(tsm);
    const uint32_t b_s = (base_s + 16u + 1023u) & ~1023u;
    unsigned char *bbuf = tsm + (b_s - base_s);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int n_mma = blockDim.x / (8 * NG);

    if (w == 0) {
        tc05::alloc(slot, NCOLS);
        tc05::relinquish();
    }
    if (tid == 0) tc05::mbar_init(mbar, 1);
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t taddr = *slot;
    if (w < 4) {   // A = ones in columns [N, NCOLS) of this warp's lane quadrant
        uint32_t one[16];
#pragma unroll
        for (int i = 0; i < 16; i++) one[i] = 0x3F800000u;
        for (int c = N; c < NCOLS; c += 16) tc05::st16(tc05::lane_addr(taddr, w, c), one);
        tc05::wait_st();
    }

    const size_t idx = (size_t)blockIdx.x * blockDim.x + tid;
    const float4 x0 = in[idx];
    float4 x = x0, tot = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned char *mine = bbuf + (w / NG) * (NG * 1024) + (w % NG) * 1024 + (lane & 3) * 4;
    const int cq = lane >> 2;
    const uint32_t idesc = tc05::idesc_tf32(128, N);
    bool bad = false;
    int r = 0;
    for (; r < reps; r++) {
        const float v[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const uint32_t hi = to_tf32(v[c]);
            const uint32_t lo = to_tf32(v[c] - __uint_as_float(hi));
            *reinterpret_cast<uint32_t *>(mine + c * 128 + ((cq ^ c) << 4)) = hi;
            *reinterpret_cast<uint32_t *>(mine + (c + 4) * 128 + ((cq ^ (c + 4)) << 4)) = lo;
        }
        tc05::fence_proxy_async_smem();
        tc05::fence_before();
        if (__syncthreads_or(bad)) break;
        if (tid == 0 && !no_mma) {
            tc05::fence_after();
            for (int s = 0; s < n_mma; s++) {
                const uint32_t bs = b_s + (uint32_t)((s >> 2) * NG * 1024 + (s & 3) * 32);
                tc05::mma_tf32_ts(taddr, taddr + N, tc05::desc_sw128(bs, 1024), idesc, s > 0);
            }
            tc05::commit(mbar);
        }
        if (!__all_sync(0xffffffffu, tc05::mbar_wait(mbar, r & 1, wait_limit))) {
            bad = true;
            continue;
        }
        tc05::fence_after();
        float hs[4] = {0.f, 0.f, 0.f, 0.f}, ls[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < N / 16; j++) {
            float d[16];
            tc05::ld16_wait(tc05::lane_addr(taddr, w & 3, 16 * j), d);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                hs[c] += d[c] + d[8 + c];
                ls[c] += d[4 + c] + d[12 + c];
            }
        }
        tc05::fence_before();
        tot = make_float4(hs[0] + ls[0], hs[1] + ls[1], hs[2] + ls[2], hs[3] + ls[3]);
        x.x = x0.x + tot.x * tiny;
        x.y = x0.y + tot.y * tiny;
        x.z = x0.z + tot.z * tiny;
        x.w = x0.w + tot.w * tiny;
    }
    if (bad) {   // let the MMAs in flight finish (bounded) before TMEM is released
        (void)tc05::mbar_wait(mbar, (r - 1) & 1, wait_limit);   // phase r - 1 gave up
        tot = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                          __int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    }
    __syncthreads();
    tc05::fence_after();
    if (w == 0) tc05::dealloc(taddr, NCOLS);
    out[idx] = tot;
}

template <int VAR>
static cudaError_t launch_r(const float *in, int threads, int n_blocks, int reps, float *out,
                            cudaStream_t s) {
    const int smem = (256 + (threads / 32) * 32 * 12) * 4;
    auto k = reduce4_kernel<VAR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<n_blocks, threads, smem, s>>>(reinterpret_cast<const float4 *>(in),
                                      reinterpret_cast<float4 *>(out), reps, 0.f);
    return cudaGetLastError();
}

static cudaError_t launch_half(const float *in, int threads, int n_blocks, int reps, float *out,
                               cudaStream_t s) {
    const int smem = (((threads + 63) / 64) * 256 + 8) * 2;
    reduce4_half_kernel<<<n_blocks, threads, smem, s>>>(reinterpret_cast<const float4 *>(in),
                                                        reinterpret_cast<float4 *>(out), reps, 0.f);
    return cudaGetLastError();
}

// Shared memory is padded so that no more CTAs are resident on an SM than
// its 512 TMEM columns can serve at once (tcgen05.alloc would otherwise
// wait for a resident CTA to finish).
template <int NG>
static cudaError_t launch_tc(const float *in, int threads, int n_blocks, int reps, float *out,
                             cudaStream_t s, bool self_test) {
    int dev = 0, sm_smem = 0, reserved = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int fit = 512 / TcShape<NG>::NCOLS;
    int smem = tc_smem_bytes(threads);
    const int floor_smem = sm_smem / (fit + 1) - reserved + 16;
    if (smem < floor_smem) smem = floor_smem;
    auto k = reduce4_tc05_kernel<NG>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<n_blocks, threads, smem, s>>>(reinterpret_cast<const float4 *>(in),
                                      reinterpret_cast<float4 *>(out), reps, 0.f,
                                      self_test ? TC_SELFTEST_LIMIT : TC_WAIT_LIMIT,
                                      self_test ? 1 : 0);
    return cudaGetLastError();
}

// Thread groups for the tcgen05 form: the most (up to 8) that divide the
// block's warps evenly; a block needs an even number of warps (N >= 16).
static int tc_groups(int threads) {
    const int W = threads / 32;
    return W % 8 == 0 ? 8 : (W % 4 == 0 ? 4 : (W % 2 == 0 ? 2 : 0));
}

// ---------------------------------------------------------------------------
// ALU throughput probes for the roofline of the scoring kernels: chains of
// dependent FP32 fused multiply-adds (8 independent chains a thread) or of
// special-function-unit operations (ex2.approx or rsqrt.approx), long enough
// that issue throughput, not latency, bounds them.  out[thread] keeps the
// results alive.
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(256) alu_kernel(float *out, int reps, float b, float c) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    if constexpr (KIND == 3) {
        // packed FP32 pairs: one instruction, two fused multiply-adds
        float2 p[8];
#pragma unroll
        for (int k = 0; k < 8; k++) p[k] = make_float2(a[k], a[k] + 0.5f);
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
        for (int r = 0; r < reps; r++) {
#pragma unroll
            for (int u = 0; u < 16; u++) {
#pragma unroll
                for (int k = 0; k < 8; k++) p[k] = __ffma2_rn(p[k], b2, c2);
            }
        }
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = p[k].x + p[k].y;
    } else {
        for (int r = 0; r < reps; r++) {
#pragma unroll
            for (int u = 0; u < 16; u++) {
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    if constexpr (KIND == 0) {
                        a[k] = fmaf(a[k], b, c);
                    } else if constexpr (KIND == 1) {
                        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(-a[k]));
                    } else {
                        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(a[k] + c));
                    }
                }
            }
        }
    }
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) t += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

cudaError_t launch_alu_bench(int kind, int n_blocks, int threads, int reps, float *out,
                             cudaStream_t s) {
    switch (kind) {
        case 0: alu_kernel<0><<<n_blocks, threads, 0, s>>>(out, reps, 0.999f, 1e-3f); break;
        case 1: alu_kernel<1><<<n_blocks, threads, 0, s>>>(out, reps, 0.f, 0.f); break;
        case 2: alu_kernel<2><<<n_blocks, threads, 0, s>>>(out, reps, 0.f, 1.f); break;
        case 3: alu_kernel<3><<<n_blocks, threads, 0, s>>>(out, reps, 0.999f, 1e-3f); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// L2 read probe.  KIND 0: coalesced streaming reads (thread t reads float4
// t, t + T, ... modulo n4, T the threads of the launch).  KIND 1: the scoring
// kernels' gather pattern: per repetition a pseudo-random cell of cell4
// float4 (an integer hash of thread and repetition) and 96 bytes of it - two
// float4 of one of its leading maps and the four trailing float4 (the grid's
// type map and its e and d maps).  Each thread writes the sum of the x
// components it read.
template <int KIND>
__global__ void __launch_bounds__(256) l2_kernel(const float4 *buf, long long n4, int cell4,
                                                 int reps, float *out) {
    const long long T = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if constexpr (KIND == 0) {
        long long i = t % n4;
        const long long step = T % n4;
#pragma unroll 8
        for (int r = 0; r < reps; r++) {
            acc += __ldg(buf + i).x;
            i += step;
            if (i >= n4) i -= n4;
        }
    } else {
        const uint32_t n_cells = (uint32_t)(n4 / cell4);
        const int m = (int)(t % (cell4 / 2 - 2));
#pragma unroll 4
        for (int r = 0; r < reps; r++) {
            uint32_t h = (uint32_t)t * 0x9E3779B1u ^ (uint32_t)r * 0x85EBCA77u;
            h ^= h >> 15;
            h *= 0x2C1B3C6Du;
            h ^= h >> 12;
            const float4 *cp = buf + (size_t)__umulhi(h, n_cells) * cell4;
            acc += __ldg(cp + 2 * m).x + __ldg(cp + 2 * m + 1).x + __ldg(cp + cell4 - 4).x +
                   __ldg(cp + cell4 - 3).x + __ldg(cp + cell4 - 2).x + __ldg(cp + cell4 - 1).x;
        }
    }
    out[t] = acc;
}

cudaError_t launch_l2_bench(int kind, const float *buf, long long n4, int cell4, int n_blocks,
                            int threads, int reps, float *out, cudaStream_t s) {
    const float4 *b = reinterpret_cast<const float4 *>(buf);
    switch (kind) {
        case 0: l2_kernel<0><<<n_blocks, threads, 0, s>>>(b, n4, cell4, reps, out); break;
        case 1: l2_kernel<1><<<n_blocks, threads, 0, s>>>(b, n4, cell4, reps, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce4_bench(int variant, const float *in, int threads, int n_blocks,
                                 int reps, float *out, cudaStream_t s) {
    switch (variant) {
        case ADGB_REDUCE4_PAPER_FS:
            return launch_r<ADGB_REDUCE4_PAPER_FS>(in, threads, n_blocks, reps, out, s);
        case ADGB_REDUCE_SHFL:
            return launch_r<ADGB_REDUCE_SHFL>(in, threads, n_blocks, reps, out, s);
        case ADGB_REDUCE_MMA_TF32X2:
            return launch_r<ADGB_REDUCE_MMA_TF32X2>(in, threads, n_blocks, reps, out, s);
        case ADGB_REDUCE_MMA_BF16X3:
            return launch_r<ADGB_REDUCE_MMA_BF16X3>(in, threads, n_blocks, reps, out, s);
        case ADGB_REDUCE4_PAPER_HALF:
            return launch_half(in, threads, n_blocks, reps, out, s);
        case ADGB_REDUCE4_TCGEN05_TF32X2:
        case ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST: {
            const bool st = variant == ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST;
            switch (tc_groups(threads)) {
                case 8: return launch_tc<8>(in, threads, n_blocks, reps, out, s, st);
                case 4: return launch_tc<4>(in, threads, n_blocks, reps, out, s, st);
                case 2: return launch_tc<2>(in, threads, n_blocks, reps, out, s, st);
            }
            return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace adgb
