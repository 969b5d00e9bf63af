// Block reduce-and-broadcast of one four-element vector per thread: the test
// kernel of Sec. 5.2.  Variants:
//  - the per-component shuffle + shared-memory atomic reduction profiled in
//    Sec. 3 (warp shuffles, one atomic add per warp, three barriers, called
//    once per component);
//  - this library's FP32 shuffle form (reduce-scatter inside each warp, one
//    barrier, every warp finishes the cross-warp sum itself);
//  - the tensor-core forms (warp_sum8 with TF32x2 / BF16x3 operands) at
//    both levels, also with a single barrier.
// `reps` repeats the reduction inside the kernel so that its cost, not the
// loads and stores around it, dominates the measured time; with tiny = 0
// every repetition reduces the same input.
#include "adgb_internal.cuh"
#include "reduce.cuh"

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
    }
    return cudaErrorInvalidValue;
}

}  // namespace adgb
