// pd_reduce.cuh -- deterministic block and grid reductions used by the fused dot products.
#pragma once

#include <cuda_runtime.h>

namespace pd {

// Sum over the block; the result is valid in thread 0.  red: shared scratch of
// blockDim.x / 32 doubles.  Fixed tree -> deterministic for a fixed launch shape.
__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

// FP32 values: the butterfly within each warp runs in FP32 (FP64 is a slow pipe
// on this GPU) and only the per-warp sums are added in FP64.  Result in thread 0.
__device__ __forceinline__ double block_sum(float v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) s += red[i];
    __syncthreads();
    return s;
}

// Grid-wide deterministic reduction of one value per block (the "last block
// finishes" pattern): every block writes its partial, the block that retires
// last sums the partials in index order and writes *out, then resets the
// retirement counter to zero for the next launch.
__device__ __forceinline__ void grid_finish(double block_value, int nblocks, int bid, double *partial,
                                            double *out, unsigned int *retire, double *red)
{
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        partial[bid] = block_value;
        __threadfence();
        unsigned int t = atomicAdd(retire, 1u);
        s_last = (t == (unsigned int)(nblocks - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += __ldcg(&partial[i]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        *out = s;
        *retire = 0u;
    }
}

}  // namespace pd
