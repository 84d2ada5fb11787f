// reduce.cuh -- fixed-order FP64 block reductions used by the domain sums.
//
// Every sum here has one fixed association order (per-thread serial sums, a
// butterfly over lanes with offsets 16, 8, 4, 2, 1, then warps added 0..W-1
// by one thread), so results are bit-reproducible run to run and do not
// depend on which other work shares the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace slbm {

__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums acc[0..4] over the block and writes them to out[0..4] (thread 0).
// blockDim.x must be a multiple of 32 and at most 1024.
__device__ __forceinline__ void block_sum5_to(const double (&acc)[5], double *out) {
    __shared__ double sw[32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double w[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) w[c] = warp_sum_fixed(acc[c]);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 5; ++c) sw[warp][c] = w[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += sw[i][c];
            out[c] = s;
        }
    }
    __syncthreads();
}

// One block: out[c] = sum over chunks of partial[chunk*5 + c], thread t
// summing chunks t, t + blockDim, ... in order, then block_sum5_to.
__global__ void reduce_partials_kernel(const double *partial, int64_t chunks, double *out);

}  // namespace slbm
