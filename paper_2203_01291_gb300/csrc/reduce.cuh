// Block-wide sums of per-thread partials (the update kernels of the CG and
// the update fused into the preconditioner's forward transform), in FP64 or
// as a compensated float pair converted to FP64 once (see cb.cuh, F2).
#pragma once

#include "cb.cuh"

namespace hol {

// Block sum of a double (blockDim a multiple of 32, <= 1024); valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// Block sum of a compensated float pair, converted to FP64 once (thread 0).
__device__ __forceinline__ double block_sum_f2(F2 v)
{
    __shared__ float red_hi[32], red_lo[32];
    v = f2_warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red_hi[w] = v.hi;
        red_lo[w] = v.lo;
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        F2 t{0.0f, 0.0f};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = f2_add(t, F2{red_hi[k], red_lo[k]});
        s = f2_to_double(t);
    }
    return s;
}

}  // namespace hol
