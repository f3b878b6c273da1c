// Device helpers shared by the per-step kernels and the persistent solve kernel.
#pragma once

#include <cuda_runtime.h>

namespace lamg {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a CSR row by a group of TPR lanes (all 32 lanes of the warp must call it); lanes of
// one group hold entries e0, e0 + TPR, ... of the row. The group total is returned to every
// lane of the group.
template <int TPR>
__device__ __forceinline__ double row_sum(int e0, int e1, const int32_t *__restrict__ ci,
                                          const double *__restrict__ val, const double *x) {
    double s = 0.0;
    for (int e = e0; e < e1; e += TPR) s += val[e] * x[ci[e]];
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Sum of NV values over the block; the totals are valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) sh[k][w] = v[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = warp_sum(lane < nw ? sh[k][lane] : 0.0);
    }
    __syncthreads();
}

}  // namespace lamg
