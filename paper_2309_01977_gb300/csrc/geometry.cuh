// Device helpers shared by the libspect kernels: the rotated-frame sample
// point of Eq. (1)'s T_rot and a deterministic block reduction.
#pragma once

#include <cuda_runtime.h>

namespace spect {

// Sample point of rotated voxel (i, j) for angle (ct, st) = (cos, sin) and
// the angle's centre cj = c + s of the shifted detector axis (T_trans of
// Eq. 1; cj = c without a shift):
//   u = c + ct (i - c) - st (j - cj),   v = c + st (i - c) + ct (j - cj).
// Every kernel that needs the point of the same (angle, i, j) calls this
// function, so the forward bilinear weights and the gathered transpose
// weights are bitwise equal.
__device__ __forceinline__ void sample_point(float ct, float st, float c, float cj, int i, int j, float& u, float& v)
{
    const float di = (float)i - c;
    const float dj = (float)j - cj;
    u = fmaf(ct, di, fmaf(-st, dj, c));
    v = fmaf(st, di, fmaf(ct, dj, c));
}

// Sum of v over the block, valid in thread 0.  Fixed reduction tree, so the
// result does not depend on scheduling.  `red` holds one double per warp.
__device__ __forceinline__ double block_sum_f64(double v, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) r += red[w];
    }
    __syncthreads();
    return r;
}

}  // namespace spect
