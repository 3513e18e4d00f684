// Host-side tiling and dispatch of the plane-blur kernels.
#include <cuda_runtime.h>

#include "internal.h"

namespace spect {

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static PlaneTiling make_tiling(int n, int nz, int rh, int ktile)
{
    PlaneTiling t{};
    t.ktile = ktile;
    t.ntiles = (nz + ktile - 1) / ktile;
    t.rh = rh;
    t.ktpad = round_up(ktile, kStrip);
    t.npad = round_up(n, kStrip);
    t.wp = (t.ktpad + 2 * rh) | 1;
    t.qs = t.ktpad | 1;
    const int items = t.ktpad * (t.npad / kStrip);
    t.ipt = (items + kFwdThreads - 1) / kFwdThreads;
    t.smem = sizeof(float) * ((size_t)n * t.wp + (size_t)(t.npad + 2 * rh) * t.qs);
    return t;
}

PlaneTiling plane_tiling(int n, int nz, int rh, size_t smem_cap)
{
    PlaneTiling t = make_tiling(n, nz, rh, nz);
    if (t.smem <= smem_cap && t.ipt <= kMaxIpt) return t;
    for (int kt = round_up(nz, kStrip) - kStrip; kt >= kStrip; kt -= kStrip) {
        t = make_tiling(n, nz, rh, kt);
        if (t.smem <= smem_cap && t.ipt <= kMaxIpt) return t;
    }
    t.smem = 0;  // does not fit
    return t;
}

int forward_max_blocks_per_sm(const PlaneTiling& t)
{
    switch (t.ipt) {
        case 1: return forward_occupancy_ipt<1>(t.smem);
        case 2: return forward_occupancy_ipt<2>(t.smem);
        default: return forward_occupancy_ipt<3>(t.smem);
    }
}

cudaError_t launch_forward(const ForwardArgs& a, int grid_x, cudaStream_t st)
{
    switch (a.t.ipt) {
        case 1: return forward_launch_ipt<1>(a, grid_x, st);
        case 2: return forward_launch_ipt<2>(a, grid_x, st);
        default: return forward_launch_ipt<3>(a, grid_x, st);
    }
}

cudaError_t launch_blur_back(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    switch (a.t.ipt) {
        case 1: return blur_back_launch_ipt<1>(a, grid_x, st);
        case 2: return blur_back_launch_ipt<2>(a, grid_x, st);
        default: return blur_back_launch_ipt<3>(a, grid_x, st);
    }
}

}  // namespace spect
