// Host-side tiling and dispatch of the plane-blur kernels.
#include <cuda_runtime.h>

#include <algorithm>

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
    t.qs = (t.npad + 2 * rh) | 1;
    // j-blur strips: ktpad columns x npad/kStrip row strips; the smallest
    // number of strips per thread that fits in kFwdThreads threads
    const int items = t.ktpad * (t.npad / kStrip);
    t.ipt = kMaxIpt + 1;
    for (int ipt = 1; ipt <= kMaxIpt; ++ipt) {
        const int thr = round_up((items + ipt - 1) / ipt, 32);
        if (thr <= kFwdThreads) {
            t.ipt = ipt;
            t.threads = std::max(64, thr);
            break;
        }
    }
    // P, Q and the forward's per-plane tap-row table (8 words per row)
    t.smem = sizeof(float) * ((size_t)n * t.wp + (size_t)t.ktpad * t.qs + 8 * (size_t)n);
    return t;
}

// Columns of the volume a tiling stages per plane (tile plus in-volume halo).
static long staged_columns(const PlaneTiling& t, int nz)
{
    long cols = 0;
    for (int tile = 0; tile < t.ntiles; ++tile) {
        const int kw0 = tile * t.ktile - t.rh;
        cols += std::min(nz, kw0 + t.ktpad + 2 * t.rh) - std::max(0, kw0);
    }
    return cols;
}

// Among the z tilings whose buffers fit `cap`: the one that stages the
// fewest volume columns per plane (halo columns are staged twice), with at
// most two j-blur strips per thread when possible (each strip per thread
// repeats the unrolled blur code).
PlaneTiling plane_tiling(int n, int nz, int rh, size_t cap, size_t /*unused*/)
{
    PlaneTiling best{};
    long best_cols = 0;
    for (int pass = 0; pass < 2 && best.smem == 0; ++pass) {
        const int ipt_limit = pass == 0 ? 2 : kMaxIpt;
        for (int nt = 1; nt <= (nz + kStrip - 1) / kStrip; ++nt) {
            const int kt = nt == 1 ? nz : round_up((nz + nt - 1) / nt, kStrip);
            if (nt > 1 && (nt - 1) * kt >= nz) continue;  // same as a smaller count
            PlaneTiling t = make_tiling(n, nz, rh, kt);
            if (t.smem > cap || t.ipt > ipt_limit) continue;
            const long cols = staged_columns(t, nz);
            if (best.smem == 0 || cols < best_cols || (cols == best_cols && t.ipt < best.ipt)) {
                best = t;
                best_cols = cols;
            }
        }
    }
    return best;  // smem == 0: does not fit
}

int forward_max_blocks_per_sm(const PlaneTiling& t)
{
    switch (t.ipt) {
        case 1: return forward_occupancy_ipt<1>(t.threads, t.smem);
        case 2: return forward_occupancy_ipt<2>(t.threads, t.smem);
        case 3: return forward_occupancy_ipt<3>(t.threads, t.smem);
        default: return forward_occupancy_ipt<4>(t.threads, t.smem);
    }
}

cudaError_t launch_forward(const ForwardArgs& a, int grid_x, cudaStream_t st)
{
    switch (a.t.ipt) {
        case 1: return forward_launch_ipt<1>(a, grid_x, st);
        case 2: return forward_launch_ipt<2>(a, grid_x, st);
        case 3: return forward_launch_ipt<3>(a, grid_x, st);
        default: return forward_launch_ipt<4>(a, grid_x, st);
    }
}

cudaError_t launch_blur_back(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    switch (a.t.ipt) {
        case 1: return blur_back_launch_ipt<1>(a, grid_x, st);
        case 2: return blur_back_launch_ipt<2>(a, grid_x, st);
        case 3: return blur_back_launch_ipt<3>(a, grid_x, st);
        default: return blur_back_launch_ipt<4>(a, grid_x, st);
    }
}

}  // namespace spect
