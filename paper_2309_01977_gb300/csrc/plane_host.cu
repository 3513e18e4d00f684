// Host-side tiling and dispatch of the plane-blur kernels.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"

namespace spect {

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static PlaneTiling make_tiling(int n, int nz, int rmax, int ktile)
{
    PlaneTiling t{};
    t.ktile = ktile;
    t.ntiles = (nz + ktile - 1) / ktile;
    t.rh = rmax + (rmax & 1);
    t.ktpad = round_up(ktile, kStrip);
    t.npad = round_up(n, kStrip);
    t.sp = ((t.ktpad + 2 * t.rh) / 2) | 1;
    t.sq = ((t.npad + 2 * t.rh) / 2) | 1;
    // j-blur strips: ktpad/2 column pairs x npad/kStrip row strips; the
    // smallest number of strips per thread that fits in kFwdThreads threads
    const int items = (t.ktpad / 2) * (t.npad / kStrip);
    t.ipt = kMaxIpt + 1;
    for (int ipt = 1; ipt <= kMaxIpt; ++ipt) {
        const int thr = round_up((items + ipt - 1) / ipt, 32);
        if (thr <= kFwdThreads) {
            t.ipt = ipt;
            t.threads = std::max(64, thr);
            break;
        }
    }
    // P and Q quads, the forward's per-plane tap-row table (32 bytes per
    // row) and the two-plane tap buffer
    const size_t pq = 16 * ((size_t)(t.npad / 2) * t.sp + (size_t)(t.ktpad / 2) * t.sq);
    const size_t taps = 2 * (kMaxR + 1) * sizeof(float);
    t.smem = pq + 32 * (size_t)n + taps;
    t.off_taps_f = (int)(pq + 32 * (size_t)n);
    t.off_taps_b = (int)pq;
    t.smem_f = t.smem;
    t.smem_b = pq + taps;
    return t;
}

// Attenuation buffers of one plane (rows of the columns a CTA reads: the
// staged window for the forward, the tile for the back blur, widened to
// 16-byte boundaries), where they fit under `limit` bytes.
static void attach_atten_buffers(PlaneTiling& t, int n, int nz, size_t limit)
{
    const int win = t.ktpad + 2 * t.rh;
    const int cols_f = t.ntiles == 1 ? nz : std::min(nz, round_up(win + 3, 4));
    const int cols_b = t.ntiles == 1 ? nz : t.ktile;
    const size_t off_f = (t.smem_f + 15) & ~(size_t)15, off_b = (t.smem_b + 15) & ~(size_t)15;
    const size_t end_f = off_f + (size_t)n * cols_f * sizeof(float), end_b = off_b + (size_t)n * cols_b * sizeof(float);
    t.a_cols_f = t.a_cols_b = 0;
    if (end_f + 8 <= limit) {
        t.a_cols_f = cols_f;
        t.off_a_f = (int)off_f;
        t.off_bar_f = (int)end_f;
        t.smem_f = end_f + 8;
    }
    if (end_b + 8 <= limit) {
        t.a_cols_b = cols_b;
        t.off_a_b = (int)off_b;
        t.off_bar_b = (int)end_b;
        t.smem_b = end_b + 8;
    }
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
// fewest volume columns per plane (halo columns are staged once per tile),
// then the fewest j-blur strips (16 column pairs) per thread (each strip per
// thread repeats the unrolled blur code and its 32 accumulators).  At 192^3
// (PSF radius 19) two 96-column tiles with two strips per thread beat three
// 64-column tiles with one: back blur 2.15 vs 4.16 ms, forward 28.2 vs
// 30.4 ms per batch-of-4 launch on GB300.  Then the attenuation buffers,
// where they fit under `limit`.
PlaneTiling plane_tiling(int n, int nz, int rmax, size_t cap, size_t limit)
{
    PlaneTiling best{};
    long best_cols = 0;
    for (int nt = 1; nt <= (nz + kStrip - 1) / kStrip; ++nt) {
        const int kt = nt == 1 ? nz : round_up((nz + nt - 1) / nt, kStrip);
        if (nt > 1 && (nt - 1) * kt >= nz) continue;  // same as a smaller count
        PlaneTiling t = make_tiling(n, nz, rmax, kt);
        if (t.smem > cap || t.ipt > kMaxIpt) continue;
        const long cols = staged_columns(t, nz);
        if (best.smem == 0 || cols < best_cols || (cols == best_cols && t.ipt < best.ipt)) {
            best = t;
            best_cols = cols;
        }
    }
    if (best.smem) attach_atten_buffers(best, n, nz, limit);
    return best;  // smem == 0: does not fit
}

int forward_max_blocks_per_sm(const PlaneTiling& t)
{
    switch (t.ipt) {
        case 1: return forward_occupancy_ipt<1>(t.threads, t.smem_f);
        case 2: return forward_occupancy_ipt<2>(t.threads, t.smem_f);
        case 3: return forward_occupancy_ipt<3>(t.threads, t.smem_f);
        default: return forward_occupancy_ipt<4>(t.threads, t.smem_f);
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
