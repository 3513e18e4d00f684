// Transpose of the bilinear rotation (T_rot^T of Eq. 1) as a per-voxel
// gather, optionally fused with the OSEM update.
//
// For angle a and voxel column q = (x, y), the rotated-grid samples p whose
// bilinear footprint covers q lie in the box of half-width |cos|+|sin|
// around R(-theta)(q - c) + (c, cj) (cj: the angle's shifted detector centre).  The plan stores, per (angle, column), up to
// kMaxCand (offset of p's row in a rotated-frame volume, weight) pairs, the
// weight recomputed with the forward's own arithmetic so that it equals the
// forward weight bit for bit.  A convex region of area 4 and perimeter 8
// holds at most 4 + 8/2 + 1 = 9 lattice points, hence kMaxCand = 9.
#include <cuda_runtime.h>

#include "geometry.cuh"
#include "internal.h"
#include "update.cuh"

namespace spect {

__global__ void gather_table_kernel(const float4* __restrict__ cs_tab, int n, int nz, int2* __restrict__ tab)
{
    const int angle = blockIdx.y;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n * n) return;
    const int x = col / n, y = col - x * n;
    const float c = 0.5f * (float)(n - 1);
    const float4 cs = cs_tab[angle];
    const float dx = (float)x - c, dy = (float)y - c;
    const float pi = c + cs.x * dx + cs.y * dy;
    const float pj = cs.z - cs.y * dx + cs.x * dy;
    const float ext = fabsf(cs.x) + fabsf(cs.y) + 1e-3f;
    const int ia = max(0, (int)ceilf(pi - ext)), ib = min(n - 1, (int)floorf(pi + ext));
    const int ja = max(0, (int)ceilf(pj - ext)), jb = min(n - 1, (int)floorf(pj + ext));
    int2* out = tab + ((size_t)angle * n * n + col) * kMaxCand;
    int count = 0;
    for (int i = ia; i <= ib; ++i)
        for (int j = ja; j <= jb; ++j) {
            float u, v;
            sample_point(cs.x, cs.y, c, cs.z, i, j, u, v);
            const float fu = floorf(u), fv = floorf(v);
            const int xa = (int)fu, ya = (int)fv;
            const float ax = u - fu, by = v - fv;
            const float wx = (x == xa) ? (1.f - ax) : (x == xa + 1 ? ax : 0.f);
            const float wy = (y == ya) ? (1.f - by) : (y == ya + 1 ? by : 0.f);
            if (wx != 0.f && wy != 0.f && count < kMaxCand) {
                out[count] = make_int2((i * n + j) * nz, __float_as_int(wx * wy));
                ++count;
            }
        }
    for (; count < kMaxCand; ++count) out[count] = make_int2(0, 0);
}

cudaError_t launch_gather_tables(const float4* cs, int n, int nz, int n_angles, int2* tab, cudaStream_t st)
{
    dim3 grid((n * n + 127) / 128, n_angles);
    gather_table_kernel<<<grid, 128, 0, st>>>(cs, n, nz, tab);
    return cudaGetLastError();
}

// One warp per (voxel column, block of 32 float4 along z); with short columns
// (nz/4 < 32) a warp covers several columns, lanes_per_col lanes each.
// Angles are taken two at a time so that the table and volume loads of both
// are in flight together; the sum runs over angles in order, then over each
// angle's entries in table order, so it is deterministic.
__global__ void __launch_bounds__(256) gather_kernel(GatherArgs a)
{
    const int n = a.n, nz = a.nz, zw = nz >> 2;
    const int lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long col;
    int z4;
    if (a.lanes_per_col == 32) {
        const int zb = (zw + 31) >> 5;
        col = gw / zb;
        z4 = (int)(gw - col * zb) * 32 + lane;
    } else {
        col = gw * (32 / a.lanes_per_col) + lane / a.lanes_per_col;
        z4 = lane % a.lanes_per_col;
    }
    if (col >= (long)n * n || z4 >= zw) return;
    const int b = blockIdx.y;
    const size_t vol = (size_t)n * n * nz;
    const float* __restrict__ bb = a.bvol + (size_t)b * a.n_sel * vol + 4 * z4;
    const int2* __restrict__ tab = a.tab;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int g = 0; g < a.n_sel; g += 2) {
        const bool two = g + 1 < a.n_sel;
        const int2* t0 = tab + ((size_t)a.sel[g] * n * n + col) * kMaxCand;
        const int2* t1 = tab + ((size_t)a.sel[two ? g + 1 : g] * n * n + col) * kMaxCand;
        int2 e0[kMaxCand], e1[kMaxCand];
#pragma unroll
        for (int e = 0; e < kMaxCand; ++e) {
            e0[e] = __ldg(t0 + e);
            e1[e] = two ? __ldg(t1 + e) : make_int2(0, 0);
        }
        float4 v0[kMaxCand], v1[kMaxCand];
        const float* b0 = bb + (size_t)g * vol;
        const float* b1 = bb + (size_t)(g + 1) * vol;
#pragma unroll
        for (int e = 0; e < kMaxCand; ++e) {
            v0[e] = e0[e].y != 0 ? __ldg(reinterpret_cast<const float4*>(b0 + e0[e].x)) : make_float4(0.f, 0.f, 0.f, 0.f);
            v1[e] = e1[e].y != 0 ? __ldg(reinterpret_cast<const float4*>(b1 + e1[e].x)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < kMaxCand; ++e) {
            if (e0[e].y != 0) {
                const float w = __int_as_float(e0[e].y);
                acc.x = fmaf(w, v0[e].x, acc.x);
                acc.y = fmaf(w, v0[e].y, acc.y);
                acc.z = fmaf(w, v0[e].z, acc.z);
                acc.w = fmaf(w, v0[e].w, acc.w);
            }
        }
#pragma unroll
        for (int e = 0; e < kMaxCand; ++e) {
            if (e1[e].y != 0) {
                const float w = __int_as_float(e1[e].y);
                acc.x = fmaf(w, v1[e].x, acc.x);
                acc.y = fmaf(w, v1[e].y, acc.y);
                acc.z = fmaf(w, v1[e].z, acc.z);
                acc.w = fmaf(w, v1[e].w, acc.w);
            }
        }
    }
    float4* o = reinterpret_cast<float4*>(a.out + (size_t)b * vol + (size_t)col * nz) + z4;
    if (a.upd.mode != kUpdNone) {
        *o = update4(a.upd, *o, acc, ((size_t)col * nz >> 2) + z4);
    } else if (a.accumulate) {
        float4 f = *o;
        f.x += acc.x;
        f.y += acc.y;
        f.z += acc.z;
        f.w += acc.w;
        *o = f;
    } else {
        *o = acc;
    }
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t st)
{
    const int zw = a.nz >> 2;
    long warps;
    if (a.lanes_per_col == 32)
        warps = (long)a.n * a.n * ((zw + 31) / 32);
    else
        warps = ((long)a.n * a.n + (32 / a.lanes_per_col) - 1) / (32 / a.lanes_per_col);
    const long blocks = (warps * 32 + 255) / 256;
    dim3 grid((unsigned)blocks, a.batch);
    gather_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
