// Transpose of the bilinear rotation (T_rot^T of Eq. 1) as a per-voxel gather,
// optionally fused with the OSEM update.
#include <cuda_runtime.h>

#include "geometry.cuh"
#include "internal.h"

namespace spect {


// Transpose of the bilinear rotation, gathered per voxel column (x, y): the
// rotated-grid samples p whose bilinear footprint covers (x, y) lie in the
// box of half-width |cos|+|sin| around R(-theta)(q - c) + c.  Each weight is
// recomputed with the forward's arithmetic, so it equals the forward weight.
__global__ void __launch_bounds__(kGatherThreads) gather_kernel(GatherArgs a)
{
    extern __shared__ __align__(16) unsigned char gsm[];
    constexpr int T = kGatherTile, TT = kGatherTile * kGatherTile;
    int* cnt = reinterpret_cast<int*>(gsm);                               // [n_sel][TT]
    int* off = cnt + a.n_sel * TT;                                        // [n_sel][TT][kMaxCand]
    float* wt = reinterpret_cast<float*>(off + a.n_sel * TT * kMaxCand);  // [n_sel][TT][kMaxCand]
    const int n = a.n, nz = a.nz;
    const int tiles_x = (n + T - 1) / T;
    const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
    const int zpart = blockIdx.y, b = blockIdx.z;
    const int x0 = tx * T, y0 = ty * T;
    const float c = 0.5f * (float)(n - 1);

    for (int e = threadIdx.x; e < a.n_sel * TT; e += kGatherThreads) {
        const int g = e / TT, col = e - g * TT;
        const int x = x0 + col / T, y = y0 + col % T;
        int count = 0;
        if (x < n && y < n) {
            const float2 cs = a.cs[a.sel[g]];
            const float dx = (float)x - c, dy = (float)y - c;
            const float pi = c + cs.x * dx + cs.y * dy;
            const float pj = c - cs.y * dx + cs.x * dy;
            const float ext = fabsf(cs.x) + fabsf(cs.y) + 1e-3f;
            const int ia = max(0, (int)ceilf(pi - ext)), ib = min(n - 1, (int)floorf(pi + ext));
            const int ja = max(0, (int)ceilf(pj - ext)), jb = min(n - 1, (int)floorf(pj + ext));
            for (int i = ia; i <= ib; ++i)
                for (int j = ja; j <= jb; ++j) {
                    float u, v;
                    sample_point(cs.x, cs.y, c, i, j, u, v);
                    const float fu = floorf(u), fv = floorf(v);
                    const int xa = (int)fu, ya = (int)fv;
                    const float ax = u - fu, by = v - fv;
                    const float wx = (x == xa) ? (1.f - ax) : (x == xa + 1 ? ax : 0.f);
                    const float wy = (y == ya) ? (1.f - by) : (y == ya + 1 ? by : 0.f);
                    if (wx != 0.f && wy != 0.f && count < kMaxCand) {
                        off[(g * TT + col) * kMaxCand + count] = (i * n + j) * nz;
                        wt[(g * TT + col) * kMaxCand + count] = wx * wy;
                        ++count;
                    }
                }
        }
        cnt[g * TT + col] = count;
    }
    __syncthreads();

    const int nz4 = nz >> 2;
    const int zc = (nz4 + a.zsplit - 1) / a.zsplit;
    const int z4a = zpart * zc, z4b = min(nz4, z4a + zc);
    const int zl = z4b - z4a;
    if (zl <= 0) return;
    const size_t vol = (size_t)n * n * nz;
    const float* bb = a.bvol + (size_t)b * a.n_sel * vol;
    for (int p = threadIdx.x; p < TT * zl; p += kGatherThreads) {
        const int col = p / zl, z4 = z4a + (p - col * zl);
        const int x = x0 + col / T, y = y0 + col % T;
        if (x >= n || y >= n) continue;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int g = 0; g < a.n_sel; ++g) {
            const int m = cnt[g * TT + col];
            const float* base = bb + (size_t)g * vol + 4 * z4;
            for (int e = 0; e < m; ++e) {
                const float w = wt[(g * TT + col) * kMaxCand + e];
                const float4 v = __ldg(reinterpret_cast<const float4*>(base + off[(g * TT + col) * kMaxCand + e]));
                acc.x = fmaf(w, v.x, acc.x);
                acc.y = fmaf(w, v.y, acc.y);
                acc.z = fmaf(w, v.z, acc.z);
                acc.w = fmaf(w, v.w, acc.w);
            }
        }
        float4* o = reinterpret_cast<float4*>(a.out + (size_t)b * vol + ((size_t)x * n + y) * nz) + z4;
        if (a.sens) {
            const float4 sv = __ldg(reinterpret_cast<const float4*>(a.sens + ((size_t)x * n + y) * nz) + z4);
            float4 f = *o;
            f.x = sv.x > 0.f ? f.x * acc.x / sv.x : f.x;
            f.y = sv.y > 0.f ? f.y * acc.y / sv.y : f.y;
            f.z = sv.z > 0.f ? f.z * acc.z / sv.z : f.z;
            f.w = sv.w > 0.f ? f.w * acc.w / sv.w : f.w;
            *o = f;
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
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t st)
{
    constexpr int TT = kGatherTile * kGatherTile;
    const size_t smem = (size_t)a.n_sel * TT * (sizeof(int) + kMaxCand * (sizeof(int) + sizeof(float)));
    static unsigned long long mask = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(mask & (1ull << (dev & 63)))) {
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        mask |= 1ull << (dev & 63);
    }
    const int tiles = (a.n + kGatherTile - 1) / kGatherTile;
    dim3 grid(tiles * tiles, a.zsplit, a.batch);
    gather_kernel<<<grid, kGatherThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
