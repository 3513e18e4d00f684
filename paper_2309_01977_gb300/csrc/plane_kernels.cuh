// Projector kernels of libspect (sm_103a).
//
// Forward  (Eq. 1, one CTA per (depth chunk, z tile, angle, batch)):
//   for each depth plane i of the chunk
//     stage   P[j][k] = A_a[i][j][k] * bilinear(f)(u(i,j), v(i,j), k)    (T_rot, T_att)
//     z-blur  Q[k][j] = sum_u w_i(u) P[j][k-u]                          (T_cdr, along z)
//     j-blur  acc[j][k] += sum_t w_i(t) Q[k][j-t]                       (T_cdr, along y; P_x)
//   Q is stored transposed (one row per axial column), so both blur passes
//   read consecutive shared-memory words.
//   The accumulator lives in registers for the whole depth loop.  With
//   several depth chunks per angle, each CTA stores a partial projection and
//   a separate reduction kernel adds the partials in chunk order (so the
//   result is deterministic) and, for OSEM, forms the ratio y / (p + s).
//
// Back (the transpose, in two launches):
//   blur_back: B_a[i][j][k] = A_a[i][j][k] * (K_i r_a)[j][k]  (K_i symmetric, zero padded)
//   gather   : x[q] = sum_a sum_p W_a(p -> q) B_a[p]  where W_a are the forward's
//              bilinear weights, enumerated from the voxel side (no atomics).
//   The gather can fuse the OSEM update x <- x * bp / sens.
#pragma once
#include <cuda_runtime.h>

#include "geometry.cuh"
#include "internal.h"

namespace spect {

// ---------------------------------------------------------------- blur strips

// kStrip outputs of a 1-D blur along consecutive shared-memory words:
//   o[q] = sum_u w(|u|) src[q + R - u],  src pointing R words before output 0.
// Sliding window: each loaded value feeds up to 2R+1 register accumulators.
template <int R>
__device__ __forceinline__ void blur_strip(const float* __restrict__ src, float (&o)[kStrip], const float (&w)[R + 1])
{
#pragma unroll
    for (int m = 0; m < kStrip + 2 * R; ++m) {
        const float v = src[m];
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            const int u = q + R - m;
            if (u >= -R && u <= R) o[q] = fmaf(w[u < 0 ? -u : u], v, o[q]);
        }
    }
}

template <int R>
__device__ __forceinline__ void load_taps(const float* __restrict__ row, float (&w)[R + 1])
{
#pragma unroll
    for (int q = 0; q <= R; ++q) w[q] = __ldg(row + kMaxR + q);
}

// z-blur of every row of P into Q (transposed: Q[col][rh + j]), for the
// tile's padded output columns.  Lanes take consecutive rows j: the reads
// (odd P stride) and the writes (consecutive words) are free of bank
// conflicts.
// This thread's first z-blur strip (row j, strip sidx), computed once per
// kernel: word offsets of its input in P and of its output in Q.
struct ZItem {
    int poff, qoff;
    bool valid;
};

__device__ __forceinline__ ZItem z_item(const PlaneTiling& t, int n, int it)
{
    ZItem z;
    z.valid = it < n * (t.ktpad / kStrip);
    const int j = it % n, sidx = it / n;
    z.poff = j * t.wp + t.rh + sidx * kStrip;
    z.qoff = sidx * kStrip * t.qs + t.rh + j;
    return z;
}

template <int R>
__device__ __forceinline__ void zblur_one(const float* P, float* Q, const PlaneTiling& t, const ZItem& z,
                                          const float (&w)[R + 1])
{
    float o[kStrip];
#pragma unroll
    for (int q = 0; q < kStrip; ++q) o[q] = 0.f;
    blur_strip<R>(P + z.poff - R, o, w);
    float* dst = Q + z.qoff;
#pragma unroll
    for (int q = 0; q < kStrip; ++q) dst[q * t.qs] = o[q];
}

// z-blur of every row of P into Q (transposed: Q[col][rh + j]), for the
// tile's padded output columns.  Lanes take consecutive rows j: the reads
// (odd P stride) and the writes (consecutive words) are free of bank
// conflicts.  `z0` is this thread's first strip; further strips (only when
// there are more strips than threads) are indexed here.
template <int R>
__device__ __forceinline__ void zblur_plane(const float* P, float* Q, const PlaneTiling& t, int n, const ZItem& z0,
                                            const float (&w)[R + 1])
{
    if (z0.valid) zblur_one<R>(P, Q, t, z0, w);
    for (int it = threadIdx.x + blockDim.x; it < n * (t.ktpad / kStrip); it += blockDim.x)
        zblur_one<R>(P, Q, t, z_item(t, n, it), w);
}

// j-blur strips of this thread: strip q covers column kk = it % ktpad and
// rows js*kStrip .. +kStrip-1 with it = threadIdx.x + q * blockDim.x;
// jq[q] is the strip's word offset in Q (or -1 when the thread has none).
template <int R, int IPT>
__device__ __forceinline__ void fwd_blur_plane(const float* P, float* Q, const PlaneTiling& t, int n, const ZItem& z0,
                                               const int (&jq)[IPT], const float* __restrict__ taps_row,
                                               float (&acc)[IPT][kStrip])
{
    float w[R + 1];
    load_taps<R>(taps_row, w);
    zblur_plane<R>(P, Q, t, n, z0, w);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < IPT; ++q)
        if (jq[q] >= 0) blur_strip<R>(Q + jq[q] - R, acc[q], w);
}

#define SPECT_R_CASES(M) \
    M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18) M(19) M(20)

// ---------------------------------------------------------------- forward

// Zero the columns of P that lie outside the volume (they are the z-blur's
// zero padding) and, in every column of the transposed Q, the halo rows
// outside [0, n) (the j-blur's zero padding).
__device__ __forceinline__ void zero_pads(float* P, float* Q, const PlaneTiling& t, int n, int nz, int kw0, bool p_all)
{
    const int W = t.ktpad + 2 * t.rh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < n; j += nw)
        for (int col = lane; col < W; col += 32) {
            const int k = kw0 + col;
            if (p_all || k < 0 || k >= nz) P[j * t.wp + col] = 0.f;
        }
    for (int col = warp; col < t.ktpad; col += nw)
        for (int r = lane; r < t.qs; r += 32)
            if (r < t.rh || r >= t.rh + n) Q[(size_t)col * t.qs + r] = 0.f;
}

// Bilinear taps of rotated row (i, j) of one plane, computed once per row
// by one thread and kept in shared memory: element offsets of the four tap
// rows in the volume and their weights.  Taps outside the grid get weight 0
// and offset 0, so every load stays in bounds.
struct TapRow {
    int off[4];
    float w[4];
};

__device__ __forceinline__ void tap_rows(TapRow* rows, int n, int nz, int i, float2 cs, float c)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float u, v;
        sample_point(cs.x, cs.y, c, i, j, u, v);
        const float fu = floorf(u), fv = floorf(v);
        const int x0 = (int)fu, y0 = (int)fv;
        const float ax = u - fu, by = v - fv;
        const bool vx0 = x0 >= 0 && x0 < n, vx1 = x0 + 1 >= 0 && x0 + 1 < n;
        const bool vy0 = y0 >= 0 && y0 < n, vy1 = y0 + 1 >= 0 && y0 + 1 < n;
        TapRow t;
        t.w[0] = (vx0 && vy0) ? (1.f - ax) * (1.f - by) : 0.f;
        t.w[1] = (vx1 && vy0) ? ax * (1.f - by) : 0.f;
        t.w[2] = (vx0 && vy1) ? (1.f - ax) * by : 0.f;
        t.w[3] = (vx1 && vy1) ? ax * by : 0.f;
        t.off[0] = (vx0 && vy0) ? (x0 * n + y0) * nz : 0;
        t.off[1] = (vx1 && vy0) ? ((x0 + 1) * n + y0) * nz : 0;
        t.off[2] = (vx0 && vy1) ? (x0 * n + y0 + 1) * nz : 0;
        t.off[3] = (vx1 && vy1) ? ((x0 + 1) * n + y0 + 1) * nz : 0;
        rows[j] = t;
    }
}

// P[j][k - kw0] = A[j][k] * sum_taps w * f[tap][k] for k in [klo, khi),
// from the row table, one row per warp at a time.  Columns go in chunks of
// 128 (four per lane): the loads of a chunk use immediate offsets from five
// per-row pointers.  In a partial last chunk the column index is clamped so
// that the loads stay in bounds and control flow stays uniform; only the
// stores are masked.
__device__ __forceinline__ void stage_plane(float* P, const PlaneTiling& t, const TapRow* rows,
                                            const float* __restrict__ xb, const float* __restrict__ arow, int n,
                                            int nz, int kw0, int klo, int khi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncols = khi - klo;
    for (int j = warp; j < n; j += nw) {
        const TapRow tr = rows[j];
        const float w0 = tr.w[0], w1 = tr.w[1], w2 = tr.w[2], w3 = tr.w[3];
        const float* __restrict__ f0 = xb + tr.off[0] + klo;
        const float* __restrict__ f1 = xb + tr.off[1] + klo;
        const float* __restrict__ f2 = xb + tr.off[2] + klo;
        const float* __restrict__ f3 = xb + tr.off[3] + klo;
        const float* __restrict__ ar = arow ? arow + (size_t)j * nz + klo : nullptr;
        float* prow = P + j * t.wp + (klo - kw0);
        for (int c0 = 0; c0 < ncols; c0 += 128) {
            float v[4];
            if (c0 + 128 <= ncols) {
                // full chunk: lane-relative immediate offsets
                const int c = c0 + lane;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[q] = w0 * __ldg(f0 + c + 32 * q);
                    v[q] = fmaf(w1, __ldg(f1 + c + 32 * q), v[q]);
                    v[q] = fmaf(w2, __ldg(f2 + c + 32 * q), v[q]);
                    v[q] = fmaf(w3, __ldg(f3 + c + 32 * q), v[q]);
                }
                if (ar) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] *= __ldg(ar + c + 32 * q);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) prow[c + 32 * q] = v[q];
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = min(c0 + lane + 32 * q, ncols - 1);
                    v[q] = w0 * __ldg(f0 + c);
                    v[q] = fmaf(w1, __ldg(f1 + c), v[q]);
                    v[q] = fmaf(w2, __ldg(f2 + c), v[q]);
                    v[q] = fmaf(w3, __ldg(f3 + c), v[q]);
                    if (ar) v[q] *= __ldg(ar + c);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = c0 + lane + 32 * q;
                    if (c < ncols) prow[c] = v[q];
                }
            }
        }
    }
}

template <int IPT>
__global__ void __launch_bounds__(kFwdThreads, 1) forward_kernel(ForwardArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const PlaneTiling& t = a.t;
    const int n = a.n, nz = a.nz;
    float* P = smem;
    float* Q = smem + (size_t)n * t.wp;
    TapRow* rows = reinterpret_cast<TapRow*>(Q + (size_t)t.ktpad * t.qs);
    const int tid = threadIdx.x;
    const int chunk = blockIdx.x % a.chunks, tile = blockIdx.x / a.chunks;
    const int sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const float2 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const int kt0 = tile * t.ktile;
    const int KT = min(t.ktile, nz - kt0);
    const int kw0 = kt0 - t.rh;
    const int W = t.ktpad + 2 * t.rh;
    const int klo = max(0, kw0), khi = min(nz, kw0 + W);

    zero_pads(P, Q, t, n, nz, kw0, false);

    // this thread's blur strips, fixed for the whole depth loop
    const ZItem z0 = z_item(t, n, tid);
    const int njs = t.npad / kStrip;
    int jq[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = tid + q * blockDim.x;
        const int kk = it % t.ktpad, js = it / t.ktpad;
        jq[q] = it < t.ktpad * njs ? kk * t.qs + t.rh + js * kStrip : -1;
    }

    float acc[IPT][kStrip];
#pragma unroll
    for (int q = 0; q < IPT; ++q)
#pragma unroll
        for (int r = 0; r < kStrip; ++r) acc[q][r] = 0.f;

    const float* xb = a.x + (size_t)b * n * n * nz;
    // planes chunk, chunk + chunks, ...: every chunk mixes planes near and
    // far from the detector, whose blur widths differ several-fold
    for (int i = chunk; i < n; i += a.chunks) {
        // ---- stage the rotated, attenuated plane (T_rot, T_att)
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        tap_rows(rows, n, nz, i, cs, c);
        __syncthreads();
        stage_plane(P, t, rows, xb, arow, n, nz, kw0, klo, khi);
        __syncthreads();
        // ---- blur along z and y, accumulate over depth (T_cdr, P_x)
        const float* trow = a.taps + (size_t)i * kTapW;
        switch (__ldg(a.rad + i)) {
#define SPECT_FWD_CASE(RR) \
    case RR: fwd_blur_plane<RR, IPT>(P, Q, t, n, z0, jq, trow, acc); break;
            SPECT_R_CASES(SPECT_FWD_CASE)
#undef SPECT_FWD_CASE
            default: break;
        }
        // The next staging writes P only; Q is rewritten after the next
        // barrier, which every thread reaches after its j-blur above.
    }

    // Raw depth sums of this chunk: to the output when the chunk is the
    // whole depth and no ratio is wanted, else to the partial planes.
    const size_t item = (size_t)b * a.n_sel + sidx;
    float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = tid + q * blockDim.x;
        if (it < t.ktpad * njs) {
            const int kk = it % t.ktpad, js = it / t.ktpad;
            if (kk < KT) {
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n) dst[(size_t)j * nz + kt0 + kk] = acc[q][r];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- back: blur

template <int R, int IPT>
__device__ __forceinline__ void back_blur_plane(const float* P, float* Q, const PlaneTiling& t, const BlurBackArgs& a,
                                                const ZItem& z0, int i, int angle, int kt0, int KT,
                                                float* __restrict__ bvol)
{
    const int n = a.n, nz = a.nz;
    const int njs = t.npad / kStrip;
    const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
    float w[R + 1];
    load_taps<R>(a.taps + (size_t)i * kTapW, w);
    zblur_plane<R>(P, Q, t, n, z0, w);
    __syncthreads();
    float* __restrict__ brow = bvol + (size_t)i * n * nz;
    // rolled loop over this thread's strips: one copy of the unrolled j-blur
#pragma unroll 1
    for (int it = threadIdx.x; it < t.ktpad * njs; it += blockDim.x) {
        {
            const int kk = it % t.ktpad, js = it / t.ktpad;
            float o[kStrip];
#pragma unroll
            for (int r = 0; r < kStrip; ++r) o[r] = 0.f;
            blur_strip<R>(Q + (size_t)kk * t.qs + t.rh + js * kStrip - R, o, w);
            if (kk < KT) {
                const int k = kt0 + kk;
                // all attenuation loads of the strip first, then the stores
                float aw[kStrip];
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    aw[r] = (arow && j < n) ? __ldg(arow + (size_t)j * nz + k) : 1.f;
                }
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n) brow[(size_t)j * nz + k] = o[r] * aw[r];
                }
            }
        }
    }
}

template <int IPT>
__global__ void __launch_bounds__(kFwdThreads, 1) blur_back_kernel(BlurBackArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const PlaneTiling& t = a.t;
    const int n = a.n, nz = a.nz;
    float* P = smem;
    float* Q = smem + (size_t)n * t.wp;
    const int tid = threadIdx.x;
    const int chunk = blockIdx.x % a.chunks, tile = blockIdx.x / a.chunks;
    const int sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const int kt0 = tile * t.ktile;
    const int KT = min(t.ktile, nz - kt0);
    const int kw0 = kt0 - t.rh;
    const int W = t.ktpad + 2 * t.rh;
    const size_t item = (size_t)b * a.n_sel + sidx;

    // The projection window of this angle, zero outside the detector.
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    zero_pads(P, Q, t, n, nz, kw0, false);
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < n; j += blockDim.x >> 5)
        for (int col = lane; col < W; col += 32) {
            const int k = kw0 + col;
            if (k >= 0 && k < nz) P[j * t.wp + col] = pr ? __ldg(pr + (size_t)j * nz + k) : 1.f;
        }
    __syncthreads();
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const ZItem z0 = z_item(t, n, tid);
    // planes chunk, chunk + chunks, ...: every chunk mixes planes near and
    // far from the detector, whose blur widths differ several-fold
    for (int i = chunk; i < n; i += a.chunks) {
        switch (__ldg(a.rad + i)) {
#define SPECT_BACK_CASE(RR) \
    case RR: back_blur_plane<RR, IPT>(P, Q, t, a, z0, i, angle, kt0, KT, bvol); break;
            SPECT_R_CASES(SPECT_BACK_CASE)
#undef SPECT_BACK_CASE
            default: break;
        }
        __syncthreads();  // Q is rewritten by the next plane's z-blur
    }
}

// ---------------------------------------------------------------- launchers

// Raise the dynamic shared-memory limit of kernel `fn` to what the device
// allows next to the kernel's static shared memory, once per device.
template <class F>
inline cudaError_t allow_big_smem(F fn, unsigned long long& mask)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (mask & bit) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) mask |= bit;
    return e;
}

// Devices on which a kernel's shared-memory limit has been raised (shared by
// the occupancy query at plan creation and the launches, so that launches
// inside a stream capture find it done).
template <int IPT>
unsigned long long g_forward_smem_mask = 0;
template <int IPT>
unsigned long long g_blur_back_smem_mask = 0;

template <int IPT>
cudaError_t forward_launch_ipt(const ForwardArgs& a, int grid_x, cudaStream_t st)
{
    cudaError_t e = allow_big_smem(forward_kernel<IPT>, g_forward_smem_mask<IPT>);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    forward_kernel<IPT><<<grid, a.t.threads, a.t.smem, st>>>(a);
    return cudaGetLastError();
}

template <int IPT>
int forward_occupancy_ipt(int threads, size_t smem)
{
    if (allow_big_smem(forward_kernel<IPT>, g_forward_smem_mask<IPT>) != cudaSuccess) {
        cudaGetLastError();  // do not leave the failure to a later launch check
        return 0;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_kernel<IPT>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <int IPT>
cudaError_t blur_back_launch_ipt(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    cudaError_t e = allow_big_smem(blur_back_kernel<IPT>, g_blur_back_smem_mask<IPT>);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    blur_back_kernel<IPT><<<grid, a.t.threads, a.t.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
