// Projector kernels of libspect (sm_103a).
//
// Forward  (Eq. 1, one CTA per (depth chunk, z tile, angle, batch)):
//   for each depth plane i of the chunk
//     stage   P[j][k] = A_a[i][j][k] * bilinear(f)(u(i,j), v(i,j), k)    (T_rot, T_att)
//     z-blur  Q[j][k] = sum_u w_i(u) P[j][k-u]                          (T_cdr, along z)
//     j-blur  acc[j][k] += sum_t w_i(t) Q[j-t][k]                       (T_cdr, along y; P_x)
//   The accumulator lives in registers for the whole depth loop.  With
//   several depth chunks per angle, each CTA stores a partial projection and
//   the last CTA to arrive adds the partials in chunk order, so the result
//   is deterministic.
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

// 16 outputs along a shared-memory row: dst[q] = sum_u w(|u|) src[q + R - u],
// src pointing R columns before the first output.
template <int R>
__device__ __forceinline__ void zblur_strip(const float* __restrict__ src, float* __restrict__ dst, const float (&w)[R + 1])
{
    float o[kStrip];
#pragma unroll
    for (int q = 0; q < kStrip; ++q) o[q] = 0.f;
#pragma unroll
    for (int m = 0; m < kStrip + 2 * R; ++m) {
        const float v = src[m];
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            const int u = q + R - m;
            if (u >= -R && u <= R) o[q] = fmaf(w[u < 0 ? -u : u], v, o[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kStrip; ++q) dst[q] = o[q];
}

// 16 outputs down a shared-memory column (row stride `stride`), added to acc.
template <int R>
__device__ __forceinline__ void jblur_strip(const float* __restrict__ src, int stride, float (&acc)[kStrip],
                                            const float (&w)[R + 1])
{
#pragma unroll
    for (int m = 0; m < kStrip + 2 * R; ++m) {
        const float v = src[m * stride];
#pragma unroll
        for (int q = 0; q < kStrip; ++q) {
            const int u = q + R - m;
            if (u >= -R && u <= R) acc[q] = fmaf(w[u < 0 ? -u : u], v, acc[q]);
        }
    }
}

template <int R>
__device__ __forceinline__ void load_taps(const float* __restrict__ row, float (&w)[R + 1])
{
#pragma unroll
    for (int q = 0; q <= R; ++q) w[q] = __ldg(row + kMaxR + q);
}

// z-blur of every row of P into the interior rows of Q, for the tile's
// padded output columns.  Lanes take consecutive rows (odd strides: no bank
// conflicts).
template <int R>
__device__ __forceinline__ void zblur_plane(const float* P, float* Q, const PlaneTiling& t, int n,
                                            const float (&w)[R + 1])
{
    const int nst = t.ktpad / kStrip;
    for (int it = threadIdx.x; it < n * nst; it += kFwdThreads) {
        const int j = it % n, sidx = it / n;
        zblur_strip<R>(P + j * t.wp + t.rh + sidx * kStrip - R, Q + (t.rh + j) * t.qs + sidx * kStrip, w);
    }
}

template <int R, int IPT>
__device__ __forceinline__ void fwd_blur_plane(const float* P, float* Q, const PlaneTiling& t, int n,
                                               const float* __restrict__ taps_row, float (&acc)[IPT][kStrip])
{
    float w[R + 1];
    load_taps<R>(taps_row, w);
    zblur_plane<R>(P, Q, t, n, w);
    __syncthreads();
    const int njs = t.npad / kStrip;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = threadIdx.x + q * kFwdThreads;
        if (it < t.ktpad * njs) {
            const int kk = it % t.ktpad, js = it / t.ktpad;
            jblur_strip<R>(Q + (t.rh + js * kStrip - R) * t.qs + kk, t.qs, acc[q], w);
        }
    }
}

#define SPECT_R_CASES(M) \
    M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18) M(19) M(20)

// ---------------------------------------------------------------- forward

struct ForwardEmit {
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
};

// Write projection value p of bin (j, k), or the OSEM ratio y/(p+s).
__device__ __forceinline__ void forward_emit(const ForwardArgs& a, int angle, size_t out_base, int j, int k, float p,
                                             ForwardEmit& e)
{
    const size_t o = out_base + (size_t)j * a.nz + k;
    if (a.y) {
        const float yv = __ldg(a.y + ((size_t)angle * a.n + j) * a.nz + k);
        const float den = p + a.s;
        const float r = den > 0.f ? yv / den : 0.f;
        a.out[o] = r;
        e.d0 += (double)den;
        e.d1 += (double)yv;
        e.d2 += den > 0.f ? (double)yv * (double)p / (double)den : 0.0;
    } else {
        a.out[o] = p;
    }
}

template <int IPT>
__global__ void __launch_bounds__(kFwdThreads, 1) forward_kernel(ForwardArgs a)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ double red[kFwdThreads / 32];
    __shared__ int s_last;
    const PlaneTiling& t = a.t;
    const int n = a.n, nz = a.nz;
    float* P = smem;
    float* Q = smem + (size_t)n * t.wp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

    // Zero the columns of P outside the volume and the halo rows of Q once.
    for (int idx = tid; idx < n * W; idx += kFwdThreads) {
        const int j = idx / W, col = idx - j * W, k = kw0 + col;
        if (k < 0 || k >= nz) P[j * t.wp + col] = 0.f;
    }
    const int qrows = t.npad + 2 * t.rh;
    for (int idx = tid; idx < qrows * t.qs; idx += kFwdThreads) {
        const int r = idx / t.qs;
        if (r < t.rh || r >= t.rh + n) Q[idx] = 0.f;
    }

    float acc[IPT][kStrip];
#pragma unroll
    for (int q = 0; q < IPT; ++q)
#pragma unroll
        for (int r = 0; r < kStrip; ++r) acc[q][r] = 0.f;

    const float* xb = a.x + (size_t)b * n * n * nz;
    const int i0 = chunk * a.ppc, i1 = min(n, i0 + a.ppc);
    for (int i = i0; i < i1; ++i) {
        // ---- stage the rotated, attenuated plane (T_rot, T_att)
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        for (int j = warp; j < n; j += kFwdThreads / 32) {
            float u, v;
            sample_point(cs.x, cs.y, c, i, j, u, v);
            const float fu = floorf(u), fv = floorf(v);
            const int x0 = (int)fu, y0 = (int)fv;
            const float ax = u - fu, by = v - fv;
            const float w00 = (1.f - ax) * (1.f - by), w10 = ax * (1.f - by);
            const float w01 = (1.f - ax) * by, w11 = ax * by;
            const bool vx0 = x0 >= 0 && x0 < n, vx1 = x0 + 1 >= 0 && x0 + 1 < n;
            const bool vy0 = y0 >= 0 && y0 < n, vy1 = y0 + 1 >= 0 && y0 + 1 < n;
            const float* r00 = xb + (vx0 && vy0 ? ((size_t)x0 * n + y0) * nz : 0);
            const float* r10 = xb + (vx1 && vy0 ? ((size_t)(x0 + 1) * n + y0) * nz : 0);
            const float* r01 = xb + (vx0 && vy1 ? ((size_t)x0 * n + y0 + 1) * nz : 0);
            const float* r11 = xb + (vx1 && vy1 ? ((size_t)(x0 + 1) * n + y0 + 1) * nz : 0);
            const bool b00 = vx0 && vy0, b10 = vx1 && vy0, b01 = vx0 && vy1, b11 = vx1 && vy1;
            float* prow = P + j * t.wp - kw0;
            const float* ar = arow ? arow + (size_t)j * nz : nullptr;
            for (int k = klo + lane; k < khi; k += 32) {
                float val = 0.f;
                if (b00) val = fmaf(w00, __ldg(r00 + k), val);
                if (b10) val = fmaf(w10, __ldg(r10 + k), val);
                if (b01) val = fmaf(w01, __ldg(r01 + k), val);
                if (b11) val = fmaf(w11, __ldg(r11 + k), val);
                if (ar) val *= __ldg(ar + k);
                prow[k] = val;
            }
        }
        __syncthreads();
        // ---- blur along z and y, accumulate over depth (T_cdr, P_x)
        const float* trow = a.taps + (size_t)i * kTapW;
        switch (__ldg(a.rad + i)) {
#define SPECT_FWD_CASE(RR) \
    case RR: fwd_blur_plane<RR, IPT>(P, Q, t, n, trow, acc); break;
            SPECT_R_CASES(SPECT_FWD_CASE)
#undef SPECT_FWD_CASE
            default: break;
        }
        // The next staging writes P only; Q is rewritten after the next
        // barrier, which every thread reaches after its j-blur above.
    }

    const int njs = t.npad / kStrip;
    const size_t item = (size_t)b * a.n_sel + sidx;
    ForwardEmit e;
    if (a.chunks == 1) {
        const size_t out_base = item * n * nz;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int it = tid + q * kFwdThreads;
            if (it < t.ktpad * njs) {
                const int kk = it % t.ktpad, js = it / t.ktpad;
                if (kk < KT) {
#pragma unroll
                    for (int r = 0; r < kStrip; ++r) {
                        const int j = js * kStrip + r;
                        if (j < n) forward_emit(a, angle, out_base, j, kt0 + kk, acc[q][r], e);
                    }
                }
            }
        }
    } else {
        float* part = a.partials + (item * a.chunks + chunk) * (size_t)n * nz;
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            const int it = tid + q * kFwdThreads;
            if (it < t.ktpad * njs) {
                const int kk = it % t.ktpad, js = it / t.ktpad;
                if (kk < KT) {
#pragma unroll
                    for (int r = 0; r < kStrip; ++r) {
                        const int j = js * kStrip + r;
                        if (j < n) part[(size_t)j * nz + kt0 + kk] = acc[q][r];
                    }
                }
            }
        }
        __threadfence();
        __syncthreads();
        unsigned* ctr = a.counters + item * t.ntiles + tile;
        if (tid == 0) s_last = (atomicAdd(ctr, 1u) == (unsigned)(a.chunks - 1));
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        const float* p0 = a.partials + item * a.chunks * (size_t)n * nz;
        const size_t out_base = item * n * nz;
        for (int idx = tid; idx < n * KT; idx += kFwdThreads) {
            const int j = idx / KT, k = kt0 + (idx - j * KT);
            const size_t off = (size_t)j * nz + k;
            float sum = 0.f;
            for (int cc = 0; cc < a.chunks; ++cc) sum += __ldcg(p0 + (size_t)cc * n * nz + off);
            forward_emit(a, angle, out_base, j, k, sum, e);
        }
        if (tid == 0) *ctr = 0u;  // ready for the next launch
    }
    if (a.y && a.diag) {
        const double s0 = block_sum_f64(e.d0, red);
        const double s1 = block_sum_f64(e.d1, red);
        const double s2 = block_sum_f64(e.d2, red);
        if (tid == 0) {
            double* d = a.diag + (item * t.ntiles + tile) * 3;
            d[0] = s0;
            d[1] = s1;
            d[2] = s2;
        }
    }
}

// ---------------------------------------------------------------- back: blur

template <int R, int IPT>
__device__ __forceinline__ void back_blur_plane(const float* P, float* Q, const PlaneTiling& t, const BlurBackArgs& a,
                                                int i, int angle, int kt0, int KT, float* __restrict__ bvol)
{
    const int n = a.n, nz = a.nz;
    float w[R + 1];
    load_taps<R>(a.taps + (size_t)i * kTapW, w);
    zblur_plane<R>(P, Q, t, n, w);
    __syncthreads();
    const int njs = t.npad / kStrip;
    const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
    float* brow = bvol + (size_t)i * n * nz;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = threadIdx.x + q * kFwdThreads;
        if (it < t.ktpad * njs) {
            const int kk = it % t.ktpad, js = it / t.ktpad;
            float o[kStrip];
#pragma unroll
            for (int r = 0; r < kStrip; ++r) o[r] = 0.f;
            jblur_strip<R>(Q + (t.rh + js * kStrip - R) * t.qs + kk, t.qs, o, w);
            if (kk < KT) {
                const int k = kt0 + kk;
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n) {
                        float v = o[r];
                        if (arow) v *= __ldg(arow + (size_t)j * nz + k);
                        brow[(size_t)j * nz + k] = v;
                    }
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
    for (int idx = tid; idx < n * W; idx += kFwdThreads) {
        const int j = idx / W, col = idx - j * W, k = kw0 + col;
        float v = 0.f;
        if (k >= 0 && k < nz) v = pr ? __ldg(pr + (size_t)j * nz + k) : 1.f;
        P[j * t.wp + col] = v;
    }
    const int qrows = t.npad + 2 * t.rh;
    for (int idx = tid; idx < qrows * t.qs; idx += kFwdThreads) {
        const int r = idx / t.qs;
        if (r < t.rh || r >= t.rh + n) Q[idx] = 0.f;
    }
    __syncthreads();
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const int i0 = chunk * a.ppc, i1 = min(n, i0 + a.ppc);
    for (int i = i0; i < i1; ++i) {
        switch (__ldg(a.rad + i)) {
#define SPECT_BACK_CASE(RR) \
    case RR: back_blur_plane<RR, IPT>(P, Q, t, a, i, angle, kt0, KT, bvol); break;
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

template <int IPT>
cudaError_t forward_launch_ipt(const ForwardArgs& a, int grid_x, cudaStream_t st)
{
    static unsigned long long mask = 0;
    cudaError_t e = allow_big_smem(forward_kernel<IPT>, mask);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    forward_kernel<IPT><<<grid, kFwdThreads, a.t.smem, st>>>(a);
    return cudaGetLastError();
}

template <int IPT>
int forward_occupancy_ipt(size_t smem)
{
    static unsigned long long mask = 0;
    if (allow_big_smem(forward_kernel<IPT>, mask) != cudaSuccess) {
        cudaGetLastError();  // do not leave the failure to a later launch check
        return 0;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_kernel<IPT>, kFwdThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <int IPT>
cudaError_t blur_back_launch_ipt(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    static unsigned long long mask = 0;
    cudaError_t e = allow_big_smem(blur_back_kernel<IPT>, mask);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    blur_back_kernel<IPT><<<grid, kFwdThreads, a.t.smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
