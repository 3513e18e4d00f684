// Projector kernels of libspect (sm_103a).
//
// Forward  (Eq. 1, one CTA per (depth chunk, z tile, angle, batch)):
//   for each depth plane i of the chunk
//     stage   P[j][k] = A_a[i][j][k] * bilinear(f)(u(i,j), v(i,j), k)    (T_rot, T_att)
//     z-blur  Z[j][k] = sum_u w_i(u) P[j][k-u]                          (T_cdr, along z)
//     j-blur  acc[j][k] += sum_t w_i(t) Z[j-t][k]                       (T_cdr, along y; P_x)
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
//
// Packed arithmetic.  Both blur passes run on pairs of independent outputs
// with the sm_100-family paired FP32 FMA (__ffma2_rn: two IEEE fmaf in one
// instruction, so each result is bitwise a scalar fmaf): the z-blur on two
// rows (j, j+1) at once, the j-blur on two columns (k, k+1) at once.  The
// plane buffers therefore hold 2 x 2 quads (one float4 per row pair and
// column pair):
//   P  (staged plane, z-blur input):  [row pair][column pair], quad
//      (P[j][k], P[j+1][k], P[j][k+1], P[j+1][k+1]), so one half of a quad
//      is the pair of rows at one column;
//   Q  (z-blurred plane, j-blur input): [column pair][row pair], quad
//      (Z[j][k], Z[j][k+1], Z[j+1][k], Z[j+1][k+1]), so one half of a quad
//      is the pair of columns at one row.
// Lanes of a warp take consecutive row pairs (z-blur) or column pairs
// (j-blur), and both strides are odd in 16-byte units, so the 128-bit
// shared-memory accesses of the blurs are free of bank conflicts.  The halo
// rh (the plan's largest PSF radius, rounded up to even) fixes the parity of
// a strip's window start, and so its quad boundaries, by R at compile time.
//
// Latency.  The attenuation plane of the next depth plane is copied into
// shared memory by bulk copies (TMA, completing on an mbarrier) while the
// current plane is blurred, and the next plane's taps travel through one
// register; every wait is bounded and a timeout is reported in the plan's
// error word.
#pragma once
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "geometry.cuh"
#include "internal.h"

namespace spect {

// ---------------------------------------------------------------- blur strips

__device__ __forceinline__ float2 lo_half(const float4& q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 hi_half(const float4& q) { return make_float2(q.z, q.w); }

// kStrip output pairs of a 1-D blur:
//   o[q] += sum_m w(|q + R - m|) x[m],   m = 0 .. kStrip + 2R - 1,
// where input pair x[m] is half (m + (R & 1)) & 1 of quad (m + (R & 1)) / 2
// of `src` (src starts one half early when R is odd).  Sliding window: each
// loaded pair feeds up to 2R + 1 register accumulators.
template <int R>
__device__ __forceinline__ void blur_pairs(const float4* __restrict__ src, float2 (&o)[kStrip],
                                           const float2 (&w)[R + 1])
{
    constexpr int odd = R & 1;
    constexpr int nq = (kStrip + 2 * R + odd + 1) / 2;
#pragma unroll
    for (int qd = 0; qd < nq; ++qd) {
        const float4 v4 = src[qd];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = 2 * qd + h - odd;
            if (m < 0 || m >= kStrip + 2 * R) continue;
            const float2 v = h ? hi_half(v4) : lo_half(v4);
#pragma unroll
            for (int q = 0; q < kStrip; ++q) {
                const int u = q + R - m;
                if (u >= -R && u <= R) o[q] = __ffma2_rn(w[u < 0 ? -u : u], v, o[q]);
            }
        }
    }
}

// Taps w(0..R) of a plane from its shared-memory copy (see TapPrefetch).
template <int R>
__device__ __forceinline__ void load_taps(const float* half_row, float2 (&w)[R + 1])
{
#pragma unroll
    for (int q = 0; q <= R; ++q) {
        const float v = half_row[q];
        w[q] = make_float2(v, v);
    }
}

// The taps of the next plane travel through one register per thread (threads
// 0..kMaxR): loaded from global memory when a plane starts, stored to the
// other half of a two-row shared buffer when it ends, so that the load's
// latency hides behind the plane's work.  Rows hold w(0..kMaxR).
struct TapPrefetch {
    float v = 0.f;
    __device__ __forceinline__ void load(const float* __restrict__ taps, int plane)
    {
        if (threadIdx.x <= kMaxR) v = __ldg(taps + (size_t)plane * kTapW + kMaxR + threadIdx.x);
    }
    __device__ __forceinline__ void store(float* buf, int plane) const
    {
        if (threadIdx.x <= kMaxR) buf[(plane & 1) * (kMaxR + 1) + threadIdx.x] = v;
    }
};

// Ask L2 to fetch columns [klo, khi) of every row of an attenuation plane
// ahead of its use (used when the plane does not fit in shared memory).
// The byte range of a row is widened to 16-byte boundaries, which stay
// inside the row because rows start on 16-byte boundaries (nz % 4 == 0).
__device__ __forceinline__ void prefetch_plane_l2(const float* plane, int n, int nz, int klo, int khi)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const size_t lo = reinterpret_cast<size_t>(plane + (size_t)j * nz + klo) & ~(size_t)15;
        const size_t hi = (reinterpret_cast<size_t>(plane + (size_t)j * nz + khi) + 15) & ~(size_t)15;
        prefetch_l2(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
    }
}

// Quad offset of a strip's window for radius R, from the quad offset of the
// strip's first output position (an even position).
template <int R>
__device__ __forceinline__ int window(int first_out_quad)
{
    return first_out_quad - (R + (R & 1)) / 2;
}

// z-blur item `it`: row pair jp, strip sidx of kStrip axial outputs.
// pq: quad offset in P of the item's first output position;
// qq: quad offset in Q of its first output (column pair 8*sidx, row pair jp).
struct ZItem {
    int pq, qq;
    bool valid;
};

__device__ __forceinline__ ZItem z_item(const PlaneTiling& t, int it)
{
    ZItem z;
    const int rp = t.npad >> 1;
    z.valid = it < rp * (t.ktpad / kStrip);
    const int jp = it % rp, sidx = it / rp;
    z.pq = jp * t.sp + ((t.rh + sidx * kStrip) >> 1);
    z.qq = sidx * (kStrip / 2) * t.sq + (t.rh >> 1) + jp;
    return z;
}

template <int R>
__device__ __forceinline__ void zblur_one(const float4* P, float4* Q, const PlaneTiling& t, const ZItem& z,
                                          const float2 (&w)[R + 1])
{
    float2 o[kStrip];
#pragma unroll
    for (int q = 0; q < kStrip; ++q) o[q] = make_float2(0.f, 0.f);
    blur_pairs<R>(P + window<R>(z.pq), o, w);
    // o[q] = (Z[j][k0+q], Z[j+1][k0+q]); a Q quad holds a column pair of two rows
    float4* dst = Q + z.qq;
#pragma unroll
    for (int q = 0; q < kStrip; q += 2) dst[(q >> 1) * t.sq] = make_float4(o[q].x, o[q + 1].x, o[q].y, o[q + 1].y);
}

// z-blur of the staged plane P into Q.  `z0` is this thread's first item;
// further items (more items than threads) are indexed here.
template <int R>
__device__ __forceinline__ void zblur_plane(const float4* P, float4* Q, const PlaneTiling& t, const ZItem& z0,
                                            const float2 (&w)[R + 1])
{
    if (z0.valid) zblur_one<R>(P, Q, t, z0, w);
    const int items = (t.npad >> 1) * (t.ktpad / kStrip);
    for (int it = threadIdx.x + blockDim.x; it < items; it += blockDim.x) zblur_one<R>(P, Q, t, z_item(t, it), w);
}

// j-blur item `it`: column pair kp = it % (ktpad/2), strip js of kStrip rows;
// the quad offset in Q of the strip's first output position, or -1.
__device__ __forceinline__ int j_item(const PlaneTiling& t, int it)
{
    const int cp = t.ktpad >> 1;
    if (it >= cp * (t.npad / kStrip)) return -1;
    const int kp = it % cp, js = it / cp;
    return kp * t.sq + ((t.rh + js * kStrip) >> 1);
}

template <int R, int IPT>
__device__ __forceinline__ void fwd_blur_plane(const float4* P, float4* Q, const PlaneTiling& t, const ZItem& z0,
                                               const int (&jq)[IPT], const float* taps_row,
                                               float2 (&acc)[IPT][kStrip])
{
    float2 w[R + 1];
    load_taps<R>(taps_row, w);
    zblur_plane<R>(P, Q, t, z0, w);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < IPT; ++q)
        if (jq[q] >= 0) blur_pairs<R>(Q + window<R>(jq[q]), acc[q], w);
}

// Planes [lo, hi) of depth chunk `chunk`: the chunks split the prefix sums
// of the per-plane work estimate (staging plus both blur passes, which grow
// with 2R_i + 1) into equal parts.  A contiguous range keeps each CTA on one
// or two blur widths at a time, so an SM's instruction working set is one or
// two unrolled blur variants rather than all of them.  The prefix sums
// increase, so lo (hi) is the number of planes whose prefix lies below the
// chunk's start (end): counted by the whole CTA, one plane per thread.
// Every thread of the CTA must call this.
__device__ __forceinline__ void chunk_range(const int* __restrict__ work, int n, int chunks, int chunk, int& lo,
                                            int& hi)
{
    const long long total = __ldg(work + n);
    const long long start = total * chunk, end = total * (chunk + 1);
    lo = hi = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const long long v = i < n ? (long long)__ldg(work + i) * chunks : end;
        lo += __syncthreads_count(v < start);
        hi += __syncthreads_count(v < end);
    }
}

// The plane range of depth chunk `chunk`: from the host's boundary table
// (the contiguous split whose heaviest chunk is lightest) when it covers
// this chunk count, else chunk_range.  Every thread of the CTA must call it.
__device__ __forceinline__ void chunk_planes(const int* __restrict__ bounds, const int* __restrict__ work, int n,
                                             int chunks, int chunk, int& lo, int& hi)
{
    if (bounds && chunks <= kBoundChunks) {
        lo = __ldg(bounds + bound_offset(chunks) + chunk);
        hi = __ldg(bounds + bound_offset(chunks) + chunk + 1);
        return;
    }
    chunk_range(work, n, chunks, chunk, lo, hi);
}

#define SPECT_R_CASES(M) \
    M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18) M(19) M(20)

// ---------------------------------------------------------------- forward

// Zero the column pairs of P outside the volume (the z-blur's zero padding)
// and, in every column pair of Q, the row-pair halo outside the rows the
// z-blur writes (the j-blur's zero padding).
__device__ __forceinline__ void zero_pads(float4* P, float4* Q, const PlaneTiling& t, int nz, int kw0)
{
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int wq = (t.ktpad >> 1) + t.rh;  // column pairs of the window
    const int rp = t.npad >> 1, hq = t.rh >> 1;
    for (int idx = threadIdx.x; idx < rp * wq; idx += blockDim.x) {
        const int jp = idx / wq, cq = idx - jp * wq;
        const int k = kw0 + 2 * cq;
        if (k < 0 || k >= nz) P[jp * t.sp + cq] = z4;
    }
    const int qrows = rp + 2 * hq;
    for (int idx = threadIdx.x; idx < (t.ktpad >> 1) * qrows; idx += blockDim.x) {
        const int kp = idx / qrows, r = idx - kp * qrows;
        if (r < hq || r >= hq + rp) Q[kp * t.sq + r] = z4;
    }
}

// Bilinear taps of rotated row (i, j) of one plane, computed once per row
// by one thread and kept in shared memory: element offsets of the four tap
// rows in the volume and their weights.  Taps outside the grid get weight 0
// and offset 0, so every load stays in bounds.
struct TapRow {
    int off[4];
    float w[4];
};

__device__ __forceinline__ void tap_rows(TapRow* rows, int n, int nz, int i, float4 cs, float c)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float u, v;
        sample_point(cs.x, cs.y, c, cs.z, i, j, u, v);
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

// Sources of one rotated row (i, j) from column klo on: the four tap rows of
// the volume, their weights and the attenuation row (global memory, or the
// shared-memory copy of the plane).
struct RowSrc {
    const float* f[4];
    float w[4];
    const float* a;
};

__device__ __forceinline__ RowSrc row_src(const TapRow* rows, int j, const float* xb, const float* arow, int astride,
                                          int aoff, int klo)
{
    RowSrc r;
    const TapRow tr = rows[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        r.f[q] = xb + tr.off[q] + klo;
        r.w[q] = tr.w[q];
    }
    r.a = arow ? arow + (size_t)j * astride + aoff : nullptr;
    return r;
}

// The row's values at columns klo + c and klo + c + 1 (c even).  The first
// product is a plain multiply and the rest fmaf, in tap order, with the
// attenuation applied last, in the same order for every column.
template <bool kSmemA>
__device__ __forceinline__ float2 row_pair_value(const RowSrc& r, int c)
{
    const float2 f0 = __ldg(reinterpret_cast<const float2*>(r.f[0] + c));
    float2 v = make_float2(r.w[0] * f0.x, r.w[0] * f0.y);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        const float2 f = __ldg(reinterpret_cast<const float2*>(r.f[q] + c));
        v = __ffma2_rn(make_float2(r.w[q], r.w[q]), f, v);
    }
    if (r.a) {
        const float2 a = kSmemA ? *reinterpret_cast<const float2*>(r.a + c)
                                : __ldg(reinterpret_cast<const float2*>(r.a + c));
        v = make_float2(v.x * a.x, v.y * a.y);
    }
    return v;
}

// The row's values at columns klo + c .. klo + c + 3 (c a multiple of 4;
// 16-byte aligned loads), each with the arithmetic of row_pair_value.
template <bool kSmemA>
__device__ __forceinline__ float4 row_quad_value(const RowSrc& r, int c)
{
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(r.f[0] + c));
    float2 lo = make_float2(r.w[0] * f0.x, r.w[0] * f0.y), hi = make_float2(r.w[0] * f0.z, r.w[0] * f0.w);
#pragma unroll
    for (int q = 1; q < 4; ++q) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(r.f[q] + c));
        const float2 w = make_float2(r.w[q], r.w[q]);
        lo = __ffma2_rn(w, make_float2(f.x, f.y), lo);
        hi = __ffma2_rn(w, make_float2(f.z, f.w), hi);
    }
    if (r.a) {
        const float4 a = kSmemA ? *reinterpret_cast<const float4*>(r.a + c)
                                : __ldg(reinterpret_cast<const float4*>(r.a + c));
        lo = make_float2(lo.x * a.x, lo.y * a.y);
        hi = make_float2(hi.x * a.z, hi.y * a.w);
    }
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// P quads of every row pair over columns [klo, khi) (both even), from the
// row table: one row pair per warp at a time, lanes on consecutive column
// pairs.  Rows at or past n are zero.  In a partial last pass the column is
// clamped so that the loads stay in bounds; only the stores are masked.
// arow: attenuation of row 0 at column klo is arow[aoff], rows astride apart.
template <bool kSmemA>
__device__ __forceinline__ void stage_plane(float4* P, const PlaneTiling& t, const TapRow* rows,
                                            const float* __restrict__ xb, const float* arow, int astride, int aoff,
                                            int n, int kw0, int klo, int khi)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncols = khi - klo;
    // A row that fits one pass of 16-byte loads (4 columns per lane), with
    // every source row and the attenuation row 16-byte aligned at klo: half
    // the load instructions of the 8-byte path below, the same values.
    const bool wide = ncols <= 128 && (ncols & 3) == 0 && (klo & 3) == 0 && (aoff & 3) == 0 && (astride & 3) == 0;
    if (wide) {
        for (int jp = warp; jp < (t.npad >> 1); jp += nw) {
            float4* prow = P + jp * t.sp + ((klo - kw0) >> 1);
            const int j0 = 2 * jp, j1 = 2 * jp + 1;
            const int c4 = 4 * lane;
            if (j0 >= n) {
                if (c4 < ncols) {
                    prow[c4 >> 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    prow[(c4 >> 1) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                continue;
            }
            const RowSrc r0 = row_src(rows, j0, xb, arow, astride, aoff, klo);
            const RowSrc r1 = row_src(rows, j1 < n ? j1 : j0, xb, arow, astride, aoff, klo);
            const int x4 = min(c4, ncols - 4);
            const float4 v0 = row_quad_value<kSmemA>(r0, x4);
            float4 v1 = row_quad_value<kSmemA>(r1, x4);
            if (j1 >= n) v1 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c4 < ncols) {
                prow[c4 >> 1] = make_float4(v0.x, v1.x, v0.y, v1.y);
                prow[(c4 >> 1) + 1] = make_float4(v0.z, v1.z, v0.w, v1.w);
            }
        }
        return;
    }
    for (int jp = warp; jp < (t.npad >> 1); jp += nw) {
        float4* prow = P + jp * t.sp + ((klo - kw0) >> 1);
        const int j0 = 2 * jp, j1 = 2 * jp + 1;
        if (j0 >= n) {
            for (int c = 2 * lane; c < ncols; c += 64) prow[c >> 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const RowSrc r0 = row_src(rows, j0, xb, arow, astride, aoff, klo);
        const RowSrc r1 = row_src(rows, j1 < n ? j1 : j0, xb, arow, astride, aoff, klo);
        // two 64-column passes at a time, so that all their loads are in
        // flight together
        for (int c0 = 0; c0 < ncols; c0 += 128) {
            const int ca = c0 + 2 * lane, cb = ca + 64;
            const int xa = min(ca, ncols - 2), xbb = min(cb, ncols - 2);
            const float2 a0 = row_pair_value<kSmemA>(r0, xa), b0 = row_pair_value<kSmemA>(r0, xbb);
            float2 a1 = row_pair_value<kSmemA>(r1, xa), b1 = row_pair_value<kSmemA>(r1, xbb);
            if (j1 >= n) a1 = b1 = make_float2(0.f, 0.f);
            if (ca < ncols) prow[ca >> 1] = make_float4(a0.x, a1.x, a0.y, a1.y);
            if (cb < ncols) prow[cb >> 1] = make_float4(b0.x, b1.x, b0.y, b1.y);
        }
    }
}

// Thread 0: bulk copies of the rows of one attenuation plane, columns
// [a_lo, a_lo + a_cols) (a_lo and a_cols multiples of 4, so every copy is
// 16-byte aligned and a multiple of 16 bytes), into `buf` (row stride
// a_cols), completing on `bar`.
__device__ __forceinline__ void load_atten_plane(uint32_t buf, const float* plane, int n, int nz, int a_lo, int a_cols,
                                                 uint32_t bar)
{
    const uint32_t row_bytes = (uint32_t)a_cols * 4u;
    mbar_expect_tx(bar, row_bytes * (uint32_t)n);
    if (a_lo == 0 && a_cols == nz) {
        bulk_load(buf, plane, row_bytes * (uint32_t)n, bar);
    } else {
        for (int j = 0; j < n; ++j) bulk_load(buf + (uint32_t)j * row_bytes, plane + (size_t)j * nz + a_lo, row_bytes, bar);
    }
}

template <int IPT>
__global__ void __launch_bounds__(kFwdThreads, 1) forward_kernel(ForwardArgs a)
{
    extern __shared__ __align__(16) float4 smem4[];
    const PlaneTiling& t = a.t;
    const int n = a.n, nz = a.nz;
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
    float4* P = smem4;
    float4* Q = P + (size_t)(t.npad >> 1) * t.sp;
    TapRow* rows = reinterpret_cast<TapRow*>(Q + (size_t)(t.ktpad >> 1) * t.sq);
    float* taps_s = reinterpret_cast<float*>(sm + t.off_taps_f);  // [2][kMaxR + 1]
    const int tid = threadIdx.x;
    const int chunk = blockIdx.x % a.chunks, tile = blockIdx.x / a.chunks;
    const int sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    // this angle's PSF tables (a non-circular orbit has one per angle)
    const float* taps_g = a.taps + (size_t)angle * a.taps_stride;
    const int* rad_g = a.rad + (size_t)angle * a.rad_stride;
    const int* work_g = a.work + (size_t)angle * a.rad_stride;
    const int* bounds_g = a.bounds ? a.bounds + (size_t)angle * a.rad_stride : nullptr;
    const float4 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const int kt0 = tile * t.ktile;
    const int KT = min(t.ktile, nz - kt0);
    const int kw0 = kt0 - t.rh;
    const int W = t.ktpad + 2 * t.rh;
    const int klo = max(0, kw0), khi = min(nz, kw0 + W);
    const float* aplane = a.atten ? a.atten + (size_t)angle * n * n * nz : nullptr;
    // attenuation planes through shared memory when the buffer fits
    const bool abuf = aplane && t.a_cols_f > 0;
    const int a_lo = klo & ~3, a_cols = min(nz, (khi + 3) & ~3) - a_lo;
    float* As = reinterpret_cast<float*>(sm + t.off_a_f);
    const uint32_t bar = smem_u32(sm + t.off_bar_f);

    zero_pads(P, Q, t, nz, kw0);
    if (abuf && tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }

    // this thread's blur items, fixed for the whole depth loop
    const ZItem z0 = z_item(t, tid);
    int jq[IPT];
#pragma unroll
    for (int q = 0; q < IPT; ++q) jq[q] = j_item(t, tid + q * blockDim.x);

    float2 acc[IPT][kStrip];
#pragma unroll
    for (int q = 0; q < IPT; ++q)
#pragma unroll
        for (int r = 0; r < kStrip; ++r) acc[q][r] = make_float2(0.f, 0.f);

    const float* xb = a.x + (size_t)b * n * n * nz;
    int i_lo, i_hi;
    chunk_planes(bounds_g, work_g, n, a.chunks, chunk, i_lo, i_hi);
    TapPrefetch tp;
    if (i_lo < i_hi) {
        tp.load(taps_g, i_lo);
        tp.store(taps_s, i_lo);  // visible after the first barrier below
    }
    __syncthreads();  // barrier initialised
    if (abuf && tid == 0 && i_lo < i_hi)
        load_atten_plane(smem_u32(As), aplane + (size_t)i_lo * n * nz, n, nz, a_lo, a_cols, bar);
    uint32_t parity = 0;
    bool timed_out = false;
    for (int i = i_lo; i < i_hi; ++i) {
        if (i + 1 < i_hi) {
            tp.load(taps_g, i + 1);
            if (aplane && !abuf) prefetch_plane_l2(aplane + (size_t)(i + 1) * n * nz, n, nz, klo, khi);
        }
        // ---- stage the rotated, attenuated plane (T_rot, T_att)
        tap_rows(rows, n, nz, i, cs, c);
        bool ok = true;
        if (abuf) {
            ok = mbar_wait(bar, parity);  // A_i has landed
            parity ^= 1;
        }
        if (!sync_ok(ok, a.err)) {
            timed_out = true;
            break;
        }
        if (abuf)
            stage_plane<true>(P, t, rows, xb, As, a_cols, klo - a_lo, n, kw0, klo, khi);
        else
            stage_plane<false>(P, t, rows, xb, aplane ? aplane + (size_t)i * n * nz : nullptr, nz, klo, n, kw0, klo,
                               khi);
        __syncthreads();
        // every read of A_i is done: fetch A_{i+1} behind the blur
        if (abuf && tid == 0 && i + 1 < i_hi) {
            fence_async_smem();
            load_atten_plane(smem_u32(As), aplane + (size_t)(i + 1) * n * nz, n, nz, a_lo, a_cols, bar);
        }
        // ---- blur along z and y, accumulate over depth (T_cdr, P_x)
        const float* trow = taps_s + (i & 1) * (kMaxR + 1);
        switch (__ldg(rad_g + i)) {
#define SPECT_FWD_CASE(RR) \
    case RR: fwd_blur_plane<RR, IPT>(P, Q, t, z0, jq, trow, acc); break;
            SPECT_R_CASES(SPECT_FWD_CASE)
#undef SPECT_FWD_CASE
            default: break;
        }
        // The next plane's taps go to the other half of taps_s, last read
        // before this plane's second barrier.  The next staging writes P and
        // the row table only; Q is rewritten after the next two barriers,
        // which every thread reaches after its j-blur above.
        if (i + 1 < i_hi) tp.store(taps_s, i + 1);
    }
    // after a timed-out wait, give the copy in flight one more bounded wait
    // before the CTA (and its shared memory) goes away
    if (timed_out) mbar_wait(bar, parity ^ 1);

    // Raw depth sums of this chunk: to the output when the chunk is the
    // whole depth and no ratio is wanted, else to the partial planes.
    const size_t item = (size_t)b * a.n_sel + sidx;
    float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
    const int cp = t.ktpad >> 1;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int it = tid + q * blockDim.x;
        if (jq[q] >= 0) {
            const int kk = 2 * (it % cp), js = it / cp;
            if (kk < KT) {
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n) *reinterpret_cast<float2*>(dst + (size_t)j * nz + kt0 + kk) = acc[q][r];
                }
            }
        }
    }
}

// ---------------------------------------------------------------- back: blur

// One plane of the back blur: z-blur of the staged projection into Q, then
// the j-blur strips, each multiplied by A_i and stored.  A_i comes from the
// shared buffer (kSmemA: As, after waiting on `bar` with `parity`) or from
// global memory (aglob, or no attenuation when it is null).  Returns false
// when the wait timed out.
template <int R, int IPT, bool kSmemA>
__device__ __forceinline__ bool back_blur_plane(const float4* P, float4* Q, const PlaneTiling& t,
                                                const BlurBackArgs& a, const ZItem& z0, const float* taps_row, int i,
                                                const float* aglob, const float* As, uint32_t bar, uint32_t parity,
                                                int kt0, int KT, float* __restrict__ bvol)
{
    const int n = a.n, nz = a.nz;
    const int cp = t.ktpad >> 1;
    float2 w[R + 1];
    load_taps<R>(taps_row, w);
    zblur_plane<R>(P, Q, t, z0, w);
    __syncthreads();
    float* __restrict__ brow = bvol + (size_t)i * n * nz;
    // A_i was requested when the previous plane ended; the z-blur covered it
    const bool ok = kSmemA ? mbar_wait(bar, parity) : true;
    // rolled loop over this thread's strips: one copy of the unrolled j-blur
#pragma unroll 1
    for (int it = threadIdx.x; it < cp * (t.npad / kStrip); it += blockDim.x) {
        const int kk = 2 * (it % cp), js = it / cp;
        float2 o[kStrip];
#pragma unroll
        for (int r = 0; r < kStrip; ++r) o[r] = make_float2(0.f, 0.f);
        blur_pairs<R>(Q + window<R>(j_item(t, it)), o, w);
        if (kk < KT) {
            const int k = kt0 + kk;
            if (kSmemA) {
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n) {
                        const float2 av = *reinterpret_cast<const float2*>(As + (size_t)j * KT + kk);
                        *reinterpret_cast<float2*>(brow + (size_t)j * nz + k) = make_float2(o[r].x * av.x, o[r].y * av.y);
                    }
                }
            } else {
                // all attenuation loads of the strip first, then the stores
                float2 aw[kStrip];
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    aw[r] = (aglob && j < n) ? __ldg(reinterpret_cast<const float2*>(aglob + (size_t)j * nz + k))
                                             : make_float2(1.f, 1.f);
                }
#pragma unroll
                for (int r = 0; r < kStrip; ++r) {
                    const int j = js * kStrip + r;
                    if (j < n)
                        *reinterpret_cast<float2*>(brow + (size_t)j * nz + k) =
                            make_float2(o[r].x * aw[r].x, o[r].y * aw[r].y);
                }
            }
        }
    }
    return ok;
}

template <int IPT, bool kSmemA>
__global__ void __launch_bounds__(kFwdThreads, 1) blur_back_kernel(BlurBackArgs a)
{
    extern __shared__ __align__(16) float4 smem4[];
    const PlaneTiling& t = a.t;
    const int n = a.n, nz = a.nz;
    unsigned char* sm = reinterpret_cast<unsigned char*>(smem4);
    float4* P = smem4;
    float4* Q = P + (size_t)(t.npad >> 1) * t.sp;
    float* taps_s = reinterpret_cast<float*>(sm + t.off_taps_b);  // [2][kMaxR + 1]
    const int tid = threadIdx.x;
    const int chunk = blockIdx.x % a.chunks, tile = blockIdx.x / a.chunks;
    const int sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    // this angle's PSF tables (a non-circular orbit has one per angle)
    const float* taps_g = a.taps + (size_t)angle * a.taps_stride;
    const int* rad_g = a.rad + (size_t)angle * a.rad_stride;
    const int* work_g = a.work + (size_t)angle * a.rad_stride;
    const int* bounds_g = a.bounds ? a.bounds + (size_t)angle * a.rad_stride : nullptr;
    const int kt0 = tile * t.ktile;
    const int KT = min(t.ktile, nz - kt0);
    const int kw0 = kt0 - t.rh;
    const int W = t.ktpad + 2 * t.rh;
    const int klo = max(0, kw0), khi = min(nz, kw0 + W);
    const size_t item = (size_t)b * a.n_sel + sidx;
    const float* aplane = a.atten ? a.atten + (size_t)angle * n * n * nz : nullptr;
    // attenuation planes (the tile's columns) through shared memory when the
    // buffer fits (the launcher picks kSmemA = atten && a_cols_b > 0)
    constexpr bool abuf = kSmemA;
    float* As = reinterpret_cast<float*>(sm + t.off_a_b);
    const uint32_t bar = smem_u32(sm + t.off_bar_b);

    // The projection window of this angle (all ones without a projection),
    // times the angle's T_fov weights when the plan has them, zero outside
    // the detector.
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    const float* fv = a.fov ? a.fov + (size_t)angle * n * nz : nullptr;
    zero_pads(P, Q, t, nz, kw0);
    {
        // one quad (two rows, two columns) per item; four items of a thread
        // load together
        const int ncp = (khi - klo) >> 1, items = (t.npad >> 1) * ncp;
        for (int it0 = 0; it0 < items; it0 += 4 * blockDim.x) {
            float2 v[4][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = it0 + u * blockDim.x + tid;
                const int jp = it / max(ncp, 1), cq = it - jp * ncp;
                const int k = klo + 2 * cq;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * jp + h;
                    v[u][h] = make_float2(0.f, 0.f);
                    if (it < items && j < n)
                        v[u][h] = pr ? __ldg(reinterpret_cast<const float2*>(pr + (size_t)j * nz + k)) : make_float2(1.f, 1.f);
                }
            }
            if (fv) {  // T_fov weights of the same elements, loaded together
                float2 m[4][2];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int it = it0 + u * blockDim.x + tid;
                    const int jp = it / max(ncp, 1), cq = it - jp * ncp;
                    const int k = klo + 2 * cq;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = 2 * jp + h;
                        m[u][h] = (it < items && j < n) ? __ldg(reinterpret_cast<const float2*>(fv + (size_t)j * nz + k))
                                                        : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int h = 0; h < 2; ++h) v[u][h] = make_float2(v[u][h].x * m[u][h].x, v[u][h].y * m[u][h].y);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int it = it0 + u * blockDim.x + tid;
                if (it < items) {
                    const int jp = it / ncp, cq = it - jp * ncp;
                    P[jp * t.sp + ((klo - kw0) >> 1) + cq] = make_float4(v[u][0].x, v[u][1].x, v[u][0].y, v[u][1].y);
                }
            }
        }
    }
    int i_lo, i_hi;
    chunk_planes(bounds_g, work_g, n, a.chunks, chunk, i_lo, i_hi);
    TapPrefetch tp;
    if (i_lo < i_hi) {
        tp.load(taps_g, i_lo);
        tp.store(taps_s, i_lo);
    }
    if (abuf && tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    if (aplane && !abuf && i_lo < i_hi) prefetch_plane_l2(aplane + (size_t)i_lo * n * nz, n, nz, kt0, kt0 + KT);
    __syncthreads();
    if (abuf && tid == 0 && i_lo < i_hi)
        load_atten_plane(smem_u32(As), aplane + (size_t)i_lo * n * nz, n, nz, kt0, KT, bar);
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const ZItem z0 = z_item(t, tid);
    uint32_t parity = 0;
    bool timed_out = false;
    for (int i = i_lo; i < i_hi; ++i) {
        if (i + 1 < i_hi) {
            tp.load(taps_g, i + 1);
            if (aplane && !abuf) prefetch_plane_l2(aplane + (size_t)(i + 1) * n * nz, n, nz, kt0, kt0 + KT);
        }
        const float* trow = taps_s + (i & 1) * (kMaxR + 1);
        const float* aglob = aplane ? aplane + (size_t)i * n * nz : nullptr;
        bool ok = true;
        switch (__ldg(rad_g + i)) {
#define SPECT_BACK_CASE(RR) \
    case RR: ok = back_blur_plane<RR, IPT, kSmemA>(P, Q, t, a, z0, trow, i, aglob, As, bar, parity, kt0, KT, bvol); break;
            SPECT_R_CASES(SPECT_BACK_CASE)
#undef SPECT_BACK_CASE
            default: break;
        }
        // the next plane's taps go to the half of taps_s read one plane ago
        if (i + 1 < i_hi) tp.store(taps_s, i + 1);
        // Q is rewritten by the next plane's z-blur; A_i has been read
        if (!sync_ok(ok, a.err)) {
            timed_out = true;
            break;
        }
        if (abuf) {
            parity ^= 1;
            if (tid == 0 && i + 1 < i_hi) {
                fence_async_smem();
                load_atten_plane(smem_u32(As), aplane + (size_t)(i + 1) * n * nz, n, nz, kt0, KT, bar);
            }
        }
    }
    // after a timed-out wait, give the copy in flight one more bounded wait
    // before the CTA (and its shared memory) goes away
    if (abuf && timed_out) mbar_wait(bar, parity);
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
template <int IPT, bool kSmemA>
unsigned long long g_blur_back_smem_mask = 0;

template <int IPT>
cudaError_t forward_launch_ipt(const ForwardArgs& a, int grid_x, cudaStream_t st)
{
    cudaError_t e = allow_big_smem(forward_kernel<IPT>, g_forward_smem_mask<IPT>);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    forward_kernel<IPT><<<grid, a.t.threads, a.t.smem_f, st>>>(a);
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

template <int IPT, bool kSmemA>
cudaError_t blur_back_launch_variant(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    cudaError_t e = allow_big_smem(blur_back_kernel<IPT, kSmemA>, g_blur_back_smem_mask<IPT, kSmemA>);
    if (e != cudaSuccess) return e;
    dim3 grid(grid_x, a.n_sel, a.batch);
    blur_back_kernel<IPT, kSmemA><<<grid, a.t.threads, a.t.smem_b, st>>>(a);
    return cudaGetLastError();
}

template <int IPT>
cudaError_t blur_back_launch_ipt(const BlurBackArgs& a, int grid_x, cudaStream_t st)
{
    if (a.atten && a.t.a_cols_b > 0) return blur_back_launch_variant<IPT, true>(a, grid_x, st);
    return blur_back_launch_variant<IPT, false>(a, grid_x, st);
}

}  // namespace spect
