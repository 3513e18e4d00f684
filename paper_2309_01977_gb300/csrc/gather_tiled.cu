// Transpose of the bilinear rotation (T_rot^T of Eq. 1), tiled: the sums of
// gather_kernel, with the rotated-frame rows that a tile of output columns
// needs staged in shared memory by bulk copies.
//
// Output columns q = (x, y) are grouped in 8 x 8 tiles.  For angle a, the
// footprint of a tile is the set of rotated-frame rows p = (i, j) with a
// nonzero bilinear weight toward some column of the tile; for each i it is
// held as the whole run j in [jlo_i, jlo_i + len_i), which is contiguous in
// the rotated-frame volume B_a[i][j][z].  The plan stores, per (angle,
// tile):
//   a descriptor  {i0, ni, rows} and (jlo_i, len_i) for i = i0 .. i0+ni-1;
//   per row y of the tile, the footprint samples whose weights reach it, in
//   lists by the column of their lower weight, each entry {row of the
//   footprint in its shared-memory copy, weight to that column, weight to
//   the next}.  The weights are the products gather_kernel's table forms
//   (recomputed by the forward's own arithmetic); a sample is read from
//   shared memory once per tile row and added to both its columns, half the
//   reads of a per-column walk.  Each column's sum runs over its samples in
//   list order (row-major within a list), so it differs from gather_kernel's
//   by the rounding of the summation order only.
// The gather CTA of (tile, z segment, batch entry) walks the subset's
// angles through `stages` footprint buffers: while it sums angle g, the
// bulk copies of the next angles fill the other buffers.  Every wait is
// bounded.
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "geometry.cuh"
#include "internal.h"
#include "update.cuh"

namespace spect {

// ---------------------------------------------------------------- tables

// One CTA per (tile, angle): first one thread per column of the tile (the
// footprint), then one per strip list.
__global__ void gather_tiled_table_kernel(const float4* __restrict__ cs_tab, int n, int nz, int T, int tiles_x,
                                          int2* __restrict__ tab, int* __restrict__ desc, int* __restrict__ rows_max,
                                          int* __restrict__ err)
{
    __shared__ int s_imin, s_imax;
    __shared__ int s_jlo[kFpMaxRows], s_jhi[kFpMaxRows], s_off[kFpMaxRows];
    const int tile = blockIdx.x, angle = blockIdx.y;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int cl = threadIdx.x;
    const int x = tx * T + cl / T, y = ty * T + cl % T;
    const bool live = cl < T * T && x < n && y < n;
    if (threadIdx.x == 0) {
        s_imin = 1 << 30;
        s_imax = -1;
    }
    for (int r = threadIdx.x; r < kFpMaxRows; r += blockDim.x) {
        s_jlo[r] = 1 << 30;
        s_jhi[r] = -1;
    }
    __syncthreads();

    // candidates of this column, enumerated exactly as gather_table_kernel
    int ci[kMaxCand], cj[kMaxCand];
    int count = 0;
    if (live) {
        const float c = 0.5f * (float)(n - 1);
        const float4 cs = cs_tab[angle];
        const float dx = (float)x - c, dy = (float)y - c;
        const float pi = c + cs.x * dx + cs.y * dy;
        const float pj = cs.z - cs.y * dx + cs.x * dy;
        const float ext = fabsf(cs.x) + fabsf(cs.y) + 1e-3f;
        const int ia = max(0, (int)ceilf(pi - ext)), ib = min(n - 1, (int)floorf(pi + ext));
        const int ja = max(0, (int)ceilf(pj - ext)), jb = min(n - 1, (int)floorf(pj + ext));
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
                    ci[count] = i;
                    cj[count] = j;
                    ++count;
                }
            }
    }
    for (int e = 0; e < count; ++e) {
        atomicMin(&s_imin, ci[e]);
        atomicMax(&s_imax, ci[e]);
    }
    __syncthreads();
    const int i0 = s_imin <= s_imax ? s_imin : 0;
    const int ni = s_imin <= s_imax ? s_imax - s_imin + 1 : 0;
    const bool fits = ni <= kFpMaxRows;
    for (int e = 0; e < count && fits; ++e) {
        atomicMin(&s_jlo[ci[e] - i0], cj[e]);
        atomicMax(&s_jhi[ci[e] - i0], cj[e]);
    }
    __syncthreads();
    int* d = desc + ((size_t)angle * gridDim.x + tile) * kFpDescInts;
    if (threadIdx.x == 0) {
        int rows = 0;
        for (int r = 0; r < (fits ? ni : 0); ++r) {
            const int len = s_jhi[r] >= s_jlo[r] ? s_jhi[r] - s_jlo[r] + 1 : 0;
            s_off[r] = rows;
            d[4 + 2 * r] = len ? s_jlo[r] : 0;
            d[5 + 2 * r] = len;
            rows += len;
        }
        d[0] = i0;
        d[1] = fits ? ni : 0;
        d[2] = rows;
        d[3] = 0;
        atomicMax(rows_max, rows);
        if (!fits) atomicExch(err, SPECT_EINVAL);
    }
    __syncthreads();
    // Strip lists: thread (w, l) of the first kGtT * kGtLists builds list l
    // of tile row w, the footprint's samples (i, j) in row-major order whose
    // lower bilinear column is xa = tx T + l - 1 and whose rows ya, ya + 1
    // include the tile row y: weights (1 - ax) wy to column xa and ax wy to
    // xa + 1, each the product gather_kernel's table forms (zero where the
    // column lies outside the tile or the volume).  Entries go to the list's
    // kGtMaxList slots as they are found; a longer list is reported and the
    // plan takes the per-column gather.
    const int lt = threadIdx.x;
    const bool lister = fits && lt < kGtT * kGtLists;
    const int w = lt / kGtLists, l = lt % kGtLists;
    const int yr = ty * T + w, xa_l = tx * T + l - 1;
    auto walk = [&](int2* __restrict__ out) {
        int count = 0;
        if (!lister || yr >= n) return 0;
        const float c = 0.5f * (float)(n - 1);
        const float4 cs = cs_tab[angle];
        for (int r = 0; r < ni; ++r) {
            if (s_jhi[r] < s_jlo[r]) continue;
            for (int j = s_jlo[r]; j <= s_jhi[r]; ++j) {
                float u, v;
                sample_point(cs.x, cs.y, c, cs.z, i0 + r, j, u, v);
                const float fu = floorf(u), fv = floorf(v);
                const int xa = (int)fu, ya = (int)fv;
                if (xa != xa_l) continue;
                const float ax = u - fu, by = v - fv;
                const float wy = (yr == ya) ? (1.f - by) : (yr == ya + 1 ? by : 0.f);
                if (wy == 0.f) continue;
                const float w0 = (l >= 1 && xa < n) ? (1.f - ax) * wy : 0.f;
                const float w1 = (l + 1 <= T && xa + 1 < n) ? ax * wy : 0.f;
                if (w0 == 0.f && w1 == 0.f) continue;
                if (count < kGtMaxList) {
                    out[2 * count] = make_int2(s_off[r] + j - s_jlo[r], __float_as_int(w0));
                    out[2 * count + 1] = make_int2(__float_as_int(w1), 0);
                }
                ++count;
            }
        }
        return count;
    };
    int* hdr = reinterpret_cast<int*>(tab) + ((size_t)angle * gridDim.x + tile) * (kGtSliceBytes / 4);
    int2* ent = reinterpret_cast<int2*>(hdr + kGtT * kGtHdr);
    if (lister) {
        const int cnt = walk(ent + 2 * (size_t)kGtMaxList * (w * kGtLists + l));
        if (cnt > kGtMaxList) atomicExch(err, SPECT_EINVAL);
        hdr[w * kGtHdr + l] = min(cnt, kGtMaxList);
    }
}

cudaError_t launch_gather_tiled_tables(const float4* cs, int n, int nz, int n_angles, int T, int2* tab, int* desc,
                                       int* rows_max, int* err, cudaStream_t st)
{
    const int tiles_x = (n + T - 1) / T;
    dim3 grid(tiles_x * tiles_x, n_angles);
    if (T != kGtT) return cudaErrorInvalidValue;
    gather_tiled_table_kernel<<<grid, ((kGtT * kGtLists + 31) / 32) * 32, 0, st>>>(cs, n, nz, T, tiles_x, tab, desc, rows_max,
                                                                          err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gather

namespace {

// The footprint descriptor of one (angle, tile), as the issuing warp holds
// it: every lane the header, lane l the run of footprint row l
// (kFpMaxRows = 32, so one row per lane covers every footprint).  Read from
// the CTA's shared-memory copy of its descriptors.
struct Footprint {
    int i0, ni, rows;  // first rotated row, rows i, footprint rows in all
    int jlo, len;      // this lane's row: first j and length of its run
};

__device__ __forceinline__ Footprint read_footprint(const int* d)
{
    const int lane = threadIdx.x & 31;
    Footprint f;
    f.i0 = d[0];
    f.ni = d[1];
    f.rows = d[2];
    // in bounds for every lane (kFpDescInts = 4 + 2 * 32); rows past ni are
    // ignored at the copies
    f.jlo = d[4 + 2 * lane];
    f.len = d[5 + 2 * lane];
    return f;
}

// The issuing warp fills buffer `buf` for one angle: lane 0 announces the bytes on
// `bar` and copies the tile's table slice (after the footprint rows, at row
// rows_cap); lane l copies footprint row-run l.  zs == nz: one copy per run
// of rows (contiguous); else one copy per row of the z segment
// [z0, z0 + zs).
__device__ __forceinline__ void issue_footprint(const GatherTiledArgs& a, const Footprint& f,
                                                const int2* __restrict__ tab, const float* __restrict__ bslot,
                                                uint32_t buf, uint32_t bar)
{
    const int lane = threadIdx.x & 31;
    const int z0 = blockIdx.z * a.zs;
    const uint32_t row_bytes = (uint32_t)a.zs * 4u;
    const uint32_t tab_bytes = (uint32_t)kGtSliceBytes;
    if (lane == 0) {
        mbar_expect_tx(bar, (uint32_t)f.rows * row_bytes + tab_bytes);
        bulk_load(buf + (uint32_t)a.rows_cap * row_bytes, tab, tab_bytes, bar);
    }
    __syncwarp();
    // offset of this lane's run: exclusive prefix of the lengths over the warp
    const int len = lane < f.ni ? f.len : 0;
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int start = incl - len;
    if (len > 0) {
        const float* src = bslot + ((size_t)(f.i0 + lane) * a.n + f.jlo) * a.nz + z0;
        if (a.zs == a.nz) {
            bulk_load(buf + (uint32_t)start * row_bytes, src, (uint32_t)len * row_bytes, bar);
        } else {
            for (int q = 0; q < len; ++q)
                bulk_load(buf + (uint32_t)(start + q) * row_bytes, src + (size_t)q * a.nz, row_bytes, bar);
        }
    }
}

}  // namespace

// a4 += w v, two packed FMAs.
__device__ __forceinline__ void fma4(float4& a4, float w, const float4& v)
{
    const float2 lo = __ffma2_rn(make_float2(w, w), make_float2(v.x, v.y), make_float2(a4.x, a4.y));
    const float2 hi = __ffma2_rn(make_float2(w, w), make_float2(v.z, v.w), make_float2(a4.z, a4.w));
    a4 = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// 288 threads: warp w < 8 owns row w of the 8 x 8 tile (columns x = 8 tx +
// k, y = 8 ty + w, k = 0 .. 7, in accumulators acc[k]), lane l holding
// float4 l of the z segment (lanes past zs/4 idle); warp 8 issues the
// footprint copies (about a dozen bulk copies an angle, which take about as
// long to issue as an angle's sums), so that they overlap the sums.  Two
// CTAs per SM (their shared memory allows two; 18 warps cap the registers
// at 96).
template <int T>
__global__ void __launch_bounds__(kGatherTiledThreads, 2) gather_tiled_kernel(GatherTiledArgs a)
{
    static_assert(T == kGtT, "strip tables are built for 8 x 8 tiles");
    extern __shared__ __align__(16) float4 gsm[];
    const int tile = blockIdx.x, b = blockIdx.y;
    const int tiles_x = (a.n + T - 1) / T;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == kGatherSumWarps;
    const int zw = a.zs >> 2;  // float4 per row segment
    const int z0 = blockIdx.z * a.zs;
    const size_t vol = (size_t)a.n * a.n * a.nz;
    constexpr int ncols = T * T;
    constexpr int kCols = (ncols + 7) / 8;  // columns per warp
    const size_t buf_f4 = (size_t)a.rows_cap * zw + kGtSliceBytes / 16;  // rows, then the strip table
    const int S = a.stages;  // footprint buffers: angle g uses buffer g % S
    // shared memory: S footprint buffers, S + 1 mbarriers (the buffers',
    // then the descriptors'), the CTA's footprint descriptors and angle ids
    float4* bufs = gsm;
    uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + S * buf_f4);
    int* sdesc = reinterpret_cast<int*>(gsm + S * buf_f4 + (S + 2) / 2);
    int* s_sel = sdesc + a.n_sel * kFpDescInts;
    const float* bvol_b = a.bvol + (size_t)b * a.n_sel * vol;
    const size_t tab_stride = (size_t)a.n_tiles * (kGtSliceBytes / 8);  // int2 per angle

    if (threadIdx.x == 0) {
        for (int q = 0; q <= S; ++q) mbar_init(smem_u32(bars + q), 1);
        mbar_init_fence();
    }
    __syncthreads();
    // The producer warp copies the CTA's descriptors (one per angle of the
    // group, lane g the one of angle g; n_sel <= 32, checked at launch) into
    // shared memory, then issues the first footprints.
    auto issue = [&](int g) {
        const int q = g % S;
        issue_footprint(a, read_footprint(sdesc + g * kFpDescInts),
                        a.tab + (size_t)s_sel[g] * tab_stride + (size_t)tile * (kGtSliceBytes / 8),
                        bvol_b + (size_t)g * vol, smem_u32(bufs + q * buf_f4), smem_u32(bars + q));
    };
    bool desc_ok = true;
    if (producer) {
        const uint32_t dbar = smem_u32(bars + S);
        if (lane == 0) mbar_expect_tx(dbar, (uint32_t)a.n_sel * kFpDescInts * 4u);
        __syncwarp();
        if (lane < a.n_sel) {
            const int ag = __ldg(a.sel + lane);
            s_sel[lane] = ag;
            bulk_load(smem_u32(sdesc + lane * kFpDescInts), a.desc + ((size_t)ag * a.n_tiles + tile) * kFpDescInts,
                      kFpDescInts * 4u, dbar);
        }
        desc_ok = mbar_wait(dbar, 0);
        __syncwarp();
        if (desc_ok)
            for (int g = 0; g < S - 1 && g < a.n_sel; ++g) issue(g);
    }

    float4 acc[kCols];
#pragma unroll
    for (int k = 0; k < kCols; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = true;
    int g = 0;
    for (; g < a.n_sel; ++g) {
        // buffer (g + S - 1) % S was last read by angle g - 1, before the
        // barrier that ended it
        if (producer && desc_ok && g + S - 1 < a.n_sel) {
            fence_async_smem();
            issue(g + S - 1);
        }
        const int q = g % S;
        const bool landed = producer ? desc_ok : mbar_wait(smem_u32(bars + q), (uint32_t)((g / S) & 1));
        const float4* buf = bufs + q * buf_f4;
        const float4* tabs = buf + (size_t)a.rows_cap * zw;
        if (!producer && landed && lane < zw) {
            // This warp's tile row, list by list: list l holds the samples
            // whose lower column is l - 1, each read once and added to
            // columns l - 1 and l.
            const int* hdr = reinterpret_cast<const int*>(tabs) + warp * kGtHdr;
            const int4* ent = reinterpret_cast<const int4*>(reinterpret_cast<const int*>(tabs) + kGtT * kGtHdr) +
                              warp * (kGtLists * kGtMaxList);
            // Fixed slots, filled under a predicate: the loads of different
            // slots are independent, so many are in flight at once.  The
            // list lengths and footprint rows come from the plan's tables;
            // one outside its buffer is reported (SPECT_EINVAL) and skipped
            // rather than read.
            bool bad = false;
#pragma unroll
            for (int l = 0; l < kGtLists; ++l) {
                const int cnt = hdr[l];
                bad |= cnt > kGtMaxList;
#pragma unroll
                for (int k = 0; k < kGtMaxList; ++k) {
                    if (k >= cnt) continue;
                    const int4 en = ent[l * kGtMaxList + k];
                    if ((unsigned)en.x >= (unsigned)a.rows_cap) {
                        bad = true;
                        continue;
                    }
                    const float4 v = buf[(size_t)en.x * zw + lane];
                    if (l >= 1) fma4(acc[l - 1], __int_as_float(en.y), v);
                    if (l < kGtT) fma4(acc[l], __int_as_float(en.z), v);
                }
            }
            if (bad) atomicExch(a.err, SPECT_EINVAL);
        }
        ok = __syncthreads_and(landed);  // and buffer q is free for angle g + S
        if (!ok) break;
    }
    if (!ok) {
        // a timed-out wait: record it, and give the copies in flight (angles
        // g .. g + S - 2) one more bounded wait before the CTA's shared memory
        // goes away
        if (threadIdx.x == 0) atomicExch(a.err, SPECT_ETIMEDOUT);
        for (int h = g; h < g + S - 1 && h < a.n_sel; ++h) mbar_wait(smem_u32(bars + h % S), (uint32_t)((h / S) & 1));
        return;
    }

    // epilogue: store, accumulate, or the fused OSEM update.  The image
    // values and sensitivities of kEpi columns are loaded before any of their
    // stores: in program order a store could alias the next column's loads,
    // and each column would wait out its own memory round trip.
    if (producer) return;
    constexpr int kEpi = kCols < 4 ? kCols : 4;
    const bool upd = a.upd.mode != kUpdNone;
    const bool need_x = upd || a.accumulate;
    float4* out_b = reinterpret_cast<float4*>(a.out + (size_t)b * vol);
#pragma unroll
    for (int k0 = 0; k0 < kCols; k0 += kEpi) {
        float4 xv[kEpi], sv[kEpi];
        size_t i4[kEpi];
        bool live[kEpi];
#pragma unroll
        for (int u = 0; u < kEpi; ++u) {
            const int cl = warp + 8 * (k0 + u);
            const int x = tx * T + cl / T, y = ty * T + cl % T;
            live[u] = cl < ncols && x < a.n && y < a.n && lane < zw;
            i4[u] = ((((size_t)x * a.n + y) * a.nz + z0) >> 2) + lane;  // float4 of the volume
            xv[u] = sv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live[u] && need_x) xv[u] = out_b[i4[u]];
            if (live[u] && upd) sv[u] = __ldg(reinterpret_cast<const float4*>(a.upd.sens) + i4[u]);
        }
#pragma unroll
        for (int u = 0; u < kEpi; ++u) {
            if (!live[u]) continue;
            const float4 s4 = acc[k0 + u];
            if (upd)
                out_b[i4[u]] = update4_sv(a.upd, xv[u], s4, sv[u], i4[u]);
            else if (a.accumulate)
                out_b[i4[u]] = make_float4(xv[u].x + s4.x, xv[u].y + s4.y, xv[u].z + s4.z, xv[u].w + s4.w);
            else
                out_b[i4[u]] = s4;
        }
    }
}

size_t gather_tiled_smem(int rows_cap, int zs, int T, int stages, int n_sel)
{
    const size_t bufs = stages * ((size_t)rows_cap * zs * sizeof(float) + (size_t)kGtSliceBytes);
    const size_t bars = 16 * (size_t)((stages + 2) / 2);
    return bufs + bars + (size_t)n_sel * (kFpDescInts + 1) * sizeof(int);
}

template <int T>
cudaError_t launch_gather_tiled_t(const GatherTiledArgs& a, cudaStream_t st)
{
    static unsigned long long mask = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!(mask & (1ull << (dev & 63)))) {
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(gather_tiled_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) return e;
        mask |= 1ull << (dev & 63);
    }
    if (a.n_sel > 32) return cudaErrorInvalidValue;  // warp 0 holds one angle id per lane
    dim3 grid(a.n_tiles, a.batch, a.nz / a.zs);
    gather_tiled_kernel<T><<<grid, kGatherTiledThreads, gather_tiled_smem(a.rows_cap, a.zs, T, a.stages, a.n_sel), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather_tiled(const GatherTiledArgs& a, cudaStream_t st)
{
    return a.T == kGtT ? launch_gather_tiled_t<kGtT>(a, st) : cudaErrorInvalidValue;
}

}  // namespace spect
