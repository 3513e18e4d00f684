// Depth-dependent PSF as banded-Toeplitz BF16 GEMMs on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory), FP32 accumulation.
//
// Per depth plane i, the 2-D blur of Eq. (1)'s T_cdr is K_i P = T_i P T_i^T
// with T_i the symmetric banded Toeplitz matrix of the plane's Gaussian taps.
// Both products are issued with K-major operands only:
//   GEMM 1   D1[k][j]  = sum_k' T_i[k][k'] P[j][k']          (blur along z)
//   GEMM 2   D2[k][j] += sum_j' X[k][j'] T_i[j][j']  with X = D1
// so D2 = (T_i P T_i^T)^T, and the forward keeps D2 in TMEM across the depth
// loop (P_x).  The taps are BF16, renormalised to unit sum; the data operands
// (P, and X read back from TMEM) are split into two BF16 parts, v = v_hi +
// v_lo (v_lo = bf16(v - v_hi)), and each GEMM runs two MMA chains,
// T * v_hi + T * v_lo.  Measured on the 128^3 x 120-angle 4 x 8 OSEM against
// the FP64 oracle: image 6.5e-4 and projections 8.5e-5 relative L2 (bar
// 1e-3).  The alternatives measured: three chains with the taps split too,
// 3.4e-6 (but 8 us slower per kernel); the taps split and the data rounded
// once, 1.3e-3; one chain, 2.5e-3 with renormalised taps, 4.0e-3 without.
// Rotation, attenuation, the ratio and the update stay FP32 on the CUDA
// cores.
//
// Shared-memory operands are K-major tiles with the 128-byte swizzle (see
// sw_off), so that both the staging (lanes along z) and the TMEM read-back
// (lanes along the tile rows) store without bank conflicts.  The per-plane
// Toeplitz tile (32 KB) arrives by one TMA bulk copy.
//
// Every wait on an mbarrier is bounded: when the bound runs out the kernel
// records SPECT_ETIMEDOUT in the plan's error word, releases its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "async_copy.cuh"
#include "geometry.cuh"
#include "internal.h"

namespace spect {

namespace {

constexpr int kTcThreads = 512;                 // 16 warps: 4 TMEM lane quadrants x 4 column parts
constexpr int kTcM = 128;                       // MMA M = axial size padded to 128
constexpr int kTile = kTcM * kTcM * 2;          // one 128x128 BF16 tile, bytes

// K-major operand tiles with the 128-byte swizzle: rows of 64 BF16 (128 B);
// 8 rows form a 1 KB atom in which 16-byte chunk c of row r is stored at
// chunk c ^ (r % 8); K beyond 64 continues in the next K block, R rows * 128 B
// further.  Tiles start on 1 KB boundaries.  Byte offset of element (r, k):
__device__ __forceinline__ uint32_t sw_off(int r, int k, int R)
{
    const int kb = k >> 6, kk = k & 63;
    return (uint32_t)(kb * R * 128 + ((r >> 3) << 10) + ((r & 7) << 7) + ((((kk >> 3) ^ (r & 7))) << 4) +
                      ((kk & 7) << 1));
}

// Shared-memory matrix descriptor of such a tile: start address, stride
// between 8-row groups (SBO) 1024 B, leading offset unused for swizzled
// K-major tiles, descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sw_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Start address of K step ks (16 elements) of a tile with R rows.
__device__ __forceinline__ uint32_t sw_kstep(uint32_t tile, int ks, int R)
{
    return tile + (uint32_t)((ks >> 2) * R * 128 + (ks & 3) * 32);
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

struct TcSmem {
    uint32_t tap;   // T (one tile)
    uint32_t b1;    // GEMM 1 B operand [n][128]: hi part, then the lo part at + b1_lo
    uint32_t a2;    // GEMM 2 A operand [128][n]: hi part, then the lo part at + a2_lo
    uint32_t b1_lo, a2_lo;  // byte distance from the hi to the lo part
    uint32_t bar_t, bar_1, bar_2;
};

// Two values as BF16 hi parts and BF16 residuals: v = hi + lo to ~2^-17.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    hi = pack_bf16x2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(a - ha, b - hb);
}

// GEMM 1: D1 = T_hi B_hi^T + T_lo B_hi^T + T_hi B_lo^T over K = 128.
__device__ __forceinline__ void issue_gemm1(const TcSmem& s, uint32_t d1, uint32_t idesc, int n)
{
    tc_fence_after();
    for (int h = 0; h < 2; ++h) {
        const uint32_t tb = s.b1 + (h ? s.b1_lo : 0);
#pragma unroll
        for (int ks = 0; ks < kTcM / 16; ++ks)
            tc_mma(d1, sw_desc(sw_kstep(s.tap, ks, kTcM)), sw_desc(sw_kstep(tb, ks, n)), idesc, (h | ks) != 0);
    }
    tc_commit(s.bar_1);
}

// GEMM 2: D2 (+)= A_hi T^T + A_lo T^T over K = n.
__device__ __forceinline__ void issue_gemm2(const TcSmem& s, uint32_t d2, uint32_t idesc, int n, bool accumulate)
{
    tc_fence_after();
    for (int h = 0; h < 2; ++h) {
        const uint32_t ta = s.a2 + (h ? s.a2_lo : 0);
        for (int ks = 0; ks < n / 16; ++ks)
            tc_mma(d2, sw_desc(sw_kstep(ta, ks, kTcM)), sw_desc(sw_kstep(s.tap, ks, kTcM)), idesc,
                   (accumulate || h || ks) ? 1u : 0u);
    }
    tc_commit(s.bar_2);
}

// D1 (TMEM, lanes k, columns j) -> BF16 hi/lo -> A2 (K-major [k][j], K = n).
// Warp w reads TMEM lanes 32*(w%4).. (its lane quadrant) and the 16-column
// chunks c with c/16 = w/4 (mod 4).
__device__ __forceinline__ void d1_to_a2(const TcSmem& s, uint32_t d1, int n)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = 32 * (warp & 3) + lane;
    for (int c = 16 * (warp >> 2); c < n; c += 64) {
        float v[16];
        tc_ld16(d1 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
        uint32_t h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
        const uint32_t o0 = s.a2 + sw_off(k, c, kTcM), o1 = s.a2 + sw_off(k, c + 8, kTcM);
        st_shared_v4(o0, h[0], h[1], h[2], h[3]);
        st_shared_v4(o1, h[4], h[5], h[6], h[7]);
        st_shared_v4(o0 + s.a2_lo, l[0], l[1], l[2], l[3]);
        st_shared_v4(o1 + s.a2_lo, l[4], l[5], l[6], l[7]);
    }
}

// Byte offset of the barriers after the operand tiles.
__host__ __device__ constexpr int bf16_tail_offset(int n)
{
    return kTile + 2 * n * kTcM * 2 + 2 * kTcM * ((n + 63) / 64 * 64) * 2;
}

struct TcState {
    TcSmem s;
    uint32_t tmem;
    uint32_t* tmem_slot;
};

__device__ __forceinline__ bool tc_setup(TcState& st, unsigned char* smem, int n, uint32_t ncols)
{
    // tiles: T (128 x 128); B1 hi, lo (n x 128); A2 hi, lo (128 x K with
    // K = n rounded up to whole 64-column swizzle blocks); all 1 KB aligned
    st.s.tap = smem_u32(smem);
    st.s.b1 = st.s.tap + kTile;
    st.s.b1_lo = n * kTcM * 2;
    st.s.a2 = st.s.b1 + 2 * st.s.b1_lo;
    st.s.a2_lo = kTcM * ((n + 63) / 64 * 64) * 2;
    unsigned char* tail = smem + bf16_tail_offset(n);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
    st.tmem_slot = reinterpret_cast<uint32_t*>(tail + 32);
    st.s.bar_t = smem_u32(bars + 0);
    st.s.bar_1 = smem_u32(bars + 1);
    st.s.bar_2 = smem_u32(bars + 2);
    if (threadIdx.x == 0) {
        mbar_init(st.s.bar_t, 1);
        mbar_init(st.s.bar_1, 1);
        mbar_init(st.s.bar_2, 1);
        mbar_init_fence();
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(st.tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    st.tmem = *st.tmem_slot;
    return true;
}

__device__ __forceinline__ void tc_teardown(TcState& st, uint32_t ncols)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(ncols) : "memory");
    }
}

// Every thread reaches this with the same `ok`; on a timeout one thread
// records the status and all threads leave together.
__device__ __forceinline__ bool all_ok(bool ok, int* err)
{
    const int bad = __syncthreads_or(!ok);
    if (bad && threadIdx.x == 0 && err) atomicExch(err, SPECT_ETIMEDOUT);
    return !bad;
}

// Bilinear taps of rotated row j of plane i (as in the FP32 forward).
struct TcTapRow {
    int off[4];
    float w[4];
};

__device__ __forceinline__ void tc_tap_rows(TcTapRow* rows, int n, int nz, int i, float4 cs, float c)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float u, v;
        sample_point(cs.x, cs.y, c, cs.z, i, j, u, v);
        const float fu = floorf(u), fv = floorf(v);
        const int x0 = (int)fu, y0 = (int)fv;
        const float ax = u - fu, by = v - fv;
        const bool vx0 = x0 >= 0 && x0 < n, vx1 = x0 + 1 >= 0 && x0 + 1 < n;
        const bool vy0 = y0 >= 0 && y0 < n, vy1 = y0 + 1 >= 0 && y0 + 1 < n;
        TcTapRow t;
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

__device__ __forceinline__ void fma4(float4& acc, float w, const float4& v)
{
    acc.x = fmaf(w, v.x, acc.x);
    acc.y = fmaf(w, v.y, acc.y);
    acc.z = fmaf(w, v.z, acc.z);
    acc.w = fmaf(w, v.w, acc.w);
}

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b)
{
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// Four values as BF16 hi and lo parts into row j, columns 4l..4l+3, of B1.
__device__ __forceinline__ void put4(uint32_t b1, uint32_t b1_lo, int j, int k, int n, float4 v)
{
    uint32_t h0, l0, h1, l1;
    split_bf16x2(v.x, v.y, h0, l0);
    split_bf16x2(v.z, v.w, h1, l1);
    const uint32_t o = b1 + sw_off(j, k, n);
    st_shared_v2(o, h0, h1);
    st_shared_v2(o + b1_lo, l0, l1);
}

// B1[j][k] = A[j][k] * bilinear(f)[j][k] for k < nz, 0 for nz <= k < 128, as
// BF16 hi and lo parts.  A warp stages whole rows, lane l covering k = 4l..4l+3
// with 128-bit loads (one 512-byte row per load instruction), four rows at a
// time so that twenty loads per lane are in flight together.
__device__ __forceinline__ void tc_stage_plane(uint32_t b1, uint32_t b1_lo, const TcTapRow* rows,
                                               const float* __restrict__ xb, const float* __restrict__ arow, int n,
                                               int nz)
{
    constexpr int kRows = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = 4 * lane;
    const bool in = k < nz;
    for (int jb = warp; jb < n; jb += kRows * nw) {
        float4 v[kRows];
        int jr[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            jr[r] = jb + r * nw;
            v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (in) {
            float4 f[kRows][4], av[kRows];
            TcTapRow t[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const int j = jr[r] < n ? jr[r] : jb;  // rows past n repeat a valid row; not stored
                t[r] = rows[j];
#pragma unroll
                for (int q = 0; q < 4; ++q) f[r][q] = __ldg(reinterpret_cast<const float4*>(xb + t[r].off[q] + k));
                av[r] = arow ? __ldg(reinterpret_cast<const float4*>(arow + (size_t)j * nz + k))
                             : make_float4(1.f, 1.f, 1.f, 1.f);
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
#pragma unroll
                for (int q = 0; q < 4; ++q) fma4(v[r], t[r].w[q], f[r][q]);
                v[r].x *= av[r].x;
                v[r].y *= av[r].y;
                v[r].z *= av[r].z;
                v[r].w *= av[r].w;
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r)
            if (jr[r] < n) put4(b1, b1_lo, jr[r], k, n, v[r]);
    }
}

// Ask L2 to fetch one attenuation plane (n rows of nz floats; rows start on
// 16-byte boundaries as nz % 8 == 0) ahead of its use; a hint that nothing
// waits on.
__device__ __forceinline__ void tc_prefetch_plane(const float* plane, int n, int nz)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) prefetch_l2(plane + (size_t)j * nz, (uint32_t)nz * 4u);
}

// B1[j][k] = proj[j][k] (all ones when proj is NULL) times the T_fov weight
// fv[j][k] (when not NULL) for k < nz, as BF16 hi and lo parts; lanes along
// k as above.
__device__ __forceinline__ void tc_stage_proj(uint32_t b1, uint32_t b1_lo, const float* __restrict__ pr,
                                              const float* __restrict__ fv, int n, int nz)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = 4 * lane;
    for (int j = warp; j < n; j += nw) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < nz) {
            v = pr ? __ldg(reinterpret_cast<const float4*>(pr + (size_t)j * nz + k)) : make_float4(1.f, 1.f, 1.f, 1.f);
            if (fv) {
                const float4 m = __ldg(reinterpret_cast<const float4*>(fv + (size_t)j * nz + k));
                v = make_float4(v.x * m.x, v.y * m.y, v.z * m.z, v.w * m.w);
            }
        }
        put4(b1, b1_lo, j, k, n, v);
    }
}

}  // namespace

size_t bf16_smem_bytes(int n);

// ---------------------------------------------------------------- forward

__global__ void __launch_bounds__(kTcThreads, 1) forward_bf16_kernel(ForwardBf16Args a)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    const int n = a.n, nz = a.nz;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const float4 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const uint32_t ncols = a.tmem_cols;
    TcState st;
    tc_setup(st, tsm, n, ncols);
    TcTapRow* rows = reinterpret_cast<TcTapRow*>(tsm + bf16_tail_offset(n) + 64);
    const uint32_t d1 = st.tmem, d2 = st.tmem + (uint32_t)n;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const float* xb = a.x + (size_t)b * n * n * nz;
    const size_t item = (size_t)b * a.n_sel + sidx;
    float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = true;

    // Pipeline per plane i (next plane i' = i + chunks):
    //   GEMM 1(i) done -> D1 to A2 -> issue GEMM 2(i)
    //   stage plane i' into B1 while GEMM 2(i) runs
    //   GEMM 2(i) done -> TMA the Toeplitz tiles of i' -> issue GEMM 1(i')
    uint32_t ph_t = 0, ph_1 = 0, ph_2 = 0;
    int i = chunk;
    if (i < n) {
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        if (a.atten && i + a.chunks < n) tc_prefetch_plane(arow + (size_t)a.chunks * n * nz, n, nz);
        if (threadIdx.x == 0) tma_load_1d(st.s.tap, ttab + (size_t)i * kTcM * kTcM, kTile, st.s.bar_t);
        tc_tap_rows(rows, n, nz, i, cs, c);
        __syncthreads();
        tc_stage_plane(st.s.b1, st.s.b1_lo, rows, xb, arow, n, nz);
        fence_async_smem();
        ok = all_ok(mbar_wait(st.s.bar_t, ph_t), a.err);
        ph_t ^= 1u;
        if (ok && threadIdx.x == 0) issue_gemm1(st.s, d1, idesc, n);
    }
    bool first = true;
    for (; i < n && ok; i += a.chunks) {
        const int inext = i + a.chunks;
        ok = all_ok(mbar_wait(st.s.bar_1, ph_1), a.err);
        ph_1 ^= 1u;
        if (!ok) break;
        tc_fence_after();
        d1_to_a2(st.s, d1, n);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        bool ok2 = true;
        if (threadIdx.x == 0) {
            issue_gemm2(st.s, d2, idesc, n, !first);
            // GEMM 2(i) is short: as soon as it has read the Toeplitz tiles,
            // fetch those of the next plane behind the staging below
            if (inext < n) {
                ok2 = mbar_wait(st.s.bar_2, ph_2);
                if (ok2) tma_load_1d(st.s.tap, ttab + (size_t)inext * kTcM * kTcM, kTile, st.s.bar_t);
            }
        }
        first = false;
        if (inext < n) {
            // GEMM 1(i) has finished with B1; stage the next plane meanwhile
            const float* arow = a.atten ? a.atten + ((size_t)angle * n + inext) * n * nz : nullptr;
            if (a.atten && inext + a.chunks < n) tc_prefetch_plane(arow + (size_t)a.chunks * n * nz, n, nz);
            tc_tap_rows(rows, n, nz, inext, cs, c);
            __syncthreads();
            tc_stage_plane(st.s.b1, st.s.b1_lo, rows, xb, arow, n, nz);
            fence_async_smem();
        }
        ok = all_ok(ok2 && mbar_wait(st.s.bar_2, ph_2), a.err);
        ph_2 ^= 1u;
        if (!ok || inext >= n) break;
        ok = all_ok(mbar_wait(st.s.bar_t, ph_t), a.err);
        ph_t ^= 1u;
        if (ok && threadIdx.x == 0) issue_gemm1(st.s, d1, idesc, n);
    }
    if (ok && !first) {
        // D2 = (sum over the chunk's planes)^T: lanes k, columns j
        tc_fence_after();
        const int k = 32 * (warp & 3) + lane;
        for (int cc = 16 * (warp >> 2); cc < n; cc += 64) {
            float v[16];
            tc_ld16(d2 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cc, v);
            if (k < nz) {
#pragma unroll
                for (int q = 0; q < 16; ++q) dst[(size_t)(cc + q) * nz + k] = v[q];
            }
        }
    } else if (ok && first) {
        // a chunk without planes (more chunks than planes): its sum is zero
        for (int e = threadIdx.x; e < n * nz; e += blockDim.x) dst[e] = 0.f;
    }
    tc_teardown(st, ncols);
}

// ---------------------------------------------------------------- back blur

__global__ void __launch_bounds__(kTcThreads, 1) blur_back_bf16_kernel(BlurBackBf16Args a)
{
    extern __shared__ __align__(128) unsigned char tsm[];
    const int n = a.n, nz = a.nz;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const uint32_t ncols = a.tmem_cols;
    TcState st;
    tc_setup(st, tsm, n, ncols);
    const uint32_t d1 = st.tmem, d2 = st.tmem + (uint32_t)n;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const size_t item = (size_t)b * a.n_sel + sidx;
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = 32 * (warp & 3) + lane;
    bool ok = true;
    uint32_t ph_t = 0, ph_1 = 0, ph_2 = 0;

    // the projection of this angle is the B operand of every plane's GEMM 1
    int i = chunk;
    if (i < n && a.atten) tc_prefetch_plane(a.atten + ((size_t)angle * n + i) * n * nz, n, nz);
    if (i < n && threadIdx.x == 0)
        tma_load_1d(st.s.tap, ttab + (size_t)i * kTcM * kTcM, kTile, st.s.bar_t);
    tc_stage_proj(st.s.b1, st.s.b1_lo, pr, a.fov ? a.fov + (size_t)angle * n * nz : nullptr, n, nz);
    fence_async_smem();
    if (i < n) {
        ok = all_ok(mbar_wait(st.s.bar_t, ph_t), a.err);
        ph_t ^= 1u;
        if (ok && threadIdx.x == 0) issue_gemm1(st.s, d1, idesc, n);
    }
    // Pipeline per plane i: GEMM 1(i) done -> D1 to A2 -> GEMM 2(i);
    // GEMM 2(i) done -> TMA of the next tiles, then the epilogue of plane i
    // (attenuation and store of B) while the copy is in flight -> GEMM 1(i').
    for (; i < n && ok; i += a.chunks) {
        const int inext = i + a.chunks;
        ok = all_ok(mbar_wait(st.s.bar_1, ph_1), a.err);
        ph_1 ^= 1u;
        if (!ok) break;
        tc_fence_after();
        d1_to_a2(st.s, d1, n);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) issue_gemm2(st.s, d2, idesc, n, false);
        ok = all_ok(mbar_wait(st.s.bar_2, ph_2), a.err);
        ph_2 ^= 1u;
        if (!ok) break;
        if (inext < n && threadIdx.x == 0)
            tma_load_1d(st.s.tap, ttab + (size_t)inext * kTcM * kTcM, kTile, st.s.bar_t);
        tc_fence_after();
        // B[i][j][k] = A[i][j][k] * (K_i r)[j][k]; D2 holds (K_i r)^T (lanes k)
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        if (a.atten && inext < n) tc_prefetch_plane(arow + (size_t)a.chunks * n * nz, n, nz);
        float* brow = bvol + (size_t)i * n * nz;
        for (int cc = 16 * (warp >> 2); cc < n; cc += 64) {
            float aw[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) aw[q] = (arow && k < nz) ? __ldg(arow + (size_t)(cc + q) * nz + k) : 1.f;
            float v[16];
            tc_ld16(d2 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cc, v);
            if (k < nz) {
#pragma unroll
                for (int q = 0; q < 16; ++q) brow[(size_t)(cc + q) * nz + k] = v[q] * aw[q];
            }
        }
        tc_fence_before();
        __syncthreads();  // D2 is overwritten by the next GEMM 2
        if (inext >= n) break;
        ok = all_ok(mbar_wait(st.s.bar_t, ph_t), a.err);
        ph_t ^= 1u;
        if (ok && threadIdx.x == 0) issue_gemm1(st.s, d1, idesc, n);
    }
    tc_teardown(st, ncols);
}

namespace {
// devices on which the kernels' shared-memory limits have been raised
unsigned long long g_fwd_bf16_mask = 0, g_back_bf16_mask = 0;

template <class F>
cudaError_t raise_smem(F fn, unsigned long long& mask)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (mask & (1ull << (dev & 63))) return cudaSuccess;
    // the largest footprint of any supported n, so one setting serves all plans
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bf16_smem_bytes(kTcM));
    if (e == cudaSuccess) mask |= 1ull << (dev & 63);
    return e;
}
}  // namespace

int bf16_occupancy(int n)
{
    int blocks = 0;
    const size_t smem = bf16_smem_bytes(n);
    if (raise_smem(forward_bf16_kernel, g_fwd_bf16_mask) != cudaSuccess ||
        raise_smem(blur_back_bf16_kernel, g_back_bf16_mask) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_bf16_kernel, kTcThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return blocks > 0 ? blocks : 1;
}

size_t bf16_smem_bytes(int n) { return (size_t)bf16_tail_offset(n) + 64 + 32 * (size_t)n; }

uint32_t bf16_tmem_cols(int n)
{
    uint32_t c = 32;
    while (c < (uint32_t)(2 * n)) c <<= 1;
    return c;
}

cudaError_t launch_forward_bf16(const ForwardBf16Args& a, cudaStream_t st)
{
    cudaError_t e = raise_smem(forward_bf16_kernel, g_fwd_bf16_mask);
    if (e != cudaSuccess) return e;
    dim3 grid(a.chunks, a.n_sel, a.batch);
    forward_bf16_kernel<<<grid, kTcThreads, bf16_smem_bytes(a.n), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_blur_back_bf16(const BlurBackBf16Args& a, cudaStream_t st)
{
    cudaError_t e = raise_smem(blur_back_bf16_kernel, g_back_bf16_mask);
    if (e != cudaSuccess) return e;
    dim3 grid(a.chunks, a.n_sel, a.batch);
    blur_back_bf16_kernel<<<grid, kTcThreads, bf16_smem_bytes(a.n), st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
