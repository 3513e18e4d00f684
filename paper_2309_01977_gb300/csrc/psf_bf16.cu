// Depth-dependent PSF as banded-Toeplitz BF16 GEMMs on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory), FP32 accumulation.
//
// Per depth plane i, the 2-D blur of Eq. (1)'s T_cdr is K_i P = T_i P T_i^T
// with T_i the symmetric banded Toeplitz matrix of the plane's Gaussian taps.
// Both products are issued with K-major operands only:
//   GEMM 1   D1[k][j]  = sum_k' T_i[k][k'] P[j][k']          (blur along z)
//   GEMM 2   D2[k][j] += sum_j' X[k][j'] T_i[j][j']  with X = bf16(D1)
// so D2 = (T_i P T_i^T)^T, and the forward keeps D2 in TMEM across the depth
// loop (P_x).  Every operand is split into two BF16 parts, v = v_hi + v_lo
// (v_lo = bf16(v - v_hi)), and each GEMM runs three MMA chains,
// hi*hi + hi*lo + lo*hi, dropping only lo*lo (relative ~2^-18): the
// projector then agrees with FP32 to ~1e-6 instead of the ~2e-4 of a single
// BF16 rounding, which OSEM would compound past 1e-3 over 32 subiterations.
// Rotation, attenuation, the ratio and the update stay FP32 on the CUDA
// cores.
//
// Shared-memory operands use the no-swizzle K-major core-matrix layout: 8x8
// BF16 core matrices of 128 contiguous bytes, K-adjacent core matrices 128 B
// apart (leading byte offset), 8-row groups (K/8)*128 B apart (stride byte
// offset).  The per-plane Toeplitz pair (64 KB) arrives by one TMA bulk copy.
//
// Every wait on an mbarrier is bounded: when the bound runs out the kernel
// records SPECT_ETIMEDOUT in the plan's error word, releases its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "geometry.cuh"
#include "internal.h"

namespace spect {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;                       // MMA M = axial size padded to 128
constexpr int kTile = kTcM * kTcM * 2;          // one 128x128 BF16 tile, bytes
constexpr long long kWaitCycles = 4000000000LL; // bounded mbarrier waits (~2 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of a K-major tile with K columns.
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K)
{
    return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Shared-memory matrix descriptor: no swizzle, K-major, LBO = 128 B,
// SBO = (K/8) * 128 B, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, int K)
{
    const uint64_t lbo = 128, sbo = (uint64_t)(K >> 3) * 128;
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(lbo >> 4) << 16;
    d |= (uint64_t)(sbo >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
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
    uint32_t tap;   // T_hi then T_lo (2 tiles)
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
__device__ __forceinline__ void issue_gemm1(const TcSmem& s, uint32_t d1, uint32_t idesc)
{
    tc_fence_after();
    for (int h = 0; h < 3; ++h) {
        const uint32_t ta = s.tap + (h == 1 ? kTile : 0);
        const uint32_t tb = s.b1 + (h == 2 ? s.b1_lo : 0);
#pragma unroll
        for (int ks = 0; ks < kTcM / 16; ++ks)
            tc_mma(d1, smem_desc(ta + ks * 256, kTcM), smem_desc(tb + ks * 256, kTcM), idesc, (h | ks) != 0);
    }
    tc_commit(s.bar_1);
}

// GEMM 2: D2 (+)= A_hi T_hi^T + A_hi T_lo^T + A_lo T_hi^T over K = n.
__device__ __forceinline__ void issue_gemm2(const TcSmem& s, uint32_t d2, uint32_t idesc, int n, bool accumulate)
{
    tc_fence_after();
    for (int h = 0; h < 3; ++h) {
        const uint32_t ta = s.a2 + (h == 2 ? s.a2_lo : 0);
        const uint32_t tb = s.tap + (h == 1 ? kTile : 0);
        for (int ks = 0; ks < n / 16; ++ks)
            tc_mma(d2, smem_desc(ta + ks * 256, n), smem_desc(tb + ks * 256, kTcM), idesc,
                   (accumulate || h || ks) ? 1u : 0u);
    }
    tc_commit(s.bar_2);
}

// D1 (TMEM, lanes k, columns j) -> BF16 -> A2 (K-major [k][j], K = n).
// Warp w reads lanes 32*(w%4).. and the column half w/4.
__device__ __forceinline__ void d1_to_a2(const TcSmem& s, uint32_t d1, int n)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = 32 * (warp & 3) + lane;
    const int half = n / 2;  // n % 32 == 0 for this path
    const int c0 = (warp >> 2) * half;
    for (int c = c0; c < c0 + half; c += 16) {
        float v[16];
        tc_ld16(d1 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
        uint32_t h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
        const uint32_t o0 = s.a2 + cm_off(k, c, n), o1 = s.a2 + cm_off(k, c + 8, n);
        st_shared_v4(o0, h[0], h[1], h[2], h[3]);
        st_shared_v4(o1, h[4], h[5], h[6], h[7]);
        st_shared_v4(o0 + s.a2_lo, l[0], l[1], l[2], l[3]);
        st_shared_v4(o1 + s.a2_lo, l[4], l[5], l[6], l[7]);
    }
}

struct TcState {
    TcSmem s;
    uint32_t tmem;
    uint32_t* tmem_slot;
};

__device__ __forceinline__ bool tc_setup(TcState& st, unsigned char* smem, int n, uint32_t ncols)
{
    st.s.tap = smem_u32(smem);
    st.s.b1 = st.s.tap + 2 * kTile;
    st.s.b1_lo = n * kTcM * 2;
    st.s.a2 = st.s.b1 + 2 * n * kTcM * 2;
    st.s.a2_lo = n * kTcM * 2;
    unsigned char* tail = smem + 2 * kTile + 4 * n * kTcM * 2;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
    st.tmem_slot = reinterpret_cast<uint32_t*>(tail + 32);
    st.s.bar_t = smem_u32(bars + 0);
    st.s.bar_1 = smem_u32(bars + 1);
    st.s.bar_2 = smem_u32(bars + 2);
    if (threadIdx.x == 0) {
        mbar_init(st.s.bar_t, 1);
        mbar_init(st.s.bar_1, 1);
        mbar_init(st.s.bar_2, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

__device__ __forceinline__ void tc_tap_rows(TcTapRow* rows, int n, int nz, int i, float2 cs, float c)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        float u, v;
        sample_point(cs.x, cs.y, c, i, j, u, v);
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

// B1[j][k'] = A[j][k'] * bilinear(f)[j][k'] for k' < nz, 0 for k' >= nz, as
// BF16 hi and lo parts: one task = (row j, 8 consecutive k'), rows fastest
// across lanes.
__device__ __forceinline__ void tc_stage_plane(uint32_t b1, uint32_t b1_lo, const TcTapRow* rows,
                                               const float* __restrict__ xb, const float* __restrict__ arow, int n,
                                               int nz)
{
    const int tasks = n * (kTcM / 8);
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
        const int j = t % n, kc = (t / n) * 8;
        uint32_t h[4] = {0u, 0u, 0u, 0u}, l[4] = {0u, 0u, 0u, 0u};
        if (kc < nz) {
            const TcTapRow tr = rows[j];
            float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4* src = reinterpret_cast<const float4*>(xb + tr.off[q] + kc);
                fma4(lo, tr.w[q], __ldg(src));
                fma4(hi, tr.w[q], __ldg(src + 1));
            }
            if (arow) {
                const float4* ap = reinterpret_cast<const float4*>(arow + (size_t)j * nz + kc);
                const float4 a0 = __ldg(ap), a1 = __ldg(ap + 1);
                lo.x *= a0.x; lo.y *= a0.y; lo.z *= a0.z; lo.w *= a0.w;
                hi.x *= a1.x; hi.y *= a1.y; hi.z *= a1.z; hi.w *= a1.w;
            }
            split_bf16x2(lo.x, lo.y, h[0], l[0]);
            split_bf16x2(lo.z, lo.w, h[1], l[1]);
            split_bf16x2(hi.x, hi.y, h[2], l[2]);
            split_bf16x2(hi.z, hi.w, h[3], l[3]);
        }
        const uint32_t o = b1 + cm_off(j, kc, kTcM);
        st_shared_v4(o, h[0], h[1], h[2], h[3]);
        st_shared_v4(o + b1_lo, l[0], l[1], l[2], l[3]);
    }
}

// B1[j][k'] = proj[j][k'] (all ones when proj is NULL) for k' < nz, as BF16
// hi and lo parts.
__device__ __forceinline__ void tc_stage_proj(uint32_t b1, uint32_t b1_lo, const float* __restrict__ pr, int n, int nz)
{
    const int tasks = n * (kTcM / 8);
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
        const int j = t % n, kc = (t / n) * 8;
        uint32_t h[4] = {0u, 0u, 0u, 0u}, l[4] = {0u, 0u, 0u, 0u};
        if (kc < nz) {
            float4 lo = make_float4(1.f, 1.f, 1.f, 1.f), hi = lo;
            if (pr) {
                const float4* src = reinterpret_cast<const float4*>(pr + (size_t)j * nz + kc);
                lo = __ldg(src);
                hi = __ldg(src + 1);
            }
            split_bf16x2(lo.x, lo.y, h[0], l[0]);
            split_bf16x2(lo.z, lo.w, h[1], l[1]);
            split_bf16x2(hi.x, hi.y, h[2], l[2]);
            split_bf16x2(hi.z, hi.w, h[3], l[3]);
        }
        const uint32_t o = b1 + cm_off(j, kc, kTcM);
        st_shared_v4(o, h[0], h[1], h[2], h[3]);
        st_shared_v4(o + b1_lo, l[0], l[1], l[2], l[3]);
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
    const float2 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const uint32_t ncols = a.tmem_cols;
    TcState st;
    tc_setup(st, tsm, n, ncols);
    TcTapRow* rows = reinterpret_cast<TcTapRow*>(tsm + 2 * kTile + 4 * n * kTcM * 2 + 64);
    const uint32_t d1 = st.tmem, d2 = st.tmem + (uint32_t)n;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const float* xb = a.x + (size_t)b * n * n * nz;
    uint32_t phase = 0;
    bool ok = true;
    bool first = true;
    for (int i = chunk; i < n && ok; i += a.chunks) {
        // taps of this plane (the previous GEMM 2, which read them, has completed)
        if (threadIdx.x == 0) tma_load_1d(st.s.tap, a.ttab + (size_t)i * 2 * kTcM * kTcM, 2 * kTile, st.s.bar_t);
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        tc_tap_rows(rows, n, nz, i, cs, c);
        __syncthreads();
        tc_stage_plane(st.s.b1, st.s.b1_lo, rows, xb, arow, n, nz);
        fence_async_smem();
        ok = all_ok(mbar_wait(st.s.bar_t, phase), a.err);
        if (!ok) break;
        if (threadIdx.x == 0) issue_gemm1(st.s, d1, idesc);
        ok = all_ok(mbar_wait(st.s.bar_1, phase), a.err);
        if (!ok) break;
        tc_fence_after();
        d1_to_a2(st.s, d1, n);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) issue_gemm2(st.s, d2, idesc, n, !first);
        ok = all_ok(mbar_wait(st.s.bar_2, phase), a.err);
        phase ^= 1u;
        first = false;
    }
    if (ok && !first) {
        // D2 = (sum over the chunk's planes)^T: lanes k, columns j
        tc_fence_after();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int k = 32 * (warp & 3) + lane;
        const size_t item = (size_t)b * a.n_sel + sidx;
        float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
        const int half = n / 2, c0 = (warp >> 2) * half;
        for (int cc = c0; cc < c0 + half; cc += 16) {
            float v[16];
            tc_ld16(d2 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cc, v);
            if (k < nz) {
#pragma unroll
                for (int q = 0; q < 16; ++q) dst[(size_t)(cc + q) * nz + k] = v[q];
            }
        }
    } else if (ok && first) {
        // a chunk without planes (more chunks than planes): its sum is zero
        const size_t item = (size_t)b * a.n_sel + sidx;
        float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
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
    const uint32_t ncols = a.tmem_cols;
    TcState st;
    tc_setup(st, tsm, n, ncols);
    const uint32_t d1 = st.tmem, d2 = st.tmem + (uint32_t)n;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const size_t item = (size_t)b * a.n_sel + sidx;
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    tc_stage_proj(st.s.b1, st.s.b1_lo, pr, n, nz);
    fence_async_smem();
    __syncthreads();
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = 32 * (warp & 3) + lane;
    const int half = n / 2, c0 = (warp >> 2) * half;
    uint32_t phase = 0;
    bool ok = true;
    for (int i = chunk; i < n && ok; i += a.chunks) {
        if (threadIdx.x == 0) tma_load_1d(st.s.tap, a.ttab + (size_t)i * 2 * kTcM * kTcM, 2 * kTile, st.s.bar_t);
        ok = all_ok(mbar_wait(st.s.bar_t, phase), a.err);
        if (!ok) break;
        if (threadIdx.x == 0) issue_gemm1(st.s, d1, idesc);
        ok = all_ok(mbar_wait(st.s.bar_1, phase), a.err);
        if (!ok) break;
        tc_fence_after();
        d1_to_a2(st.s, d1, n);
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) issue_gemm2(st.s, d2, idesc, n, false);
        ok = all_ok(mbar_wait(st.s.bar_2, phase), a.err);
        if (!ok) break;
        tc_fence_after();
        // B[i][j][k] = A[i][j][k] * (K_i r)[j][k]; D2 holds (K_i r)^T (lanes k)
        const float* arow = a.atten ? a.atten + ((size_t)angle * n + i) * n * nz : nullptr;
        float* brow = bvol + (size_t)i * n * nz;
        for (int cc = c0; cc < c0 + half; cc += 16) {
            float v[16];
            tc_ld16(d2 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cc, v);
            if (k < nz) {
                float aw[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) aw[q] = arow ? __ldg(arow + (size_t)(cc + q) * nz + k) : 1.f;
#pragma unroll
                for (int q = 0; q < 16; ++q) brow[(size_t)(cc + q) * nz + k] = v[q] * aw[q];
            }
        }
        tc_fence_before();
        __syncthreads();  // TMEM and the tap tiles are reused by the next plane
        phase ^= 1u;
    }
    tc_teardown(st, ncols);
}

int bf16_occupancy(int n)
{
    int blocks = 0;
    const size_t smem = bf16_smem_bytes(n);
    if (cudaFuncSetAttribute(forward_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bf16_smem_bytes(kTcM)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_bf16_kernel, kTcThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return blocks > 0 ? blocks : 1;
}

size_t bf16_smem_bytes(int n) { return (size_t)2 * kTile + (size_t)4 * n * kTcM * 2 + 64 + 32 * (size_t)n; }

uint32_t bf16_tmem_cols(int n)
{
    uint32_t c = 32;
    while (c < (uint32_t)(2 * n)) c <<= 1;
    return c;
}

cudaError_t launch_forward_bf16(const ForwardBf16Args& a, cudaStream_t st)
{
    static unsigned long long mask = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = bf16_smem_bytes(a.n);
    if (!(mask & (1ull << (dev & 63)))) {
        // the largest footprint of any supported n, so one setting serves all plans
        e = cudaFuncSetAttribute(forward_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bf16_smem_bytes(kTcM));
        if (e != cudaSuccess) return e;
        mask |= 1ull << (dev & 63);
    }
    dim3 grid(a.chunks, a.n_sel, a.batch);
    forward_bf16_kernel<<<grid, kTcThreads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_blur_back_bf16(const BlurBackBf16Args& a, cudaStream_t st)
{
    static unsigned long long mask = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t smem = bf16_smem_bytes(a.n);
    if (!(mask & (1ull << (dev & 63)))) {
        e = cudaFuncSetAttribute(blur_back_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bf16_smem_bytes(kTcM));
        if (e != cudaSuccess) return e;
        mask |= 1ull << (dev & 63);
    }
    dim3 grid(a.chunks, a.n_sel, a.batch);
    blur_back_bf16_kernel<<<grid, kTcThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
