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
// Toeplitz tile (32 KB) arrives by one TMA bulk copy into one of several
// slots, planes ahead of its use.  The kernels are software pipelines in
// which the tensor cores work on one plane while the CUDA cores stage the
// next (forward) or finish the previous one (back blur); see each kernel.
//
// Every wait on an mbarrier is bounded: when the bound runs out the kernel
// records SPECT_ETIMEDOUT in the plan's error word, releases its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
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

// Two values as BF16 hi parts and BF16 residuals: v = hi + lo to ~2^-17.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    hi = pack_bf16x2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(a - ha, b - hb);
}

// GEMM 1: D1 = T B_hi^T + T B_lo^T over K = 128 (the axial direction); B is
// n x 128 with its lo part `lo` bytes after the hi part.  Completion arrives
// on `bar`.
__device__ __forceinline__ void issue_gemm1(uint32_t tap, uint32_t b1, uint32_t lo, uint32_t d1, uint32_t idesc, int n,
                                            uint32_t bar)
{
    for (int h = 0; h < 2; ++h) {
        const uint32_t tb = b1 + (h ? lo : 0u);
#pragma unroll
        for (int ks = 0; ks < kTcM / 16; ++ks)
            tc_mma(d1, sw_desc(sw_kstep(tap, ks, kTcM)), sw_desc(sw_kstep(tb, ks, n)), idesc, (h | ks) != 0);
    }
    tc_commit(bar);
}

// GEMM 2: D2 (+)= A_hi T^T + A_lo T^T over K = n (the transaxial direction);
// A is 128 x n.  Completion arrives on `bar` unless it is 0.
__device__ __forceinline__ void issue_gemm2(uint32_t a2, uint32_t lo, uint32_t tap, uint32_t d2, uint32_t idesc, int n,
                                            bool accumulate, uint32_t bar)
{
    for (int h = 0; h < 2; ++h) {
        const uint32_t ta = a2 + (h ? lo : 0u);
        for (int ks = 0; ks < n / 16; ++ks)
            tc_mma(d2, sw_desc(sw_kstep(ta, ks, kTcM)), sw_desc(sw_kstep(tap, ks, kTcM)), idesc,
                   (accumulate || h || ks) ? 1u : 0u);
    }
    if (bar) tc_commit(bar);
}

// D1 (TMEM, lanes k, columns j) -> BF16 hi/lo -> A operand of GEMM 2
// (K-major [k][j], K = n; lo part `lo` bytes after the hi part).  Warp w
// reads TMEM lanes 32*(w%4).. (its lane quadrant) and the 16-column chunks
// c with c/16 = w/4 (mod 4).
__device__ __forceinline__ void d1_to_a2(uint32_t a2, uint32_t lo, uint32_t d1, int n)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = 32 * (warp & 3) + lane;
    for (int c = 16 * (warp >> 2); c < n; c += 64) {
        float v[16];
        tc_ld16(d1 + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)c, v);
        uint32_t h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
        const uint32_t o0 = a2 + sw_off(k, c, kTcM), o1 = a2 + sw_off(k, c + 8, kTcM);
        st_shared_v4(o0, h[0], h[1], h[2], h[3]);
        st_shared_v4(o1, h[4], h[5], h[6], h[7]);
        st_shared_v4(o0 + lo, l[0], l[1], l[2], l[3]);
        st_shared_v4(o1 + lo, l[4], l[5], l[6], l[7]);
    }
}

// Bytes of one BF16 part (hi or lo) of a plane operand: the larger of the
// GEMM 1 B operand (n rows x 128) and the GEMM 2 A operand (128 rows x n,
// rounded up to whole 64-column swizzle blocks).
__host__ __device__ constexpr uint32_t part_bytes(int n) { return (uint32_t)kTcM * ((n + 63) / 64 * 64) * 2u; }

// Shared-memory layouts (every tile 1 KB aligned), then a 64-byte block of
// up to six mbarriers and the TMEM address slot at byte 48:
//   forward:  Toeplitz slots [2] | plane buffers [2] (hi, lo) | tap-row tables [2][n]
//   back:     Toeplitz slots [3] | B1 = projection (hi, lo) | A2 (hi, lo)
constexpr int kFwdSlots = 2, kBackSlots = 3;
constexpr uint32_t kBarBytes = 64;
__host__ __device__ constexpr uint32_t fwd_rows_offset(int n) { return kFwdSlots * kTile + 4u * part_bytes(n); }
__host__ __device__ constexpr uint32_t fwd_bar_offset(int n) { return fwd_rows_offset(n) + 64u * (uint32_t)n; }
__host__ __device__ constexpr uint32_t back_bar_offset(int n) { return kBackSlots * kTile + 4u * part_bytes(n); }

// Thread 0's record of the Toeplitz-tile copies per slot (slot s completes
// on the barrier at bars + 8 s): a copy is pending from its issue until
// thread 0 has seen it land, and the parity bit of a slot is that of its
// next completion.  After a timeout, drain() waits (bounded) for the copies
// still in flight, so that none lands after the CTA has left.
struct TileLoads {
    uint32_t pend = 0, par = 0;
    __device__ __forceinline__ void load(int s, uint32_t dst, const void* src, uint32_t bars)
    {
        tma_load_1d(dst, src, (uint32_t)kTile, bars + 8u * s);
        pend |= 1u << s;
    }
    __device__ __forceinline__ bool wait(int s, uint32_t bars)
    {
        const bool ok = mbar_wait(bars + 8u * s, (par >> s) & 1u);
        if (ok) {
            par ^= 1u << s;
            pend &= ~(1u << s);
        }
        return ok;
    }
    __device__ __forceinline__ void drain(uint32_t bars, int slots)
    {
        for (int s = 0; s < slots; ++s)
            if ((pend >> s) & 1u) mbar_wait(bars + 8u * s, (par >> s) & 1u);
    }
};

// Thread 0, after a timeout: one more commit covers every product it has
// issued; wait (bounded) until they are done before the TMEM is released.
__device__ __forceinline__ void tc_drain(uint32_t bar)
{
    tc_commit(bar);
    mbar_wait(bar, 0);
}

// Initialise `count` barriers of one arrival at bars, bars + 8, ... (thread
// 0), allocate `ncols` TMEM columns (warp 0) and return their base address.
__device__ __forceinline__ uint32_t tc_begin(uint32_t bars, int count, uint32_t ncols)
{
    const uint32_t slot = bars + 48u;
    if (threadIdx.x == 0) {
        for (int q = 0; q < count; ++q) mbar_init(bars + 8u * q, 1);
        mbar_init_fence();
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t t;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(t) : "r"(slot) : "memory");
    return t;
}

__device__ __forceinline__ void tc_end(uint32_t tmem, uint32_t ncols)
{
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// Every thread reaches this with its own `ok`; on a timeout one thread
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
// time so that twenty loads per lane are in flight together.  When wait_bar
// is not 0 the buffer is still an operand of products in flight: the first
// stores wait for phase parity wait_par of that barrier, behind the first
// loads.  Returns false when that wait ran out.
__device__ __forceinline__ bool tc_stage_plane(uint32_t b1, uint32_t b1_lo, const TcTapRow* rows,
                                               const float* __restrict__ xb, const float* __restrict__ arow, int n,
                                               int nz, uint32_t wait_bar, uint32_t wait_par)
{
    bool ok = true;
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
        if (wait_bar) {
            ok = mbar_wait(wait_bar, wait_par);
            wait_bar = 0;
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r)
            if (jr[r] < n) put4(b1, b1_lo, jr[r], k, n, v[r]);
    }
    if (wait_bar) ok = mbar_wait(wait_bar, wait_par);
    return ok;
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

// ---------------------------------------------------------------- forward
//
// Planes p = 0, 1, .. of this CTA's depth chunk (plane index chunk + p *
// chunks) flow through two plane buffers X[p & 1]: the staged plane is the B
// operand of GEMM 1(p); once GEMM 1(p) is done, D1 is written back over it
// as the A operand of GEMM 2(p); once GEMM 2(p) is done, X[p & 1] takes the
// staging of plane p + 2.  Per iteration p the CUDA cores stage plane p + 1
// and hand D1(p) over, while the tensor cores run GEMM 2(p - 1) and
// GEMM 1(p); one thread then issues GEMM 2(p) and GEMM 1(p + 1) back to
// back.  The Toeplitz tile of plane p + 1 is copied into the slot of plane
// p - 1 as soon as GEMM 2(p - 1) is done, a whole staging ahead of its use.
// D2 accumulates the chunk's depth sum in TMEM (P_x).

__global__ void __launch_bounds__(kTcThreads, 1) forward_bf16_kernel(ForwardBf16Args a)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int n = a.n, nz = a.nz, tid = threadIdx.x;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const float4 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const uint32_t base = smem_u32(tsm), part = part_bytes(n);
    const uint32_t bars = base + fwd_bar_offset(n);  // Toeplitz slots s at bars + 8 s
    const uint32_t bar_1 = bars + 16, bar_2 = bars + 24, bar_d = bars + 32;
    TcTapRow* rows = reinterpret_cast<TcTapRow*>(tsm + fwd_rows_offset(n));  // [2][n]
    const uint32_t tmem = tc_begin(bars, 5, a.tmem_cols);
    const uint32_t d1 = tmem, d2 = tmem + (uint32_t)n;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const int np = chunk < n ? (n - 1 - chunk) / a.chunks + 1 : 0;
    const float* xb = a.x + (size_t)b * n * n * nz;
    const size_t item = (size_t)b * a.n_sel + sidx;
    float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
    const int warp = tid >> 5, lane = tid & 31;
    auto plane = [&](int p) { return chunk + p * a.chunks; };
    auto tap = [&](int s) { return base + (uint32_t)s * kTile; };
    auto xbuf = [&](int s) { return base + kFwdSlots * kTile + (uint32_t)s * 2u * part; };
    auto tsrc = [&](int p) { return ttab + (size_t)plane(p) * kTcM * kTcM; };
    auto arow = [&](int p) -> const float* {
        return a.atten ? a.atten + ((size_t)angle * n + plane(p)) * n * nz : nullptr;
    };
    TileLoads tl;
    bool ok = true;

    if (np > 0) {
        if (tid == 0) {
            tl.load(0, tap(0), tsrc(0), bars);
            if (np > 1) tl.load(1, tap(1), tsrc(1), bars);
        }
        if (a.atten && np > 1) tc_prefetch_plane(arow(1), n, nz);
        tc_tap_rows(rows, n, nz, plane(0), cs, c);
        __syncthreads();
        if (np > 1) tc_tap_rows(rows + n, n, nz, plane(1), cs, c);  // read after the next barrier
        tc_stage_plane(xbuf(0), part, rows, xb, arow(0), n, nz, 0u, 0u);
        fence_async_smem();
        __syncthreads();
        bool okt = true;
        if (tid == 0) {
            okt = tl.wait(0, bars);
            if (okt) {
                tc_fence_after();
                issue_gemm1(tap(0), xbuf(0), part, d1, idesc, n, bar_1);
            }
        }
        ok = all_ok(okt, a.err);
    }
    for (int p = 0; p < np && ok; ++p) {
        const bool more = p + 1 < np;
        bool okw = true;
        if (more) {
            if (p + 2 < np) {  // the table of plane p was read by its staging, before the last barrier
                tc_tap_rows(rows + (p & 1) * n, n, nz, plane(p + 2), cs, c);
                if (a.atten) tc_prefetch_plane(arow(p + 2), n, nz);
            }
            // X[(p+1)&1] last held the A operand of GEMM 2(p-1)
            okw = tc_stage_plane(xbuf((p + 1) & 1), part, rows + ((p + 1) & 1) * n, xb, arow(p + 1), n, nz,
                                 p > 0 ? bar_2 : 0u, (uint32_t)(p - 1) & 1u);
            // GEMM 2(p-1) has also released the Toeplitz slot of plane p+1
            if (tid == 0 && p > 0 && okw) tl.load((p + 1) & 1, tap((p + 1) & 1), tsrc(p + 1), bars);
        } else if (p > 0) {
            okw = mbar_wait(bar_2, (uint32_t)(p - 1) & 1u);  // keep the waits on bar_2 one phase apart
        }
        // GEMM 1(p) is done: D1 becomes the A operand of GEMM 2(p), over
        // GEMM 1(p)'s B operand in X[p&1]
        const bool ok1 = mbar_wait(bar_1, (uint32_t)p & 1u);
        tc_fence_after();
        if (ok1) d1_to_a2(xbuf(p & 1), part, d1, n);
        fence_async_smem();
        tc_fence_before();
        ok = all_ok(okw && ok1, a.err);
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            issue_gemm2(xbuf(p & 1), part, tap(p & 1), d2, idesc, n, p > 0, bar_2);
            if (more && tl.wait((p + 1) & 1, bars))
                issue_gemm1(tap((p + 1) & 1), xbuf((p + 1) & 1), part, d1, idesc, n, bar_1);
        }
        __syncwarp();  // warp 0 reconverges before its next warp-wide TMEM access
    }
    if (ok && np > 0) {
        ok = all_ok(mbar_wait(bar_2, (uint32_t)(np - 1) & 1u), a.err);
        if (ok) {
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
        }
    } else if (ok) {
        // a chunk without planes (more chunks than planes): its sum is zero
        for (int e = tid; e < n * nz; e += blockDim.x) dst[e] = 0.f;
    }
    if (!ok && tid == 0) {
        tl.drain(bars, kFwdSlots);
        tc_drain(bar_d);
    }
    tc_end(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------- back blur
//
// The projection of the angle is the B operand of every plane's GEMM 1.
// Per iteration p: GEMM 1(p) done (and with it GEMM 2(p - 1)) -> D1 to A2
// -> one thread issues GEMM 2(p) into D2[p & 1] and GEMM 1(p + 1); the CUDA
// cores meanwhile finish plane p - 1 from D2[(p - 1) & 1]: times A, stored
// as B.  Three Toeplitz slots: the tile of plane p + 2 is copied into the
// slot of plane p - 1 once GEMM 2(p - 1) is done.

__global__ void __launch_bounds__(kTcThreads, 1) blur_back_bf16_kernel(BlurBackBf16Args a)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int n = a.n, nz = a.nz, tid = threadIdx.x;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const uint32_t base = smem_u32(tsm), part = part_bytes(n);
    const uint32_t bars = base + back_bar_offset(n);  // Toeplitz slots s at bars + 8 s
    const uint32_t bar_1 = bars + 24, bar_2 = bars + 32, bar_d = bars + 40;
    const uint32_t tmem = tc_begin(bars, 6, a.tmem_cols);
    const uint32_t d1 = tmem;
    const uint32_t b1 = base + kBackSlots * kTile, a2 = b1 + 2u * part;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const int np = chunk < n ? (n - 1 - chunk) / a.chunks + 1 : 0;
    const size_t item = (size_t)b * a.n_sel + sidx;
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    const int warp = tid >> 5, lane = tid & 31;
    const int k = 32 * (warp & 3) + lane;
    const uint32_t quad = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lane quadrant
    auto plane = [&](int p) { return chunk + p * a.chunks; };
    auto tap = [&](int s) { return base + (uint32_t)s * kTile; };
    auto d2 = [&](int s) { return tmem + (uint32_t)n * (1u + (uint32_t)s); };
    auto tsrc = [&](int p) { return ttab + (size_t)plane(p) * kTcM * kTcM; };
    auto arow = [&](int p) -> const float* {
        return a.atten ? a.atten + ((size_t)angle * n + plane(p)) * n * nz : nullptr;
    };
    // A of plane p for this thread's elements (lane k, columns cc + q of its
    // at most two 16-column chunks), loaded ahead of the waits
    auto load_a = [&](int p, float (&aw)[2][16]) {
        const float* ar = arow(p);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int cc = 16 * (warp >> 2) + 64 * m;
#pragma unroll
            for (int q = 0; q < 16; ++q) aw[m][q] = (ar && cc < n && k < nz) ? __ldg(ar + (size_t)(cc + q) * nz + k) : 1.f;
        }
    };
    // B[plane p][j][k] = A * (K_i r)[j][k]; D2 holds (K_i r)^T (lanes k)
    auto finish = [&](int p, const float (&aw)[2][16]) {
        float* brow = bvol + (size_t)plane(p) * n * nz;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int cc = 16 * (warp >> 2) + 64 * m;
            if (cc < n) {
                float v[16];
                tc_ld16(d2(p & 1) + quad + (uint32_t)cc, v);
                if (k < nz) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) brow[(size_t)(cc + q) * nz + k] = v[q] * aw[m][q];
                }
            }
        }
    };
    TileLoads tl;
    bool ok = true;

    if (np > 0 && tid == 0)
        for (int s = 0; s < kBackSlots && s < np; ++s) tl.load(s, tap(s), tsrc(s), bars);
    if (np > 0 && a.atten) tc_prefetch_plane(arow(0), n, nz);
    tc_stage_proj(b1, part, pr, a.fov ? a.fov + (size_t)angle * n * nz : nullptr, n, nz);
    fence_async_smem();
    __syncthreads();
    if (np > 0) {
        bool okt = true;
        if (tid == 0) {
            okt = tl.wait(0, bars);
            if (okt) {
                tc_fence_after();
                issue_gemm1(tap(0), b1, part, d1, idesc, n, bar_1);
            }
        }
        ok = all_ok(okt, a.err);
    }
    for (int p = 0; p < np && ok; ++p) {
        float aw[2][16];
        if (p > 0) load_a(p - 1, aw);
        if (a.atten && p + 1 < np) tc_prefetch_plane(arow(p + 1), n, nz);
        // GEMM 1(p) done; so is GEMM 2(p-1), issued before it: A2, D2[(p-1)&1]
        // and the Toeplitz slot of plane p-1 are free
        const bool ok1 = mbar_wait(bar_1, (uint32_t)p & 1u);
        if (tid == 0 && ok1 && p > 0 && p + 2 < np) tl.load((p + 2) % 3, tap((p + 2) % 3), tsrc(p + 2), bars);
        tc_fence_after();
        if (ok1) d1_to_a2(a2, part, d1, n);
        fence_async_smem();
        tc_fence_before();
        ok = all_ok(ok1, a.err);
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            issue_gemm2(a2, part, tap(p % 3), d2(p & 1), idesc, n, false, p + 1 == np ? bar_2 : 0u);
            if (p + 1 < np && tl.wait((p + 1) % 3, bars)) issue_gemm1(tap((p + 1) % 3), b1, part, d1, idesc, n, bar_1);
        }
        __syncwarp();  // warp 0 reconverges before its warp-wide TMEM loads
        if (p > 0) finish(p - 1, aw);
    }
    if (ok && np > 0) {
        float aw[2][16];
        load_a(np - 1, aw);
        ok = all_ok(mbar_wait(bar_2, 0u), a.err);  // the last GEMM 2
        if (ok) {
            tc_fence_after();
            finish(np - 1, aw);
        }
    }
    if (!ok && tid == 0) {
        tl.drain(bars, kBackSlots);
        tc_drain(bar_d);
    }
    tc_end(tmem, a.tmem_cols);
}

namespace {
// devices on which the kernels' shared-memory limits have been raised
unsigned long long g_fwd_bf16_mask = 0, g_back_bf16_mask = 0;

size_t fwd_smem(int n) { return (size_t)fwd_bar_offset(n) + kBarBytes; }
size_t back_smem(int n) { return (size_t)back_bar_offset(n) + kBarBytes; }

template <class F>
cudaError_t raise_smem(F fn, size_t bytes, unsigned long long& mask)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (mask & (1ull << (dev & 63))) return cudaSuccess;
    // the largest footprint of any supported n, so one setting serves all plans
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) mask |= 1ull << (dev & 63);
    return e;
}
}  // namespace

int bf16_occupancy(int n)
{
    int blocks = 0;
    if (raise_smem(forward_bf16_kernel, fwd_smem(kTcM), g_fwd_bf16_mask) != cudaSuccess ||
        raise_smem(blur_back_bf16_kernel, back_smem(kTcM), g_back_bf16_mask) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, forward_bf16_kernel, kTcThreads, fwd_smem(n)) !=
            cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return blocks > 0 ? blocks : 1;
}

size_t bf16_smem_bytes(int n) { return std::max(fwd_smem(n), back_smem(n)); }

uint32_t bf16_tmem_cols(int n, int tiles)
{
    uint32_t c = 32;
    while (c < (uint32_t)(tiles * n)) c <<= 1;
    return c;
}

cudaError_t launch_forward_bf16(const ForwardBf16Args& a, cudaStream_t st)
{
    cudaError_t e = raise_smem(forward_bf16_kernel, fwd_smem(kTcM), g_fwd_bf16_mask);
    if (e != cudaSuccess) return e;
    dim3 grid(a.chunks, a.n_sel, a.batch);
    forward_bf16_kernel<<<grid, kTcThreads, fwd_smem(a.n), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_blur_back_bf16(const BlurBackBf16Args& a, cudaStream_t st)
{
    cudaError_t e = raise_smem(blur_back_bf16_kernel, back_smem(kTcM), g_back_bf16_mask);
    if (e != cudaSuccess) return e;
    dim3 grid(a.chunks, a.n_sel, a.batch);
    blur_back_bf16_kernel<<<grid, kTcThreads, back_smem(a.n), st>>>(a);
    return cudaGetLastError();
}

}  // namespace spect
