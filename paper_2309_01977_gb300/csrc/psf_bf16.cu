// Depth-dependent PSF as banded-Toeplitz BF16 GEMMs on the 5th-generation
// tensor cores (tcgen05, accumulators in tensor memory), FP32 accumulation.
//
// Per depth plane i, the 2-D blur of Eq. (1)'s T_cdr is K_i P = T_i P T_i^T
// with T_i the symmetric banded Toeplitz matrix of the plane's Gaussian taps.
// Both products are issued with K-major operands:
//   GEMM 1   D1[k][j]  = sum_k' T_i[k][k'] P[j][k']          (blur along z)
//   GEMM 2   D2[k][j] += sum_j' X[k][j'] T_i[j][j']  with X = D1
// so D2 = (T_i P T_i^T)^T, and the forward keeps D2 in TMEM across the depth
// loop (P_x).  GEMM 1 reads T_i and P from shared memory; GEMM 2 reads X
// from tensor memory (the workers convert D1 there) and T_i from shared
// memory.  Every operand is split into two BF16 parts, v = v_hi + v_lo
// (v_lo = bf16(v - v_hi)), and each GEMM runs three MMA chains, T_hi v_hi +
// T_lo v_hi + T_hi v_lo, dropping only T_lo v_lo (relative ~2^-18).
// Measured against the FP64 oracle: image 3.4e-6 relative L2 on the 128^3 x
// 120-angle 4 x 8 OSEM, and below 5.2e-6 from FP32 on every request class of
// the serving mix.  Two chains (data split, BF16 taps renormalised to unit
// sum) measured 6.5e-4 on the 4 x 8 OSEM but up to 2.2e-3 on serving
// requests, over the 1e-3 bar; one chain, 2.5e-3 on the 4 x 8 OSEM.
// Rotation, attenuation, the ratio and the update stay FP32 on the CUDA
// cores.
//
// Shared-memory operands are K-major tiles with the 128-byte swizzle (see
// sw_off), so that the staging (lanes along z) stores without bank
// conflicts.  The per-plane Toeplitz pair (T_hi, T_lo) arrives by TMA bulk
// copies, only the 64-column K blocks the GEMMs read, into slots refilled as
// soon as the products before have finished with them.  The kernels are
// warp-specialised pipelines in which the tensor cores work on one plane
// while the CUDA cores stage the next (forward) or finish the previous one
// (back blur); see each kernel.
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

constexpr int kWorkers = 16;                    // worker warps: 4 TMEM lane quadrants x 4 column parts
constexpr int kTcThreads = 32 * (1 + kWorkers); // warp 0 issues copies and products, warps 1..16 work
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

// K step ks (16 elements) of a tile with R rows starts (ks / 4) R 128 +
// (ks % 4) 32 bytes into the tile; as an increment of the tile's descriptor
// (whose address field counts 16-byte units; no tile crosses 256 KB, so the
// sum never carries out of the field):
__device__ __forceinline__ uint64_t sw_kstep_desc(int ks, int R)
{
    return (uint64_t)(((ks >> 2) * R * 128 + (ks & 3) * 32) >> 4);
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

// The same product with its A operand in tensor memory: A's rows are TMEM
// lanes and its K elements run along the columns, two BF16 per 32-bit
// column (the lower K index in the lower half).  Only B is read from shared
// memory, half the shared-memory traffic of a product with both operands
// there.
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
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

// Eight 32-bit values into eight consecutive TMEM columns of this thread's
// lane, and the wait for this thread's stores.
__device__ __forceinline__ void tc_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Two values as BF16 hi parts and BF16 residuals: v = hi + lo to ~2^-17.
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    hi = pack_bf16x2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xffff0000u);
    lo = pack_bf16x2(a - ha, b - hb);
}

// One MMA chain of GEMM 1, D1 (+)= T B^T over K = 128 (tile addresses of
// one BF16 part each).  The descriptors of a chain are formed once and
// stepped by constant increments, so that issuing a product costs the
// issuing thread a few instructions.  GEMM 1 runs K steps 0 .. kz-1 only,
// kz = ceil(nz / 16): its B operand is zero beyond the axial size, so the
// steps past it would add zeros.
__device__ __forceinline__ void gemm1_chain(uint32_t t, uint32_t b, uint32_t d1, uint32_t idesc, int n, int kz,
                                            bool acc)
{
    const uint64_t da = sw_desc(t), db = sw_desc(b);
#pragma unroll
    for (int ks = 0; ks < kTcM / 16; ++ks)
        if (ks < kz)
            tc_mma(d1, da + sw_kstep_desc(ks, kTcM), db + sw_kstep_desc(ks, n), idesc, (acc || ks) ? 1u : 0u);
}


// GEMM 1: D1 = T_hi B_hi^T + T_lo B_hi^T + T_hi B_lo^T over K = 128 (the
// axial direction); T_lo sits kTile bytes after T_hi, and B (n x 128) has its
// lo part `lo` bytes after the hi part.  Completion arrives on `bar`.
__device__ __forceinline__ void issue_gemm1(uint32_t tap, uint32_t b1, uint32_t lo, uint32_t d1, uint32_t idesc, int n,
                                            int kz, uint32_t bar)
{
    gemm1_chain(tap, b1, d1, idesc, n, kz, false);
    gemm1_chain(tap + (uint32_t)kTile, b1, d1, idesc, n, kz, true);
    gemm1_chain(tap, b1 + lo, d1, idesc, n, kz, true);
    tc_commit(bar);
}

// One chain of GEMM 2 with A in tensor memory: K step ks starts 8 columns
// (16 BF16) further along A.
__device__ __forceinline__ void gemm2_chain_ts(uint32_t a_tmem, uint32_t t, uint32_t d2, uint32_t idesc, int n, bool acc)
{
    const uint64_t db = sw_desc(t);
#pragma unroll
    for (int ks = 0; ks < kTcM / 16; ++ks)
        if (ks < n / 16) tc_mma_ts(d2, a_tmem + 8u * ks, db + sw_kstep_desc(ks, kTcM), idesc, (acc || ks) ? 1u : 0u);
}


// The worker warps w = 1..kWorkers split each TMEM accumulator: warp w may
// only access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 (its lane quadrant),
// and takes the 16-column chunks c with c / 16 = (w - 1) / 4 (mod 4), so
// the 16 workers cover every (quadrant, chunk) once.
__device__ __forceinline__ int tm_quad(int warp) { return warp & 3; }
__device__ __forceinline__ int tm_col0(int warp) { return 16 * ((warp - 1) >> 2); }


// D1 (TMEM, lanes k, columns j) -> BF16 hi/lo -> GEMM 2's A operand in TMEM
// (lanes k; the hi part from column a2hi, the lo part from a2lo, j / 2
// columns in); this worker's lanes and chunks.  Returns after this thread's
// stores are done.
__device__ __forceinline__ void d1_to_a2_tmem(uint32_t a2hi, uint32_t a2lo, uint32_t d1, int n)
{
    const int warp = threadIdx.x >> 5;
    const uint32_t quad = (uint32_t)(32 * tm_quad(warp)) << 16;
    for (int c = tm_col0(warp); c < n; c += 64) {
        float v[16];
        tc_ld16(d1 + quad + (uint32_t)c, v);
        uint32_t h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) split_bf16x2(v[2 * q], v[2 * q + 1], h[q], l[q]);
        tc_st8(a2hi + quad + (uint32_t)(c >> 1), h);
        tc_st8(a2lo + quad + (uint32_t)(c >> 1), l);
    }
    tc_wait_st();
}

// TMEM columns: `tiles` accumulators of n columns, then GEMM 2's A operand
// (hi and lo parts, up to 64 columns each) from a 64-column boundary.
__host__ __device__ constexpr uint32_t a2_tmem_col(int n, int tiles) { return (uint32_t)((tiles * n + 63) / 64 * 64); }

// Bytes of one BF16 part (hi or lo) of GEMM 1's B operand (n rows x 128 K
// elements; 1 KB aligned as n % 8 == 0).
__host__ __device__ constexpr uint32_t part_bytes(int n) { return (uint32_t)n * kTcM * 2u; }

// Shared-memory layouts (every tile 1 KB aligned), then a 128-byte block of
// mbarriers with the TMEM address slot at byte 112:
//   forward:  Toeplitz pair (hi, lo) | plane buffers [2] (hi, lo) | tap-row table [n]
//   back:     T_hi slots [2] | T_lo slot | B1 = projection (hi, lo)
constexpr uint32_t kPair = 2u * kTile;  // T_hi and T_lo of one plane
constexpr uint32_t kBarBytes = 128, kTmemSlot = 112;
__host__ __device__ constexpr uint32_t fwd_rows_offset(int n) { return kPair + 4u * part_bytes(n); }
__host__ __device__ constexpr uint32_t fwd_bar_offset(int n) { return fwd_rows_offset(n) + 32u * (uint32_t)n; }
__host__ __device__ constexpr uint32_t back_bar_offset(int n) { return 3u * kTile + 2u * part_bytes(n); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The bytes of a Toeplitz tile that the GEMMs read: its leading 64-column K
// blocks (16 KB each) up to the larger of the axial size (GEMM 1's K) and
// the plane width (GEMM 2's K).
__host__ __device__ constexpr uint32_t tile_bytes(int n, int nz)
{
    return (uint32_t)(((n > nz ? n : nz) + 63) / 64) * (uint32_t)(kTcM * 128);
}

// The issuing thread's record of the Toeplitz-tile copies per slot (slot s
// completes on the barrier at bars + 8 s): a copy is pending
// from its issue until that thread has seen it land, and the parity bit of a
// slot is that of its next completion.  After a timeout, drain() waits
// (bounded) for the copies still in flight.
struct TileLoads {
    uint32_t pend = 0, par = 0;
    __device__ __forceinline__ void load(int s, uint32_t dst, const void* src, uint32_t bytes, uint32_t bars)
    {
        tma_load_1d(dst, src, bytes, bars + 8u * s);
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

// The issuing thread's record of the Toeplitz-pair copies into the slot
// (completing on `bar`): a copy is pending from its issue until that thread
// has seen it land, and `par` is the parity of the next completion.  After a
// timeout, drain() waits (bounded) for a copy still in flight, so that none
// lands after the CTA has left.
struct PairLoads {
    uint32_t pend = 0, par = 0;
    // the leading `bytes` of T_hi (at src) and of T_lo (kTile bytes further)
    __device__ __forceinline__ void load(uint32_t dst, const uint16_t* src, uint32_t bytes, uint32_t bar)
    {
        mbar_expect_tx(bar, 2u * bytes);
        bulk_load(dst, src, bytes, bar);
        bulk_load(dst + (uint32_t)kTile, src + kTcM * kTcM, bytes, bar);
        pend = 1;
    }
    __device__ __forceinline__ bool wait(uint32_t bar)
    {
        const bool ok = mbar_wait(bar, par);
        if (ok) {
            par ^= 1u;
            pend = 0;
        }
        return ok;
    }
    __device__ __forceinline__ void drain(uint32_t bar)
    {
        if (pend) mbar_wait(bar, par);
    }
};

// The issuing thread, last: one more commit covers every product it has
// issued; wait (bounded) until they are done, so that none is in flight
// when the TMEM is released.
__device__ __forceinline__ void tc_drain(uint32_t bar)
{
    tc_commit(bar);
    mbar_wait(bar, 0);
}

// Allocate `ncols` TMEM columns (warp 0) after thread 0 has initialised the
// barriers, and return their base address to every thread.
__device__ __forceinline__ uint32_t tc_alloc(uint32_t slot, uint32_t ncols)
{
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

__device__ __forceinline__ void report_timeout(int* err)
{
    if (err) atomicExch(err, SPECT_ETIMEDOUT);
}

// Bilinear taps of one rotated row (as in the FP32 forward).
struct TcTapRow {
    int off[4];
    float w[4];
};

__device__ __forceinline__ TcTapRow tc_tap_row(int n, int nz, int i, int j, float4 cs, float c)
{
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
    return t;
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

// Worker wi (0 .. kWorkers-1) owns the rows j = wi + kWorkers r of every
// plane.  Ask L2 to fetch its rows of an attenuation plane ahead of use (one
// 16-byte-aligned request per row).
__device__ __forceinline__ void prefetch_rows(const float* plane, int n, int nz, int wi)
{
    const int lane = threadIdx.x & 31;
    for (int j = wi + kWorkers * lane; j < n; j += kWorkers * 32) prefetch_l2(plane + (size_t)j * nz, (uint32_t)nz * 4u);
}

// B1[j][k] = A[j][k] * bilinear(f)[j][k] (plane i) for this worker's rows j,
// k < nz, 0 for nz <= k < 128, as BF16 hi and lo parts.  Lanes compute the
// rows' taps into the shared table first; then lane l covers k = 4l..4l+3
// with 128-bit loads (one 512-byte row per load instruction), four rows at a
// time so that twenty loads per lane are in flight together.
__device__ __forceinline__ void stage_rows(uint32_t b1, uint32_t b1_lo, TcTapRow* rows, const float* __restrict__ xb,
                                           const float* __restrict__ arow, int n, int nz, int i, float4 cs, float c,
                                           int wi)
{
    constexpr int kRows = 4;
    const int lane = threadIdx.x & 31;
    const int nr = (n - wi + kWorkers - 1) / kWorkers;  // rows of this worker
    __syncwarp();  // this warp's reads of its table entries are done
    if (lane < nr) rows[wi + kWorkers * lane] = tc_tap_row(n, nz, i, wi + kWorkers * lane, cs, c);
    __syncwarp();
    const int k = 4 * lane;
    const bool in = k < nz;
    for (int r0 = 0; r0 < nr; r0 += kRows) {
        float4 v[kRows];
        int jr[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            jr[r] = wi + kWorkers * (r0 + r);
            v[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (in) {
            float4 f[kRows][4], av[kRows];
            TcTapRow t[kRows];
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const int j = jr[r] < n ? jr[r] : wi;  // rows past n repeat a valid row; not stored
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

// B1[j][k] = proj[j][k] (all ones when proj is NULL) times the T_fov weight
// fv[j][k] (when not NULL) for this worker's rows j and k < nz, as BF16 hi
// and lo parts; lanes along k as above.
__device__ __forceinline__ void stage_proj_rows(uint32_t b1, uint32_t b1_lo, const float* __restrict__ pr,
                                                const float* __restrict__ fv, int n, int nz, int wi)
{
    const int k = 4 * (threadIdx.x & 31);
    for (int j = wi; j < n; j += kWorkers) {
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
// operand of GEMM 1(p) into D1, and X[p & 1] takes the staging of plane
// p + 2 once GEMM 1(p) is done.  The workers hand D1 over, as BF16 hi and lo
// parts, to GEMM 2's A operand A2 in tensor memory (once GEMM 2(p - 1) has
// read it); GEMM 2(p) accumulates the chunk's depth sum in D2 (P_x); once it
// is done, the Toeplitz slot takes plane p + 1's pair.  Warp 0 (one thread)
// issues the copies and the products; the 16 worker warps stage plane p + 1
// while the tensor cores run plane p, and meet the issuer on mbarriers only,
// so a fast warp has its loads in flight while the others finish.
//
// Barriers (bars + 8 q): q = 0 Toeplitz pair; 1 GEMM 1; 2 GEMM 2; 3, 4 plane
// staged into X[0], X[1] (every worker thread arrives); 5 D1 handed over
// (every worker thread); 6 final drain.

__global__ void __launch_bounds__(kTcThreads, 1) forward_bf16_kernel(ForwardBf16Args a)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int n = a.n, nz = a.nz, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const float4 cs = a.cs[angle];
    const float c = 0.5f * (float)(n - 1);
    const uint32_t base = smem_u32(tsm), part = part_bytes(n);
    const uint32_t bars = base + fwd_bar_offset(n);
    const uint32_t bar_t = bars, bar_1 = bars + 8, bar_2 = bars + 16, bar_s = bars + 24, bar_a = bars + 40,
                   bar_d = bars + 48;
    TcTapRow* rows = reinterpret_cast<TcTapRow*>(tsm + fwd_rows_offset(n));  // [n]
    if (tid == 0) {
        for (int q = 0; q < 7; ++q) mbar_init(bars + 8u * q, (q >= 3 && q <= 5) ? 32u * kWorkers : 1u);
        mbar_init_fence();
    }
    const uint32_t tmem = tc_alloc(bars + kTmemSlot, a.tmem_cols);  // D1, D2, A2 (hi, lo)
    const uint32_t d1 = tmem, d2 = tmem + (uint32_t)n;
    const uint32_t a2hi = tmem + a2_tmem_col(n, 2), a2lo = a2hi + 64u;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const int kz = (nz + 15) / 16;  // GEMM 1's K steps
    const uint32_t tbytes = tile_bytes(n, nz);  // per Toeplitz tile copy
    const uint32_t tap = base;
    const int np = chunk < n ? (n - 1 - chunk) / a.chunks + 1 : 0;
    const float* xb = a.x + (size_t)b * n * n * nz;
    const size_t item = (size_t)b * a.n_sel + sidx;
    float* dst = a.partials ? a.partials + (item * a.chunks + chunk) * (size_t)n * nz : a.out + item * (size_t)n * nz;
    auto plane = [&](int p) { return chunk + p * a.chunks; };
    auto xbuf = [&](int s) { return base + kPair + (uint32_t)s * 2u * part; };
    auto tsrc = [&](int p) { return ttab + (size_t)plane(p) * 2 * kTcM * kTcM; };
    auto arow = [&](int p) -> const float* {
        return a.atten ? a.atten + ((size_t)angle * n + plane(p)) * n * nz : nullptr;
    };

    if (np == 0) {
        // a chunk without planes (more chunks than planes): its sum is zero
        for (int e = tid; e < n * nz; e += blockDim.x) dst[e] = 0.f;
    } else if (warp == 0) {
        if (lane == 0) {
            PairLoads tl;
            tl.load(tap, tsrc(0), tbytes, bar_t);
            bool ok = true;
            for (int p = 0; p < np && ok; ++p) {
                ok = mbar_wait(bar_s + 8u * (p & 1), (uint32_t)(p >> 1) & 1u) && tl.wait(bar_t);
                if (!ok) break;
                tc_fence_after();
                issue_gemm1(tap, xbuf(p & 1), part, d1, idesc, n, kz, bar_1);
                ok = mbar_wait(bar_a, (uint32_t)p & 1u);
                if (!ok) break;
                tc_fence_after();
                gemm2_chain_ts(a2hi, tap, d2, idesc, n, p > 0);
                gemm2_chain_ts(a2hi, tap + (uint32_t)kTile, d2, idesc, n, true);
                gemm2_chain_ts(a2lo, tap, d2, idesc, n, true);
                tc_commit(bar_2);
                // GEMM 2(p) done: the Toeplitz slot takes plane p+1's pair
                ok = mbar_wait(bar_2, (uint32_t)p & 1u);
                if (ok && p + 1 < np) tl.load(tap, tsrc(p + 1), tbytes, bar_t);
            }
            if (!ok) {
                report_timeout(a.err);
                tl.drain(bar_t);
            }
            tc_drain(bar_d);
        }
        __syncwarp();
    } else {
        const int wi = warp - 1;
        if (a.atten && np > 1) prefetch_rows(arow(1), n, nz, wi);
        stage_rows(xbuf(0), part, rows, xb, arow(0), n, nz, plane(0), cs, c, wi);
        bool ok = true;
        fence_async_smem();
        mbar_arrive(bar_s);
        for (int p = 0; p < np && ok; ++p) {
            if (p + 1 < np) {
                if (a.atten && p + 2 < np) prefetch_rows(arow(p + 2), n, nz, wi);
                // X[(p+1)&1] was last read by GEMM 1(p-1), which this warp
                // saw done before its previous hand-over
                stage_rows(xbuf((p + 1) & 1), part, rows, xb, arow(p + 1), n, nz, plane(p + 1), cs, c, wi);
                fence_async_smem();
                mbar_arrive(bar_s + 8u * ((p + 1) & 1));
            }
            // GEMM 1(p) is done, and GEMM 2(p-1) has read A2: D1 becomes the
            // A operand of GEMM 2(p)
            ok = ok && mbar_wait(bar_1, (uint32_t)p & 1u);
            if (ok && p > 0) ok = mbar_wait(bar_2, (uint32_t)(p - 1) & 1u);
            if (!ok) break;
            tc_fence_after();
            d1_to_a2_tmem(a2hi, a2lo, d1, n);
            tc_fence_before();
            mbar_arrive(bar_a);
        }
        if (ok) ok = mbar_wait(bar_2, (uint32_t)(np - 1) & 1u);  // the last GEMM 2
        if (ok) {
            // D2 = (sum over the chunk's planes)^T: lanes k, columns j
            tc_fence_after();
            const int k = 32 * tm_quad(warp) + lane;
            for (int cc = tm_col0(warp); cc < n; cc += 64) {
                float v[16];
                tc_ld16(d2 + ((uint32_t)(32 * tm_quad(warp)) << 16) + (uint32_t)cc, v);
                if (k < nz) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) dst[(size_t)(cc + q) * nz + k] = v[q];
                }
            }
        } else if (lane == 0) {
            report_timeout(a.err);
        }
    }
    tc_end(tmem, a.tmem_cols);
}

// ---------------------------------------------------------------- back blur
//
// The projection of the angle is the B operand of every plane's GEMM 1.
// Plane p: GEMM 1(p) into D1; the workers hand D1 over, as BF16 hi and lo
// parts, to GEMM 2's A operand A2 in tensor memory; GEMM 2(p) into D2[p & 1];
// the workers finish the plane from D2 (times A, stored as B) while the
// tensor cores run plane p + 1.  The issuer starts GEMM 2(p) once
// A2 holds plane p and the workers have finished plane p - 2 from the same
// D2 buffer.  T_hi has two slots and is copied a plane ahead; T_lo has one:
// GEMM 2 runs its T_lo chain first, so that plane p + 1's T_lo is copied
// while GEMM 2(p)'s T_hi chains and GEMM 1(p + 1)'s run.
//
// Barriers (bars + 8 q): q = 0, 1 T_hi slots; 2 T_lo slot; 3 GEMM 1; 4, 5
// GEMM 2 into D2[0], D2[1]; 6 GEMM 2's T_lo chain; 7 projection staged
// (every worker thread arrives); 8 A2 handed over (every worker thread); 9,
// 10 plane finished from D2[0], D2[1] (every worker thread); 11 final drain.

__global__ void __launch_bounds__(kTcThreads, 1) blur_back_bf16_kernel(BlurBackBf16Args a)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int n = a.n, nz = a.nz, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x, sidx = blockIdx.y, b = blockIdx.z;
    const int angle = a.sel[sidx];
    const uint16_t* ttab = a.ttab + (size_t)angle * a.ttab_stride;  // this angle's tiles
    const uint32_t base = smem_u32(tsm), part = part_bytes(n);
    const uint32_t bars = base + back_bar_offset(n);
    const uint32_t bar_t = bars, bar_1 = bars + 24, bar_2 = bars + 32, bar_l = bars + 48, bar_s = bars + 56,
                   bar_a = bars + 64, bar_f = bars + 72, bar_d = bars + 88;
    if (tid == 0) {
        for (int q = 0; q < 12; ++q) mbar_init(bars + 8u * q, (q >= 7 && q <= 10) ? 32u * kWorkers : 1u);
        mbar_init_fence();
    }
    const uint32_t tmem = tc_alloc(bars + kTmemSlot, a.tmem_cols);  // D1, D2[0], D2[1], A2 (hi, lo)
    const uint32_t d1 = tmem;
    const uint32_t a2hi = tmem + a2_tmem_col(n, 3), a2lo = a2hi + 64u;
    const uint32_t t_lo = base + 2u * kTile, b1 = base + 3u * kTile;
    const uint32_t idesc = idesc_bf16(kTcM, n);
    const int kz = (nz + 15) / 16;  // GEMM 1's K steps
    const uint32_t tbytes = tile_bytes(n, nz);  // per Toeplitz tile copy
    const int np = chunk < n ? (n - 1 - chunk) / a.chunks + 1 : 0;
    const size_t item = (size_t)b * a.n_sel + sidx;
    const float* pr = a.proj ? a.proj + (size_t)b * a.proj_bstride + (size_t)sidx * n * nz : nullptr;
    float* bvol = a.bvol + item * (size_t)n * n * nz;
    auto plane = [&](int p) { return chunk + p * a.chunks; };
    auto t_hi = [&](int s) { return base + (uint32_t)s * kTile; };
    auto d2 = [&](int s) { return tmem + (uint32_t)(1 + s) * (uint32_t)n; };
    auto src_hi = [&](int p) { return ttab + (size_t)plane(p) * 2 * kTcM * kTcM; };
    auto src_lo = [&](int p) { return ttab + ((size_t)plane(p) * 2 + 1) * kTcM * kTcM; };
    auto arow = [&](int p) -> const float* {
        return a.atten ? a.atten + ((size_t)angle * n + plane(p)) * n * nz : nullptr;
    };

    if (np > 0 && warp == 0) {
        if (lane == 0) {
            TileLoads tl;  // slots 0, 1: T_hi; slot 2: T_lo
            tl.load(0, t_hi(0), src_hi(0), tbytes, bar_t);
            tl.load(2, t_lo, src_lo(0), tbytes, bar_t);
            if (np > 1) tl.load(1, t_hi(1), src_hi(1), tbytes, bar_t);
            bool ok = mbar_wait(bar_s, 0u);
            for (int p = 0; p < np && ok; ++p) {
                const int s = p & 1;
                // GEMM 2(p-1) done: its T_hi slot takes plane p+1's
                if (p > 0) {
                    ok = mbar_wait(bar_2 + 8u * ((p - 1) & 1), (uint32_t)((p - 1) >> 1) & 1u);
                    if (!ok) break;
                    if (p + 1 < np) tl.load((p + 1) & 1, t_hi((p + 1) & 1), src_hi(p + 1), tbytes, bar_t);
                }
                // GEMM 1(p): the T_hi chains, then the T_lo chain
                ok = tl.wait(s, bar_t);
                if (!ok) break;
                tc_fence_after();
                gemm1_chain(t_hi(s), b1, d1, idesc, n, kz, false);
                gemm1_chain(t_hi(s), b1 + part, d1, idesc, n, kz, true);
                ok = tl.wait(2, bar_t);
                if (!ok) break;
                gemm1_chain(t_lo, b1, d1, idesc, n, kz, true);
                tc_commit(bar_1);
                ok = mbar_wait(bar_a, (uint32_t)p & 1u);  // A2 holds plane p
                // D2[p&1] was last read by the finish of plane p-2
                if (ok && p >= 2) ok = mbar_wait(bar_f + 8u * s, (uint32_t)((p - 2) >> 1) & 1u);
                if (!ok) break;
                tc_fence_after();
                gemm2_chain_ts(a2hi, t_lo, d2(s), idesc, n, false);
                tc_commit(bar_l);
                gemm2_chain_ts(a2hi, t_hi(s), d2(s), idesc, n, true);
                gemm2_chain_ts(a2lo, t_hi(s), d2(s), idesc, n, true);
                tc_commit(bar_2 + 8u * s);
                // the T_lo chain done: the slot takes plane p+1's T_lo
                ok = mbar_wait(bar_l, (uint32_t)p & 1u);
                if (ok && p + 1 < np) tl.load(2, t_lo, src_lo(p + 1), tbytes, bar_t);
            }
            if (!ok) {
                report_timeout(a.err);
                tl.drain(bar_t, 3);
            }
            tc_drain(bar_d);
        }
        __syncwarp();
    } else if (np > 0) {
        const int wi = warp - 1;
        const int k = 32 * tm_quad(warp) + lane, col0 = tm_col0(warp);
        const uint32_t quad = (uint32_t)(32 * tm_quad(warp)) << 16;
        // A of plane p for this thread's elements (lane k, columns cc + q of
        // its at most two 16-column chunks), loaded ahead of the waits
        auto load_a = [&](int p, float (&aw)[2][16]) {
            const float* ar = arow(p);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int cc = col0 + 64 * m;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    aw[m][q] = (ar && cc < n && k < nz) ? __ldg(ar + (size_t)(cc + q) * nz + k) : 1.f;
            }
        };
        // B[plane p][j][k] = A * (K_i r)[j][k]; D2 holds (K_i r)^T (lanes k)
        auto finish = [&](int p, const float (&aw)[2][16]) {
            float* brow = bvol + (size_t)plane(p) * n * nz;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int cc = col0 + 64 * m;
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
        if (a.atten) prefetch_rows(arow(0), n, nz, wi);
        stage_proj_rows(b1, part, pr, a.fov ? a.fov + (size_t)angle * n * nz : nullptr, n, nz, wi);
        fence_async_smem();
        mbar_arrive(bar_s);
        bool ok = true;
        for (int p = 0; p < np && ok; ++p) {
            float aw[2][16];
            if (p > 0) load_a(p - 1, aw);
            if (a.atten && p + 1 < np) prefetch_rows(arow(p + 1), n, nz, wi);
            // GEMM 1(p) done; GEMM 2(p-1) done: A2 is free and D2[(p-1)&1] ready
            ok = mbar_wait(bar_1, (uint32_t)p & 1u);
            if (ok && p > 0) ok = mbar_wait(bar_2 + 8u * ((p - 1) & 1), (uint32_t)((p - 1) >> 1) & 1u);
            if (!ok) break;
            tc_fence_after();
            d1_to_a2_tmem(a2hi, a2lo, d1, n);
            tc_fence_before();
            mbar_arrive(bar_a);
            if (p > 0) {
                finish(p - 1, aw);
                tc_fence_before();
                mbar_arrive(bar_f + 8u * ((p - 1) & 1));
            }
        }
        if (ok) {
            float aw[2][16];
            load_a(np - 1, aw);
            ok = mbar_wait(bar_2 + 8u * ((np - 1) & 1), (uint32_t)((np - 1) >> 1) & 1u);  // the last GEMM 2
            if (ok) {
                tc_fence_after();
                finish(np - 1, aw);
            }
        }
        if (!ok && lane == 0) report_timeout(a.err);
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
    while (c < a2_tmem_col(n, tiles) + 128u) c <<= 1;
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
