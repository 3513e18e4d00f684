// Internal declarations shared by the libspect translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "spect.h"

namespace spect {

constexpr int kMaxR = 20;            // largest supported PSF radius (taps 2*kMaxR+1)
constexpr int kTapW = 2 * kMaxR + 1; // row width of the device taps table
constexpr int kStrip = 16;           // outputs per thread along one blur strip
constexpr int kFwdThreads = 512;     // most threads of the forward / blur kernels
constexpr int kMaxCand = 9;          // rotated-grid samples that can touch one voxel
constexpr int kMaxIpt = 4;           // largest j-blur strips per thread
constexpr int kTcTile = 128 * 128;   // BF16 Toeplitz tile, elements
// Depth-chunk boundaries precomputed for 1..kBoundChunks chunks per angle
// (more chunks: split on the device); chunks c start at bound_offset(c).
constexpr int kBoundChunks = 64;
constexpr int kBoundInts = kBoundChunks * (kBoundChunks + 1) / 2 + kBoundChunks;
__host__ __device__ constexpr int bound_offset(int c) { return (c - 1) * (c + 2) / 2; }
// Per PSF table ints: radii [n], forward and back work prefixes [n + 1]
// each, forward and back chunk boundaries [kBoundInts] each.
__host__ __device__ constexpr int psf_int_stride(int n) { return 3 * n + 2 + 2 * kBoundInts; }


// Shape of one plane-blur launch: which columns of z a CTA owns and the
// shared-memory layout of its buffers.
struct PlaneTiling {
    int ktile;    // output columns per z tile (multiple of kStrip unless it is nz)
    int ntiles;   // z tiles
    int rh;       // halo = largest PSF radius of the plan, rounded up to even
    int ktpad;    // ktile rounded up to kStrip
    int npad;     // n rounded up to kStrip
    int sp;       // P stride between row pairs, in 16-byte quads (odd): >= (ktpad + 2*rh) / 2
    int sq;       // Q stride between column pairs, in quads (odd): >= (npad + 2*rh) / 2
    int threads;  // CTA size (multiple of 32, <= kFwdThreads)
    int ipt;      // j-blur strips per thread (1..kMaxIpt)
    size_t smem;  // P, Q, the forward's tap-row table and the tap buffer, bytes
    // Attenuation planes staged in shared memory by bulk copies, one plane
    // ahead: row width in floats (0 when the buffer does not fit and A is
    // read from global memory), and byte offsets of the tap buffer, the
    // attenuation buffer and its mbarrier; per kernel (f: forward, b: back).
    int a_cols_f, off_taps_f, off_a_f, off_bar_f;
    int a_cols_b, off_taps_b, off_a_b, off_bar_b;
    size_t smem_f, smem_b;  // dynamic shared memory of each kernel
};

struct ForwardArgs {
    const float* x;        // [batch][n][n][nz]
    const float* atten;    // [n_angles][n][n][nz] or nullptr
    const float4* cs;      // [n_angles] (cos, sin, cj = c + T_trans shift, 0)
    const float* taps;     // [n][kTapW] centred at kMaxR
    const int* rad;        // [n]
    const int* work;       // [n+1] prefix sums of the per-plane work estimate
    const int* bounds;     // [kBoundInts] depth-chunk boundaries (see bound_offset)
    size_t taps_stride;    // floats between the angles' tap tables (0: one table)
    int rad_stride;        // ints between the angles' radius / work tables (0: one table)
    const int* sel;        // [n_sel] angle ids
    int n, nz, n_sel, batch;
    int chunks;            // depth chunks: contiguous plane ranges of equal work
    PlaneTiling t;
    float* out;            // [batch][n_sel][n][nz] raw depth sums when partials == nullptr
    float* partials;       // else [batch*n_sel*chunks][n][nz] per-chunk sums
    int* err;              // SPECT_ETIMEDOUT when a bounded wait runs out
};

// Sum of the depth-chunk partials in chunk order, and optionally the OSEM
// ratio r = y / (p + s) with FP64 count sums.
struct ReduceArgs {
    const float* partials; // [items*chunks][plane]
    int chunks;
    int items, n_sel;      // items = batch * n_sel
    int plane;             // n * nz (multiple of 4)
    float* out;            // [items][plane]: p, or r in ratio mode
    const float* y;        // [n_angles][plane] or nullptr
    const int* sel;        // angle ids (ratio mode)
    float s;
    float scale;           // forward-model scale a (multi-photopeak): r = a y / (a p + s); 1 otherwise
    const float* s_ptr;    // when not NULL, s is read from this device word
    const float* fov;      // [n_angles][plane] T_fov weights applied to p, or nullptr
    double* diag_blocks;   // [gridDim.x][3] or nullptr: sums of (p+s), y, y*p/(p+s)
};

struct BlurBackArgs {
    const float* proj;     // first projection of the group, or nullptr for all-ones projections
    size_t proj_bstride;   // elements between batch entries of proj
    const float* fov;      // [n_angles][n][nz] T_fov weights applied to proj, or nullptr
    const float* atten;    // [n_angles][n][n][nz] or nullptr
    const float* taps;
    const int* rad;
    const int* work;       // [n+1] prefix sums of the per-plane work estimate
    const int* bounds;     // [kBoundInts] depth-chunk boundaries (see bound_offset)
    size_t taps_stride;    // as ForwardArgs
    int rad_stride;
    const int* sel;        // [n_sel] angle ids
    int n, nz, n_sel, batch;
    int chunks;            // depth chunks: contiguous plane ranges of equal work
    PlaneTiling t;
    float* bvol;           // [batch][n_sel][n][n][nz] rotated-frame volumes A . (K_i r)
    int* err;              // SPECT_ETIMEDOUT when a bounded wait runs out
};

// Image update at the end of a subiteration (update.cuh).
constexpr int kUpdNone = 0, kUpdOsem = 1, kUpdOsl = 2, kUpdBsrem = 3;
struct UpdateSpec {
    int mode;              // kUpd*
    const float* sens;     // H_m^T 1 of the subset
    const float* grad;     // prior gradient grad V(x), or nullptr (zero)
    const float* sens_all; // BSREM: H^T 1 over all angles
    float beta_n;          // prior weight of the subiteration, beta / M
    float step;            // BSREM: alpha_t * M
    const float* bp_add;   // added to the back projection before the update (other photopeaks), or nullptr
};

struct GatherArgs {
    const float* bvol;     // [batch][n_sel][n][n][nz]
    const int2* tab;       // [n_angles][n*n][kMaxCand] (row offset, weight bits)
    const int* sel;        // [n_sel] angle ids
    int n, nz, n_sel, batch;
    int lanes_per_col;     // 32, or the power of two >= nz/4 when nz/4 < 32
    float* out;            // [batch][n][n][nz]
    int accumulate;        // add into out instead of overwriting
    UpdateSpec upd;        // mode != kUpdNone: update x (`out`) with the finished back projection
};

// Tiled gather (gather_tiled.cu): T x T output columns per CTA, footprint
// rows of each angle staged in shared memory by bulk copies.
constexpr int kFpMaxRows = 32;                    // rotated rows i per footprint
constexpr int kFpDescInts = 4 + 2 * kFpMaxRows;   // {i0, ni, rows, 0}, then (jlo, len) per i
// Tiled gather strip tables, per (angle, 8 x 8 tile): for each tile row (a
// warp) the rotated-grid samples whose bilinear weights reach the row, in
// kGtLists lists by the tile column of their lower weight (-1 .. 7), each of
// at most kGtMaxList entries (a 1 x 2 cell of the rotated unit grid holds at
// most three samples): a header of kGtHdr ints per row (the list lengths),
// then per row kGtLists x kGtMaxList int4 entries {footprint row, weight to
// column s, weight to s + 1, 0}.
constexpr int kGtT = 8;
constexpr int kGtLists = kGtT + 1;
constexpr int kGtMaxList = 3;
constexpr int kGtHdr = 12;
constexpr int kGtSliceBytes = kGtT * kGtHdr * 4 + kGtT * kGtLists * kGtMaxList * 16;
constexpr int kGatherMaxAngles = 16;                                // angles per back blur + gather launch
constexpr int kGatherSumWarps = 8;                                  // tiled gather: warps that sum
constexpr int kGatherTiledThreads = 32 * (kGatherSumWarps + 1);      // and one that issues the copies

struct GatherTiledArgs {
    const float* bvol;     // [batch][n_sel][n][n][nz]
    const int2* tab;       // [n_angles][n_tiles] strip tables of kGtSliceBytes (see gather_tiled.cu)
    const int* desc;       // [n_angles][n_tiles][kFpDescInts]
    const int* sel;        // [n_sel] angle ids
    int n, nz, n_sel, batch;
    int T, n_tiles;        // tile side (4 or 8), tiles
    int zs;                // z segment per CTA (divides nz, multiple of 4, <= 128)
    int rows_cap;          // largest footprint, rows
    int stages;            // footprint buffers (angles in flight + 1)
    float* out;            // [batch][n][n][nz]
    int accumulate;
    UpdateSpec upd;        // as GatherArgs
    int* err;
};

// Tensor-core PSF path (SPECT_FLAG_PSF_BF16): n % 32 == 0, n <= 128,
// nz % 8 == 0, nz <= 128; per-plane Toeplitz tiles ttab[i][hi|lo][128*128]
// (BF16 bits, K-major core-matrix layout).
struct ForwardBf16Args {
    const float* x;
    const float* atten;
    const float4* cs;
    const uint16_t* ttab;
    size_t ttab_stride;    // elements between the angles' Toeplitz tile sets (0: one set)
    const int* sel;
    int n, nz, n_sel, batch, chunks;
    uint32_t tmem_cols;
    float* out;            // raw depth sums when partials == nullptr
    float* partials;       // else [batch*n_sel*chunks][n][nz]
    int* err;              // SPECT_ETIMEDOUT when a bounded wait runs out
};

struct BlurBackBf16Args {
    const float* proj;
    size_t proj_bstride;
    const float* fov;      // T_fov weights applied to proj, or nullptr
    const float* atten;
    const uint16_t* ttab;
    size_t ttab_stride;    // elements between the angles' Toeplitz tile sets (0: one set)
    const int* sel;
    int n, nz, n_sel, batch, chunks;
    uint32_t tmem_cols;
    float* bvol;
    int* err;
};

cudaError_t launch_forward_bf16(const ForwardBf16Args& a, cudaStream_t st);
cudaError_t launch_blur_back_bf16(const BlurBackBf16Args& a, cudaStream_t st);
size_t bf16_smem_bytes(int n);
uint32_t bf16_tmem_cols(int n, int tiles);  // TMEM columns: `tiles` n-column accumulators and GEMM 2's A operand
int bf16_occupancy(int n);

PlaneTiling plane_tiling(int n, int nz, int rmax, size_t cap, size_t limit);
cudaError_t launch_forward(const ForwardArgs& a, int grid_x, cudaStream_t st);
cudaError_t launch_blur_back(const BlurBackArgs& a, int grid_x, cudaStream_t st);
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t st);
cudaError_t launch_gather_tables(const float4* cs, int n, int nz, int n_angles, int2* tab, cudaStream_t st);
cudaError_t launch_gather_tiled_tables(const float4* cs, int n, int nz, int n_angles, int T, int2* tab, int* desc,
                                       int* rows_max, int* err, cudaStream_t st);
cudaError_t launch_gather_tiled(const GatherTiledArgs& a, cudaStream_t st);
size_t gather_tiled_smem(int rows_cap, int zs, int T, int stages, int n_sel);  // n_sel: angles per launch
int forward_max_blocks_per_sm(const PlaneTiling& t);

// Per-IPT instantiations (one translation unit each, compiled in parallel).
template <int IPT> cudaError_t forward_launch_ipt(const ForwardArgs& a, int grid_x, cudaStream_t st);
template <int IPT> int forward_occupancy_ipt(int threads, size_t smem);
template <int IPT> cudaError_t blur_back_launch_ipt(const BlurBackArgs& a, int grid_x, cudaStream_t st);

// misc kernels
cudaError_t launch_attenuation(const float* mu, const float4* cs, int n, int nz, int n_angles,
                               float voxel_cm, int f64, float* atten, cudaStream_t st);
cudaError_t launch_diag_finalize(const double* part, int n_part, double* out3, cudaStream_t st);
cudaError_t launch_forward_reduce(const ReduceArgs& a, int blocks, cudaStream_t st);
constexpr int kReduceBlocks = 1024;  // largest grid of the reduction kernel
cudaError_t launch_poisson_ll(const float* y, const float* p, float s, size_t count, double* block_part,
                              int n_blocks, double* ll, float* grad, cudaStream_t st);
cudaError_t launch_fill(float* dst, size_t count, float value, cudaStream_t st);
cudaError_t launch_wait_selftest(long long limit, int* err, cudaStream_t st);
cudaError_t launch_update(float* x, const float* bp, const UpdateSpec& u, size_t count, cudaStream_t st);
constexpr int kMaxPeaks = 8;
cudaError_t launch_wsum(float* out, const float* const* in, const float* w, int terms, size_t count, cudaStream_t st);
cudaError_t launch_prior_grad(const float* x, float* grad, int n, int nz, int prior, float delta, float gamma,
                              cudaStream_t st);

}  // namespace spect

// Sets the thread-local message returned by spect_last_error().
void spect_internal_set_error(const char* msg);
// Adds kernels launched outside spect_api.cu to spect_kernel_launches().
void spect_internal_count_launches(unsigned long long kernels);

// Scratch of the calls queued on one stream of a plan: calls on different
// streams never share it, so they may run concurrently.
struct spect_plan_scratch {
    cudaStream_t stream = nullptr;
    float* partials = nullptr;    // forward depth-chunk partials [partial_planes][n][nz]
    float* bvol = nullptr;        // back-projection rotated-frame volumes [bvol_cap][vol]
    float* ratio = nullptr;       // [max_subset][n][nz]
    float* bp = nullptr;          // one volume: back projection of large subsets, other peaks
    double* diag_part = nullptr;  // [kReduceBlocks][3]
    double* ll_part = nullptr;    // poisson block partials [1024]
    float* grad = nullptr;        // MAP: prior gradient (allocated by the first MAP call on the stream)
    float* msens = nullptr;       // multi-photopeak: weighted subset sensitivity (first call)
};

struct spect_plan {
    spect_geom geom{};
    int n = 0, nz = 0, na = 0, M = 1;
    int rmax = 0;
    int device = 0, num_sms = 0;
    std::vector<double> angles;
    std::vector<std::vector<int>> subsets;  // host angle lists
    std::vector<int> rad;                   // host PSF radius per depth plane (per table)
    int psf_tables = 1;                     // PSF tables: n_angles for a non-circular orbit, else 1
    int max_subset = 0;
    spect::PlaneTiling tiling{};
    int fwd_occ = 1;         // resident forward CTAs per SM

    // device memory
    float4* d_cs = nullptr;                   // [na] (cos, sin, cj = c + T_trans shift, 0)
    float* d_fov = nullptr;                   // [na][n][nz] T_fov weights, or none
    float* d_taps = nullptr;
    int* d_rad = nullptr;
    int* d_sel_all = nullptr;                 // [na] = 0..na-1
    std::vector<int*> d_sel;                  // per subset
    float* d_atten = nullptr;                 // [na][vol]
    float* d_sens = nullptr;                  // [M][vol]
    size_t partial_planes = 0;                // capacity of a scratch's depth-chunk partials, planes
    int2* d_gtab = nullptr;                   // adjoint-rotation gather tables: [na][n*n][kMaxCand], or
                                              // tiled [na][gt_tiles] strip tables of kGtSliceBytes
    int* d_gdesc = nullptr;                   // tiled gather footprints [na][gt_tiles][kFpDescInts]
    float* d_sens_all = nullptr;              // BSREM: H^T 1 over all angles (first BSREM call)
    bool sens_all_ok = false;                 // d_sens_all matches the current attenuation map
    cudaEvent_t sens_all_ready = nullptr;     // recorded after d_sens_all was computed
    cudaStream_t sens_all_stream = nullptr;   // the stream it was computed on
    int* d_gwork = nullptr;                   // tiled gather: largest footprint (rows)
    bool gather_tiled = false;                // footprints staged in shared memory
    int gt_T = 0, gt_tiles = 0, gt_zs = 0, gt_rows = 0, gt_stages = 2;
    bool bf16 = false;                        // tensor-core PSF path
    uint16_t* d_ttab = nullptr;               // [tables][n][hi, lo][128*128] BF16 Toeplitz tiles
    int* d_err = nullptr;                     // kernel status word (bounded waits)
    size_t bvol_cap = 0;                      // capacity of a scratch's rotated-frame volumes
    // per-stream scratch (the creation stream's first), and the lock every
    // call holds while it reads or changes host-side plan state and queues
    // its work
    std::vector<std::unique_ptr<spect_plan_scratch>> scratch;
    std::mutex mtx;
    size_t device_bytes = 0;
    size_t atten_bytes = 0;
    std::vector<void*> allocations;

    // optional per-launch CUDA-event timing (spect_profile_enable)
    struct ProfRec {
        const char* name;
        cudaEvent_t start, stop;
    };
    bool prof = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<unsigned long long, double>> totals;
};
