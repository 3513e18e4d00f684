// C ABI of libspect: plans, forward/back projection, sensitivity, OSEM and
// the Poisson likelihood.  Host logic only; the kernels live in
// proj_kernels.cu and misc_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "async_copy.cuh"
#include <nvtx3/nvToolsExt.h>

#include "internal.h"

using namespace spect;

namespace {
thread_local std::string g_last_error;
}  // namespace

void spect_internal_set_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void spect_internal_count_launches(unsigned long long kernels) { g_launches += kernels; }

namespace {

cudaEvent_t take_event(spect_plan* p)
{
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Launch `kernels` kernels through `launch`, counting them and, when the
// plan profiles, bracketing them with CUDA events on the launch stream.
template <class F>
cudaError_t timed(spect_plan* p, const char* name, cudaStream_t st, int kernels, F&& launch)
{
    cudaEvent_t e0 = nullptr;
    if (p && p->prof && p->pending.size() < 1000000) {
        e0 = take_event(p);
        if (e0) cudaEventRecord(e0, st);
    }
    cudaError_t e = launch();
    if (e == cudaSuccess) g_launches += (unsigned long long)kernels;
    if (e0) {
        cudaEvent_t e1 = take_event(p);
        if (e1) {
            cudaEventRecord(e1, st);
            p->pending.push_back({name, e0, e1});
        } else {
            p->event_pool.push_back(e0);
        }
    }
    return e;
}

// Boundaries out[0..c] of the split of planes 0..n-1 (work prefix sums w)
// into c contiguous depth chunks whose heaviest chunk is as light as
// possible: the smallest feasible cap by bisection, then greedy filling
// that leaves at least one plane for every later chunk.  With c >= n the
// chunks hold one plane each and the rest are empty.
void chunk_bounds(const int* w, int n, int c, int* out)
{
    if (c >= n) {
        for (int j = 0; j <= c; ++j) out[j] = std::min(j, n);
        return;
    }
    long long lo = 0, hi = w[n];
    for (int i = 0; i < n; ++i) lo = std::max<long long>(lo, w[i + 1] - w[i]);
    auto feasible = [&](long long cap) {
        int parts = 1;
        long long s = 0;
        for (int i = 0; i < n; ++i) {
            const long long x = w[i + 1] - w[i];
            if (s + x > cap) {
                ++parts;
                s = x;
            } else {
                s += x;
            }
        }
        return parts <= c;
    };
    while (lo < hi) {
        const long long mid = (lo + hi) / 2;
        if (feasible(mid)) hi = mid;
        else lo = mid + 1;
    }
    int pos = 0;
    for (int j = 0; j < c; ++j) {
        out[j] = pos;
        if (j == c - 1) break;
        const int rem = c - j - 1;
        ++pos;  // at least one plane
        while (pos < n && w[pos + 1] - w[out[j]] <= lo && n - (pos + 1) >= rem) ++pos;
    }
    out[c] = n;
}

int fail(int status, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(SPECT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Makes the plan's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
int dev_alloc(spect_plan* p, T** out, size_t count)
{
    *out = nullptr;
    if (count == 0) return SPECT_OK;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SPECT_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    p->allocations.push_back(ptr);
    p->device_bytes += count * sizeof(T);
    *out = static_cast<T*>(ptr);
    return SPECT_OK;
}

void free_plan(spect_plan* p)
{
    if (!p) return;
    for (auto& r : p->pending) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    if (p->sens_all_ready) cudaEventDestroy(p->sens_all_ready);
    for (void* a : p->allocations) cudaFree(a);
    delete p;
}

size_t vol_elems(const spect_plan* p) { return (size_t)p->n * p->n * p->nz; }

// Round-to-nearest-even FP32 -> BF16 bits (finite inputs).
uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

float bf16_value(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Per-plane banded Toeplitz tiles T_i[r][c] = w_i(r - c) (|r - c| <= R_i) of
// the tensor-core PSF path, as BF16 hi and lo parts (w = hi + lo to ~2^-17),
// in the K-major 128-byte-swizzled layout of a 128 x 128 tile: K blocks of
// 64 columns (16 KB apart), rows of 128 B, 8-row atoms of 1 KB in which the
// 16-byte chunk c of row r sits at chunk c ^ (r % 8).
void build_toeplitz_bf16(const spect_geom& g, int n, double offset, std::vector<uint16_t>& all)
{
    const int T = 128;
    const size_t base = all.size();
    all.resize(base + (size_t)n * 2 * T * T, 0);
    uint16_t* out = all.data() + base;
    for (int i = 0; i < n; ++i) {
        const double d = (double)n - i - 0.5 + offset;
        const double s = (double)g.psf_sigma0 + (double)g.psf_slope * d;
        const int r = (int)std::ceil((double)g.psf_nsigma * s);
        std::vector<double> w(2 * r + 1);
        double sum = 0.0;
        for (int t = -r; t <= r; ++t) sum += (w[t + r] = std::exp(-(double)t * t / (2.0 * s * s)));
        for (double& v : w) v /= sum;
        uint16_t* hi = out + (size_t)i * 2 * T * T;
        uint16_t* lo = hi + (size_t)T * T;
        for (int row = 0; row < T; ++row)
            for (int col = std::max(0, row - r); col <= std::min(T - 1, row + r); ++col) {
                const double wv = w[row - col + r];
                const uint16_t h = bf16_bits((float)wv);
                const uint16_t l = bf16_bits((float)(wv - (double)bf16_value(h)));
                const int kb = col >> 6, kk = col & 63;
                const size_t byte = (size_t)kb * T * 128 + ((size_t)(row >> 3) << 10) + ((row & 7) << 7) +
                                    ((((kk >> 3) ^ (row & 7))) << 4) + ((kk & 7) << 1);
                const size_t e = byte >> 1;
                hi[e] = h;
                lo[e] = l;
            }
    }
}
size_t plane_elems(const spect_plan* p) { return (size_t)p->n * p->nz; }

// Host PSF table (Eq. 1, T_cdr): sigma_i = sigma0 + slope * (n - i - 0.5 + offset),
// R_i = ceil(nsigma * sigma_i), taps exp(-t^2 / (2 sigma_i^2)) normalised in FP64.
// One angle's table (detector offset `offset`), appended to taps / rad.
void build_psf(const spect_geom& g, int n, bool psf, double offset, std::vector<float>& all_taps,
               std::vector<int>& all_rad, int& rmax)
{
    const size_t tb = all_taps.size(), rb = all_rad.size();
    all_taps.resize(tb + (size_t)n * kTapW, 0.f);
    all_rad.resize(rb + (size_t)n, 0);
    float* taps = all_taps.data() + tb;
    int* rad = all_rad.data() + rb;
    for (int i = 0; i < n; ++i) {
        if (!psf) {
            taps[(size_t)i * kTapW + kMaxR] = 1.f;
            continue;
        }
        const double d = (double)n - i - 0.5 + offset;
        const double s = (double)g.psf_sigma0 + (double)g.psf_slope * d;
        const int r = (int)std::ceil((double)g.psf_nsigma * s);
        rad[i] = r;
        rmax = std::max(rmax, r);
        if (r > kMaxR) continue;
        double w[kTapW];
        double sum = 0.0;
        for (int t = -r; t <= r; ++t) {
            w[t + r] = std::exp(-(double)t * t / (2.0 * s * s));
            sum += w[t + r];
        }
        for (int t = -r; t <= r; ++t) taps[(size_t)i * kTapW + kMaxR + t] = (float)(w[t + r] / sum);
    }
}

// ---------------------------------------------------------------- launches

int chunk_target(const spect_plan* p, long items)
{
    const long target = (long)p->num_sms * p->fwd_occ;
    if (items >= target) return 1;
    return (int)std::max<long>(1, std::min<long>(std::max(1, p->n / 2), target / items));
}

// proj (or, with y, the ratio y / (p + s)) = H_sel x.  The depth split
// depends on the subset size only (never on the batch), so a volume
// projects to bitwise the same values alone or in a batch.  diag_blocks
// (ratio mode only) receives per-block FP64 sums; *n_diag their count.
int run_forward(spect_plan* p, spect_plan_scratch& sc, const float* x, float* out, const int* sel_dev, int n_sel,
                int batch, const float* y, float s, double* diag_blocks, int* n_diag, cudaStream_t st,
                const float* s_ptr = nullptr, float scale = 1.f)
{
    const PlaneTiling& t = p->tiling;
    // never more chunks than the partial buffer holds for one batch entry
    const int chunks = (int)std::min<size_t>(chunk_target(p, (long)n_sel * (p->bf16 ? 1 : t.ntiles)),
                                             std::max<size_t>(1, p->partial_planes / (size_t)n_sel));
    // the reduction pass also applies T_fov
    const bool use_partials = chunks > 1 || y != nullptr || p->d_fov != nullptr;
    const size_t vol = vol_elems(p), plane = plane_elems(p);
    int bper = batch;
    if (use_partials)
        bper = (int)std::max<size_t>(1, std::min<size_t>(batch, p->partial_planes / ((size_t)n_sel * chunks)));
    if (n_diag) *n_diag = 0;
    for (int b0 = 0; b0 < batch; b0 += bper) {
        const int nb = std::min(bper, batch - b0);
        cudaError_t e;
        if (p->bf16) {
            ForwardBf16Args a{};
            a.x = x + (size_t)b0 * vol;
            a.atten = p->d_atten;
            a.cs = p->d_cs;
            a.ttab = p->d_ttab;
            a.ttab_stride = p->psf_tables > 1 ? (size_t)p->n * 2 * kTcTile : 0;
            a.sel = sel_dev;
            a.n = p->n;
            a.nz = p->nz;
            a.n_sel = n_sel;
            a.batch = nb;
            a.chunks = chunks;
            a.tmem_cols = bf16_tmem_cols(p->n, 2);  // D1, D2
            a.out = out + (size_t)b0 * n_sel * plane;
            a.partials = use_partials ? sc.partials : nullptr;
            a.err = p->d_err;
            e = timed(p, "forward_bf16", st, 1, [&] { return launch_forward_bf16(a, st); });
        } else {
            ForwardArgs a{};
            a.x = x + (size_t)b0 * vol;
            a.atten = p->d_atten;
            a.cs = p->d_cs;
            a.taps = p->d_taps;
            a.rad = p->d_rad;
            a.work = p->d_rad + p->n;  // forward work prefix
            a.bounds = p->d_rad + 3 * p->n + 2;
            a.taps_stride = p->psf_tables > 1 ? (size_t)p->n * kTapW : 0;
            a.rad_stride = p->psf_tables > 1 ? psf_int_stride(p->n) : 0;
            a.sel = sel_dev;
            a.n = p->n;
            a.nz = p->nz;
            a.n_sel = n_sel;
            a.batch = nb;
            a.chunks = chunks;
            a.t = t;
            a.out = out + (size_t)b0 * n_sel * plane;
            a.partials = use_partials ? sc.partials : nullptr;
            a.err = p->d_err;
            e = timed(p, "forward", st, 1, [&] { return launch_forward(a, chunks * t.ntiles, st); });
        }
        if (e != cudaSuccess) return cuda_fail(e, "forward kernel launch");
        if (!use_partials) continue;
        ReduceArgs r{};
        r.partials = sc.partials;
        r.chunks = chunks;
        r.items = nb * n_sel;
        r.n_sel = n_sel;
        r.plane = (int)plane;
        r.out = out + (size_t)b0 * n_sel * plane;
        r.y = y;
        r.sel = sel_dev;
        r.s = s;
        r.scale = scale;
        r.s_ptr = s_ptr;
        r.fov = p->d_fov;
        r.diag_blocks = (y && diag_blocks) ? diag_blocks : nullptr;
        const size_t total4 = (size_t)r.items * plane / 4;
        const int blocks = (int)std::max<size_t>(1, std::min<size_t>(kReduceBlocks, (total4 + 255) / 256));
        e = timed(p, "forward_reduce", st, 1, [&] { return launch_forward_reduce(r, blocks, st); });
        if (e != cudaSuccess) return cuda_fail(e, "reduce kernel launch");
        if (n_diag) *n_diag = blocks;
    }
    return SPECT_OK;
}

// x_out (per batch entry) = sum over sel of H_a^T proj_a, optionally fused with
// the OSEM update x_out <- x_out * bp / sens (then batch must be 1).
int run_back(spect_plan* p, spect_plan_scratch& sc, const float* proj, float* x_out, const int* sel_dev, int n_sel,
             int batch, const UpdateSpec* upd, cudaStream_t st, bool accumulate = false)
{
    const size_t vol = vol_elems(p), plane = plane_elems(p);
    const int gmax = (int)std::min<size_t>(kGatherMaxAngles, p->bvol_cap);
    const bool fused = upd && n_sel <= gmax;
    // Angle groups of a fixed size (independent of the batch, so that each
    // volume is summed in the same order alone or in a batch), and as many
    // batch entries per launch as the rotated-frame buffer holds.
    const int G = std::min(gmax, n_sel);
    const int bper = std::max(1, std::min(batch, (int)(p->bvol_cap / G)));
    for (int b0 = 0; b0 < batch; b0 += bper) {
        float* out_b = (upd && !fused) ? sc.bp : x_out + (size_t)b0 * vol;
        const int nb = std::min(bper, batch - b0);
        for (int g0 = 0; g0 < n_sel; g0 += G) {
            const int ng = std::min(G, n_sel - g0);
            cudaError_t e;
            if (p->bf16) {
                BlurBackBf16Args bb{};
                bb.proj = proj ? proj + ((size_t)b0 * n_sel + g0) * plane : nullptr;
                bb.proj_bstride = (size_t)n_sel * plane;
                bb.fov = p->d_fov;
                bb.atten = p->d_atten;
                bb.ttab = p->d_ttab;
                bb.ttab_stride = p->psf_tables > 1 ? (size_t)p->n * 2 * kTcTile : 0;
                bb.sel = sel_dev + g0;
                bb.n = p->n;
                bb.nz = p->nz;
                bb.n_sel = ng;
                bb.batch = nb;
                bb.chunks = chunk_target(p, (long)nb * ng);
                bb.tmem_cols = bf16_tmem_cols(p->n, 3);  // D1, D2 twice
                bb.bvol = sc.bvol;
                bb.err = p->d_err;
                e = timed(p, "blur_back_bf16", st, 1, [&] { return launch_blur_back_bf16(bb, st); });
            } else {
                BlurBackArgs bb{};
                bb.proj = proj ? proj + ((size_t)b0 * n_sel + g0) * plane : nullptr;
                bb.proj_bstride = (size_t)n_sel * plane;
                bb.fov = p->d_fov;
                bb.atten = p->d_atten;
                bb.taps = p->d_taps;
                bb.rad = p->d_rad;
                bb.work = p->d_rad + 2 * p->n + 1;  // blur_back work prefix
                bb.bounds = p->d_rad + 3 * p->n + 2 + kBoundInts;
                bb.taps_stride = p->psf_tables > 1 ? (size_t)p->n * kTapW : 0;
                bb.rad_stride = p->psf_tables > 1 ? psf_int_stride(p->n) : 0;
                bb.sel = sel_dev + g0;
                bb.n = p->n;
                bb.nz = p->nz;
                bb.n_sel = ng;
                bb.batch = nb;
                bb.t = p->tiling;
                const int chunks = chunk_target(p, (long)nb * ng * p->tiling.ntiles);
                bb.chunks = chunks;
                bb.bvol = sc.bvol;
                bb.err = p->d_err;
                e = timed(p, "blur_back", st, 1, [&] { return launch_blur_back(bb, chunks * p->tiling.ntiles, st); });
            }
            if (e != cudaSuccess) return cuda_fail(e, "blur_back kernel launch");
            if (p->gather_tiled) {
                GatherTiledArgs gt{};
                gt.bvol = sc.bvol;
                gt.tab = p->d_gtab;
                gt.desc = p->d_gdesc;
                gt.sel = sel_dev + g0;
                gt.n = p->n;
                gt.nz = p->nz;
                gt.n_sel = ng;
                gt.batch = nb;
                gt.T = p->gt_T;
                gt.n_tiles = p->gt_tiles;
                gt.zs = p->gt_zs;
                gt.rows_cap = p->gt_rows;
                gt.stages = p->gt_stages;
                gt.out = out_b;
                gt.accumulate = g0 > 0 || accumulate;
                if (fused) gt.upd = *upd;
                gt.err = p->d_err;
                e = timed(p, fused ? "gather_update" : "gather", st, 1, [&] { return launch_gather_tiled(gt, st); });
                if (e != cudaSuccess) return cuda_fail(e, "gather kernel launch");
                continue;
            }
            GatherArgs ga{};
            ga.bvol = sc.bvol;
            ga.tab = p->d_gtab;
            ga.sel = sel_dev + g0;
            ga.n = p->n;
            ga.nz = p->nz;
            ga.n_sel = ng;
            ga.batch = nb;
            {
                int l = 1;
                while (l < p->nz / 4 && l < 32) l <<= 1;
                ga.lanes_per_col = l;
            }
            ga.out = out_b;
            ga.accumulate = g0 > 0 || accumulate;
            if (fused) ga.upd = *upd;
            e = timed(p, fused ? "gather_update" : "gather", st, 1, [&] { return launch_gather(ga, st); });
            if (e != cudaSuccess) return cuda_fail(e, "gather kernel launch");
        }
        if (upd && !fused) {
            cudaError_t e = timed(p, "update", st, 1, [&] { return launch_update(x_out + (size_t)b0 * vol, sc.bp, *upd, vol, st); });
            if (e != cudaSuccess) return cuda_fail(e, "update kernel launch");
        }
    }
    return SPECT_OK;
}

int check_plan(const spect_plan* p)
{
    if (!p) return fail(SPECT_EINVAL, "plan is NULL");
    return SPECT_OK;
}

// The scratch of the calls on stream st, created (cudaMalloc) by the first
// call on st.  The caller holds p->mtx and has made the plan's device
// current.  A stream under capture cannot allocate: its scratch has to
// exist before the capture begins.
int scratch_for(spect_plan* p, cudaStream_t st, spect_plan_scratch** out)
{
    *out = nullptr;
    for (auto& s : p->scratch)
        if (s->stream == st) {
            *out = s.get();
            return SPECT_OK;
        }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    if (cap != cudaStreamCaptureStatusNone)
        return fail(SPECT_ESTATE, "the stream is being captured and this plan has no scratch for it yet: call "
                                  "spect_plan_reserve_stream (or any call on the stream) before the capture");
    std::unique_ptr<spect_plan_scratch> s(new (std::nothrow) spect_plan_scratch());
    if (!s) return fail(SPECT_ENOMEM, "host allocation failed");
    s->stream = st;
    const size_t vol = vol_elems(p), plane = plane_elems(p);
    int rc;
    if ((rc = dev_alloc(p, &s->partials, p->partial_planes * plane)) ||
        (rc = dev_alloc(p, &s->bvol, p->bvol_cap * vol)) ||
        (rc = dev_alloc(p, &s->ratio, (size_t)p->max_subset * plane)) ||
        (rc = dev_alloc(p, &s->bp, vol)) ||
        (rc = dev_alloc(p, &s->diag_part, (size_t)kReduceBlocks * 3)) ||
        (rc = dev_alloc(p, &s->ll_part, 1024)))
        return rc;  // what was allocated stays on the plan's list and is freed with it
    *out = s.get();
    p->scratch.push_back(std::move(s));
    return SPECT_OK;
}

// Free one device allocation of the plan (a released stream's scratch).
void dev_free(spect_plan* p, void* ptr, size_t bytes)
{
    if (!ptr) return;
    auto it = std::find(p->allocations.begin(), p->allocations.end(), ptr);
    if (it == p->allocations.end()) return;
    p->allocations.erase(it);
    p->device_bytes -= bytes;
    cudaFree(ptr);
}

int subset_of(const spect_plan* p, int subset, const int** sel_dev, int* n_sel)
{
    if (subset == -1) {
        *sel_dev = p->d_sel_all;
        *n_sel = p->na;
        return SPECT_OK;
    }
    if (subset < 0 || subset >= p->M) return fail(SPECT_EINVAL, "subset %d out of range [-1, %d)", subset, p->M);
    *sel_dev = p->d_sel[subset];
    *n_sel = (int)p->subsets[subset].size();
    return SPECT_OK;
}

int osem_core(spect_plan* plan, const float* y, float s, const float* s_dev, float* x_inout, int first_subiter,
              int n_subiters, double* diag_dev, void* stream)
{
    if (int rc = check_plan(plan)) return rc;
    if (!y || !x_inout) return fail(SPECT_EINVAL, "y and x_inout must be device pointers");
    if (!aligned16(y) || !aligned16(x_inout)) return fail(SPECT_EINVAL, "y and x_inout must be 16-byte aligned");
    if (first_subiter < 0 || n_subiters < 0) return fail(SPECT_EINVAL, "negative subiteration range");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    const size_t vol = vol_elems(plan);
    for (int t = first_subiter; t < first_subiter + n_subiters; ++t) {
        const int m = t % plan->M;
        const int ns = (int)plan->subsets[m].size();
        int n_diag = 0;
        int rc = run_forward(plan, *sc, x_inout, sc->ratio, plan->d_sel[m], ns, 1, y, s,
                             diag_dev ? sc->diag_part : nullptr, &n_diag, st, s_dev);
        if (rc) return rc;
        if (diag_dev) {
            cudaError_t e = timed(plan, "diag", st, 1, [&] {
                return launch_diag_finalize(sc->diag_part, n_diag, diag_dev + 3 * (size_t)(t - first_subiter), st);
            });
            if (e != cudaSuccess) return cuda_fail(e, "diag kernel launch");
        }
        UpdateSpec u{};
        u.mode = kUpdOsem;
        u.sens = plan->d_sens + (size_t)m * vol;
        rc = run_back(plan, *sc, sc->ratio, x_inout, plan->d_sel[m], ns, 1, &u, st);
        if (rc) return rc;
    }
    return SPECT_OK;
}

// OSMAPOSL / BSREM subiterations (Eq. PGA, Table 1): per subiteration the
// ratio y / (H_m x + s), the prior gradient of the current image, then the
// back projection with the MAP update fused into the gather.
int map_core(spect_plan* plan, const float* y, float s, float* x_inout, int first_subiter, int n_subiters,
             const spect_map_params* mp, void* stream)
{
    if (int rc = check_plan(plan)) return rc;
    if (!mp) return fail(SPECT_EINVAL, "params is NULL");
    if (mp->algorithm != SPECT_ALG_OSMAPOSL && mp->algorithm != SPECT_ALG_BSREM)
        return fail(SPECT_EINVAL, "unknown algorithm %d", mp->algorithm);
    if (mp->prior < SPECT_PRIOR_NONE || mp->prior > SPECT_PRIOR_RDP) return fail(SPECT_EINVAL, "unknown prior %d", mp->prior);
    if (mp->prior == SPECT_PRIOR_QUADRATIC && !(mp->delta > 0.f)) return fail(SPECT_EINVAL, "delta must be > 0");
    if (mp->prior == SPECT_PRIOR_RDP && !(mp->gamma >= 0.f)) return fail(SPECT_EINVAL, "gamma must be >= 0");
    if (!(mp->beta >= 0.f)) return fail(SPECT_EINVAL, "beta must be >= 0");
    if (mp->algorithm == SPECT_ALG_BSREM && !(mp->alpha0 > 0.f)) return fail(SPECT_EINVAL, "alpha0 must be > 0");
    if (!y || !x_inout) return fail(SPECT_EINVAL, "y and x_inout must be device pointers");
    if (!aligned16(y) || !aligned16(x_inout)) return fail(SPECT_EINVAL, "y and x_inout must be 16-byte aligned");
    if (first_subiter < 0 || n_subiters < 0) return fail(SPECT_EINVAL, "negative subiteration range");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    int rc;
    if ((rc = scratch_for(plan, st, &sc))) return rc;
    const size_t vol = vol_elems(plan);
    if (!sc->grad && ((rc = dev_alloc(plan, &sc->grad, vol)))) return rc;
    if (mp->algorithm == SPECT_ALG_BSREM && !plan->sens_all_ok) {
        // H^T 1 over all angles, once per attenuation map, on this stream;
        // calls on other streams wait for it through an event
        if (!plan->d_sens_all && ((rc = dev_alloc(plan, &plan->d_sens_all, vol)))) return rc;
        if (!plan->sens_all_ready) {
            cudaError_t e = cudaEventCreateWithFlags(&plan->sens_all_ready, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "create event");
        }
        rc = run_back(plan, *sc, nullptr, plan->d_sens_all, plan->d_sel_all, plan->na, 1, nullptr, st);
        if (rc) return rc;
        cudaError_t e = cudaEventRecord(plan->sens_all_ready, st);
        if (e != cudaSuccess) return cuda_fail(e, "record event");
        plan->sens_all_stream = st;
        plan->sens_all_ok = true;
    } else if (mp->algorithm == SPECT_ALG_BSREM && plan->sens_all_stream != st) {
        cudaError_t e = cudaStreamWaitEvent(st, plan->sens_all_ready, 0);
        if (e != cudaSuccess) return cuda_fail(e, "wait for H^T 1");
    }
    const float c = 1.f / (float)plan->M;
    for (int t = first_subiter; t < first_subiter + n_subiters; ++t) {
        const int m = t % plan->M;
        const int ns = (int)plan->subsets[m].size();
        rc = run_forward(plan, *sc, x_inout, sc->ratio, plan->d_sel[m], ns, 1, y, s, nullptr, nullptr, st);
        if (rc) return rc;
        UpdateSpec u{};
        u.mode = mp->algorithm == SPECT_ALG_OSMAPOSL ? kUpdOsl : kUpdBsrem;
        u.sens = plan->d_sens + (size_t)m * vol;
        u.beta_n = mp->beta * c;
        if (mp->prior != SPECT_PRIOR_NONE) {
            cudaError_t e = timed(plan, "prior_grad", st, 1, [&] {
                return launch_prior_grad(x_inout, sc->grad, plan->n, plan->nz, mp->prior, mp->delta, mp->gamma, st);
            });
            if (e != cudaSuccess) return cuda_fail(e, "prior gradient kernel");
            u.grad = sc->grad;
        }
        if (u.mode == kUpdBsrem) {
            u.sens_all = plan->d_sens_all;
            u.step = mp->alpha0 / (1.f + (float)(t / plan->M)) / c;
        }
        rc = run_back(plan, *sc, sc->ratio, x_inout, plan->d_sel[m], ns, 1, &u, st);
        if (rc) return rc;
    }
    return SPECT_OK;
}

// OSEM for a multi-photopeak extended system matrix (Eq. extended_sm):
// per subiteration each peak's ratio r'_n = a_n y_n / (a_n H_n,m x + s_n),
// the weighted sensitivity sum_n a_n H_n,m^T 1, the back projections of the
// first peaks accumulated into a scratch volume, and the last peak's back
// projection fused with the update x <- x (sum_n H_n,m^T r'_n) / (sum_n a_n H_n,m^T 1).
// plans[0]'s back-projection buffer holds the partial sum (so plans[0] must
// differ from the last plan).
int multi_core(spect_plan* const* plans, const float* scales, int P, const float* const* y, const float* s,
               float* x, int first, int count, void* stream)
{
    if (!plans || !scales || !y || !s) return fail(SPECT_EINVAL, "plans, scales, y and s must not be NULL");
    if (P < 1 || P > kMaxPeaks) return fail(SPECT_EINVAL, "n_peaks must be in [1, %d]", kMaxPeaks);
    if (!x || !aligned16(x)) return fail(SPECT_EINVAL, "x_inout must be a 16-byte aligned device pointer");
    if (first < 0 || count < 0) return fail(SPECT_EINVAL, "negative subiteration range");
    spect_plan* p0 = plans[0];
    for (int n = 0; n < P; ++n) {
        spect_plan* q = plans[n];
        if (!q) return fail(SPECT_EINVAL, "plan %d is NULL", n);
        if (q->n != p0->n || q->nz != p0->nz || q->na != p0->na || q->M != p0->M || q->device != p0->device)
            return fail(SPECT_EINVAL, "plan %d: peaks must share volume, angles, subsets and device", n);
        if (n > 0 && q == p0) return fail(SPECT_EINVAL, "plan %d repeats plans[0]", n);
        if (!y[n] || !aligned16(y[n])) return fail(SPECT_EINVAL, "y[%d] must be a 16-byte aligned device pointer", n);
        if (!(scales[n] > 0.f) || !(s[n] >= 0.f)) return fail(SPECT_EINVAL, "peak %d: scale must be > 0, s >= 0", n);
    }
    DeviceGuard guard(p0->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plans' device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t vol = vol_elems(p0);
    int rc;
    // each peak's scratch of this stream; the plans are locked one at a time
    // (never two together), around the host work of each step
    spect_plan_scratch* sc[kMaxPeaks];
    for (int n = 0; n < P; ++n) {
        std::lock_guard<std::mutex> lock(plans[n]->mtx);
        if ((rc = scratch_for(plans[n], st, &sc[n]))) return rc;
        if (n == 0 && !sc[0]->msens && ((rc = dev_alloc(p0, &sc[0]->msens, vol)))) return rc;
    }
    for (int t = first; t < first + count; ++t) {
        const int m = t % p0->M;
        const int ns = (int)p0->subsets[m].size();
        const float* sens[kMaxPeaks];
        for (int n = 0; n < P; ++n) {
            std::lock_guard<std::mutex> lock(plans[n]->mtx);
            rc = run_forward(plans[n], *sc[n], x, sc[n]->ratio, plans[n]->d_sel[m], ns, 1, y[n], s[n], nullptr, nullptr,
                             st, nullptr, scales[n]);
            if (rc) return rc;
            sens[n] = plans[n]->d_sens + (size_t)m * vol;
        }
        {
            std::lock_guard<std::mutex> lock(p0->mtx);
            cudaError_t e = timed(p0, "sens_sum", st, 1, [&] { return launch_wsum(sc[0]->msens, sens, scales, P, vol, st); });
            if (e != cudaSuccess) return cuda_fail(e, "weighted sum kernel");
        }
        for (int n = 0; n + 1 < P; ++n) {
            std::lock_guard<std::mutex> lock(plans[n]->mtx);
            rc = run_back(plans[n], *sc[n], sc[n]->ratio, sc[0]->bp, plans[n]->d_sel[m], ns, 1, nullptr, st, n > 0);
            if (rc) return rc;
        }
        UpdateSpec u{};
        u.mode = kUpdOsem;
        u.sens = sc[0]->msens;
        u.bp_add = P > 1 ? sc[0]->bp : nullptr;
        std::lock_guard<std::mutex> lock(plans[P - 1]->mtx);
        rc = run_back(plans[P - 1], *sc[P - 1], sc[P - 1]->ratio, x, plans[P - 1]->d_sel[m], ns, 1, &u, st);
        if (rc) return rc;
    }
    return SPECT_OK;
}

// Attenuation cache A_a (T_att) from mu and the per-subset sensitivities
// H_m^T 1 (compute_normalization_factor); queued on st.
int refresh_mu(spect_plan* p, spect_plan_scratch& sc, const float* mu_dev, cudaStream_t st)
{
    const size_t vol = vol_elems(p);
    if (p->d_atten) {
        cudaError_t e = timed(p, "attenuation", st, 1, [&] {
            return launch_attenuation(mu_dev, p->d_cs, p->n, p->nz, p->na, p->geom.voxel_cm,
                                      (p->geom.flags & SPECT_FLAG_ATTEN_F64) ? 1 : 0, p->d_atten, st);
        });
        if (e != cudaSuccess) return cuda_fail(e, "attenuation kernel");
    }
    for (int m = 0; m < p->M; ++m) {
        const int rc = run_back(p, sc, nullptr, p->d_sens + (size_t)m * vol, p->d_sel[m], (int)p->subsets[m].size(),
                                1, nullptr, st);
        if (rc) return rc;
    }
    return SPECT_OK;
}

}  // namespace

// An NVTX range over one library call (host side: argument checks and the
// queueing of its kernels), named after the call, so that a profiler's
// timeline shows which call issued which kernels.  NVTX is header-only and
// costs a branch when no tool is attached.
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
    CallRange(const CallRange&) = delete;
    CallRange& operator=(const CallRange&) = delete;
};

extern "C" {

const char* spect_version(void) { return "libspect 0.1 (sm_103a)"; }

const char* spect_last_error(void) { return g_last_error.c_str(); }

const char* spect_status_str(int status)
{
    switch (status) {
        case SPECT_OK: return "SPECT_OK";
        case SPECT_EINVAL: return "SPECT_EINVAL";
        case SPECT_ENOMEM: return "SPECT_ENOMEM";
        case SPECT_ECUDA: return "SPECT_ECUDA";
        case SPECT_EBUDGET: return "SPECT_EBUDGET";
        case SPECT_ETIMEDOUT: return "SPECT_ETIMEDOUT";
        case SPECT_ECANCELLED: return "SPECT_ECANCELLED";
        case SPECT_ESTATE: return "SPECT_ESTATE";
        case SPECT_ENOTFOUND: return "SPECT_ENOTFOUND";
        default: return "SPECT_UNKNOWN";
    }
}

int spect_plan_create(const spect_geom* geom, const float* mu_dev, void* stream, spect_plan** out)
{
    CallRange range("spect_plan_create");
    if (!out) return fail(SPECT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!geom) return fail(SPECT_EINVAL, "geom is NULL");
    const spect_geom& g = *geom;
    if (g.nx != g.ny) return fail(SPECT_EINVAL, "nx (%d) != ny (%d): square transaxial grid required", g.nx, g.ny);
    if (g.nx < 2 || g.nx > 1024) return fail(SPECT_EINVAL, "nx = %d outside [2, 1024]", g.nx);
    if (g.nz < 4 || g.nz > 4096 || g.nz % 4 != 0) return fail(SPECT_EINVAL, "nz = %d must be a multiple of 4 in [4, 4096]", g.nz);
    if (g.n_angles < 1 || g.n_angles > 4096) return fail(SPECT_EINVAL, "n_angles = %d outside [1, 4096]", g.n_angles);
    if ((long long)g.nx * g.ny * g.nz * 16 >= (1ll << 31))
        return fail(SPECT_EINVAL, "volume %dx%dx%d too large (element offsets of 16 volumes must fit 31 bits)", g.nx, g.ny, g.nz);
    if (g.n_subsets < 1 || g.n_subsets > g.n_angles)
        return fail(SPECT_EINVAL, "n_subsets = %d outside [1, n_angles]", g.n_subsets);
    const unsigned known = SPECT_FLAG_ATTEN | SPECT_FLAG_PSF | SPECT_FLAG_PSF_BF16 | SPECT_FLAG_ATTEN_F64;
    if (g.flags & ~known) return fail(SPECT_EINVAL, "unknown flag bits 0x%x", g.flags & ~known);
    if (g.flags & SPECT_FLAG_PSF_BF16) {
        if (!(g.flags & SPECT_FLAG_PSF)) return fail(SPECT_EINVAL, "SPECT_FLAG_PSF_BF16 needs SPECT_FLAG_PSF");
        if (g.nx % 32 != 0 || g.nx > 128 || g.nz % 8 != 0 || g.nz > 128)
            return fail(SPECT_EINVAL, "the BF16 tensor-core PSF needs nx %% 32 == 0, nx <= 128, nz %% 8 == 0, nz <= 128 "
                                      "(got %d x %d)", g.nx, g.nz);
    }
    const bool atten = (g.flags & SPECT_FLAG_ATTEN) != 0;
    const bool psf = (g.flags & SPECT_FLAG_PSF) != 0;
    if (atten) {
        if (!mu_dev) return fail(SPECT_EINVAL, "SPECT_FLAG_ATTEN needs a mu map");
        if (!aligned16(mu_dev)) return fail(SPECT_EINVAL, "mu must be 16-byte aligned");
        if (!(g.voxel_cm > 0.f) || !std::isfinite(g.voxel_cm)) return fail(SPECT_EINVAL, "voxel_cm must be > 0");
    }
    if (psf) {
        if (!(g.psf_sigma0 > 0.f) || !(g.psf_slope >= 0.f) || !(g.psf_nsigma > 0.f) || !std::isfinite(g.psf_slope) ||
            !std::isfinite(g.psf_sigma0) || !std::isfinite(g.psf_nsigma) || !std::isfinite(g.det_offset))
            return fail(SPECT_EINVAL, "PSF needs sigma0 > 0, slope >= 0, nsigma > 0 (finite)");
        if ((double)g.psf_sigma0 + (double)g.psf_slope * ((double)g.nx - 0.5 + (double)g.det_offset) <= 0.0 ||
            (double)g.psf_sigma0 + (double)g.psf_slope * (0.5 + (double)g.det_offset) <= 0.0)
            return fail(SPECT_EINVAL, "PSF sigma must stay positive over depth");
    }

    spect_plan* p = new (std::nothrow) spect_plan();
    if (!p) return fail(SPECT_ENOMEM, "host allocation failed");
    p->geom = g;
    p->geom.angles_rad = nullptr;
    p->geom.det_offsets = nullptr;
    p->geom.det_shifts = nullptr;
    p->geom.fov_mask = nullptr;
    p->n = g.nx;
    p->nz = g.nz;
    p->na = g.n_angles;
    p->M = g.n_subsets;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = SPECT_OK;
    cudaError_t e;
    if ((e = cudaGetDevice(&p->device)) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaGetDevice"); }
    if ((e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device)) != cudaSuccess) {
        free_plan(p);
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }

    // angles: FP32 cos, sin (computed in FP64; exact 0 and +-1 at the
    // quarter turns of the default angles 2 pi a / n_angles, where the FP64
    // library values carry ~1e-16 residues) and the centre of the angle's
    // detector axis, c + the T_trans shift
    p->angles.resize(p->na);
    std::vector<float4> cs(p->na);
    for (int a = 0; a < p->na; ++a) {
        const double th = g.angles_rad ? g.angles_rad[a] : 2.0 * M_PI * (double)a / (double)p->na;
        if (!std::isfinite(th)) { free_plan(p); return fail(SPECT_EINVAL, "angle %d is not finite", a); }
        const double sh = g.det_shifts ? (double)g.det_shifts[a] : 0.0;
        if (!std::isfinite(sh) || std::fabs(sh) > 4.0 * p->n)
            { free_plan(p); return fail(SPECT_EINVAL, "detector shift %d is not finite or beyond 4 n", a); }
        p->angles[a] = th;
        double ct = std::cos(th), st = std::sin(th);
        if (!g.angles_rad && (4L * a) % p->na == 0) {
            static const double qc[4] = {1.0, 0.0, -1.0, 0.0}, qs[4] = {0.0, 1.0, 0.0, -1.0};
            const int q = (int)((4L * a / p->na) % 4);
            ct = qc[q];
            st = qs[q];
        }
        cs[a] = make_float4((float)ct, (float)st, (float)(0.5 * (double)(p->n - 1) + sh), 0.f);
    }
    if (g.fov_mask) {
        const size_t cnt = (size_t)p->na * p->n * p->nz;
        for (size_t q = 0; q < cnt; ++q)
            if (!std::isfinite(g.fov_mask[q]) || g.fov_mask[q] < 0.f) {
                free_plan(p);
                return fail(SPECT_EINVAL, "fov_mask[%zu] is not a finite value >= 0", q);
            }
    }
    // PSF tables: one per angle for a non-circular orbit, else one
    std::vector<float> taps;
    std::vector<int> rad;
    p->psf_tables = g.det_offsets ? p->na : 1;
    p->rmax = 0;
    for (int a = 0; a < p->psf_tables; ++a) {
        const double off = g.det_offsets ? (double)g.det_offsets[a] : (double)g.det_offset;
        if (!std::isfinite(off)) { free_plan(p); return fail(SPECT_EINVAL, "detector offset %d is not finite", a); }
        build_psf(g, p->n, psf, off, taps, rad, p->rmax);
    }
    p->rad = rad;
    if (p->rmax > kMaxR) {
        free_plan(p);
        return fail(SPECT_EINVAL, "PSF radius %d exceeds the supported %d (reduce psf_nsigma or the slope)", p->rmax, kMaxR);
    }
    p->subsets.assign(p->M, {});
    for (int a = 0; a < p->na; ++a) p->subsets[a % p->M].push_back(a);
    for (auto& s : p->subsets) p->max_subset = std::max(p->max_subset, (int)s.size());

    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    // leave room for the 1 KB the hardware reserves per CTA and static shared memory
    const size_t cap1 = (size_t)std::min(smem_optin, 227 * 1024) - 2048;
    p->tiling = plane_tiling(p->n, p->nz, p->rmax, cap1, (size_t)smem_optin);
    if (p->tiling.smem == 0) { free_plan(p); return fail(SPECT_EINVAL, "plane %dx%d too large for shared memory", p->n, p->nz); }
    p->bf16 = (g.flags & SPECT_FLAG_PSF_BF16) != 0;
    p->fwd_occ = p->bf16 ? bf16_occupancy(p->n) : std::max(1, forward_max_blocks_per_sm(p->tiling));

    const size_t vol = vol_elems(p), plane = plane_elems(p);
    const size_t target = (size_t)p->num_sms * p->fwd_occ;
    p->partial_planes = std::max<size_t>(2 * target, (size_t)p->max_subset);
    p->bvol_cap = (size_t)std::max(p->max_subset, 16);
    if ((rc = dev_alloc(p, &p->d_cs, p->na)) ||
        (rc = dev_alloc(p, &p->d_taps, taps.size())) ||
        (rc = dev_alloc(p, &p->d_rad, (size_t)p->psf_tables * psf_int_stride(p->n))) ||
        (rc = dev_alloc(p, &p->d_sel_all, (size_t)p->na)) ||
        (rc = dev_alloc(p, &p->d_sens, (size_t)p->M * vol)) ||
        (rc = dev_alloc(p, &p->d_gwork, 1)) ||
        (rc = dev_alloc(p, &p->d_err, 1))) {
        free_plan(p);
        return rc;
    }
    if (atten) {
        if ((rc = dev_alloc(p, &p->d_atten, (size_t)p->na * vol))) { free_plan(p); return rc; }
        p->atten_bytes = (size_t)p->na * vol * sizeof(float);
    }
    p->d_sel.assign(p->M, nullptr);
    for (int m = 0; m < p->M; ++m)
        if ((rc = dev_alloc(p, &p->d_sel[m], p->subsets[m].size()))) { free_plan(p); return rc; }

    std::vector<int> all(p->na);
    for (int a = 0; a < p->na; ++a) all[a] = a;
#define SPECT_CK(call, what)                                   \
    do {                                                       \
        cudaError_t _e = (call);                               \
        if (_e != cudaSuccess) {                               \
            cudaStreamSynchronize(st);                         \
            free_plan(p);                                      \
            return cuda_fail(_e, what);                        \
        }                                                      \
    } while (0)
    std::vector<uint16_t> ttab;
    if (p->bf16) {
        for (int a = 0; a < p->psf_tables; ++a)
            build_toeplitz_bf16(g, p->n, g.det_offsets ? (double)g.det_offsets[a] : (double)g.det_offset, ttab);
        if ((rc = dev_alloc(p, &p->d_ttab, ttab.size()))) { free_plan(p); return rc; }
    }
    SPECT_CK(cudaMemcpyAsync(p->d_cs, cs.data(), cs.size() * sizeof(float4), cudaMemcpyHostToDevice, st), "copy angles");
    if (g.fov_mask) {
        if ((rc = dev_alloc(p, &p->d_fov, (size_t)p->na * plane))) { cudaStreamSynchronize(st); free_plan(p); return rc; }
        SPECT_CK(cudaMemcpyAsync(p->d_fov, g.fov_mask, (size_t)p->na * plane * sizeof(float), cudaMemcpyHostToDevice, st),
                 "copy field-of-view weights");
    }
    SPECT_CK(cudaMemsetAsync(p->d_err, 0, sizeof(int), st), "clear status");
    if (p->bf16)
        SPECT_CK(cudaMemcpyAsync(p->d_ttab, ttab.data(), ttab.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st),
                 "copy Toeplitz tiles");
    SPECT_CK(cudaMemcpyAsync(p->d_taps, taps.data(), taps.size() * sizeof(float), cudaMemcpyHostToDevice, st), "copy taps");
    // radii, then per kernel the prefix sums of a per-plane work estimate
    // for the depth chunks: a fixed cost per plane (staging, barriers,
    // attenuation loads) plus a cost per tap, in the ratios fitted to
    // per-CTA timers on GB300 at 128^3 (1,500 CTAs of 2 to 26 planes, RMS
    // error 4 % / 8 %): 28 taps' worth per plane for the forward (4.28 us +
    // 0.155 us per tap) and 15 for the back blur (2.41 us + 0.157 us per tap)
    const size_t rstride = psf_int_stride(p->n);  // per table: radii, work prefixes, chunk boundaries
    std::vector<int> radw(p->psf_tables * rstride, 0);
    for (int a = 0; a < p->psf_tables; ++a) {
        int* rw = radw.data() + a * rstride;
        int* wf = rw + p->n;
        int* wb = wf + p->n + 1;
        for (int i = 0; i < p->n; ++i) {
            rw[i] = rad[(size_t)a * p->n + i];
            wf[i + 1] = wf[i] + 28 + (2 * rw[i] + 1);
            wb[i + 1] = wb[i] + 15 + (2 * rw[i] + 1);
        }
        int* bf = wb + p->n + 1;
        int* bb = bf + kBoundInts;
        for (int c = 1; c <= kBoundChunks; ++c) {
            chunk_bounds(wf, p->n, c, bf + bound_offset(c));
            chunk_bounds(wb, p->n, c, bb + bound_offset(c));
        }
    }
    SPECT_CK(cudaMemcpyAsync(p->d_rad, radw.data(), radw.size() * sizeof(int), cudaMemcpyHostToDevice, st), "copy radii");
    SPECT_CK(cudaMemcpyAsync(p->d_sel_all, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st), "copy angles");
    // Gather tables.  Tiled (footprints staged in shared memory) for planes
    // of at least 128 x 128 with nz <= 128 (smaller planes are faster with
    // the per-column gather): 8 x 8 tiles, whole columns (each run of
    // footprint rows is one contiguous copy) and two footprint buffers (one
    // angle in flight; a third buffer measured slower on GB300).
    p->gather_tiled = p->n >= 128 && p->nz <= 128;
    if (p->gather_tiled) {
        p->gt_T = kGtT;
        const int tx = (p->n + p->gt_T - 1) / p->gt_T;
        p->gt_tiles = tx * tx;
        if ((rc = dev_alloc(p, &p->d_gtab, (size_t)p->na * p->gt_tiles * (kGtSliceBytes / 8))) ||
            (rc = dev_alloc(p, &p->d_gdesc, (size_t)p->na * p->gt_tiles * kFpDescInts))) {
            free_plan(p);
            return rc;
        }
        SPECT_CK(cudaMemsetAsync(p->d_gwork, 0, sizeof(int), st), "clear footprint size");
        SPECT_CK(timed(p, "gather_tables", st, 1, [&] {
                     return launch_gather_tiled_tables(p->d_cs, p->n, p->nz, p->na, p->gt_T, p->d_gtab, p->d_gdesc,
                                                       p->d_gwork, p->d_err, st);
                 }),
                 "gather table kernel");
        int rows = 0, err = 0;
        SPECT_CK(cudaMemcpyAsync(&rows, p->d_gwork, sizeof(int), cudaMemcpyDeviceToHost, st), "read footprint size");
        SPECT_CK(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
        SPECT_CK(cudaStreamSynchronize(st), "gather tables");
        p->gt_rows = std::max(rows, 1);
        p->gt_zs = p->nz;
        p->gt_stages = 2;
        if (err != 0 || gather_tiled_smem(p->gt_rows, p->gt_zs, p->gt_T, 2, kGatherMaxAngles) > (size_t)smem_optin) {
            // footprints too large for shared memory, or a strip list past
            // its slots: the per-column gather, whose tables replace these
            p->gather_tiled = false;
            dev_free(p, p->d_gtab, (size_t)p->na * p->gt_tiles * kGtSliceBytes);
            dev_free(p, p->d_gdesc, (size_t)p->na * p->gt_tiles * kFpDescInts * sizeof(int));
            p->d_gtab = nullptr;
            p->d_gdesc = nullptr;
            SPECT_CK(cudaMemsetAsync(p->d_err, 0, sizeof(int), st), "clear status");
        }
    }
    if (!p->gather_tiled) {
        if ((rc = dev_alloc(p, &p->d_gtab, (size_t)p->na * p->n * p->n * kMaxCand))) {
            free_plan(p);
            return rc;
        }
        SPECT_CK(timed(p, "gather_tables", st, 1,
                       [&] { return launch_gather_tables(p->d_cs, p->n, p->nz, p->na, p->d_gtab, st); }),
                 "gather table kernel");
    }
    for (int m = 0; m < p->M; ++m)
        SPECT_CK(cudaMemcpyAsync(p->d_sel[m], p->subsets[m].data(), p->subsets[m].size() * sizeof(int),
                                 cudaMemcpyHostToDevice, st), "copy subsets");
    // the creation stream's scratch, then A_a and the sensitivities
    spect_plan_scratch* sc = nullptr;
    rc = scratch_for(p, st, &sc);
    if (!rc) rc = refresh_mu(p, *sc, mu_dev, st);
    if (rc) { cudaStreamSynchronize(st); free_plan(p); return rc; }
    SPECT_CK(cudaStreamSynchronize(st), "plan creation");
    SPECT_CK(cudaGetLastError(), "plan creation");
#undef SPECT_CK
    *out = p;
    return SPECT_OK;
}

int spect_plan_destroy(spect_plan* plan)
{
    if (!plan) return SPECT_OK;
    DeviceGuard guard(plan->device);
    free_plan(plan);
    return SPECT_OK;
}

int spect_plan_query(const spect_plan* plan, spect_plan_info* info)
{
    if (int rc = check_plan(plan)) return rc;
    if (!info) return fail(SPECT_EINVAL, "info is NULL");
    info->n = plan->n;
    info->nz = plan->nz;
    info->n_angles = plan->na;
    info->n_subsets = plan->M;
    info->max_subset_size = plan->max_subset;
    info->psf_rmax = plan->rmax;
    info->device_bytes = plan->device_bytes;
    info->atten_cache_bytes = plan->atten_bytes;
    info->ztile = plan->tiling.ktile;
    info->n_ztiles = plan->tiling.ntiles;
    info->threads = plan->tiling.threads;
    info->smem_bytes = (int)plan->tiling.smem;
    return SPECT_OK;
}

int spect_subset_size(const spect_plan* plan, int subset)
{
    if (int rc = check_plan(plan)) return rc;
    if (subset == -1) return plan->na;
    if (subset < 0 || subset >= plan->M) return fail(SPECT_EINVAL, "subset %d out of range", subset);
    return (int)plan->subsets[subset].size();
}

int spect_subset_angles(const spect_plan* plan, int subset, int* out)
{
    if (int rc = check_plan(plan)) return rc;
    if (!out) return fail(SPECT_EINVAL, "out is NULL");
    if (subset == -1) {
        for (int a = 0; a < plan->na; ++a) out[a] = a;
        return SPECT_OK;
    }
    if (subset < 0 || subset >= plan->M) return fail(SPECT_EINVAL, "subset %d out of range", subset);
    std::copy(plan->subsets[subset].begin(), plan->subsets[subset].end(), out);
    return SPECT_OK;
}

int spect_forward(spect_plan* plan, const float* x, float* proj, int subset, int batch, void* stream)
{
    CallRange range("spect_forward");
    if (int rc = check_plan(plan)) return rc;
    if (!x || !proj) return fail(SPECT_EINVAL, "x and proj must be device pointers");
    if (!aligned16(x) || !aligned16(proj)) return fail(SPECT_EINVAL, "x and proj must be 16-byte aligned");
    if (batch < 1 || batch > 65535) return fail(SPECT_EINVAL, "batch = %d outside [1, 65535]", batch);
    const int* sel;
    int ns;
    if (int rc = subset_of(plan, subset, &sel, &ns)) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    return run_forward(plan, *sc, x, proj, sel, ns, batch, nullptr, 0.f, nullptr, nullptr, st);
}

int spect_back(spect_plan* plan, const float* proj, float* x_out, int subset, int batch, void* stream)
{
    CallRange range("spect_back");
    if (int rc = check_plan(plan)) return rc;
    if (!proj || !x_out) return fail(SPECT_EINVAL, "proj and x_out must be device pointers");
    if (!aligned16(proj) || !aligned16(x_out)) return fail(SPECT_EINVAL, "proj and x_out must be 16-byte aligned");
    if (batch < 1 || batch > 65535) return fail(SPECT_EINVAL, "batch = %d outside [1, 65535]", batch);
    const int* sel;
    int ns;
    if (int rc = subset_of(plan, subset, &sel, &ns)) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    return run_back(plan, *sc, proj, x_out, sel, ns, batch, nullptr, st);
}

int spect_sensitivity(spect_plan* plan, int subset, float* out, void* stream)
{
    CallRange range("spect_sensitivity");
    if (int rc = check_plan(plan)) return rc;
    if (!out || !aligned16(out)) return fail(SPECT_EINVAL, "out must be a 16-byte aligned device pointer");
    const int* sel;
    int ns;
    if (int rc = subset_of(plan, subset, &sel, &ns)) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t vol = vol_elems(plan);
    if (subset >= 0) {
        cudaError_t e = cudaMemcpyAsync(out, plan->d_sens + (size_t)subset * vol, vol * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy sensitivity");
        return SPECT_OK;
    }
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    return run_back(plan, *sc, nullptr, out, sel, ns, 1, nullptr, st);
}

int spect_osem_run(spect_plan* plan, const float* y, float s, float* x_inout, int first_subiter, int n_subiters,
                   double* diag_dev, void* stream)
{
    CallRange range("spect_osem_run");
    if (!std::isfinite(s) || s < 0.f) return fail(SPECT_EINVAL, "s must be finite and >= 0");
    return osem_core(plan, y, s, nullptr, x_inout, first_subiter, n_subiters, diag_dev, stream);
}

int spect_osem_run_dev(spect_plan* plan, const float* y, const float* s_dev, float* x_inout, int first_subiter,
                       int n_subiters, double* diag_dev, void* stream)
{
    CallRange range("spect_osem_run_dev");
    if (!s_dev) return fail(SPECT_EINVAL, "s_dev must be a device pointer");
    return osem_core(plan, y, 0.f, s_dev, x_inout, first_subiter, n_subiters, diag_dev, stream);
}

int spect_plan_set_mu(spect_plan* plan, const float* mu_dev, void* stream)
{
    CallRange range("spect_plan_set_mu");
    if (int rc = check_plan(plan)) return rc;
    if (plan->d_atten && (!mu_dev || !aligned16(mu_dev)))
        return fail(SPECT_EINVAL, "the plan models attenuation: mu must be a 16-byte aligned device pointer");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    plan->sens_all_ok = false;  // BSREM's H^T 1 follows the attenuation map
    return refresh_mu(plan, *sc, mu_dev, st);
}

int spect_map_run(spect_plan* plan, const float* y, float s, float* x_inout, int first_subiter, int n_subiters,
                  const spect_map_params* params, void* stream)
{
    CallRange range("spect_map_run");
    return map_core(plan, y, s, x_inout, first_subiter, n_subiters, params, stream);
}

int spect_multi_osem_run(spect_plan* const* plans, const float* scales, int n_peaks, const float* const* y,
                         const float* s, float* x_inout, int first_subiter, int n_subiters, void* stream)
{
    CallRange range("spect_multi_osem_run");
    return multi_core(plans, scales, n_peaks, y, s, x_inout, first_subiter, n_subiters, stream);
}

int spect_prior_grad(const float* x, int n, int nz, int prior, float delta, float gamma, float* grad_out,
                     void* stream)
{
    if (!x || !grad_out) return fail(SPECT_EINVAL, "x and grad_out must be device pointers");
    if (n <= 0 || nz <= 0) return fail(SPECT_EINVAL, "bad volume size %d x %d x %d", n, n, nz);
    if (prior != SPECT_PRIOR_QUADRATIC && prior != SPECT_PRIOR_RDP) return fail(SPECT_EINVAL, "unknown prior %d", prior);
    if (prior == SPECT_PRIOR_QUADRATIC && !(delta > 0.f)) return fail(SPECT_EINVAL, "delta must be > 0");
    if (prior == SPECT_PRIOR_RDP && !(gamma >= 0.f)) return fail(SPECT_EINVAL, "gamma must be >= 0");
    cudaError_t e = launch_prior_grad(x, grad_out, n, nz, prior, delta, gamma, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "prior gradient kernel");
    return SPECT_OK;
}

int spect_poisson_ll(spect_plan* plan, const float* y, const float* p, float s, size_t count, double* ll_dev,
                     float* grad_proj, void* stream)
{
    CallRange range("spect_poisson_ll");
    if (int rc = check_plan(plan)) return rc;
    if (!y || !p || !ll_dev) return fail(SPECT_EINVAL, "y, p and ll must be device pointers");
    if (!aligned16(y) || !aligned16(p) || (grad_proj && !aligned16(grad_proj)))
        return fail(SPECT_EINVAL, "y, p and grad must be 16-byte aligned");
    if (!std::isfinite(s)) return fail(SPECT_EINVAL, "s must be finite");
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>(1024, (count + 255) / 256));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    if (int rc = scratch_for(plan, st, &sc)) return rc;
    cudaError_t e = timed(plan, "poisson_ll", st, 2, [&] {
        return launch_poisson_ll(y, p, s, count, sc->ll_part, blocks, ll_dev, grad_proj, st);
    });
    if (e != cudaSuccess) return cuda_fail(e, "poisson kernel launch");
    return SPECT_OK;
}

int spect_plan_reserve_stream(spect_plan* plan, void* stream)
{
    if (int rc = check_plan(plan)) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    std::lock_guard<std::mutex> lock(plan->mtx);
    spect_plan_scratch* sc;
    return scratch_for(plan, static_cast<cudaStream_t>(stream), &sc);
}

int spect_plan_release_stream(spect_plan* plan, void* stream)
{
    if (int rc = check_plan(plan)) return rc;
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    for (size_t k = 0; k < plan->scratch.size(); ++k) {
        spect_plan_scratch* s = plan->scratch[k].get();
        if (s->stream != st) continue;
        cudaError_t e = cudaStreamSynchronize(st);  // its last use has finished
        if (e != cudaSuccess) return cuda_fail(e, "synchronize the released stream");
        const size_t vol = vol_elems(plan), plane = plane_elems(plan);
        dev_free(plan, s->partials, plan->partial_planes * plane * sizeof(float));
        dev_free(plan, s->bvol, plan->bvol_cap * vol * sizeof(float));
        dev_free(plan, s->ratio, (size_t)plan->max_subset * plane * sizeof(float));
        dev_free(plan, s->bp, vol * sizeof(float));
        dev_free(plan, s->diag_part, (size_t)kReduceBlocks * 3 * sizeof(double));
        dev_free(plan, s->ll_part, 1024 * sizeof(double));
        dev_free(plan, s->grad, vol * sizeof(float));
        dev_free(plan, s->msens, vol * sizeof(float));
        plan->scratch.erase(plan->scratch.begin() + (long)k);
        return SPECT_OK;
    }
    return SPECT_OK;  // the stream had no scratch
}

int spect_plan_check(spect_plan* plan)
{
    if (int rc = check_plan(plan)) return rc;
    DeviceGuard guard(plan->device);
    std::lock_guard<std::mutex> lock(plan->mtx);
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read kernel status");
    if (err != 0) {
        cudaMemset(plan->d_err, 0, sizeof(int));
        return fail(err, "a kernel of this plan gave up a bounded wait (%s)", spect_status_str(err));
    }
    return SPECT_OK;
}

int spect_plan_selftest_timeout(spect_plan* plan, long long limit_cycles, void* stream)
{
    if (int rc = check_plan(plan)) return rc;
    if (limit_cycles < 1 || limit_cycles > kWaitCycles)
        return fail(SPECT_EINVAL, "limit_cycles must be in [1, %lld]", (long long)kWaitCycles);
    DeviceGuard guard(plan->device);
    if (!guard.ok) return fail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(plan->mtx);
    cudaError_t e = timed(plan, "wait_selftest", st, 1, [&] { return launch_wait_selftest(limit_cycles, plan->d_err, st); });
    if (e != cudaSuccess) return cuda_fail(e, "self-test kernel launch");
    return SPECT_OK;
}

int spect_profile_enable(spect_plan* plan, int on)
{
    if (int rc = check_plan(plan)) return rc;
    std::lock_guard<std::mutex> lock(plan->mtx);
    plan->prof = on != 0;
    return SPECT_OK;
}

int spect_profile_read(spect_plan* plan, spect_kernel_time* out, int max_entries, int reset)
{
    if (int rc = check_plan(plan)) return rc;
    if (max_entries < 0 || (max_entries > 0 && !out)) return fail(SPECT_EINVAL, "bad output array");
    DeviceGuard guard(plan->device);
    std::lock_guard<std::mutex> lock(plan->mtx);
    for (auto& r : plan->pending) {
        cudaError_t e = cudaEventSynchronize(r.stop);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "profile events");
        auto& tot = plan->totals[r.name];
        tot.first += 1;
        tot.second += ms;
        plan->event_pool.push_back(r.start);
        plan->event_pool.push_back(r.stop);
    }
    plan->pending.clear();
    int n = 0;
    for (auto& kv : plan->totals) {
        if (n >= max_entries) break;
        std::snprintf(out[n].name, sizeof out[n].name, "%s", kv.first.c_str());
        out[n].launches = kv.second.first;
        out[n].total_ms = kv.second.second;
        ++n;
    }
    if (reset) plan->totals.clear();
    return n;
}

unsigned long long spect_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
