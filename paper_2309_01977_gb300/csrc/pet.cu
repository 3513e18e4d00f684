// Listmode PET system matrix H = T_eta T_omega P_Sigma T_rr (Sec. 2.1.1,
// Eq. (2)) and listmode OSEM (Table 1) on sm_103a.
//
// P_Sigma is Joseph's method: one thread per line of response walks the
// voxel planes of the line's principal axis and interpolates the image
// bilinearly in the other two axes.  The image (tens of MB) stays in L2
// across the walk, so the walk is bound by L2 gather throughput, not HBM.
// The listmode OSEM subiteration is a single pass over its events: each
// thread integrates its line through the blurred image, forms
// mult / (p + s) and spreads it back along the same samples with atomic adds
// (the expectation needs no other event, so no ratio array is written).
// T_rr is three separable 1-D passes; the last pass of the back projection
// applies the multiplicative update.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "pet.h"

namespace {

constexpr int kPetMaxR = 24;          // largest T_rr radius per axis
constexpr int kPetThreads = 256;
constexpr int kPetMaxBlocks = 152 * 32;

struct RrTaps {
    int r;                       // radius (0: identity)
    float w[2 * kPetMaxR + 1];   // w[t + r], t in [-r, r]
};

struct PetGrid {
    int n[3];
    float v[3];
    long long stride[3];  // elements between neighbours along x, y, z
    long long total;      // voxels
};

enum PetMode { kModeFwd = 0, kModeMult = 1, kModeBack = 2, kModeEm = 3 };

// The walk of one line: principal axis a, planes q0 .. q0 + count - 1, the
// in-plane index coordinates (u, w) on axes b < c at plane q0 and their
// increments per plane, and the step length (mm).
struct Walk {
    int a, b, c, q0, count;
    float u0, du, w0, dw, step;
    int i0, i1;       // samples visited (the time-of-flight window, else 0 .. count - 1)
    float l0, dl;     // arc length of sample 0 from the line's midpoint and its step (mm)
};

// Time of flight: bins of `width` mm centred at (b - (nb - 1)/2) width on the
// arc length from the line's midpoint (positive towards the second end);
// the Gaussian timing kernel integrated over the bin, truncated at
// nsigma sigma + width / 2.
struct TofParams {
    int nb;             // bins (0: no time of flight)
    float width, sigma, nsigma;
    float half_win;     // nsigma sigma + width / 2: the table covers [-half_win, half_win]
    float inv_h;        // table entries per mm
};

// The bin-integrated timing weight as a function of the distance x from the
// bin centre, tabulated at kTofTab + 1 points over [-half_win, half_win] and
// read with linear interpolation: the step is (2 nsigma + width / sigma)
// sigma / kTofTab, and the error (interpolation plus single-precision
// entries) stays near 4e-7 of the peak weight for bin widths of 0.5 to 2
// sigma.
constexpr int kTofTab = 4096;
constexpr size_t kTofSmem = (kTofTab + 1) * sizeof(float);

// Element i of a three-element array with constant indices only, so that
// the array stays in registers.
template <class T>
__device__ __forceinline__ T sel3(const T (&v)[3], int i)
{
    return i == 0 ? v[0] : i == 1 ? v[1] : v[2];
}

template <bool kTof>
__device__ __forceinline__ bool walk_setup(const float* __restrict__ lor, const PetGrid& g, Walk& k,
                                           const TofParams& tp, int bin, float& cb)
{
    const float2 l0 = __ldg(reinterpret_cast<const float2*>(lor));
    const float2 l1 = __ldg(reinterpret_cast<const float2*>(lor) + 1);
    const float2 l2 = __ldg(reinterpret_cast<const float2*>(lor) + 2);
    const float p1[3] = {l0.x, l0.y, l1.x};
    const float p2[3] = {l1.y, l2.x, l2.y};
    // integer decisions in single precision, rounded op by op
    float sc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) sc[c] = __fdiv_rn(fabsf(__fsub_rn(p2[c], p1[c])), g.v[c]);
    int a = 0;
    if (sc[1] > sc[0]) a = 1;
    if (sc[2] > sel3(sc, a)) a = 2;
    if (!(sel3(sc, a) > 0.f)) return false;
    const float va = sel3(g.v, a);
    const int na = sel3(g.n, a);
    const float half = __fmul_rn(0.5f, (float)(na - 1));
    const float org = -__fmul_rn(half, va);
    const float s1 = __fdiv_rn(__fsub_rn(sel3(p1, a), org), va);
    const float s2 = __fdiv_rn(__fsub_rn(sel3(p2, a), org), va);
    float lo = ceilf(s1 < s2 ? s1 : s2), hi = floorf(s1 < s2 ? s2 : s1);
    if (lo < 0.f) lo = 0.f;
    if (hi > (float)(na - 1)) hi = (float)(na - 1);
    if (!(lo <= hi)) return false;
    k.a = a;
    k.b = a == 0 ? 1 : 0;
    k.c = a == 2 ? 1 : 2;
    k.q0 = (int)lo;
    k.count = (int)hi - k.q0 + 1;
    // sample positions in double precision from the single-precision ends
    // (double operations spelled out where the time-of-flight window, an
    // integer, depends on their rounding)
    double e1[3], e2[3], len2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double v = (double)g.v[c];
        const double o = __dmul_rn(-0.5 * (double)(g.n[c] - 1), v);
        e1[c] = __ddiv_rn(__dsub_rn((double)p1[c], o), v);
        e2[c] = __ddiv_rn(__dsub_rn((double)p2[c], o), v);
        const double d = __dsub_rn((double)p2[c], (double)p1[c]);
        len2 = __dadd_rn(len2, __dmul_rn(d, d));
    }
    const double da = __dsub_rn(sel3(e2, a), sel3(e1, a));
    const double t0 = __ddiv_rn(__dsub_rn((double)k.q0, sel3(e1, a)), da);
    const double db = sel3(e2, k.b) - sel3(e1, k.b), dc = sel3(e2, k.c) - sel3(e1, k.c);
    k.u0 = (float)(sel3(e1, k.b) + t0 * db);
    k.w0 = (float)(sel3(e1, k.c) + t0 * dc);
    k.du = (float)(db / da);
    k.dw = (float)(dc / da);
    const double len = __dsqrt_rn(len2);
    k.step = (float)((double)va * len / fabs((double)sel3(p2, a) - (double)sel3(p1, a)));
    k.i0 = 0;
    k.i1 = k.count - 1;
    if (kTof) {
        const double l0 = __dmul_rn(__dsub_rn(t0, 0.5), len);
        const double dl = __ddiv_rn(len, da);
        const double width = (double)tp.width;
        const double c = __dmul_rn(__dsub_rn((double)bin, __dmul_rn(0.5, (double)(tp.nb - 1))), width);
        const double w = __dadd_rn(__dmul_rn((double)tp.nsigma, (double)tp.sigma), __dmul_rn(0.5, width));
        double lo = __ddiv_rn(__dsub_rn(__dsub_rn(c, w), l0), dl);
        double hi = __ddiv_rn(__dsub_rn(__dadd_rn(c, w), l0), dl);
        if (dl < 0.0) {
            const double t = lo;
            lo = hi;
            hi = t;
        }
        lo = ceil(lo);
        hi = floor(hi);
        if (lo < 0.0) lo = 0.0;
        if (lo > (double)k.count) lo = (double)k.count;
        if (hi > (double)(k.count - 1)) hi = (double)(k.count - 1);
        if (hi < -1.0) hi = -1.0;
        k.i0 = (int)lo;
        k.i1 = (int)hi;
        k.l0 = (float)l0;
        k.dl = (float)dl;
        cb = (float)c;
    }
    return true;
}

// Visits the in-image bilinear taps of every sample, one image row of the
// b axis at a time: fn(idx, ok0, ok1, w0, w1) for the taps idx (along c at
// iw) and idx + stride_c (at iw + 1), each present only where ok.
template <bool kTof, class F>
__device__ __forceinline__ void walk(const Walk& k, const PetGrid& g, const TofParams& tp, float cb,
                                     const float* tof_tab, F&& fn)
{
    const long long sa = sel3(g.stride, k.a), sb = sel3(g.stride, k.b), sc = sel3(g.stride, k.c);
    const int nb = sel3(g.n, k.b), nc = sel3(g.n, k.c);
    for (int i = k.i0; i <= k.i1; ++i) {
        float wt = 1.f;
        if (kTof) {
            const float x = (fmaf((float)i, k.dl, k.l0) - cb + tp.half_win) * tp.inv_h;
            const float xc = fminf(fmaxf(x, 0.f), (float)kTofTab);
            const int j = min((int)xc, kTofTab - 1);
            const float fr = xc - (float)j;
            const float t0 = tof_tab[j], t1 = tof_tab[j + 1];
            wt = fmaf(fr, t1 - t0, t0);
        }
        const float u = fmaf((float)i, k.du, k.u0);
        const float w = fmaf((float)i, k.dw, k.w0);
        const float fu = floorf(u), fw = floorf(w);
        // outside the image by a full voxel: no tap reads anything
        if (!(fu >= -1.f && fu <= (float)(nb - 1) && fw >= -1.f && fw <= (float)(nc - 1))) continue;
        const int iu = (int)fu, iw = (int)fw;
        const float tu = u - fu, tw = w - fw;
        const long long base = (long long)(k.q0 + i) * sa + (long long)iu * sb + (long long)iw * sc;
        const bool w0ok = iw >= 0, w1ok = iw + 1 < nc;
        const float ru = (1.f - tu) * wt, su = tu * wt;
        if (iu >= 0) fn(base, w0ok, w1ok, ru * (1.f - tw), ru * tw);
        if (iu + 1 < nb) fn(base + sb, w0ok, w1ok, su * (1.f - tw), su * tw);
    }
}

// w0 img[idx] + w1 img[idx + sc] over the present taps.  Two taps next to
// each other in memory (sc == 1) inside one aligned 16-byte quad of the
// image are read with one vector load.
__device__ __forceinline__ float gather_pair(const float* __restrict__ img, long long idx, long long sc,
                                             long long total, bool ok0, bool ok1, float w0, float w1)
{
    const long long q = idx & ~3LL;
    const int r = (int)(idx & 3);
    if (sc == 1 && ok0 && ok1 && r < 3 && q + 3 < total) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(img + q));
        const float a = r == 0 ? v.x : r == 1 ? v.y : v.z;
        const float b = r == 0 ? v.y : r == 1 ? v.z : v.w;
        return fmaf(w1, b, w0 * a);
    }
    float acc = 0.f;
    if (ok0) acc = w0 * __ldg(img + idx);
    if (ok1) acc = fmaf(w1, __ldg(img + idx + sc), acc);
    return acc;
}

// bp[idx] += v0, bp[idx + sc] += v1 over the present taps: one 16-byte
// vector atomic when both fall in one aligned quad (the other two lanes add
// +0, which leaves every non-negative value unchanged), else scalar atomics.
__device__ __forceinline__ void scatter_pair(float* bp, long long idx, long long sc, long long total, bool ok0,
                                             bool ok1, float v0, float v1)
{
    const long long q = idx & ~3LL;
    const int r = (int)(idx & 3);
    if (sc == 1 && ok0 && ok1 && r < 3 && q + 3 < total) {
        const float4 v = make_float4(r == 0 ? v0 : 0.f, r == 0 ? v1 : r == 1 ? v0 : 0.f,
                                     r == 1 ? v1 : r == 2 ? v0 : 0.f, r == 2 ? v1 : 0.f);
        atomicAdd(reinterpret_cast<float4*>(bp + q), v);
        return;
    }
    if (ok0) atomicAdd(bp + idx, v0);
    if (ok1) atomicAdd(bp + idx + sc, v1);
}

struct LmArgs {
    const float* img;     // image read by the walk (blurred x, or mu)
    float* bp;            // back-projection accumulator
    const float* lors;    // [n][6]
    const float* mult;    // [n] or nullptr (1)
    const float* vals;    // kModeBack: q [n]; kModeMult: eta [n] or nullptr
    const float* s;       // kModeEm: [n] or nullptr (0)
    float* out;           // kModeFwd / kModeMult: [n]
    double* diag;         // kModeEm: 2 doubles (sum p/(p+s), events used) or nullptr
    const int* tof_bin;   // [n] time-of-flight bins (kTof kernels)
    const float* tof_tab; // [kTofTab + 1] timing weights (kTof kernels)
    long long first, stride, count;  // events first + t * stride, t < count
    PetGrid g;
    TofParams tof;
};

__device__ __forceinline__ void block_add2(double a, double b, double* dst)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    __shared__ double red[2][kPetThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = a;
        red[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < kPetThreads / 32; ++i) {
            sa += red[0][i];
            sb += red[1][i];
        }
        atomicAdd(dst, sa);
        atomicAdd(dst + 1, sb);
    }
}

template <int kMode, bool kTof>
__global__ void __launch_bounds__(kPetThreads) pet_lm_kernel(LmArgs a)
{
    extern __shared__ float tof_s[];  // kTof: the timing-weight table
    if (kTof) {
        for (int i = threadIdx.x; i <= kTofTab; i += blockDim.x) tof_s[i] = __ldg(a.tof_tab + i);
        __syncthreads();
    }
    double cons = 0.0, used = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < a.count;
         t += (long long)gridDim.x * blockDim.x) {
        const long long e = a.first + t * a.stride;
        Walk k;
        float cb = 0.f;
        const bool hit = walk_setup<kTof>(a.lors + 6 * e, a.g, k, a.tof, kTof ? __ldg(a.tof_bin + e) : 0, cb);
        if (kMode == kModeBack) {
            const float val = __ldg(a.vals + e) * (a.mult ? __ldg(a.mult + e) : 1.f);
            if (!hit || val == 0.f) continue;
            const float sv = val * k.step;
            const long long sc = sel3(a.g.stride, k.c);
            walk<kTof>(k, a.g, a.tof, cb, tof_s, [&](long long idx, bool o0, bool o1, float w0, float w1) {
                scatter_pair(a.bp, idx, sc, a.g.total, o0, o1, sv * w0, sv * w1);
            });
            continue;
        }
        float acc = 0.f;
        if (hit && (kMode != kModeMult || a.img != nullptr)) {
            const long long sc = sel3(a.g.stride, k.c);
            walk<kTof>(k, a.g, a.tof, cb, tof_s, [&](long long idx, bool o0, bool o1, float w0, float w1) {
                acc += gather_pair(a.img, idx, sc, a.g.total, o0, o1, w0, w1);
            });
        }
        const float line = hit ? acc * k.step : 0.f;
        if (kMode == kModeFwd) {
            a.out[e] = a.mult ? __ldg(a.mult + e) * line : line;
        } else if (kMode == kModeMult) {
            const float om = a.img ? expf(-line) : 1.f;
            a.out[e] = (a.vals ? __ldg(a.vals + e) : 1.f) * om;
        } else {  // kModeEm
            const float m = __ldg(a.mult + e);
            const float p = m * line;
            const float den = p + (a.s ? __ldg(a.s + e) : 0.f);
            if (!(den > 0.f)) continue;
            cons += (double)p / (double)den;
            used += 1.0;
            const float sv = m / den * k.step;
            if (hit) {
                const long long sc = sel3(a.g.stride, k.c);
                walk<kTof>(k, a.g, a.tof, cb, tof_s, [&](long long idx, bool o0, bool o1, float w0, float w1) {
                    scatter_pair(a.bp, idx, sc, a.g.total, o0, o1, sv * w0, sv * w1);
                });
            }
        }
    }
    if (kMode == kModeEm && a.diag) block_add2(cons, used, a.diag);
}

// One separable T_rr pass along axis AX (0 = x, 1 = y, 2 = z), zero padding.
// With `sens` set the pass is the last one of a back projection and writes
// x <- x * out / (sens / M) where sens / M > 0 (x unchanged elsewhere).
template <int AX>
__global__ void __launch_bounds__(kPetThreads) pet_rr_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                             RrTaps taps, int nx, int ny, int nz,
                                                             const float* __restrict__ sens, float inv_m)
{
    const long long total = (long long)nx * ny * nz;
    const int n_ax = AX == 0 ? nx : AX == 1 ? ny : nz;
    const long long st = AX == 0 ? (long long)ny * nz : AX == 1 ? nz : 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int pos = AX == 0 ? (int)(i / ((long long)ny * nz)) : AX == 1 ? (int)((i / nz) % ny) : (int)(i % nz);
        float acc = 0.f;
        for (int t = -taps.r; t <= taps.r; ++t) {
            const int p = pos - t;
            if (p < 0 || p >= n_ax) continue;
            acc = fmaf(taps.w[t + taps.r], __ldg(in + i - (long long)t * st), acc);
        }
        if (sens) {
            const float sm = __ldg(sens + i) * inv_m;
            if (sm > 0.f) out[i] = out[i] * acc / sm;
        } else {
            out[i] = acc;
        }
    }
}

// x <- x * bp / (sens / M) without T_rr.
__global__ void __launch_bounds__(kPetThreads) pet_update_kernel(float* __restrict__ x, const float* __restrict__ bp,
                                                                 const float* __restrict__ sens, float inv_m,
                                                                 long long total)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float sm = __ldg(sens + i) * inv_m;
        if (sm > 0.f) x[i] = x[i] * __ldg(bp + i) / sm;
    }
}

int pfail(int status, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    spect_internal_set_error(buf);
    return status;
}

int pcuda(cudaError_t e, const char* what)
{
    cudaGetLastError();
    return pfail(SPECT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void* p, unsigned a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

unsigned blocks_for(long long count)
{
    const long long b = (count + kPetThreads - 1) / kPetThreads;
    return (unsigned)(b < 1 ? 1 : b > kPetMaxBlocks ? kPetMaxBlocks : b);
}

struct DevGuard {
    int prev = -1;
    bool ok = true;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DevGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct pet_plan {
    pet_geom geom{};
    int device = 0;
    PetGrid grid{};
    RrTaps taps[3]{};
    bool rr = false;
    TofParams tof{};
    long long voxels = 0;
    float* mu = nullptr;
    float* tof_tab = nullptr;  // [kTofTab + 1] timing weights
    float* t1 = nullptr;
    float* t2 = nullptr;
    float* fb = nullptr;
    float* bp = nullptr;
    double* diag = nullptr;
    int diag_cap = 0;  // subiterations the diag buffer holds
    std::vector<void*> allocations;
    bool prof = false;
    struct Pending {
        std::string name;
        cudaEvent_t start, stop;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    std::map<std::string, std::pair<unsigned long long, double>> totals;
};

namespace {

template <class T>
int palloc(pet_plan* p, T** out, size_t count)
{
    *out = nullptr;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pfail(SPECT_ENOMEM, "cudaMalloc of %zu bytes failed", count * sizeof(T));
    }
    p->allocations.push_back(ptr);
    *out = static_cast<T*>(ptr);
    return SPECT_OK;
}

cudaEvent_t take_event(pet_plan* p)
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

// Launch through `fn`, count the kernels and time them when profiling.
template <class F>
int launch(pet_plan* p, const char* name, cudaStream_t st, int kernels, F&& fn)
{
    cudaEvent_t e0 = nullptr;
    if (p->prof && p->pending.size() < 1000000) {
        e0 = take_event(p);
        if (e0) cudaEventRecord(e0, st);
    }
    fn();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pcuda(e, name);
    spect_internal_count_launches((unsigned long long)kernels);
    if (e0) {
        cudaEvent_t e1 = take_event(p);
        if (e1) {
            cudaEventRecord(e1, st);
            p->pending.push_back({name, e0, e1});
        } else {
            p->event_pool.push_back(e0);
        }
    }
    return SPECT_OK;
}

// out = T_rr in (three passes through t1, t2), or the update of x (sens set).
int rr_apply(pet_plan* p, const float* in, float* out, const float* sens, cudaStream_t st)
{
    const int nx = p->geom.nx, ny = p->geom.ny, nz = p->geom.nz;
    const unsigned blocks = blocks_for(p->voxels);
    const float inv_m = 1.f / (float)p->geom.n_subsets;
    return launch(p, sens ? "rr_update" : "rr_blur", st, 3, [&] {
        pet_rr_kernel<0><<<blocks, kPetThreads, 0, st>>>(in, p->t1, p->taps[0], nx, ny, nz, nullptr, 0.f);
        pet_rr_kernel<1><<<blocks, kPetThreads, 0, st>>>(p->t1, p->t2, p->taps[1], nx, ny, nz, nullptr, 0.f);
        pet_rr_kernel<2><<<blocks, kPetThreads, 0, st>>>(p->t2, out, p->taps[2], nx, ny, nz, sens, inv_m);
    });
}

LmArgs base_args(const pet_plan* p, const float* lors, long long n)
{
    LmArgs a{};
    a.lors = lors;
    a.first = 0;
    a.stride = 1;
    a.count = n;
    a.g = p->grid;
    a.tof = p->tof;
    a.tof_tab = p->tof_tab;
    return a;
}

int check_tof(const pet_plan* p, const int* tof_bin, int64_t n)
{
    if (tof_bin && p->tof.nb == 0) return pfail(SPECT_EINVAL, "tof_bin given to a plan without time of flight");
    if (tof_bin && n > 0 && !aligned(tof_bin, 4)) return pfail(SPECT_EINVAL, "tof_bin must be 4-byte aligned");
    return SPECT_OK;
}

int check_lors(const pet_plan* p, const float* lors, int64_t n)
{
    if (!p) return pfail(SPECT_EINVAL, "plan is NULL");
    if (n < 0) return pfail(SPECT_EINVAL, "negative LOR count");
    if (n > 0 && (!lors || !aligned(lors, 8))) return pfail(SPECT_EINVAL, "lors must be an 8-byte aligned device pointer");
    return SPECT_OK;
}

int check_image(const float* x, const char* what)
{
    if (!x || !aligned(x, 16)) return pfail(SPECT_EINVAL, "%s must be a 16-byte aligned device pointer", what);
    return SPECT_OK;
}

}  // namespace

extern "C" {

int pet_plan_create(const pet_geom* geom, const float* mu_dev, void* stream, pet_plan** out)
{
    if (!out) return pfail(SPECT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!geom) return pfail(SPECT_EINVAL, "geom is NULL");
    const pet_geom& g = *geom;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.nx > 4096 || g.ny > 4096 || g.nz > 4096)
        return pfail(SPECT_EINVAL, "image size must be in [1, 4096] per axis");
    if (!(g.vx > 0.f) || !(g.vy > 0.f) || !(g.vz > 0.f)) return pfail(SPECT_EINVAL, "voxel sizes must be > 0");
    if (g.n_subsets < 1) return pfail(SPECT_EINVAL, "n_subsets must be >= 1");
    const bool rr = g.rr_sigma_mm > 0.f;
    if (rr && !(g.rr_nsigma > 0.f)) return pfail(SPECT_EINVAL, "rr_nsigma must be > 0");
    if (mu_dev && !aligned(mu_dev, 16)) return pfail(SPECT_EINVAL, "mu must be a 16-byte aligned device pointer");
    if (g.n_tof_bins < 0 || g.n_tof_bins > 4096) return pfail(SPECT_EINVAL, "n_tof_bins must be in [0, 4096]");
    if (g.n_tof_bins > 0 && (!(g.tof_bin_mm > 0.f) || !(g.tof_sigma_mm > 0.f) || !(g.tof_nsigma > 0.f)))
        return pfail(SPECT_EINVAL, "time of flight needs tof_bin_mm, tof_sigma_mm and tof_nsigma > 0");
    pet_plan* p = new pet_plan();
    p->geom = g;
    p->rr = rr;
    p->tof.nb = g.n_tof_bins;
    std::vector<float> tof_tab;
    if (g.n_tof_bins > 0) {
        p->tof.width = g.tof_bin_mm;
        p->tof.sigma = g.tof_sigma_mm;
        p->tof.nsigma = g.tof_nsigma;
        const double hw = (double)g.tof_nsigma * g.tof_sigma_mm + 0.5 * (double)g.tof_bin_mm;
        p->tof.half_win = (float)hw;
        p->tof.inv_h = (float)(kTofTab / (2.0 * hw));
        tof_tab.resize(kTofTab + 1);
        const double s2 = std::sqrt(2.0) * (double)g.tof_sigma_mm, h = 0.5 * (double)g.tof_bin_mm;
        for (int i = 0; i <= kTofTab; ++i) {
            // Phi((x + h)/sigma) - Phi((x - h)/sigma) with Phi(t) = erfc(-t/sqrt 2) / 2
            const double x = -hw + 2.0 * hw * i / kTofTab;
            tof_tab[i] = (float)(0.5 * (std::erfc(-(x + h) / s2) - std::erfc(-(x - h) / s2)));
        }
    }
    const float v[3] = {g.vx, g.vy, g.vz};
    const int n[3] = {g.nx, g.ny, g.nz};
    for (int c = 0; c < 3; ++c) {
        p->grid.n[c] = n[c];
        p->grid.v[c] = v[c];
    }
    p->grid.stride[0] = (long long)g.ny * g.nz;
    p->grid.stride[1] = g.nz;
    p->grid.stride[2] = 1;
    p->voxels = (long long)g.nx * g.ny * g.nz;
    p->grid.total = p->voxels;
    // T_rr taps per axis, in double, stored as float
    for (int c = 0; c < 3; ++c) {
        RrTaps& t = p->taps[c];
        if (!rr) {
            t.r = 0;
            t.w[0] = 1.f;
            continue;
        }
        const double s = (double)g.rr_sigma_mm / (double)v[c];
        const double rd = std::ceil((double)g.rr_nsigma * s);
        if (rd > kPetMaxR) {
            delete p;
            return pfail(SPECT_EINVAL, "T_rr radius %.0f voxels exceeds %d", rd, kPetMaxR);
        }
        t.r = (int)rd;
        double w[2 * kPetMaxR + 1], sum = 0.0;
        for (int q = -t.r; q <= t.r; ++q) {
            w[q + t.r] = std::exp(-(double)q * q / (2.0 * s * s));
            sum += w[q + t.r];
        }
        for (int q = 0; q <= 2 * t.r; ++q) t.w[q] = (float)(w[q] / sum);
    }
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return pcuda(cudaGetLastError(), "cudaGetDevice");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = SPECT_OK;
    const size_t nv = (size_t)p->voxels;
    if (!rc) rc = palloc(p, &p->t1, nv);
    if (!rc) rc = palloc(p, &p->t2, nv);
    if (!rc) rc = palloc(p, &p->fb, nv);
    if (!rc) rc = palloc(p, &p->bp, nv);
    if (!rc) {
        p->diag_cap = 64;
        rc = palloc(p, &p->diag, 2 * (size_t)p->diag_cap);
    }
    if (!rc && !tof_tab.empty()) {
        rc = palloc(p, &p->tof_tab, tof_tab.size());
        if (!rc) {
            cudaError_t e = cudaMemcpy(p->tof_tab, tof_tab.data(), tof_tab.size() * sizeof(float),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) rc = pcuda(e, "copy of the timing table");
        }
    }
    if (!rc && mu_dev) {
        rc = palloc(p, &p->mu, nv);
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(p->mu, mu_dev, nv * sizeof(float), cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) rc = pcuda(e, "copy of mu");
        }
    }
    if (rc) {
        pet_plan_destroy(p);
        return rc;
    }
    *out = p;
    return SPECT_OK;
}

int pet_plan_destroy(pet_plan* p)
{
    if (!p) return SPECT_OK;
    DevGuard guard(p->device);
    cudaDeviceSynchronize();
    for (void* a : p->allocations) cudaFree(a);
    for (auto& r : p->pending) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    delete p;
    return SPECT_OK;
}

int pet_mult(pet_plan* p, const float* lors, const float* eta, int64_t n, float* mult_out, void* stream)
{
    if (int rc = check_lors(p, lors, n)) return rc;
    if (n > 0 && (!mult_out || !aligned(mult_out, 4))) return pfail(SPECT_EINVAL, "mult_out must be a device pointer");
    if (n == 0) return SPECT_OK;
    DevGuard guard(p->device);
    if (!guard.ok) return pfail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    LmArgs a = base_args(p, lors, n);
    a.img = p->mu;
    a.vals = eta;
    a.out = mult_out;
    return launch(p, "joseph_mult", st, 1,
                  [&] { pet_lm_kernel<kModeMult, false><<<blocks_for(n), kPetThreads, 0, st>>>(a); });
}

int pet_forward(pet_plan* p, const float* x, const float* lors, const float* mult, const int* tof_bin, int64_t n,
                float* out, void* stream)
{
    if (int rc = check_lors(p, lors, n)) return rc;
    if (int rc = check_tof(p, tof_bin, n)) return rc;
    if (int rc = check_image(x, "x")) return rc;
    if (n > 0 && !out) return pfail(SPECT_EINVAL, "out is NULL");
    if (n == 0) return SPECT_OK;
    DevGuard guard(p->device);
    if (!guard.ok) return pfail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float* img = x;
    if (p->rr) {
        if (int rc = rr_apply(p, x, p->fb, nullptr, st)) return rc;
        img = p->fb;
    }
    LmArgs a = base_args(p, lors, n);
    a.img = img;
    a.mult = mult;
    a.out = out;
    a.tof_bin = tof_bin;
    return launch(p, tof_bin ? "joseph_fwd_tof" : "joseph_fwd", st, 1, [&] {
        if (tof_bin)
            pet_lm_kernel<kModeFwd, true><<<blocks_for(n), kPetThreads, kTofSmem, st>>>(a);
        else
            pet_lm_kernel<kModeFwd, false><<<blocks_for(n), kPetThreads, 0, st>>>(a);
    });
}

int pet_back(pet_plan* p, const float* q, const float* lors, const float* mult, const int* tof_bin, int64_t n,
             float* x_out, void* stream)
{
    if (int rc = check_lors(p, lors, n)) return rc;
    if (int rc = check_tof(p, tof_bin, n)) return rc;
    if (int rc = check_image(x_out, "x_out")) return rc;
    if (n > 0 && !q) return pfail(SPECT_EINVAL, "q is NULL");
    DevGuard guard(p->device);
    if (!guard.ok) return pfail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* acc = p->rr ? p->bp : x_out;
    cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)p->voxels * sizeof(float), st);
    if (e != cudaSuccess) return pcuda(e, "clear of the back projection");
    if (n > 0) {
        LmArgs a = base_args(p, lors, n);
        a.bp = acc;
        a.vals = q;
        a.mult = mult;
        a.tof_bin = tof_bin;
        if (int rc = launch(p, tof_bin ? "joseph_back_tof" : "joseph_back", st, 1, [&] {
                if (tof_bin)
                    pet_lm_kernel<kModeBack, true><<<blocks_for(n), kPetThreads, kTofSmem, st>>>(a);
                else
                    pet_lm_kernel<kModeBack, false><<<blocks_for(n), kPetThreads, 0, st>>>(a);
            }))
            return rc;
    }
    if (p->rr) return rr_apply(p, p->bp, x_out, nullptr, st);
    return SPECT_OK;
}

int pet_lm_osem_run(pet_plan* p, const float* lors, const float* mult, const float* s, const int* tof_bin,
                    int64_t n, const float* sens, float* x, int first, int count, double* diag_out, void* stream)
{
    if (int rc = check_lors(p, lors, n)) return rc;
    if (int rc = check_tof(p, tof_bin, n)) return rc;
    if (int rc = check_image(x, "x_inout")) return rc;
    if (int rc = check_image(sens, "sens")) return rc;
    if (n > 0 && !mult) return pfail(SPECT_EINVAL, "mult is NULL");
    if (first < 0 || count < 0) return pfail(SPECT_EINVAL, "negative subiteration range");
    DevGuard guard(p->device);
    if (!guard.ok) return pfail(SPECT_ECUDA, "cannot select the plan's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (diag_out && count > p->diag_cap) {
        double* d = nullptr;
        cudaError_t e = cudaMalloc(&d, 2 * (size_t)count * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return pfail(SPECT_ENOMEM, "diagnostics buffer");
        }
        p->allocations.push_back(d);
        p->diag = d;
        p->diag_cap = count;
    }
    if (diag_out && count > 0) {
        cudaError_t e = cudaMemsetAsync(p->diag, 0, 2 * (size_t)count * sizeof(double), st);
        if (e != cudaSuccess) return pcuda(e, "clear of the diagnostics");
    }
    const int M = p->geom.n_subsets;
    const float inv_m = 1.f / (float)M;
    for (int it = first; it < first + count; ++it) {
        const int m = it % M;
        const float* img = x;
        if (p->rr) {
            if (int rc = rr_apply(p, x, p->fb, nullptr, st)) return rc;
            img = p->fb;
        }
        cudaError_t e = cudaMemsetAsync(p->bp, 0, (size_t)p->voxels * sizeof(float), st);
        if (e != cudaSuccess) return pcuda(e, "clear of the back projection");
        const long long cnt = n > m ? (n - m + M - 1) / M : 0;
        if (cnt > 0) {
            LmArgs a = base_args(p, lors, cnt);
            a.first = m;
            a.stride = M;
            a.img = img;
            a.bp = p->bp;
            a.mult = mult;
            a.s = s;
            a.diag = diag_out ? p->diag + 2 * (it - first) : nullptr;
            a.tof_bin = tof_bin;
            if (int rc = launch(p, tof_bin ? "joseph_em_tof" : "joseph_em", st, 1, [&] {
                    if (tof_bin)
                        pet_lm_kernel<kModeEm, true><<<blocks_for(cnt), kPetThreads, kTofSmem, st>>>(a);
                    else
                        pet_lm_kernel<kModeEm, false><<<blocks_for(cnt), kPetThreads, 0, st>>>(a);
                }))
                return rc;
        }
        if (p->rr) {
            if (int rc = rr_apply(p, p->bp, x, sens, st)) return rc;
        } else {
            const long long nv = p->voxels;
            if (int rc = launch(p, "update", st, 1, [&] {
                    pet_update_kernel<<<blocks_for(nv), kPetThreads, 0, st>>>(x, p->bp, sens, inv_m, nv);
                }))
                return rc;
        }
    }
    if (diag_out && count > 0) {
        cudaError_t e = cudaMemcpyAsync(diag_out, p->diag, 2 * (size_t)count * sizeof(double),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return pcuda(e, "diagnostics");
    }
    return SPECT_OK;
}

int pet_profile_enable(pet_plan* p, int on)
{
    if (!p) return pfail(SPECT_EINVAL, "plan is NULL");
    p->prof = on != 0;
    return SPECT_OK;
}

int pet_profile_read(pet_plan* p, spect_kernel_time* out, int max_entries, int reset)
{
    if (!p) return pfail(SPECT_EINVAL, "plan is NULL");
    if (max_entries < 0 || (max_entries > 0 && !out)) return pfail(SPECT_EINVAL, "bad output array");
    DevGuard guard(p->device);
    for (auto& r : p->pending) {
        cudaError_t e = cudaEventSynchronize(r.stop);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess) return pcuda(e, "profile events");
        auto& tot = p->totals[r.name];
        tot.first += 1;
        tot.second += ms;
        p->event_pool.push_back(r.start);
        p->event_pool.push_back(r.stop);
    }
    p->pending.clear();
    int k = 0;
    for (auto& kv : p->totals) {
        if (k >= max_entries) break;
        std::snprintf(out[k].name, sizeof out[k].name, "%s", kv.first.c_str());
        out[k].launches = kv.second.first;
        out[k].total_ms = kv.second.second;
        ++k;
    }
    if (reset) p->totals.clear();
    return k;
}

}  // extern "C"
