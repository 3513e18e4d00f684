// Attenuation cache, FP64 count reductions and the Poisson likelihood.
#include <cuda_runtime.h>

#include "async_copy.cuh"
#include "geometry.cuh"
#include "internal.h"
#include "update.cuh"

namespace spect {

// T_att of Eq. (1) in the rotated frame of angle a: one thread per four
// detector rays (j, k..k+3) walks depth from the detector side (i = n-1)
// inward,
//   A[i] = exp(-(sum_{i'>i} tau[i'] + tau[i]/2)),  tau = voxel_cm * bilinear(mu)(u, v, k).
// The running sum is compensated (Kahan) FP32, and with f64 != 0 it is
// folded into an FP64 total every kFold steps (the last <= kFold terms are
// held as the compensated FP32 pair), so the ray's prefix sum is carried in
// FP64 at the cost of a few FP64 operations per kFold steps.  The
// exponential is FP32 in both modes.  A block covers 256 / (nz/4) rows j of
// one angle, whose bilinear taps overlap in L1.
namespace {
constexpr int kFold = 8;

struct RaySum {
    float s = 0.f, c = 0.f;  // compensated partial sum: value s - c
    double base = 0.0;       // FP64 total of the folded terms
    float base_f = 0.f;      // base rounded to FP32
    __device__ __forceinline__ float prefix() const { return base_f + (s - c); }
    __device__ __forceinline__ void add(float tau)
    {
        const float y = tau - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void fold()
    {
        base += (double)s;
        base -= (double)c;
        base_f = (float)base;
        s = c = 0.f;
    }
};
}  // namespace

__global__ void __launch_bounds__(256) attenuation_kernel(const float* __restrict__ mu, const float4* __restrict__ cs_tab,
                                                          int n, int nz, float voxel_cm, int f64,
                                                          float* __restrict__ atten)
{
    const int angle = blockIdx.y;
    const int zq = nz >> 2;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * zq) return;
    const int j = idx / zq, k = 4 * (idx - j * zq);
    const float4 cs = cs_tab[angle];
    const float c = 0.5f * (float)(n - 1);
    RaySum r[4];
    float4* out = reinterpret_cast<float4*>(atten + ((size_t)angle * n * n + j) * nz + k);
    const size_t plane4 = (size_t)n * nz / 4;
    for (int i0 = n - 1; i0 >= 0; i0 -= kFold) {
#pragma unroll
        for (int s = 0; s < kFold; ++s) {
            const int i = i0 - s;
            if (i < 0) break;
            float u, v;
            sample_point(cs.x, cs.y, c, cs.z, i, j, u, v);
            const float fu = floorf(u), fv = floorf(v);
            const int x0 = (int)fu, y0 = (int)fv;
            const float ax = u - fu, by = v - fv;
            const bool vx0 = x0 >= 0 && x0 < n, vx1 = x0 + 1 >= 0 && x0 + 1 < n;
            const bool vy0 = y0 >= 0 && y0 < n, vy1 = y0 + 1 >= 0 && y0 + 1 < n;
            float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
            auto tap = [&](bool ok, int x, int y, float w) {
                if (!ok) return;
                const float4 q = __ldg(reinterpret_cast<const float4*>(mu + ((size_t)x * n + y) * nz + k));
                m.x = fmaf(w, q.x, m.x);
                m.y = fmaf(w, q.y, m.y);
                m.z = fmaf(w, q.z, m.z);
                m.w = fmaf(w, q.w, m.w);
            };
            tap(vx0 && vy0, x0, y0, (1.f - ax) * (1.f - by));
            tap(vx1 && vy0, x0 + 1, y0, ax * (1.f - by));
            tap(vx0 && vy1, x0, y0 + 1, (1.f - ax) * by);
            tap(vx1 && vy1, x0 + 1, y0 + 1, ax * by);
            const float tau[4] = {voxel_cm * m.x, voxel_cm * m.y, voxel_cm * m.z, voxel_cm * m.w};
            float a[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = expf(-(r[q].prefix() + 0.5f * tau[q]));
                r[q].add(tau[q]);
            }
            out[(size_t)i * plane4] = make_float4(a[0], a[1], a[2], a[3]);
        }
        if (f64) {
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q].fold();
        }
    }
}

cudaError_t launch_attenuation(const float* mu, const float4* cs, int n, int nz, int n_angles, float voxel_cm, int f64,
                               float* atten, cudaStream_t st)
{
    const int threads = 256;
    dim3 grid((n * (nz / 4) + threads - 1) / threads, n_angles);
    attenuation_kernel<<<grid, threads, 0, st>>>(mu, cs, n, nz, voxel_cm, f64, atten);
    return cudaGetLastError();
}

// Sum the per-(angle, tile) FP64 partials of one subiteration in a fixed order.
__global__ void diag_finalize_kernel(const double* __restrict__ part, int n_part, double* __restrict__ out3)
{
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int p = 0; p < n_part; ++p) s += part[3 * p + threadIdx.x];
        out3[threadIdx.x] = s;
    }
}

cudaError_t launch_diag_finalize(const double* part, int n_part, double* out3, cudaStream_t st)
{
    diag_finalize_kernel<<<1, 32, 0, st>>>(part, n_part, out3);
    return cudaGetLastError();
}

// Sum of the depth-chunk partial projections (chunk order, deterministic),
// times the T_fov weights of the angle when the plan has them, and, with y,
// the OSEM ratio r = y / (p + s) (0 where p + s == 0) and the
// FP64 count sums of (p + s), y and y * p / (p + s) per block.
// The FP64 count sums run only when requested (kDiag): FP64 throughput on
// GB300 is a small fraction of FP32.
template <bool kDiag>
__global__ void __launch_bounds__(256) forward_reduce_kernel(ReduceArgs a)
{
    __shared__ double red[32];
    const int plane4 = a.plane >> 2;
    const size_t total4 = (size_t)a.items * plane4;
    const float s = a.s_ptr ? __ldg(a.s_ptr) : a.s;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total4; e += (size_t)gridDim.x * blockDim.x) {
        const int item = (int)(e / plane4);
        const int off4 = (int)(e - (size_t)item * plane4);
        const float4* src = reinterpret_cast<const float4*>(a.partials) + (size_t)item * a.chunks * plane4 + off4;
        // the partials summed in chunk order, up to 12 of their loads in
        // flight together (the order of the sums, and so the result, is that
        // of a plain loop)
        float4 p = __ldcg(src);
        int c = 1;
        for (; c < a.chunks; c += 12) {
            float4 v[12];
#pragma unroll
            for (int u = 0; u < 12; ++u)
                if (c + u < a.chunks) v[u] = __ldcg(src + (size_t)(c + u) * plane4);
#pragma unroll
            for (int u = 0; u < 12; ++u) {
                if (c + u < a.chunks) {
                    p.x += v[u].x;
                    p.y += v[u].y;
                    p.z += v[u].z;
                    p.w += v[u].w;
                }
            }
        }
        if (a.fov) {  // T_fov of the item's angle
            const float4 m = __ldg(reinterpret_cast<const float4*>(a.fov) +
                                   (size_t)a.sel[item % a.n_sel] * plane4 + off4);
            p = make_float4(p.x * m.x, p.y * m.y, p.z * m.z, p.w * m.w);
        }
        float4 o = p;
        if (a.y) {
            const int angle = a.sel[item % a.n_sel];
            const float4 yv = __ldg(reinterpret_cast<const float4*>(a.y) + (size_t)angle * plane4 + off4);
            const float pv[4] = {p.x, p.y, p.z, p.w};
            const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
            float rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float den = a.scale * pv[q] + s;
                rv[q] = den > 0.f ? a.scale * yy[q] / den : 0.f;
                if (kDiag) {
                    d0 += (double)den;
                    d1 += (double)yy[q];
                    d2 += (double)(rv[q] * pv[q]);
                }
            }
            o = make_float4(rv[0], rv[1], rv[2], rv[3]);
        }
        reinterpret_cast<float4*>(a.out)[e] = o;
    }
    if (kDiag) {
        const double s0 = block_sum_f64(d0, red);
        const double s1 = block_sum_f64(d1, red);
        const double s2 = block_sum_f64(d2, red);
        if (threadIdx.x == 0) {
            a.diag_blocks[3 * blockIdx.x + 0] = s0;
            a.diag_blocks[3 * blockIdx.x + 1] = s1;
            a.diag_blocks[3 * blockIdx.x + 2] = s2;
        }
    }
}

cudaError_t launch_forward_reduce(const ReduceArgs& a, int blocks, cudaStream_t st)
{
    if (a.diag_blocks)
        forward_reduce_kernel<true><<<blocks, 256, 0, st>>>(a);
    else
        forward_reduce_kernel<false><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Poisson log-likelihood (Table 1): sum_b y_b log(p_b + s) - (p_b + s), in
// FP64 per block, plus the gradient with respect to p, y/(p+s) - 1.
__global__ void poisson_ll_kernel(const float* __restrict__ y, const float* __restrict__ p, float s, size_t count,
                                  double* __restrict__ block_part, float* __restrict__ grad)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x; b < count; b += (size_t)gridDim.x * blockDim.x) {
        const float yv = __ldg(y + b);
        const float lam = __ldg(p + b) + s;
        double term = -(double)lam;
        if (yv != 0.f) term += (double)yv * (double)logf(lam);
        acc += term;
        if (grad) grad[b] = (lam > 0.f ? yv / lam : 0.f) - 1.f;
    }
    const double tot = block_sum_f64(acc, red);
    if (threadIdx.x == 0) block_part[blockIdx.x] = tot;
}

__global__ void sum_blocks_kernel(const double* __restrict__ part, int n, double* __restrict__ out)
{
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < n; ++b) s += part[b];
        out[0] = s;
    }
}

cudaError_t launch_poisson_ll(const float* y, const float* p, float s, size_t count, double* block_part, int n_blocks,
                              double* ll, float* grad, cudaStream_t st)
{
    poisson_ll_kernel<<<n_blocks, 256, 0, st>>>(y, p, s, count, block_part, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_blocks_kernel<<<1, 32, 0, st>>>(block_part, n_blocks, ll);
    return cudaGetLastError();
}

__global__ void fill_kernel(float* __restrict__ dst, size_t count, float value)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = value;
}

// Self-test of the bounded-wait path that every mbarrier wait of the
// projector kernels takes: thread 0 waits on a barrier that nothing arrives
// on, gives up after `limit` cycles, and the CTA reports SPECT_ETIMEDOUT
// through the status word with the same helper as those kernels.  No copy
// is in flight, so the CTA leaves at once.
__global__ void wait_selftest_kernel(long long limit, int* err)
{
    __shared__ __align__(8) unsigned long long bar_word;
    const uint32_t bar = smem_u32(&bar_word);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = threadIdx.x == 0 ? mbar_wait_for(bar, 0, limit) : true;
    sync_ok(ok, err);
}

cudaError_t launch_wait_selftest(long long limit, int* err, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 64, 0, st>>>(limit, err);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* dst, size_t count, float value, cudaStream_t st)
{
    size_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) return cudaSuccess;
    fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(dst, count, value);
    return cudaGetLastError();
}

}  // namespace spect

namespace spect {

// The subiteration's image update (update.cuh) where the back projection
// was gathered into a separate buffer.
__global__ void update_kernel(float* __restrict__ x, const float* __restrict__ bp, UpdateSpec u, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float gv = u.grad ? u.grad[i] : 0.f;
        const float sa = u.sens_all ? u.sens_all[i] : 0.f;
        const float b = u.bp_add ? bp[i] + u.bp_add[i] : bp[i];
        x[i] = update1(u, x[i], b, u.sens[i], gv, sa);
    }
}

cudaError_t launch_update(float* x, const float* bp, const UpdateSpec& u, size_t count, cudaStream_t st)
{
    size_t blocks = (count + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks == 0) return cudaSuccess;
    update_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, bp, u, count);
    return cudaGetLastError();
}

// out = sum_t w[t] in[t] (the weighted subset sensitivity of several photopeaks).
struct WsumArgs {
    const float* in[kMaxPeaks];
    float w[kMaxPeaks];
};

__global__ void wsum_kernel(float* __restrict__ out, WsumArgs a, int terms, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        float v = a.w[0] * a.in[0][i];
        for (int t = 1; t < terms; ++t) v = fmaf(a.w[t], a.in[t][i], v);
        out[i] = v;
    }
}

cudaError_t launch_wsum(float* out, const float* const* in, const float* w, int terms, size_t count, cudaStream_t st)
{
    if (terms < 1 || terms > kMaxPeaks) return cudaErrorInvalidValue;
    WsumArgs a{};
    for (int t = 0; t < terms; ++t) {
        a.in[t] = in[t];
        a.w[t] = w[t];
    }
    size_t blocks = (count + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks == 0) return cudaSuccess;
    wsum_kernel<<<(unsigned)blocks, 256, 0, st>>>(out, a, terms, count);
    return cudaGetLastError();
}

// Gradient of a nearest-neighbour prior (Sec. 2.1.3, Table 1):
//   V(x) = sum_r sum_s w_rs phi(x_r, x_s),  s over the 26 neighbours of r
//   inside the volume, w_rs = 1 / |r - s|;
//   dV/dx_r = 2 sum_s w_rs dphi(x_r, x_s)/dx_r  (phi symmetric), with
//   quadratic  phi = ((a - b)/delta)^2 / 4:  dphi/da = (a - b) / (2 delta^2);
//   RDP  phi = (a - b)^2 / (a + b + gamma|a - b|):
//        dphi/da = (a - b)(a + 3b + gamma|a - b|) / (a + b + gamma|a - b|)^2,
//   a pair whose RDP denominator is 0 contributing 0.  One thread per voxel,
//   z fastest, neighbours through L1.
__global__ void __launch_bounds__(256) prior_grad_kernel(const float* __restrict__ x, float* __restrict__ grad, int n,
                                                         int nz, int prior, float delta, float gamma)
{
    const size_t vol = (size_t)n * n * nz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= vol) return;
    const int k = (int)(idx % nz);
    const int j = (int)((idx / nz) % n);
    const int i = (int)(idx / ((size_t)nz * n));
    const float a = x[idx];
    const float inv2d2 = 1.f / (2.f * delta * delta);
    const float wt[4] = {0.f, 1.f, 1.f / sqrtf(2.f), 1.f / sqrtf(3.f)};
    float g = 0.f;
#pragma unroll
    for (int di = -1; di <= 1; ++di)
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int dk = -1; dk <= 1; ++dk) {
                if (!di && !dj && !dk) continue;
                const int i2 = i + di, j2 = j + dj, k2 = k + dk;
                if (i2 < 0 || i2 >= n || j2 < 0 || j2 >= n || k2 < 0 || k2 >= nz) continue;
                const float b = __ldg(x + ((size_t)i2 * n + j2) * nz + k2);
                const float w = wt[di * di + dj * dj + dk * dk];
                const float d = a - b;
                float t;
                if (prior == SPECT_PRIOR_QUADRATIC) {
                    t = d * inv2d2;
                } else {
                    const float ad = fabsf(d);
                    const float S = a + b + gamma * ad;
                    t = S != 0.f ? d * (a + 3.f * b + gamma * ad) / (S * S) : 0.f;
                }
                g = fmaf(2.f * w, t, g);
            }
    grad[idx] = g;
}

cudaError_t launch_prior_grad(const float* x, float* grad, int n, int nz, int prior, float delta, float gamma,
                              cudaStream_t st)
{
    const size_t vol = (size_t)n * n * nz;
    if (vol == 0) return cudaSuccess;
    prior_grad_kernel<<<(unsigned)((vol + 255) / 256), 256, 0, st>>>(x, grad, n, nz, prior, delta, gamma);
    return cudaGetLastError();
}

}  // namespace spect
