/*
 * spect.h -- C ABI of libspect, a GB300 (sm_103a) implementation of the
 * parallel-hole SPECT system matrix H, its exact transpose H^T and OSEM.
 *
 * Method: PyTomography (arXiv 2309.01977).
 *   - Sec. 2.1.1, Eq. (1): H = sum_n v_n (x) (T_fov P_x T_cdr T_att T_trans T_rot);
 *     per projection angle n the volume is rotated (bilinear) and optionally
 *     shifted along the detector axis (T_trans, non-central projections),
 *     weighted by attenuation, blurred plane by plane by a depth-dependent
 *     Gaussian, summed along the depth axis +x and optionally weighted by a
 *     field-of-view mask in projection space (T_fov).
 *   - Sec. 2.1.1: forward projection is H f, back projection is H^T g.
 *   - Table 1: Poisson gradient H^T(g/(Hf+s)) - H^T 1 and the OSEM
 *     preconditioner f / (H_m^T 1), which give the update
 *     f <- f * H_m^T(g/(H_m f + s)) / H_m^T 1 over subsets m.
 *   - Sec. 2.2 (Projectors): forward, backward, compute_normalization_factor,
 *     set_n_subsets, get_projection_subset map to spect_forward, spect_back,
 *     spect_sensitivity, spect_geom.n_subsets and the subset argument.
 *
 * Conventions (the paper leaves them open; the library fixes them):
 *   volume   f[x][y][z], z fastest, nx == ny == n, float32, contiguous;
 *   rotation about c = (n-1)/2; angle theta_a = 2*pi*a/n_angles unless given
 *            (its quarter turns with the exact cos, sin of 0 and +-1);
 *            rotated voxel (i, j) samples f at
 *              u = c + cos(t)(i-c) - sin(t)(j-c),  v = c + sin(t)(i-c) + cos(t)(j-c)
 *            bilinearly, zero outside the grid; i is depth, j the detector bin;
 *   attenuation  A[i] = exp(-(sum_{i'>i} tau[i'] + tau[i]/2)), tau = voxel_cm * (R mu),
 *            detector on the +x side;
 *   PSF      d_i = n - i - 0.5 + det_offset, sigma_i = psf_sigma0 + psf_slope * d_i
 *            (voxels), taps exp(-t^2/(2 sigma_i^2)) for |t| <= ceil(psf_nsigma*sigma_i),
 *            normalised to sum 1, applied along y and z with zero padding;
 *   projections p[a][y][z] (angle, detector bin along y, axial bin z);
 *   subsets  S_m = { a : a mod n_subsets == m }, angles in ascending order.
 *
 * Ownership: the caller owns every buffer it passes.  Device buffers are
 * float32, contiguous and 16-byte aligned, else SPECT_EINVAL.  A plan owns
 * its tables, attenuation cache, sensitivities and scratch.
 *
 * Concurrency: after creation a plan's tables, attenuation cache and
 * sensitivities are only read (spect_plan_set_mu is the exception: it
 * rewrites them, so no other call on the plan may run at the same time).
 * The plan keeps one set of scratch buffers per stream: the creation
 * stream's at creation, another stream's at the first call on it (or at
 * spect_plan_reserve_stream), so calls queued on different streams never
 * share scratch and may run concurrently on the device; calls on one
 * stream are ordered by the stream.  Calls from several host threads take
 * the plan's lock while they queue their work.  A stream under graph
 * capture cannot allocate: reserve its scratch before capturing (the
 * creation stream has it already); a captured graph uses the scratch of
 * the stream it was captured on, so replay it on that stream.  Calls on
 * different plans are independent.
 *
 * Errors: every call returns SPECT_OK (0) or a negative status; nothing
 * aborts or throws across the ABI.  spect_last_error() gives a thread-local
 * message for the last failure on the calling thread.
 *
 * Asynchrony: device work is queued on `stream` (a cudaStream_t; NULL is
 * the legacy default stream) and the call returns without waiting, except
 * where stated.
 */
#ifndef SPECT_H
#define SPECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define SPECT_OK 0
#define SPECT_EINVAL (-1)      /* bad argument, size, alignment or geometry */
#define SPECT_ENOMEM (-2)      /* device or host allocation failed */
#define SPECT_ECUDA (-3)       /* a CUDA runtime call failed */
#define SPECT_EBUDGET (-4)     /* request does not fit the memory budget */
#define SPECT_ETIMEDOUT (-5)   /* a bounded wait ran out */
#define SPECT_ECANCELLED (-6)  /* request was cancelled */
#define SPECT_ESTATE (-7)      /* call not valid in the object's state */
#define SPECT_ENOTFOUND (-8)   /* unknown request id */

/* ---------------------------------------------------------------- geometry */
#define SPECT_FLAG_ATTEN 1u      /* model attenuation (needs mu at plan creation) */
#define SPECT_FLAG_PSF 2u        /* model the depth-dependent collimator blur */
#define SPECT_FLAG_PSF_BF16 4u   /* PSF as banded-Toeplitz BF16 tensor-core GEMMs (FP32
                                    accumulate; taps and data split into BF16 hi + lo
                                    parts, three products per GEMM; image within 1e-3 of
                                    FP64; needs nx % 32 == 0, nx <= 128, nz % 8 == 0,
                                    nz <= 128) */
#define SPECT_FLAG_ATTEN_F64 8u  /* attenuation prefix sums in FP64 (else compensated FP32);
                                    the exponential is FP32 either way */

typedef struct spect_geom {
    int nx, ny, nz;           /* volume size; nx == ny required, nz % 4 == 0 */
    float voxel_cm;           /* voxel edge in cm (scales mu to optical depth) */
    int n_angles;             /* projections over 360 degrees */
    const double* angles_rad; /* host array [n_angles] or NULL for 2*pi*a/n_angles */
    float psf_sigma0;         /* sigma at the detector face, voxels */
    float psf_slope;          /* d sigma / d distance, voxels per voxel */
    float psf_nsigma;         /* truncation radius in sigmas (3 in the configs) */
    float det_offset;         /* extra detector distance, voxels */
    int n_subsets;            /* M >= 1 (ordered subsets) */
    unsigned flags;           /* SPECT_FLAG_* */
    const float* det_offsets; /* host array [n_angles] or NULL: a non-circular orbit, the
                                 detector offset of each angle in voxels (replaces
                                 det_offset; each angle gets its own PSF table, T_cdr of
                                 Eq. 1 with d_i = n - i - 0.5 + det_offsets[a]) */
    const float* det_shifts;  /* host array [n_angles] or NULL: T_trans of Eq. 1 (non-central
                                 projections), the shift s_a in voxels of angle a's rotated
                                 frame along the detector axis y (|s_a| <= 4 n): rotated
                                 voxel (i, j) samples where the central geometry puts
                                 (i, j - s_a), one bilinear interpolation (j - c becomes
                                 j - s_a - c below); the attenuation map is shifted alike */
    const float* fov_mask;    /* host array [n_angles][ny][nz] or NULL: T_fov of Eq. 1, a
                                 weight (finite, >= 0; 1 inside the field of view, 0
                                 outside) on every projection bin of every angle; the back
                                 projection applies it to its input.  Copied at plan
                                 creation. */
} spect_geom;

typedef struct spect_plan spect_plan;

/* Plan limits and figures the caller may want (spect_plan_query). */
typedef struct spect_plan_info {
    int n, nz, n_angles, n_subsets;
    int max_subset_size;      /* largest |S_m| */
    int psf_rmax;             /* largest PSF radius over depth planes */
    size_t device_bytes;      /* device memory owned by the plan */
    size_t atten_cache_bytes; /* part of it that is the per-angle A cache */
    int ztile;                /* axial columns per CTA of the plane kernels */
    int n_ztiles;             /* axial tiles per plane */
    int threads;              /* CTA size of the plane kernels */
    int smem_bytes;           /* their dynamic shared memory per CTA */
} spect_plan_info;

/* Create a plan: validates the geometry, builds the angle table, the
 * per-plane PSF taps (Eq. 1, T_cdr), the subset lists (Sec. 2.2) and, with
 * SPECT_FLAG_ATTEN, the per-angle attenuation cache A_a (T_att) from the
 * device mu map [nx][ny][nz] in 1/cm, and the per-subset sensitivities
 * H_m^T 1 (compute_normalization_factor).  Work is queued on `stream`;
 * the call synchronises that stream before it returns.  mu is only read
 * during the call.  *out is NULL on failure. */
int spect_plan_create(const spect_geom* geom, const float* mu_dev, void* stream, spect_plan** out);

/* Free the plan and its device memory (waits for its work to finish). */
int spect_plan_destroy(spect_plan* plan);

int spect_plan_query(const spect_plan* plan, spect_plan_info* info);

/* Wait for the device and report whether any kernel of this plan gave up a
 * bounded wait (SPECT_ETIMEDOUT; the flag is then cleared).  Synchronous. */
int spect_plan_check(spect_plan* plan);

/* Create this plan's scratch for `stream` now (a cudaMalloc; about one
 * volume per angle of the largest subset, at least 16 volumes, plus the
 * depth-chunk partials), so that later calls on the stream, including ones
 * inside a graph capture, allocate nothing.  No-op when it exists. */
int spect_plan_reserve_stream(spect_plan* plan, void* stream);

/* Wait for `stream`, then free this plan's scratch for it (a later call on
 * the stream creates it again).  No-op when the stream has none. */
int spect_plan_release_stream(spect_plan* plan, void* stream);

/* Self-test of failure detection.  Every wait of the projector kernels on
 * an asynchronous copy is bounded (about 4e9 SM cycles, ~2 s); when a wait
 * runs out the kernel records SPECT_ETIMEDOUT in the plan's status word,
 * leaves, and spect_plan_check reports it.  This call runs that path on
 * purpose: a one-CTA kernel waits on a barrier that nothing arrives on,
 * for limit_cycles SM cycles (1 .. 4e9), then records the timeout exactly
 * like the projector kernels.  The context stays usable.  Asynchronous on
 * `stream`.  (Not part of the paper's method.) */
int spect_plan_selftest_timeout(spect_plan* plan, long long limit_cycles, void* stream);

/* Number of angles of subset m (m == -1: all angles). */
int spect_subset_size(const spect_plan* plan, int subset);

/* Host copy of subset m's angle indices (ascending) into out[spect_subset_size]. */
int spect_subset_angles(const spect_plan* plan, int subset, int* out);

/* Forward projection (Eq. 1): proj = H_m x for each of `batch` volumes.
 * x: device [batch][nx][ny][nz]; proj: device [batch][|S_m|][ny][nz] with
 * the subset's angles in ascending order (subset == -1: all angles).
 * Deterministic: the same inputs give bitwise the same output. */
int spect_forward(spect_plan* plan, const float* x, float* proj, int subset, int batch, void* stream);

/* Back projection, the exact transpose of spect_forward:
 * x_out = H_m^T proj, overwriting x_out.  Layouts as in spect_forward. */
int spect_back(spect_plan* plan, const float* proj, float* x_out, int subset, int batch, void* stream);

/* Copy the plan's sensitivity H_m^T 1 of subset m (m == -1: all angles,
 * computed on the fly) into out [nx][ny][nz]. */
int spect_sensitivity(spect_plan* plan, int subset, float* out, void* stream);

/* OSEM (Table 1): run subiterations t = first_subiter .. first_subiter +
 * n_subiters - 1, subset m = t mod n_subsets, each doing
 *     p = H_m x;  r = y_m / (p + s)  (0 where p + s == 0);
 *     x <- x * H_m^T r / H_m^T 1    (x unchanged where H_m^T 1 == 0).
 * y: device [n_angles][ny][nz] measured counts (all angles);
 * s: constant additive scatter term; x_inout: device image, updated in place.
 * diag_dev: NULL or device double[3 * n_subiters] receiving, per subiteration
 * and before its update, the FP64 sums over the subset's bins of (p + s),
 * y and y * p / (p + s) (the last equals sum of H_m x_new: count conservation).
 * Resume by calling again with the next first_subiter. */
int spect_osem_run(spect_plan* plan, const float* y, float s, float* x_inout, int first_subiter,
                   int n_subiters, double* diag_dev, void* stream);

/* spect_osem_run with the scatter term read from device memory (*s_dev)
 * when the kernels run, so that a captured CUDA graph of the run can be
 * replayed for a new s. */
int spect_osem_run_dev(spect_plan* plan, const float* y, const float* s_dev, float* x_inout, int first_subiter,
                       int n_subiters, double* diag_dev, void* stream);

/* ---------------------------------------------------------------- MAP */

/* Nearest-neighbour priors (Sec. 2.1.3 and Table 1, prior classes):
 *   V(x) = sum_r sum_s w_rs phi(x_r, x_s), s over the 26 neighbours of voxel
 *   r inside the volume, w_rs = 1 / |r - s| (voxel units);
 *   SPECT_PRIOR_QUADRATIC  phi = ((a - b) / delta)^2 / 4
 *   SPECT_PRIOR_RDP        phi = (a - b)^2 / (a + b + gamma |a - b|)
 *                          (relative difference prior; a pair whose
 *                          denominator is 0 contributes 0). */
#define SPECT_PRIOR_NONE 0
#define SPECT_PRIOR_QUADRATIC 1
#define SPECT_PRIOR_RDP 2

/* Algorithms of Table 1 beyond OSEM, as preconditioned gradient ascent
 * (Eq. PGA) with beta_n = beta / M:
 *   SPECT_ALG_OSMAPOSL  x <- x H_m^T r / (H_m^T 1 + beta_n grad V(x)), r = y/(H_m x + s);
 *                       a voxel whose denominator is <= 0 is unchanged;
 *   SPECT_ALG_BSREM     x <- max(0, x + alpha_t M x / H^T 1 (H_m^T r - H_m^T 1 - beta_n grad V(x))),
 *                       H^T 1 over all angles, alpha_t = alpha0 / (1 + floor(t / M))
 *                       for subiteration t; a voxel with H^T 1 == 0 is unchanged. */
#define SPECT_ALG_OSMAPOSL 1
#define SPECT_ALG_BSREM 2

typedef struct spect_map_params {
    int algorithm;   /* SPECT_ALG_* */
    int prior;       /* SPECT_PRIOR_* */
    float beta;      /* prior weight (before the 1/M subset scaling) */
    float delta;     /* quadratic prior scale (> 0) */
    float gamma;     /* RDP edge-preservation parameter (>= 0) */
    float alpha0;    /* BSREM relaxation at the first iteration (> 0) */
} spect_map_params;

/* OSMAPOSL or BSREM subiterations first_subiter .. first_subiter+n_subiters-1
 * (subset m = t mod M) on x_inout (device float[nx][ny][nz], updated in
 * place), with the same y, s and plan as spect_osem_run.  The first call on
 * a plan allocates two volumes (the prior gradient and, for BSREM, H^T 1
 * over all angles, recomputed after spect_plan_set_mu).  Resume by calling
 * again with the next first_subiter.  Asynchronous on `stream`. */
int spect_map_run(spect_plan* plan, const float* y, float s, float* x_inout, int first_subiter, int n_subiters,
                  const spect_map_params* params, void* stream);

/* OSEM for several photopeaks (Sec. 2.1.1, Eq. extended_sm: H' = sum_n v_n (x)
 * a_n H_n, B_n = identity, A_n = the scalar a_n per peak): plans[n] is the
 * system matrix of peak n (its own attenuation map and PSF model; all peaks
 * share the volume, angles, subsets and device), scales[n] = a_n > 0 (detector
 * sensitivity times branching ratio), y[n] its projections (device,
 * [n_angles][ny][nz]) and s[n] >= 0 its additive term.  Subiteration t:
 *   x <- x (sum_n a_n H_n,m^T (y_n / (a_n H_n,m x + s_n))) / (sum_n a_n H_n,m^T 1)
 * (unchanged where the denominator is 0).  1 <= n_peaks <= 8; plans[0] may not
 * appear again in the list (its buffers hold partial sums); its first call
 * allocates one volume.  Asynchronous on `stream`. */
int spect_multi_osem_run(spect_plan* const* plans, const float* scales, int n_peaks, const float* const* y,
                         const float* s, float* x_inout, int first_subiter, int n_subiters, void* stream);

/* grad_out = dV/dx for prior `prior` (SPECT_PRIOR_QUADRATIC or _RDP) on a
 * device volume x[n][n][nz]; no plan, nothing allocated.  Asynchronous. */
int spect_prior_grad(const float* x, int n, int nz, int prior, float delta, float gamma, float* grad_out,
                     void* stream);

/* Reuse a plan for a new attenuation map: recompute the attenuation cache
 * and the subset sensitivities from mu_dev [nx][ny][nz] (1/cm), queued on
 * `stream` (no synchronisation).  The geometry tables are kept. */
int spect_plan_set_mu(spect_plan* plan, const float* mu_dev, void* stream);

/* Poisson log-likelihood (Table 1, PoissonLogLikelihood), FP64 sums:
 *   ll_dev[0] = sum_b y_b log(p_b + s) - (p_b + s)   (log y! dropped)
 * over `count` bins, and, if grad_proj is not NULL, its gradient with
 * respect to p: grad_proj[b] = y_b / (p_b + s) - 1 (0 - 1 where p_b + s == 0).
 * y, p, grad_proj: device float[count]; ll_dev: device double[1].
 * The plan (required) supplies the scratch for the block partial sums. */
int spect_poisson_ll(spect_plan* plan, const float* y, const float* p, float s, size_t count,
                     double* ll_dev, float* grad_proj, void* stream);

/* Poisson log-likelihood and its gradient, like spect_poisson_ll, for
 * callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment convenience.
 *
 * Who needs it: code that runs where cudaMalloc is unavailable or not
 * allowed -- a host framework that has reserved all device memory for its
 * own pool allocator, or a real-time loop that must not pay the latency of
 * an allocation or risk it failing.  spect_poisson_ll needs a plan, and a
 * plan allocates; this call needs none.
 *
 * Scratch: the per-block partial sums live in a fixed 128 KiB array built
 * into the library, so it covers at most 67,108,864 bins (count beyond that
 * returns SPECT_EINVAL and launches nothing).  Every GPU that loads the
 * library holds that array until the process exits.  The first call on a
 * device looks up the array's device address (with that device current);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: it does not survive cudaDeviceReset (or any
 * other teardown of the device's primary context), after which this call
 * must not be used.  The call itself makes no
 * allocation of any kind.  All calls on a device share the array: calls that
 * overlap on the GPU (different streams without ordering) race and give
 * wrong sums; calls ordered on one stream are safe.  Each call overwrites
 * every partial it reads, so nothing has to be cleared between calls.
 *
 * y, p, grad_proj: device float[count], 16-byte aligned (else
 * SPECT_EINVAL, as spect_poisson_ll); ll_dev: device double[1];
 * grad_proj may be NULL; count 0 gives ll = 0.  Asynchronous on `stream`. */
int spect_poisson_ll_noalloc(const float* y, const float* p, float s, size_t count, double* ll_dev,
                             float* grad_proj, void* stream);

/* ---------------------------------------------------------------- profiling */

/* Accumulated device time of one kernel kind launched through a plan. */
typedef struct spect_kernel_time {
    char name[32];            /* "forward", "blur_back", "gather", ... */
    unsigned long long launches;
    double total_ms;          /* sum of CUDA-event durations on the launch stream */
} spect_kernel_time;

/* Turn per-launch CUDA-event timing of this plan's kernels on (1) or off (0).
 * Events are recorded on the stream each kernel is launched on. */
int spect_profile_enable(spect_plan* plan, int on);

/* Wait for the recorded events, add them up per kernel kind and copy at
 * most max_entries rows into out.  Returns the number of rows (>= 0) or a
 * status.  reset != 0 clears the totals afterwards. */
int spect_profile_read(spect_plan* plan, spect_kernel_time* out, int max_entries, int reset);

/* Number of kernels libspect has launched in this process (all plans). */
unsigned long long spect_kernel_launches(void);

/* Human-readable name of a status code. */
const char* spect_status_str(int status);

/* Thread-local description of the last failure ("" if none). */
const char* spect_last_error(void);

/* Library version string. */
const char* spect_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPECT_H */
