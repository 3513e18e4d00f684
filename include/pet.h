/*
 * Listmode PET system matrix and listmode OSEM on one GB300 (sm_103a).
 *
 * PyTomography (arXiv 2309.01977), Sec. 2.1.1, Eq. (2) (PET_SM):
 *   H = T_eta T_omega P_Sigma T_rr,
 * T_rr an object-space Gaussian resolution model, P_Sigma the line integral
 * of the image along each line of response (Joseph's method, listmode, no
 * time of flight), T_omega the attenuation factor exp(-P_Sigma mu) of the
 * line and T_eta its detector-pair normalisation.  OSEM follows Table 1
 * (OSEM row) with the listmode Poisson likelihood.
 *
 * Conventions (readings where the paper is silent):
 *   - image [nx][ny][nz] FP32, z fastest; voxel sizes (vx, vy, vz) in mm;
 *     voxel (i, j, k) is centred at ((i - (nx-1)/2) vx, (j - (ny-1)/2) vy,
 *     (k - (nz-1)/2) vz) mm (the image is centred on the scanner axis).
 *   - a line of response (LOR) is 6 floats (x1, y1, z1, x2, y2, z2) in mm,
 *     the segment between two detector positions.
 *   - Joseph's method: principal axis a = argmax_c |x2_c - x1_c| / v_c (ties
 *     to the lower axis), taken in single precision; the line is sampled on
 *     every voxel plane q of axis a whose index lies between the endpoints'
 *     index coordinates (inclusive, single precision: s = (x_a - o_a) / v_a
 *     with o_a = -((n_a - 1) / 2 * v_a), planes ceil(min s) .. floor(max s)
 *     clipped to the image); at each plane the image is interpolated
 *     bilinearly in the other two axes with zero outside the image; each
 *     sample is weighted by v_a |x2 - x1| / |x2_a - x1_a| (mm).
 *   - T_rr: separable Gaussian of standard deviation rr_sigma_mm, i.e.
 *     rr_sigma_mm / v_c voxels on axis c, sampled taps exp(-t^2 / 2 s^2) for
 *     |t| <= ceil(rr_nsigma s), normalised to sum 1, zero padding; off when
 *     rr_sigma_mm <= 0.
 *   - mu in 1/mm; mult_e = eta_e exp(-(P_Sigma mu)_e) (no T_rr on mu).
 *   - listmode OSEM: subsets {e : e mod n_subsets == m}, visited m = 0..M-1;
 *     p_e = mult_e (P_Sigma T_rr f)_e,
 *       f <- f * T_rr P_Sigma^T(mult / (p + s))|_{S_m} / (sens / M),
 *     sens = T_rr P_Sigma^T mult over every LOR of the scanner (the caller
 *     computes it with pet_back); voxels with sens == 0 are unchanged,
 *     events with p + s == 0 contribute nothing.
 *
 * Memory: every pointer argument is a device pointer (the caller owns it) to
 * contiguous FP32 data, LOR arrays 8-byte aligned, images 16-byte aligned;
 * diag_out is a host pointer.  The plan owns its taps, a copy of mu and its
 * scratch images.  Calls are asynchronous on `stream` (a cudaStream_t, NULL
 * for the legacy stream) and a plan serves one stream at a time.
 * Errors: SPECT_OK (0) or a negative status of spect.h; the message is in
 * spect_last_error().  Floating-point sums that scatter (P_Sigma^T) use
 * atomic adds, so their rounding order varies from run to run.
 */
#ifndef PET_H
#define PET_H

#include <stdint.h>

#include "spect.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pet_geom {
    int nx, ny, nz;       /* image size, z fastest */
    float vx, vy, vz;     /* voxel size, mm */
    float rr_sigma_mm;    /* T_rr standard deviation, mm (<= 0: off) */
    float rr_nsigma;      /* T_rr truncation in standard deviations (3) */
    int n_subsets;        /* listmode subsets {e mod n_subsets} (>= 1) */
} pet_geom;

typedef struct pet_plan pet_plan;

/* Plan: geometry, T_rr taps, a copy of mu (NULL: no attenuation) and the
 * scratch images (4 images of nx*ny*nz floats). */
int pet_plan_create(const pet_geom* geom, const float* mu_dev, void* stream, pet_plan** out);
int pet_plan_destroy(pet_plan* plan);

/* mult_out[e] = eta[e] * exp(-(P_Sigma mu)_e) for n LORs (eta NULL: 1; a
 * plan without mu: omega = 1). */
int pet_mult(pet_plan* plan, const float* lors, const float* eta, int64_t n, float* mult_out, void* stream);

/* out[e] = mult[e] * (P_Sigma T_rr x)_e (mult NULL: 1). */
int pet_forward(pet_plan* plan, const float* x, const float* lors, const float* mult, int64_t n, float* out,
                void* stream);

/* x_out = T_rr P_Sigma^T (mult * q) over n LORs (overwrites x_out). */
int pet_back(pet_plan* plan, const float* q, const float* lors, const float* mult, int64_t n, float* x_out,
             void* stream);

/* Listmode OSEM subiterations first_subiter .. first_subiter + n_subiters - 1
 * (subset = subiteration mod n_subsets) on events lors[n] with factors
 * mult[n] and additive terms s[n] (NULL: 0); sens = T_rr P_Sigma^T mult over
 * all scanner LORs.  diag_out (host, NULL or 2 * n_subiters doubles): per
 * subiteration sum_e p_e / (p_e + s_e) over its events and the number of its
 * events with p_e + s_e > 0, in FP64; filling it synchronises the stream. */
int pet_lm_osem_run(pet_plan* plan, const float* lors, const float* mult, const float* s, int64_t n,
                    const float* sens, float* x_inout, int first_subiter, int n_subiters, double* diag_out,
                    void* stream);

/* Per-kernel CUDA-event timing on the launch stream (off by default). */
int pet_profile_enable(pet_plan* plan, int on);
/* Wait for the recorded events, add them up per kernel kind and copy at
 * most max_entries rows into out.  Returns the number of rows (>= 0) or a
 * status.  reset != 0 clears the totals afterwards. */
int pet_profile_read(pet_plan* plan, spect_kernel_time* out, int max_entries, int reset);

#ifdef __cplusplus
}
#endif

#endif
