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
 *   - time of flight (n_tof_bins > 0 and a tof_bin array): bin b is centred
 *     at c_b = (b - (n_tof_bins - 1)/2) tof_bin_mm on the arc length l from
 *     the line's midpoint (positive towards the second end); each sample is
 *     weighted by Phi((l - c_b + w/2)/sigma) - Phi((l - c_b - w/2)/sigma),
 *     w the bin width, over the window |l - c_b| <= nsigma sigma + w/2 taken
 *     as a range of sample indices in double precision.  Attenuation factors
 *     and the sensitivity image are computed without time of flight.
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
    int n_tof_bins;       /* time-of-flight bins (0: no time of flight) */
    float tof_bin_mm;     /* bin width along the line, mm */
    float tof_sigma_mm;   /* standard deviation of the Gaussian timing kernel, mm */
    float tof_nsigma;     /* kernel truncation: |l - c_b| <= tof_nsigma sigma + width / 2 (3) */
} pet_geom;

typedef struct pet_plan pet_plan;

/* Plan: geometry, T_rr taps, a copy of mu (NULL: no attenuation) and the
 * scratch images (4 images of nx*ny*nz floats). */
int pet_plan_create(const pet_geom* geom, const float* mu_dev, void* stream, pet_plan** out);
int pet_plan_destroy(pet_plan* plan);

/* mult_out[e] = eta[e] * exp(-(P_Sigma mu)_e) for n LORs (eta NULL: 1; a
 * plan without mu: omega = 1). */
int pet_mult(pet_plan* plan, const float* lors, const float* eta, int64_t n, float* mult_out, void* stream);

/* out[e] = mult[e] * (P_Sigma T_rr x)_e (mult NULL: 1; tof_bin NULL: no
 * time of flight, else the bin of every LOR). */
int pet_forward(pet_plan* plan, const float* x, const float* lors, const float* mult, const int* tof_bin, int64_t n,
                float* out, void* stream);

/* x_out = T_rr P_Sigma^T (mult * q) over n LORs (overwrites x_out; tof_bin
 * as for pet_forward). */
int pet_back(pet_plan* plan, const float* q, const float* lors, const float* mult, const int* tof_bin, int64_t n,
             float* x_out, void* stream);

/* Listmode OSEM subiterations first_subiter .. first_subiter + n_subiters - 1
 * (subset = subiteration mod n_subsets) on events lors[n] with factors
 * mult[n], additive terms s[n] (NULL: 0) and time-of-flight bins tof_bin[n]
 * (NULL: no time of flight); sens = T_rr P_Sigma^T mult over all scanner
 * LORs (without time of flight).  diag_out (host, NULL or 2 * n_subiters doubles): per
 * subiteration sum_e p_e / (p_e + s_e) over its events and the number of its
 * events with p_e + s_e > 0, in FP64; filling it synchronises the stream. */
int pet_lm_osem_run(pet_plan* plan, const float* lors, const float* mult, const float* s, const int* tof_bin,
                    int64_t n, const float* sens, float* x_inout, int first_subiter, int n_subiters,
                    double* diag_out, void* stream);

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
