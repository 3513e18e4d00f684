/*
 * FP64 CPU oracle for the listmode PET system matrix and listmode OSEM.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
 * CUDA library's PET path is checked against.  Only the test suite, the smoke
 * check and the CPU legs of the benchmark may load it; the library never calls
 * it and shares no code, header or table with it.
 *
 * Paper: PyTomography (arXiv 2309.01977), Sec. 2.1.1 "Projectors", Eq. (2)
 * (PET_SM): H = T_eta T_omega P_Sigma T_rr.  T_rr is object-space resolution
 * modelling with one Gaussian kernel, P_Sigma the line integral along each
 * line of response (Joseph's method, listmode, no time of flight), T_omega the
 * attenuation factor of the line and T_eta the detector-pair normalisation.
 * OSEM follows Table 1 (OSEM row) with the listmode Poisson likelihood.
 *
 * Conventions where the paper is silent (each one is a documented reading):
 *   - image f[i][j][k] over axes (x, y, z), k fastest; voxel sizes v[3] in mm;
 *     voxel centres at ((i - (nx-1)/2) vx, (j - (ny-1)/2) vy, (k - (nz-1)/2) vz)
 *     so the image is centred on the scanner axis.
 *   - a line of response (LOR) is the segment from p1 to p2 (mm).
 *   - Joseph's method: the principal axis a is the one with the largest
 *     |p2_a - p1_a| / v_a (ties to the lower axis).  The line is sampled on
 *     every voxel plane q of that axis whose index lies between the endpoints'
 *     index coordinates (inclusive); at each plane the image is bilinearly
 *     interpolated in the other two axes, taps outside the image read 0; every
 *     sample is weighted by the line's length between neighbouring planes,
 *     v_a |p2 - p1| / |p2_a - p1_a| (mm).  The principal axis and the plane
 *     range are integers that floating point decides; the oracle takes them
 *     in double precision from the endpoints as given (a line whose
 *     single-precision decision differs is a rounding tie, which the tests
 *     identify and leave out of the comparison).
 *   - T_rr: separable Gaussian with standard deviation sigma (mm) per axis,
 *     sigma / v_c voxels on axis c, sampled taps exp(-t^2 / 2 s^2) for
 *     |t| <= ceil(nsigma s), normalised to sum 1, zero padding, same size.
 *     A non-positive sigma turns it off.
 *   - T_omega: omega = exp(-(P_Sigma mu)) with mu in 1/mm (no T_rr on mu);
 *     T_eta: one factor eta per LOR.  mult = eta * omega.
 *   - time of flight (or_pet_set_tof): n_b bins of width D (mm) centred at
 *     c_b = (b - (n_b - 1)/2) D on the line's signed arc length l from its
 *     midpoint (positive towards p2); a sample at l in bin b is weighted by
 *     Phi((l - c_b + D/2)/sigma) - Phi((l - c_b - D/2)/sigma) (the Gaussian
 *     timing kernel integrated over the bin).  Only samples of the window
 *     |l - c_b| <= nsigma sigma + D/2 count, tested sample by sample in
 *     double precision.  The attenuation factors never use time of flight.
 *   - listmode OSEM: subsets of events {e : e mod M == m}, visited
 *     m = 0..M-1; with p_e = mult_e (P_Sigma T_rr f)_e and the additive term
 *     s_e (randoms and scatter expected on that LOR),
 *       f <- f * T_rr P_Sigma^T(mult / (p + s))|_{S_m} / (sens / M),
 *     sens = T_rr P_Sigma^T mult over every LOR of the scanner (given by the
 *     caller).  Voxels with sens == 0 are unchanged; events with p + s == 0
 *     give ratio 0.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n[3];      /* nx, ny, nz */
    double v[3];   /* voxel size, mm */
} pet_img;

/* The integer decisions of Joseph's method for one LOR, in double precision:
 * principal axis *a (largest |p2_c - p1_c| / v_c, ties to the lower axis)
 * and the planes [*q_lo, *q_hi] of that axis whose index lies between the
 * endpoints' index coordinates, inside the image (empty when q_lo > q_hi). */
static void lor_planes(const pet_img* g, const double* lor, int* a, int* q_lo, int* q_hi)
{
    double sc[3];
    for (int c = 0; c < 3; ++c) sc[c] = fabs(lor[3 + c] - lor[c]) / g->v[c];
    int ax = 0;
    if (sc[1] > sc[ax]) ax = 1;
    if (sc[2] > sc[ax]) ax = 2;
    *a = ax;
    *q_lo = 1;
    *q_hi = 0;
    if (!(sc[ax] > 0.0)) return;
    const double org = -0.5 * (double)(g->n[ax] - 1) * g->v[ax];
    const double s1 = (lor[ax] - org) / g->v[ax];
    const double s2 = (lor[3 + ax] - org) / g->v[ax];
    double lo = ceil(s1 < s2 ? s1 : s2), hi = floor(s1 < s2 ? s2 : s1);
    if (lo < 0.0) lo = 0.0;
    if (hi > (double)(g->n[ax] - 1)) hi = (double)(g->n[ax] - 1);
    if (lo > hi) return;
    *q_lo = (int)lo;
    *q_hi = (int)hi;
}

static size_t vox(const pet_img* g, int i, int j, int k)
{
    return ((size_t)i * g->n[1] + j) * g->n[2] + k;
}

/* Time-of-flight model (module state, set by or_pet_set_tof; bins == NULL
 * means no time of flight). */
typedef struct {
    int nb;
    double bin_mm, sigma_mm, nsigma;
    const int* bins;  /* per LOR index */
} pet_tof;

static pet_tof g_tof = {0, 0.0, 0.0, 0.0, NULL};

void or_pet_set_tof(int n_bins, double bin_mm, double sigma_mm, double nsigma, const int* bins)
{
    g_tof.nb = n_bins;
    g_tof.bin_mm = bin_mm;
    g_tof.sigma_mm = sigma_mm;
    g_tof.nsigma = nsigma;
    g_tof.bins = n_bins > 0 ? bins : NULL;
}

static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Visit the samples of one LOR: for every plane q of the principal axis, the
 * four bilinear taps (voxel index, weight including the step length and, with
 * time of flight, the bin's timing weight).  Taps outside the image are
 * skipped (they read 0 / receive nothing). */
typedef void (*tap_fn)(size_t idx, double w, void* ctx);

static void lor_walk(const pet_img* g, const double* lor, const pet_tof* tf, int bin, tap_fn fn, void* ctx)
{
    int a, q_lo, q_hi;
    lor_planes(g, lor, &a, &q_lo, &q_hi);
    if (q_lo > q_hi) return;
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    double e1[3], e2[3], d[3], len2 = 0.0;
    for (int t = 0; t < 3; ++t) {
        const double org = -0.5 * (g->n[t] - 1) * g->v[t];
        e1[t] = (lor[t] - org) / g->v[t];
        e2[t] = (lor[3 + t] - org) / g->v[t];
        d[t] = lor[3 + t] - lor[t];
        len2 += d[t] * d[t];
    }
    const double len = sqrt(len2);
    const double step = g->v[a] * len / fabs(d[a]);
    const double cb = tf ? ((double)bin - 0.5 * (double)(tf->nb - 1)) * tf->bin_mm : 0.0;
    for (int q = q_lo; q <= q_hi; ++q) {
        double wt_tof = 1.0;
        if (tf) {
            /* signed arc length of the sample from the line's midpoint */
            const double l = ((q - e1[a]) / (e2[a] - e1[a]) - 0.5) * len;
            if (!(fabs(l - cb) <= tf->nsigma * tf->sigma_mm + 0.5 * tf->bin_mm)) continue;
            wt_tof = std_normal_cdf((l - cb + 0.5 * tf->bin_mm) / tf->sigma_mm) -
                     std_normal_cdf((l - cb - 0.5 * tf->bin_mm) / tf->sigma_mm);
        }
        const double t = (q - e1[a]) / (e2[a] - e1[a]);
        const double u = e1[b] + t * (e2[b] - e1[b]);
        const double w = e1[c] + t * (e2[c] - e1[c]);
        const double u0 = floor(u), w0 = floor(w);
        const double fu = u - u0, fw = w - w0;
        for (int du = 0; du < 2; ++du)
            for (int dw = 0; dw < 2; ++dw) {
                const long iu = (long)u0 + du, iw = (long)w0 + dw;
                if (iu < 0 || iu >= g->n[b] || iw < 0 || iw >= g->n[c]) continue;
                const double wt = (du ? fu : 1.0 - fu) * (dw ? fw : 1.0 - fw);
                int idx[3];
                idx[a] = q;
                idx[b] = (int)iu;
                idx[c] = (int)iw;
                fn(vox(g, idx[0], idx[1], idx[2]), step * wt * wt_tof, ctx);
            }
    }
}

typedef struct {
    const double* f;
    double acc;
} fwd_ctx;

static void fwd_tap(size_t idx, double w, void* ctx)
{
    fwd_ctx* k = (fwd_ctx*)ctx;
    k->acc += w * k->f[idx];
}

typedef struct {
    double* out;
    double val;
} back_ctx;

static void back_tap(size_t idx, double w, void* ctx)
{
    back_ctx* k = (back_ctx*)ctx;
    k->out[idx] += w * k->val;
}

static pet_img make_img(int nx, int ny, int nz, const double* v)
{
    pet_img g;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    for (int c = 0; c < 3; ++c) g.v[c] = v[c];
    return g;
}

/* Principal axis and plane range of each LOR (the double-precision decisions). */
void or_pet_planes(const double* lors, long n_lors, int nx, int ny, int nz, const double* v, int* out3)
{
    const pet_img g = make_img(nx, ny, nz, v);
    for (long e = 0; e < n_lors; ++e) lor_planes(&g, lors + 6 * e, out3 + 3 * e, out3 + 3 * e + 1, out3 + 3 * e + 2);
}

static const pet_tof* tof_on(void) { return g_tof.bins ? &g_tof : NULL; }

static int tof_bin(const pet_tof* tf, long e) { return tf ? tf->bins[e] : 0; }

static void joseph_fwd(const double* f, const pet_img* g, const double* lors, long n_lors, const pet_tof* tf,
                       double* out)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (long e = 0; e < n_lors; ++e) {
        fwd_ctx k = {f, 0.0};
        lor_walk(g, lors + 6 * e, tf, tof_bin(tf, e), fwd_tap, &k);
        out[e] = k.acc;
    }
}

/* P_Sigma: line integral of f along each LOR (Joseph; with time of flight
 * when or_pet_set_tof gave bins). */
void or_joseph_fwd(const double* f, int nx, int ny, int nz, const double* v, const double* lors, long n_lors,
                   double* out)
{
    const pet_img g = make_img(nx, ny, nz, v);
    joseph_fwd(f, &g, lors, n_lors, tof_on(), out);
}

/* P_Sigma^T: each LOR's value spread back along its samples (serial, so the
 * sums are in event order). */
void or_joseph_back(const double* vals, const double* lors, long n_lors, int nx, int ny, int nz, const double* v,
                    double* out)
{
    const pet_img g = make_img(nx, ny, nz, v);
    memset(out, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (long e = 0; e < n_lors; ++e) {
        back_ctx k = {out, vals[e]};
        if (vals[e] != 0.0) lor_walk(&g, lors + 6 * e, tof_on(), tof_bin(tof_on(), e), back_tap, &k);
    }
}

/* Taps of T_rr on one axis: sigma in voxels; returns the radius R and fills
 * w[0..2R] (w must hold 2R+1).  R = 0 and w[0] = 1 when sigma <= 0. */
int or_pet_rr_radius(double sigma_vox, double nsigma)
{
    if (!(sigma_vox > 0.0)) return 0;
    return (int)ceil(nsigma * sigma_vox);
}

void or_pet_rr_taps(double sigma_vox, double nsigma, double* w)
{
    const int r = or_pet_rr_radius(sigma_vox, nsigma);
    if (r == 0) {
        w[0] = 1.0;
        return;
    }
    double sum = 0.0;
    for (int t = -r; t <= r; ++t) {
        w[t + r] = exp(-(double)t * t / (2.0 * sigma_vox * sigma_vox));
        sum += w[t + r];
    }
    for (int t = 0; t <= 2 * r; ++t) w[t] /= sum;
}

/* T_rr: separable Gaussian, x then y then z, zero padding. */
void or_pet_blur(const double* f, int nx, int ny, int nz, const double* v, double sigma_mm, double nsigma,
                 double* out)
{
    const int n[3] = {nx, ny, nz};
    const size_t total = (size_t)nx * ny * nz;
    const size_t stride[3] = {(size_t)ny * nz, (size_t)nz, 1};
    double* cur = (double*)malloc(sizeof(double) * total);
    double* nxt = (double*)malloc(sizeof(double) * total);
    memcpy(cur, f, sizeof(double) * total);
    for (int ax = 0; ax < 3; ++ax) {
        const double s = sigma_mm > 0.0 ? sigma_mm / v[ax] : 0.0;
        const int r = or_pet_rr_radius(s, nsigma);
        double* w = (double*)malloc(sizeof(double) * (2 * r + 1));
        or_pet_rr_taps(s, nsigma, w);
#pragma omp parallel for
        for (long i = 0; i < (long)nx; ++i)
            for (int j = 0; j < ny; ++j)
                for (int k = 0; k < nz; ++k) {
                    const int pos[3] = {(int)i, j, k};
                    const size_t o = ((size_t)i * ny + j) * nz + k;
                    double acc = 0.0;
                    for (int t = -r; t <= r; ++t) {
                        const int p = pos[ax] - t;
                        if (p < 0 || p >= n[ax]) continue;
                        acc += w[t + r] * cur[o - (long)t * (long)stride[ax]];
                    }
                    nxt[o] = acc;
                }
        free(w);
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    memcpy(out, cur, sizeof(double) * total);
    free(cur);
    free(nxt);
}

/* mult_e = eta_e * exp(-(P_Sigma mu)_e); eta NULL means 1, mu NULL means no
 * attenuation. */
void or_pet_mult(const double* mu, int nx, int ny, int nz, const double* v, const double* lors, long n_lors,
                 const double* eta, double* out)
{
    const pet_img g = make_img(nx, ny, nz, v);
    if (mu) joseph_fwd(mu, &g, lors, n_lors, NULL, out);
    for (long e = 0; e < n_lors; ++e) {
        const double om = mu ? exp(-out[e]) : 1.0;
        out[e] = (eta ? eta[e] : 1.0) * om;
    }
}

/* H f on a list of LORs: mult (P_Sigma T_rr f); mult NULL means 1. */
void or_pet_forward(const double* f, int nx, int ny, int nz, const double* v, double sigma_mm, double nsigma,
                    const double* lors, const double* mult, long n_lors, double* out)
{
    const size_t total = (size_t)nx * ny * nz;
    double* fb = (double*)malloc(sizeof(double) * total);
    or_pet_blur(f, nx, ny, nz, v, sigma_mm, nsigma, fb);
    or_joseph_fwd(fb, nx, ny, nz, v, lors, n_lors, out);
    if (mult)
        for (long e = 0; e < n_lors; ++e) out[e] *= mult[e];
    free(fb);
}

/* H^T q: T_rr P_Sigma^T (mult q). */
void or_pet_back(const double* q, int nx, int ny, int nz, const double* v, double sigma_mm, double nsigma,
                 const double* lors, const double* mult, long n_lors, double* out)
{
    const size_t total = (size_t)nx * ny * nz;
    double* val = (double*)malloc(sizeof(double) * (size_t)(n_lors > 0 ? n_lors : 1));
    double* bp = (double*)malloc(sizeof(double) * total);
    for (long e = 0; e < n_lors; ++e) val[e] = mult ? mult[e] * q[e] : q[e];
    or_joseph_back(val, lors, n_lors, nx, ny, nz, v, bp);
    or_pet_blur(bp, nx, ny, nz, v, sigma_mm, nsigma, out);
    free(val);
    free(bp);
}

/* Listmode OSEM, subiterations first .. first + count - 1 (subset it mod M).
 * s NULL means s = 0.  diag (NULL or 2*count doubles): per subiteration
 * sum_e p_e / (p_e + s_e) over its events and the number of its events with
 * p_e + s_e > 0. */
void or_pet_lm_osem(const double* lors, const double* mult, const double* s, long n_ev, const double* sens,
                    int nx, int ny, int nz, const double* v, double sigma_mm, double nsigma, int n_subsets,
                    double* x, int first, int count, double* diag)
{
    const size_t total = (size_t)nx * ny * nz;
    double* fb = (double*)malloc(sizeof(double) * total);
    double* bp = (double*)malloc(sizeof(double) * total);
    double* bpb = (double*)malloc(sizeof(double) * total);
    const pet_img g = make_img(nx, ny, nz, v);
    for (int it = first; it < first + count; ++it) {
        const int m = it % n_subsets;
        or_pet_blur(x, nx, ny, nz, v, sigma_mm, nsigma, fb);
        memset(bp, 0, sizeof(double) * total);
        double cons = 0.0, used = 0.0;
        for (long e = m; e < n_ev; e += n_subsets) {
            fwd_ctx k = {fb, 0.0};
            lor_walk(&g, lors + 6 * e, tof_on(), tof_bin(tof_on(), e), fwd_tap, &k);
            const double p = mult[e] * k.acc;
            const double den = p + (s ? s[e] : 0.0);
            if (!(den > 0.0)) continue;
            cons += p / den;
            used += 1.0;
            back_ctx b = {bp, mult[e] / den};
            lor_walk(&g, lors + 6 * e, tof_on(), tof_bin(tof_on(), e), back_tap, &b);
        }
        or_pet_blur(bp, nx, ny, nz, v, sigma_mm, nsigma, bpb);
        for (size_t i = 0; i < total; ++i) {
            const double sm = sens[i] / n_subsets;
            if (sm > 0.0) x[i] = x[i] * bpb[i] / sm;
        }
        if (diag) {
            diag[2 * (it - first)] = cons;
            diag[2 * (it - first) + 1] = used;
        }
    }
    free(fb);
    free(bp);
    free(bpb);
}
