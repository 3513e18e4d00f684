/*
 * FP64 CPU oracle for the parallel-hole SPECT system matrix and OSEM.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library itself never calls it and shares no code, header or table with it.
 *
 * Paper: PyTomography (arXiv 2309.01977), Sec. 2.1.1 "Projectors", Eq. (1)
 * (SPECT_SM): H = sum_n v_n (x) ( T_fov P_x T_cdr T_att T_trans T_rot ).
 * Per angle n the object is rotated (T_rot), weighted by attenuation (T_att),
 * blurred plane by plane with a depth-dependent collimator-detector response
 * (T_cdr) and summed along +x (P_x).  T_trans (non-central projections) is a
 * per-angle shift of the rotated frame along the detector's transaxial axis,
 * and T_fov a per-angle weight (mask) on the projection bins; both are
 * optional module state (or_set_trans, or_set_fov) and identities when unset
 * (the paper names them without giving their geometry).  The back projector is the literal
 * transpose of each step (the paper: back projection is H^T).  OSEM follows
 * Table 1 (OSEM row: preconditioner f / H_m^T 1, no prior) applied to the
 * Poisson gradient of Table 1 (H^T(g/(Hf+s)) - H^T 1), i.e. the classical
 * multiplicative update f <- f * H_m^T(g/(H_m f+s)) / H_m^T 1.
 *
 * Conventions where the paper is silent (each one is a documented reading):
 *   - volume f[i][j][k]: i = x (depth after rotation), j = y (detector bin),
 *     k = z (axial bin), k fastest.  Square transaxial grid nx == ny == n.
 *   - rotation centre c = (n-1)/2; rotated sample (i,j) reads f at
 *       u = c + cos(t)(i-c) - sin(t)(j-c),  v = c + sin(t)(i-c) + cos(t)(j-c)
 *     with bilinear weights and zero fill for taps outside the grid.
 *   - T_trans of angle n: the rotated frame shifted by s_n voxels along +j
 *     (the projection of the rotation axis lands s_n bins from the detector
 *     centre): sample (i,j) reads the rotated object at (i, j - s_n), i.e.
 *     j - c becomes j - s_n - c above, in one bilinear interpolation.  The
 *     attenuation map goes through the same T_trans T_rot.
 *   - T_fov of angle n: projection bin (j,k) multiplied by m_n[j][k] (1 in the
 *     field of view, 0 outside, or any weight); the back projector applies
 *     the same factor to its input (a diagonal operator is its own
 *     transpose).
 *   - default angles theta_n = 2*pi*n / n_angles, with the exact cos and sin
 *     (0, +-1) at quarter turns.
 *   - attenuation: detector on the +x side; with tau = voxel_cm * (R_n mu),
 *       A[i] = exp( -( sum_{i'>i} tau[i'] + tau[i]/2 ) )   (mid-voxel rule).
 *   - PSF: d_i = n - i - 0.5 + det_offset (voxels), or with a non-circular
 *     orbit (or_set_orbit) d_i(a) = n - i - 0.5 + det_offsets[a] for angle a
 *     (the detector's distance varies with the angle),
 *       sigma_i = sigma0 + slope * d_i,  R_i = ceil(nsigma * sigma_i),
 *       w_i(t) = exp(-t^2 / (2 sigma_i^2)) for |t| <= R_i, normalised to sum 1,
 *     2-D kernel w_i(t) w_i(u) over (j,k), zero padding at the edges.
 *   - subsets S_m = { n : n mod M == m }, visited m = 0..M-1.
 *   - OSEM: where H_m^T 1 == 0 the voxel is unchanged; where H_m f + s == 0
 *     the ratio is 0.  No epsilon anywhere.
 *   - priors (Sec. 2.1.3, Table 1, prior classes): V(f) = sum_r sum_s w_rs
 *     phi(f_r, f_s) over the 26 neighbours s of r inside the volume, with
 *     w_rs = 1 / |r - s| (inverse Euclidean distance in voxels); a term whose
 *     RDP denominator f_r + f_s + gamma |f_r - f_s| is 0 contributes 0.
 *   - MAP algorithms (Eq. PGA with the Table 1 preconditioners), beta_n =
 *     beta / M (c_n = 1/M, the subset's share of the data):
 *       OSMAPOSL  f <- f H_m^T r / (H_m^T 1 + beta_n grad V(f)); a voxel whose
 *                 denominator is <= 0 is unchanged;
 *       BSREM     f <- max(0, f + alpha_t f / (c_n H^T 1) (H_m^T r - H_m^T 1
 *                 - beta_n grad V(f))), H^T 1 over all angles, alpha_t =
 *                 alpha0 / (1 + floor(t / M)) (one relaxation step per
 *                 iteration); a voxel with H^T 1 == 0 is unchanged.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(i, j, k, n, nz) ((((size_t)(i)) * (size_t)(n) + (size_t)(j)) * (size_t)(nz) + (size_t)(k))

/* ---------------------------------------------------------------- angles */

/* cos and sin of projection angle theta_n: the given angle (radians), or by
 * default theta_n = 2 pi n / n_angles, whose quarter turns (4 n a multiple
 * of n_angles) have the exact values 0 and +-1 (the FP64 library values of
 * cos(pi/2) and sin(pi) carry residues of ~1e-16, which would leak
 * rounding-level bilinear weights into voxels the exact rotation does not
 * reach). */
static void angle_cs(int n, int n_angles, const double* angles, double* ct, double* st)
{
    if (angles) {
        *ct = cos(angles[n]);
        *st = sin(angles[n]);
        return;
    }
    if ((4L * n) % n_angles == 0) {
        static const double qc[4] = {1.0, 0.0, -1.0, 0.0}, qs[4] = {0.0, 1.0, 0.0, -1.0};
        const int q = (int)((4L * n / n_angles) % 4);
        *ct = qc[q];
        *st = qs[q];
        return;
    }
    const double theta = 2.0 * M_PI * (double)n / (double)n_angles;
    *ct = cos(theta);
    *st = sin(theta);
}

int or_n_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---------------------------------------------------------------- T_cdr */

/* Largest truncation radius over all depth planes (sigma grows with d). */
int or_psf_rmax(int n, double sigma0, double slope, double nsigma, double det_offset)
{
    int rmax = 0;
    for (int i = 0; i < n; ++i) {
        double d = (double)n - (double)i - 0.5 + det_offset;
        double s = sigma0 + slope * d;
        int r = (int)ceil(nsigma * s);
        if (r > rmax) rmax = r;
    }
    return rmax;
}

/* Per-plane sigma, radius and normalised 1-D taps (T_cdr, Eq. 1).
 * taps is [n][2*rmax+1], tap t of plane i stored at taps[i*(2*rmax+1) + rmax + t]. */
void or_psf_taps(int n, double sigma0, double slope, double nsigma, double det_offset,
                 int rmax, double* sigma_out, int* radius_out, double* taps)
{
    int width = 2 * rmax + 1;
    for (int i = 0; i < n; ++i) {
        double d = (double)n - (double)i - 0.5 + det_offset;
        double s = sigma0 + slope * d;
        int r = (int)ceil(nsigma * s);
        double* w = taps + (size_t)i * width;
        for (int t = 0; t < width; ++t) w[t] = 0.0;
        double sum = 0.0;
        for (int t = -r; t <= r; ++t) {
            double v = exp(-(double)(t * t) / (2.0 * s * s));
            w[rmax + t] = v;
            sum += v;
        }
        for (int t = -r; t <= r; ++t) w[rmax + t] /= sum;
        if (sigma_out) sigma_out[i] = s;
        if (radius_out) radius_out[i] = r;
    }
}

/* 2-D blur of one n x nz plane: out[j][k] = sum_{t,u} w(t) w(u) in[j-t][k-u],
 * zero outside the plane.  w is centred: w[r + t], |t| <= r. */
static void blur_plane(const double* in, double* out, double* tmp, int n, int nz, const double* w, int r)
{
    /* along k */
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < nz; ++k) {
            double acc = 0.0;
            for (int u = -r; u <= r; ++u) {
                int kk = k - u;
                if (kk < 0 || kk >= nz) continue;
                acc += w[r + u] * in[(size_t)j * nz + kk];
            }
            tmp[(size_t)j * nz + k] = acc;
        }
    /* along j */
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < nz; ++k) {
            double acc = 0.0;
            for (int t = -r; t <= r; ++t) {
                int jj = j - t;
                if (jj < 0 || jj >= n) continue;
                acc += w[r + t] * tmp[(size_t)jj * nz + k];
            }
            out[(size_t)j * nz + k] = acc;
        }
}

/* ---------------------------------------------------------------- T_rot */

/* Bilinear rotation and translation (T_trans T_rot, Eq. 1):
 * out[i][j][k] = f(u(i,j), v(i,j), k) with j - c replaced by j - shift - c. */
static void rotate_cs(const double* f, int n, int nz, double ct, double st, double shift, double* out)
{
    double c = 0.5 * (double)(n - 1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double dj = (double)j - shift - c;
            double u = c + ct * ((double)i - c) - st * dj;
            double v = c + st * ((double)i - c) + ct * dj;
            double fu = floor(u), fv = floor(v);
            int x0 = (int)fu, y0 = (int)fv;
            double a = u - fu, b = v - fv;
            int xs[4] = {x0, x0 + 1, x0, x0 + 1};
            int ys[4] = {y0, y0, y0 + 1, y0 + 1};
            double ws[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
            double* o = out + IDX3(i, j, 0, n, nz);
            for (int k = 0; k < nz; ++k) o[k] = 0.0;
            for (int q = 0; q < 4; ++q) {
                if (xs[q] < 0 || xs[q] >= n || ys[q] < 0 || ys[q] >= n) continue;
                const double* src = f + IDX3(xs[q], ys[q], 0, n, nz);
                for (int k = 0; k < nz; ++k) o[k] += ws[q] * src[k];
            }
        }
}

void or_rotate_shift(const double* f, int n, int nz, double theta, double shift, double* out)
{
    rotate_cs(f, n, nz, cos(theta), sin(theta), shift, out);
}

/* Bilinear rotation (T_rot, Eq. 1): out[i][j][k] = f(u(i,j), v(i,j), k). */
void or_rotate(const double* f, int n, int nz, double theta, double* out)
{
    or_rotate_shift(f, n, nz, theta, 0.0, out);
}

/* Literal transpose of or_rotate_shift: every weight of sample (i,j) is
 * scattered back to the tap it read.  out is overwritten.  Parallel over z
 * only, so the order of the scatter is the same for every thread count. */
static void rotate_adjoint_cs(const double* in, int n, int nz, double ct, double st, double shift, double* out)
{
    double c = 0.5 * (double)(n - 1);
    memset(out, 0, sizeof(double) * (size_t)n * n * nz);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double dj = (double)j - shift - c;
                double u = c + ct * ((double)i - c) - st * dj;
                double v = c + st * ((double)i - c) + ct * dj;
                double fu = floor(u), fv = floor(v);
                int x0 = (int)fu, y0 = (int)fv;
                double a = u - fu, b = v - fv;
                int xs[4] = {x0, x0 + 1, x0, x0 + 1};
                int ys[4] = {y0, y0, y0 + 1, y0 + 1};
                double ws[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
                double val = in[IDX3(i, j, k, n, nz)];
                for (int q = 0; q < 4; ++q) {
                    if (xs[q] < 0 || xs[q] >= n || ys[q] < 0 || ys[q] >= n) continue;
                    out[IDX3(xs[q], ys[q], k, n, nz)] += ws[q] * val;
                }
            }
}

void or_rotate_adjoint_shift(const double* in, int n, int nz, double theta, double shift, double* out)
{
    rotate_adjoint_cs(in, n, nz, cos(theta), sin(theta), shift, out);
}

void or_rotate_adjoint(const double* in, int n, int nz, double theta, double* out)
{
    or_rotate_adjoint_shift(in, n, nz, theta, 0.0, out);
}

/* ---------------------------------------------------------------- T_att */

/* Attenuation weights of angle theta in the rotated (and shifted) frame
 * (T_att, Eq. 1): A[i][j][k] = exp(-(sum_{i'>i} tau[i'][j][k] + tau[i][j][k]/2)),
 * tau = voxel_cm * (T_trans T_rot mu).  mu in 1/cm. */
static void attenuation_cs(const double* mu, int n, int nz, double ct, double st, double shift, double voxel_cm,
                           double* A)
{
    size_t vol = (size_t)n * n * nz;
    double* m = (double*)malloc(sizeof(double) * vol);
    rotate_cs(mu, n, nz, ct, st, shift, m);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int k = 0; k < nz; ++k) {
            double beyond = 0.0; /* sum of tau over planes closer to the detector */
            for (int i = n - 1; i >= 0; --i) {
                double tau = voxel_cm * m[IDX3(i, j, k, n, nz)];
                A[IDX3(i, j, k, n, nz)] = exp(-(beyond + 0.5 * tau));
                beyond += tau;
            }
        }
    free(m);
}

void or_attenuation_shift(const double* mu, int n, int nz, double theta, double shift, double voxel_cm, double* A)
{
    attenuation_cs(mu, n, nz, cos(theta), sin(theta), shift, voxel_cm, A);
}

void or_attenuation(const double* mu, int n, int nz, double theta, double voxel_cm, double* A)
{
    or_attenuation_shift(mu, n, nz, theta, 0.0, voxel_cm, A);
}

/* ---------------------------------------------------------------- H, H^T */

/* Non-circular orbit (Sec. 2.1.1, the per-angle detector geometry of T_cdr):
 * per-angle detector offsets in voxels, or none (every angle uses the
 * geometry's det_offset).  Test infrastructure state, set by or_set_orbit. */
static double* g_orbit = NULL;
static int g_orbit_n = 0;

void or_set_orbit(const double* det_offsets, int n_angles)
{
    free(g_orbit);
    g_orbit = NULL;
    g_orbit_n = 0;
    if (det_offsets && n_angles > 0) {
        g_orbit = (double*)malloc(sizeof(double) * (size_t)n_angles);
        memcpy(g_orbit, det_offsets, sizeof(double) * (size_t)n_angles);
        g_orbit_n = n_angles;
    }
}

/* T_trans: per-angle shift of the rotated frame along +j (voxels), or none.
 * T_fov: per-angle projection-space weights [n_angles][n][nz], or none.
 * Test infrastructure state, set by or_set_trans / or_set_fov. */
static double* g_trans = NULL;
static int g_trans_n = 0;
static double* g_fov = NULL;
static size_t g_fov_len = 0;

void or_set_trans(const double* shifts, int n_angles)
{
    free(g_trans);
    g_trans = NULL;
    g_trans_n = 0;
    if (shifts && n_angles > 0) {
        g_trans = (double*)malloc(sizeof(double) * (size_t)n_angles);
        memcpy(g_trans, shifts, sizeof(double) * (size_t)n_angles);
        g_trans_n = n_angles;
    }
}

void or_set_fov(const double* mask, int n_angles, int n, int nz)
{
    free(g_fov);
    g_fov = NULL;
    g_fov_len = 0;
    if (mask && n_angles > 0) {
        g_fov_len = (size_t)n_angles * n * nz;
        g_fov = (double*)malloc(sizeof(double) * g_fov_len);
        memcpy(g_fov, mask, sizeof(double) * g_fov_len);
    }
}

static double trans_of(int angle) { return (g_trans && angle < g_trans_n) ? g_trans[angle] : 0.0; }

/* T_fov weights of one angle ([n][nz]) or NULL. */
static const double* fov_of(int angle, size_t plane)
{
    if (!g_fov || (size_t)(angle + 1) * plane > g_fov_len) return NULL;
    return g_fov + (size_t)angle * plane;
}

typedef struct {
    int n, nz, n_angles;
    const double* angles;  /* NULL: uniform */
    double voxel_cm;
    const double* mu;      /* NULL: no attenuation */
    int use_psf;
    double sigma0, slope, nsigma, det_offset;
} or_geom;

/* Per-angle forward projection H_n f (Eq. 1): rotate, attenuate, blur each
 * depth plane with its own PSF, sum over depth. proj is [n][nz]. */
static void forward_one(const or_geom* g, const double* f, int angle, double* proj,
                        const double* taps, const int* radius, int rmax)
{
    int n = g->n, nz = g->nz;
    size_t vol = (size_t)n * n * nz, plane = (size_t)n * nz;
    double ct, st;
    angle_cs(angle, g->n_angles, g->angles, &ct, &st);
    double* rot = (double*)malloc(sizeof(double) * vol);
    double* blurred = (double*)malloc(sizeof(double) * vol);
    double* own_taps = NULL;
    int* own_rad = NULL;
    if (g->use_psf && g_orbit && angle < g_orbit_n) {      /* this angle's own PSF table */
        rmax = or_psf_rmax(n, g->sigma0, g->slope, g->nsigma, g_orbit[angle]);
        own_taps = (double*)malloc(sizeof(double) * (size_t)n * (2 * rmax + 1));
        own_rad = (int*)malloc(sizeof(int) * (size_t)n);
        or_psf_taps(n, g->sigma0, g->slope, g->nsigma, g_orbit[angle], rmax, NULL, own_rad, own_taps);
        taps = own_taps;
        radius = own_rad;
    }
    const double shift = trans_of(angle);
    rotate_cs(f, n, nz, ct, st, shift, rot);               /* T_trans T_rot */
    if (g->mu) {                                           /* T_att */
        double* A = (double*)malloc(sizeof(double) * vol);
        attenuation_cs(g->mu, n, nz, ct, st, shift, g->voxel_cm, A);
        for (size_t q = 0; q < vol; ++q) rot[q] *= A[q];
        free(A);
    }
    if (g->use_psf) {                                      /* T_cdr */
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < n; ++i) {
            double* tmp = (double*)malloc(sizeof(double) * plane);
            blur_plane(rot + (size_t)i * plane, blurred + (size_t)i * plane, tmp, n, nz,
                       taps + (size_t)i * (2 * rmax + 1) + (rmax - radius[i]), radius[i]);
            free(tmp);
        }
    } else {
        memcpy(blurred, rot, sizeof(double) * vol);
    }
    for (size_t q = 0; q < plane; ++q) proj[q] = 0.0;     /* P_x: sum along +x */
    for (int i = 0; i < n; ++i)
        for (size_t q = 0; q < plane; ++q) proj[q] += blurred[(size_t)i * plane + q];
    const double* fov = fov_of(angle, plane);              /* T_fov */
    if (fov)
        for (size_t q = 0; q < plane; ++q) proj[q] *= fov[q];
    free(rot);
    free(blurred);
    free(own_taps);
    free(own_rad);
}

/* Per-angle back projection H_n^T q, ADDED into out: the transpose of each
 * step of forward_one in reverse order (the T_fov weights, broadcast over
 * depth, blur (the zero-padded symmetric Gaussian is self-adjoint),
 * attenuate, (T_trans T_rot)^T). */
static void back_one(const or_geom* g, const double* q_in, int angle, double* out,
                     const double* taps, const int* radius, int rmax)
{
    int n = g->n, nz = g->nz;
    size_t vol = (size_t)n * n * nz, plane = (size_t)n * nz;
    double ct, st;
    angle_cs(angle, g->n_angles, g->angles, &ct, &st);
    const double shift = trans_of(angle);
    const double* fov = fov_of(angle, plane);
    double* qm = (double*)malloc(sizeof(double) * plane);
    for (size_t p = 0; p < plane; ++p) qm[p] = fov ? fov[p] * q_in[p] : q_in[p];
    const double* q = qm;
    double* b = (double*)malloc(sizeof(double) * vol);
    double* r = (double*)malloc(sizeof(double) * vol);
    double* own_taps = NULL;
    int* own_rad = NULL;
    if (g->use_psf && g_orbit && angle < g_orbit_n) {      /* this angle's own PSF table */
        rmax = or_psf_rmax(n, g->sigma0, g->slope, g->nsigma, g_orbit[angle]);
        own_taps = (double*)malloc(sizeof(double) * (size_t)n * (2 * rmax + 1));
        own_rad = (int*)malloc(sizeof(int) * (size_t)n);
        or_psf_taps(n, g->sigma0, g->slope, g->nsigma, g_orbit[angle], rmax, NULL, own_rad, own_taps);
        taps = own_taps;
        radius = own_rad;
    }
    if (g->use_psf) {
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < n; ++i) {
            double* tmp = (double*)malloc(sizeof(double) * plane);
            blur_plane(q, b + (size_t)i * plane, tmp, n, nz,
                       taps + (size_t)i * (2 * rmax + 1) + (rmax - radius[i]), radius[i]);
            free(tmp);
        }
    } else {
        for (int i = 0; i < n; ++i) memcpy(b + (size_t)i * plane, q, sizeof(double) * plane);
    }
    if (g->mu) {
        double* A = (double*)malloc(sizeof(double) * vol);
        attenuation_cs(g->mu, n, nz, ct, st, shift, g->voxel_cm, A);
        for (size_t p = 0; p < vol; ++p) b[p] *= A[p];
        free(A);
    }
    rotate_adjoint_cs(b, n, nz, ct, st, shift, r);
    for (size_t p = 0; p < vol; ++p) out[p] += r[p];
    free(qm);
    free(b);
    free(r);
    free(own_taps);
    free(own_rad);
}

static or_geom make_geom(int n, int nz, int n_angles, const double* angles, double voxel_cm,
                         const double* mu, int use_psf, double sigma0, double slope,
                         double nsigma, double det_offset)
{
    or_geom g;
    g.n = n; g.nz = nz; g.n_angles = n_angles; g.angles = angles; g.voxel_cm = voxel_cm;
    g.mu = mu; g.use_psf = use_psf; g.sigma0 = sigma0; g.slope = slope; g.nsigma = nsigma;
    g.det_offset = det_offset;
    return g;
}

/* H restricted to the listed angles: proj is [n_sel][n][nz] in list order. */
void or_forward(const double* f, int n, int nz, int n_angles, const double* angles,
                double voxel_cm, const double* mu, int use_psf, double sigma0, double slope,
                double nsigma, double det_offset, const int* sel, int n_sel, double* proj)
{
    or_geom g = make_geom(n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma, det_offset);
    int rmax = use_psf ? or_psf_rmax(n, sigma0, slope, nsigma, det_offset) : 0;
    double* taps = (double*)malloc(sizeof(double) * (size_t)n * (2 * rmax + 1));
    int* radius = (int*)malloc(sizeof(int) * (size_t)n);
    if (use_psf) or_psf_taps(n, sigma0, slope, nsigma, det_offset, rmax, NULL, radius, taps);
    for (int s = 0; s < n_sel; ++s)
        forward_one(&g, f, sel[s], proj + (size_t)s * n * nz, taps, radius, rmax);
    free(taps);
    free(radius);
}

/* H^T restricted to the listed angles: out = sum_s H_{sel[s]}^T proj[s]. */
void or_back(const double* proj, int n, int nz, int n_angles, const double* angles,
             double voxel_cm, const double* mu, int use_psf, double sigma0, double slope,
             double nsigma, double det_offset, const int* sel, int n_sel, double* out)
{
    or_geom g = make_geom(n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma, det_offset);
    int rmax = use_psf ? or_psf_rmax(n, sigma0, slope, nsigma, det_offset) : 0;
    double* taps = (double*)malloc(sizeof(double) * (size_t)n * (2 * rmax + 1));
    int* radius = (int*)malloc(sizeof(int) * (size_t)n);
    if (use_psf) or_psf_taps(n, sigma0, slope, nsigma, det_offset, rmax, NULL, radius, taps);
    memset(out, 0, sizeof(double) * (size_t)n * n * nz);
    for (int s = 0; s < n_sel; ++s)
        back_one(&g, proj + (size_t)s * n * nz, sel[s], out, taps, radius, rmax);
    free(taps);
    free(radius);
}

/* ---------------------------------------------------------------- OSEM */

/* OSEM (Table 1, OSEM row, with the Poisson gradient of Table 1):
 * for subiterations t = first .. first+count-1, subset m = t mod M:
 *   p = H_m f;  r = y_m / (p + s);  f <- f * H_m^T r / H_m^T 1.
 * y is [n_angles][n][nz] in angle order; s is a constant additive term.
 * diag (optional) gets 3 doubles per subiteration, taken before the update:
 *   sum over S_m bins of (p + s), of y, and of y * p / (p + s). */
void or_osem(const double* y, double s, int n, int nz, int n_angles, const double* angles,
             double voxel_cm, const double* mu, int use_psf, double sigma0, double slope,
             double nsigma, double det_offset, int n_subsets, int first, int count,
             double* f, double* diag)
{
    size_t vol = (size_t)n * n * nz, plane = (size_t)n * nz;
    int* sel = (int*)malloc(sizeof(int) * (size_t)n_angles);
    double* p = (double*)malloc(sizeof(double) * plane * (size_t)n_angles);
    double* ones = (double*)malloc(sizeof(double) * plane * (size_t)n_angles);
    double* bp = (double*)malloc(sizeof(double) * vol);
    double* sens = (double*)malloc(sizeof(double) * vol);
    for (int t = first; t < first + count; ++t) {
        int m = t % n_subsets, ns = 0;
        for (int a = 0; a < n_angles; ++a)
            if (a % n_subsets == m) sel[ns++] = a;
        or_forward(f, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                   det_offset, sel, ns, p);
        double sum_ps = 0.0, sum_y = 0.0, sum_yfrac = 0.0;
        for (int a = 0; a < ns; ++a)
            for (size_t q = 0; q < plane; ++q) {
                double ybin = y[(size_t)sel[a] * plane + q];
                double den = p[(size_t)a * plane + q] + s;
                sum_ps += den;
                sum_y += ybin;
                sum_yfrac += den > 0.0 ? ybin * p[(size_t)a * plane + q] / den : 0.0;
                p[(size_t)a * plane + q] = den > 0.0 ? ybin / den : 0.0;   /* ratio */
                ones[(size_t)a * plane + q] = 1.0;
            }
        if (diag) {
            diag[3 * (t - first) + 0] = sum_ps;
            diag[3 * (t - first) + 1] = sum_y;
            diag[3 * (t - first) + 2] = sum_yfrac;
        }
        or_back(p, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                det_offset, sel, ns, bp);
        or_back(ones, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                det_offset, sel, ns, sens);
        for (size_t q = 0; q < vol; ++q)
            if (sens[q] > 0.0) f[q] = f[q] * bp[q] / sens[q];
    }
    free(sel);
    free(p);
    free(ones);
    free(bp);
    free(sens);
}

/* ---------------------------------------------------------------- likelihood */

/* Poisson log-likelihood without the log(y!) constant:
 * L = sum_b y_b log(p_b + s) - (p_b + s).  A bin with y_b == 0 contributes
 * -(p_b + s) whatever p_b + s is. */
double or_poisson_ll(const double* y, const double* p, double s, size_t count)
{
    double L = 0.0;
    for (size_t b = 0; b < count; ++b) {
        double lam = p[b] + s;
        if (y[b] != 0.0) L += y[b] * log(lam);
        L -= lam;
    }
    return L;
}

/* ---------------------------------------------------------------- priors */

/* Nearest-neighbour priors of Table 1: the pair function phi(a, b) and its
 * partial derivative in its first argument.
 *   kind 1, QuadraticPrior:          phi = ((a - b) / delta)^2 / 4
 *   kind 2, RelativeDifferencePrior: phi = (a - b)^2 / (a + b + gamma |a - b|)
 */
static double prior_phi(int kind, double a, double b, double delta, double gamma)
{
    double d = a - b;
    if (kind == 1) return (d / delta) * (d / delta) / 4.0;
    double den = a + b + gamma * fabs(d);
    return den != 0.0 ? d * d / den : 0.0;
}

/* d phi(a, b) / d a.  Quadratic: (a - b) / (2 delta^2).  RDP, with
 * S = a + b + gamma |a - b|: (2 (a - b) S - (a - b)^2 (1 + gamma sign(a - b)))
 * / S^2, written out without simplification. */
static double prior_dphi_a(int kind, double a, double b, double delta, double gamma)
{
    double d = a - b;
    if (kind == 1) return d / (2.0 * delta * delta);
    double S = a + b + gamma * fabs(d);
    if (S == 0.0) return 0.0;
    double sg = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
    return (2.0 * d * S - d * d * (1.0 + gamma * sg)) / (S * S);
}

/* V(f) = sum_r sum_s w_rs phi(f_r, f_s), s over the 26 neighbours of r that
 * lie inside the volume, w_rs = 1 / |r - s|. */
double or_prior_value(const double* f, int n, int nz, int kind, double delta, double gamma)
{
    double V = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < nz; ++k)
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int dk = -1; dk <= 1; ++dk) {
                            if (!di && !dj && !dk) continue;
                            int i2 = i + di, j2 = j + dj, k2 = k + dk;
                            if (i2 < 0 || i2 >= n || j2 < 0 || j2 >= n || k2 < 0 || k2 >= nz) continue;
                            double w = 1.0 / sqrt((double)(di * di + dj * dj + dk * dk));
                            V += w * prior_phi(kind, f[IDX3(i, j, k, n, nz)], f[IDX3(i2, j2, k2, n, nz)], delta, gamma);
                        }
    return V;
}

/* dV/df_r.  f_r appears in the terms (r, s) as the first argument and in
 * the terms (s, r) as the second; phi is symmetric for both priors, so the
 * second partial of (s, r) equals the first partial of (r, s):
 *   dV/df_r = sum_s w_rs 2 dphi(f_r, f_s)/da. */
void or_prior_grad(const double* f, int n, int nz, int kind, double delta, double gamma, double* grad)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < nz; ++k) {
                double g = 0.0, fr = f[IDX3(i, j, k, n, nz)];
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int dk = -1; dk <= 1; ++dk) {
                            if (!di && !dj && !dk) continue;
                            int i2 = i + di, j2 = j + dj, k2 = k + dk;
                            if (i2 < 0 || i2 >= n || j2 < 0 || j2 >= n || k2 < 0 || k2 >= nz) continue;
                            double w = 1.0 / sqrt((double)(di * di + dj * dj + dk * dk));
                            g += w * 2.0 * prior_dphi_a(kind, fr, f[IDX3(i2, j2, k2, n, nz)], delta, gamma);
                        }
                grad[IDX3(i, j, k, n, nz)] = g;
            }
}

/* ---------------------------------------------------------------- MAP */

/* OSMAPOSL (algo 1) and BSREM (algo 2) subiterations first .. first+count-1
 * with prior `kind` (0: none), as stated in the header (Eq. PGA, Table 1). */
void or_map(const double* y, double s, int n, int nz, int n_angles, const double* angles,
            double voxel_cm, const double* mu, int use_psf, double sigma0, double slope,
            double nsigma, double det_offset, int n_subsets, int first, int count,
            int algo, int kind, double beta, double delta, double gamma, double alpha0, double* f)
{
    size_t vol = (size_t)n * n * nz, plane = (size_t)n * nz;
    int* sel = (int*)malloc(sizeof(int) * (size_t)n_angles);
    double* p = (double*)malloc(sizeof(double) * plane * (size_t)n_angles);
    double* ones = (double*)malloc(sizeof(double) * plane * (size_t)n_angles);
    double* bp = (double*)malloc(sizeof(double) * vol);
    double* sens = (double*)malloc(sizeof(double) * vol);
    double* sens_all = (double*)malloc(sizeof(double) * vol);
    double* gv = (double*)calloc(vol, sizeof(double));
    double c = 1.0 / (double)n_subsets, beta_n = beta * c;
    for (size_t q = 0; q < plane * (size_t)n_angles; ++q) ones[q] = 1.0;
    if (algo == 2) {
        for (int a = 0; a < n_angles; ++a) sel[a] = a;
        or_back(ones, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma, det_offset,
                sel, n_angles, sens_all);
    }
    for (int t = first; t < first + count; ++t) {
        int m = t % n_subsets, ns = 0;
        for (int a = 0; a < n_angles; ++a)
            if (a % n_subsets == m) sel[ns++] = a;
        or_forward(f, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                   det_offset, sel, ns, p);
        for (int a = 0; a < ns; ++a)
            for (size_t q = 0; q < plane; ++q) {
                double den = p[(size_t)a * plane + q] + s;
                p[(size_t)a * plane + q] = den > 0.0 ? y[(size_t)sel[a] * plane + q] / den : 0.0;
            }
        or_back(p, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                det_offset, sel, ns, bp);
        or_back(ones, n, nz, n_angles, angles, voxel_cm, mu, use_psf, sigma0, slope, nsigma,
                det_offset, sel, ns, sens);
        if (kind) or_prior_grad(f, n, nz, kind, delta, gamma, gv);
        double alpha = alpha0 / (1.0 + (double)(t / n_subsets));
        for (size_t q = 0; q < vol; ++q) {
            if (algo == 1) {
                double den = sens[q] + beta_n * gv[q];
                if (den > 0.0) f[q] = f[q] * bp[q] / den;
            } else {
                if (sens_all[q] > 0.0) {
                    double v = f[q] + alpha * f[q] / (c * sens_all[q]) * (bp[q] - sens[q] - beta_n * gv[q]);
                    f[q] = v > 0.0 ? v : 0.0;
                }
            }
        }
    }
    free(sel);
    free(p);
    free(ones);
    free(bp);
    free(sens);
    free(sens_all);
    free(gv);
}

