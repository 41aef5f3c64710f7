/*
 * FP64 CPU oracle for all-sky seedless clustering (Thrane & Coughlin,
 * "Seedless clustering in all-sky searches for gravitational-wave transients").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain statement of what the
 * GPU scorer must compute.  It shares no code, header, table or constant
 * generator with the CUDA library; only tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * What it computes (paper sections cited per function):
 *   template generation  Sec. III (six random numbers per Bezier template, plus
 *                        a uniform random delay, Sec. III after Eq. 6)
 *   rasterisation        Sec. III, the quadratic Bezier curve (t(xi), f(xi))
 *   statistic            Eq. 7 (Eq. 5 with the delay phase), sigma^-2 weighted
 *                        form allowed by the footnote to Eq. 5
 *   selection            Sec. III (most significant cluster), Sec. V (runs with
 *                        different seeds combined by a maximum)
 *
 * Readings of the paper used here (the paper is silent on each):
 *   - Bezier control times are pinned to the first, middle and last column, so
 *     t(xi) = M xi with M = n_t - 1 and column j sits at xi = j / M; the curve
 *     gives exactly one pixel per column, the nearest frequency bin with halves
 *     rounded up.
 *   - Random numbers: Philox4x64-10 (Salmon et al., SC'11) with counter
 *     (g, 0, 0, 0) and key (seed, 0) for template index g.  Words u0, u1, u2
 *     give the control frequency bins floor(u * n_f / 2^64); u3 gives the delay
 *     tau = tau_max * ((2 (u3 >> 12) + 1) / 2^52 - 1), open and symmetric.
 *   - Phase factor exp(+2 pi i f tau) with f = f_min + bin * df (Eq. 7).
 *   - Weighted statistic: SNR = sum_j Re[e^{i theta_j} y_j sigma_j^-2] /
 *     sqrt(sum_j sigma_j^-2); paper mode: SNR = (1/N) sum_j Re[e^{i theta_j}
 *     y_j / sigma_j] (Eq. 7 with the complex SNR p = y / sigma).
 *   - Loudest = signed maximum; ties go to the smaller template index.
 *   - Notched pixels (the black lines of Fig. 1's caption): sigma = +infinity
 *     marks a pixel removed from the analysis; it contributes nothing to S or
 *     W (z = 0, w = 0, whatever y holds there).  The paper form keeps N, the
 *     template's pixel count.  A template whose pixels are all notched has no
 *     data: its SNR is 0.
 *
 * Precision: every step is IEEE binary64 with libm cos/sin; integers are exact
 * 64-bit (128-bit for the Philox products and the bin draw).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */
/* Philox4x64-10 as defined by Salmon, Moraes, Dror and Shaw (SC'11): each
 * round multiplies words 0 and 2 by two fixed odd constants, the new state is
 * (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)), and the
 * key is bumped by two Weyl constants between rounds. */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------ template parameters */
/* Sec. III: a template is drawn from random numbers; here three control
 * frequencies (integer bins, uniform on [0, n_f)) and one delay uniform on
 * (-tau_max, +tau_max) (the isotropic-sky delay prior of Sec. III). */
void orc_track_params(uint64_t seed, uint64_t g, int n_f, double tau_max,
                      uint32_t f[3], double *tau)
{
    uint64_t ctr[4] = {g, 0, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t u[4];
    orc_philox4x64_10(ctr, key, u);
    for (int k = 0; k < 3; ++k)
        f[k] = (uint32_t)(((unsigned __int128)u[k] * (uint64_t)n_f) >> 64);
    uint64_t v = u[3] >> 12;                         /* 52 random bits */
    double unit = (double)(2 * v + 1) / 4503599627370496.0 - 1.0; /* 2^52 */
    *tau = tau_max * unit;
}

/* ------------------------------------------------------------ rasterisation */
/* Sec. III, quadratic Bezier: f(xi) = (1-xi)^2 f0 + 2 (1-xi) xi f1 + xi^2 f2.
 * With xi = j / M the value is num_j / M^2 where
 * num_j = (M-j)^2 f0 + 2 (M-j) j f1 + j^2 f2, an exact integer; the pixel is
 * the nearest bin, halves rounded up: floor((2 num_j + M^2) / (2 M^2)). */
void orc_track_bins(const uint32_t f[3], int n_t, int32_t *bins)
{
    int64_t M = (int64_t)n_t - 1;
    int64_t M2 = M * M;
    for (int64_t j = 0; j <= M; ++j) {
        int64_t a = M - j;
        int64_t num = a * a * (int64_t)f[0] + 2 * a * j * (int64_t)f[1] + j * j * (int64_t)f[2];
        bins[j] = (int32_t)((2 * num + M2) / (2 * M2));
    }
}

/* ---------------------------------------------------------------------- map */
/* The map the statistic reads: z = y sigma^-2 and w = sigma^-2 (weighted), or
 * z = y / sigma and w = 1 (paper mode), all in binary64, [n_t][n_f]. */
typedef struct {
    int n_t, n_f;
    double f_min, df;
    int paper_mode;
    double *z;   /* interleaved re, im: 2 * n_t * n_f */
    double *w;   /* n_t * n_f */
} orc_map;

orc_map *orc_map_create(const float *y_c64, const float *sigma, int sigma_per_freq,
                        int n_t, int n_f, double f_min, double df, int paper_mode)
{
    orc_map *m = (orc_map *)calloc(1, sizeof(orc_map));
    if (!m) return NULL;
    size_t np = (size_t)n_t * (size_t)n_f;
    m->n_t = n_t; m->n_f = n_f; m->f_min = f_min; m->df = df; m->paper_mode = paper_mode;
    m->z = (double *)malloc(2 * np * sizeof(double));
    m->w = (double *)malloc(np * sizeof(double));
    if (!m->z || !m->w) { free(m->z); free(m->w); free(m); return NULL; }
    for (int t = 0; t < n_t; ++t) {
        for (int k = 0; k < n_f; ++k) {
            size_t p = (size_t)t * n_f + k;
            double s = sigma_per_freq ? (double)sigma[k] : (double)sigma[p];
            double yr = (double)y_c64[2 * p], yi = (double)y_c64[2 * p + 1];
            if (isinf(s) && s > 0) {                     /* notched: no data */
                m->z[2 * p] = 0.0; m->z[2 * p + 1] = 0.0; m->w[p] = paper_mode ? 1.0 : 0.0;
            } else if (paper_mode) {
                m->z[2 * p] = yr / s; m->z[2 * p + 1] = yi / s; m->w[p] = 1.0;
            } else {
                double w = 1.0 / (s * s);
                m->z[2 * p] = yr * w; m->z[2 * p + 1] = yi * w; m->w[p] = w;
            }
        }
    }
    return m;
}

void orc_map_free(orc_map *m)
{
    if (!m) return;
    free(m->z); free(m->w); free(m);
}

/* ---------------------------------------------------------------- statistic */
/* Eq. 7: sum over the template's pixels of Re[exp(2 pi i f tau) p(t; f)].
 * Returns the SNR; also the raw sums S, W, and two magnitude sums used to
 * bound rounding in comparisons: sum_j |Re term_j| and sum_j |z_j|. */
double orc_score_track(const orc_map *m, const uint32_t f[3], double tau,
                       double *S_out, double *W_out, double *absterm_out, double *absz_out)
{
    int n_t = m->n_t;
    int32_t *bins = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_t);
    orc_track_bins(f, n_t, bins);
    double S = 0.0, W = 0.0, A = 0.0, Z = 0.0;
    for (int j = 0; j < n_t; ++j) {
        size_t p = (size_t)j * m->n_f + (size_t)bins[j];
        double fr = m->f_min + (double)bins[j] * m->df;
        double th = 2.0 * M_PI * fr * tau;
        double zr = m->z[2 * p], zi = m->z[2 * p + 1];
        double term = cos(th) * zr - sin(th) * zi;   /* Re[(cos + i sin)(zr + i zi)] */
        S += term;
        W += m->w[p];
        A += fabs(term);
        Z += sqrt(zr * zr + zi * zi);
    }
    free(bins);
    double snr = m->paper_mode ? S / (double)n_t : (W > 0.0 ? S / sqrt(W) : 0.0);
    if (S_out) *S_out = S;
    if (W_out) *W_out = W;
    if (absterm_out) *absterm_out = A;
    if (absz_out) *absz_out = Z;
    return snr;
}

void orc_score_explicit(const orc_map *m, const uint32_t *f3, const double *tau, uint64_t n,
                        double *snr, double *S, double *W, double *absterm, double *absz)
{
    for (uint64_t i = 0; i < n; ++i)
        snr[i] = orc_score_track(m, f3 + 3 * i, tau[i], S ? S + i : NULL, W ? W + i : NULL,
                                 absterm ? absterm + i : NULL, absz ? absz + i : NULL);
}

/* Score templates g = offset .. offset + T - 1 drawn with `seed`; threads take
 * contiguous slices of the range.  snr_out[i] is the SNR of template offset+i. */
typedef struct {
    const orc_map *m;
    uint64_t seed, g0, n;
    double tau_max;
    double *out;
    double *scale;   /* optional: sum_j |z_j| / norm, the scale of the comparison bound */
} orc_job;

static void *orc_range_worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    for (uint64_t i = 0; i < jb->n; ++i) {
        uint32_t f[3];
        double tau, W = 0.0, Z = 0.0;
        orc_track_params(jb->seed, jb->g0 + i, jb->m->n_f, jb->tau_max, f, &tau);
        jb->out[i] = orc_score_track(jb->m, f, tau, NULL, &W, NULL, &Z);
        if (jb->scale) jb->scale[i] = jb->m->paper_mode ? Z / (double)jb->m->n_t : (W > 0.0 ? Z / sqrt(W) : 0.0);
    }
    return NULL;
}

static int orc_range_run(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max,
                         int nthreads, double *snr_out, double *scale_out);

int orc_score_range(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T,
                    double tau_max, int nthreads, double *snr_out)
{
    return orc_range_run(m, seed, offset, T, tau_max, nthreads, snr_out, NULL);
}

/* As orc_score_range, also writing each template's comparison scale
 * sum_j |z_j| / norm (norm = sqrt(W), or N in the paper form). */
int orc_score_range_scale(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T,
                          double tau_max, int nthreads, double *snr_out, double *scale_out)
{
    return orc_range_run(m, seed, offset, T, tau_max, nthreads, snr_out, scale_out);
}

static int orc_range_run(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max,
                         int nthreads, double *snr_out, double *scale_out)
{
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > T) nthreads = T ? (int)T : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    orc_job *jobs = (orc_job *)malloc(sizeof(orc_job) * (size_t)nthreads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    uint64_t base = T / (uint64_t)nthreads, rem = T % (uint64_t)nthreads, start = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t n = base + ((uint64_t)t < rem ? 1 : 0);
        jobs[t].m = m; jobs[t].seed = seed; jobs[t].g0 = offset + start; jobs[t].n = n;
        jobs[t].tau_max = tau_max; jobs[t].out = snr_out + start;
        jobs[t].scale = scale_out ? scale_out + start : NULL;
        start += n;
    }
    int rc = 0, started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, orc_range_worker, &jobs[t]) != 0) { rc = -2; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return rc;
}

/* ---------------------------------------------------------------- selection */
/* Most significant cluster (Sec. III) generalised to the K largest: order by
 * SNR descending, then template index ascending. */
typedef struct { double snr; uint64_t g; } orc_rec;

static int orc_rec_cmp(const void *a, const void *b)
{
    const orc_rec *x = (const orc_rec *)a, *y = (const orc_rec *)b;
    if (x->snr > y->snr) return -1;
    if (x->snr < y->snr) return 1;
    if (x->g < y->g) return -1;
    if (x->g > y->g) return 1;
    return 0;
}

int orc_topk(const double *snr, uint64_t T, uint64_t offset, int K,
             double *snr_k, uint64_t *g_k)
{
    if (K < 0 || (uint64_t)K > T) return -1;
    orc_rec *r = (orc_rec *)malloc(sizeof(orc_rec) * (size_t)(T ? T : 1));
    if (!r) return -2;
    for (uint64_t i = 0; i < T; ++i) { r[i].snr = snr[i]; r[i].g = offset + i; }
    qsort(r, (size_t)T, sizeof(orc_rec), orc_rec_cmp);
    for (int i = 0; i < K; ++i) { snr_k[i] = r[i].snr; g_k[i] = r[i].g; }
    free(r);
    return 0;
}

/* ------------------------------------------------- interpolated statistic */
/* Refinement of loud templates (the follow-up of Sec. V): the control
 * frequencies become real numbers (in bins) and the delay stays continuous.
 * The curve's frequency at column j is x_j = ((M-j)^2 f0 + 2 (M-j) j f1 + j^2 f2) / M^2
 * (bins, clamped to [0, n_f - 1]).  The map between bins is interpolated
 * linearly in frequency: with k = floor(x_j) (at most n_f - 2) and a = x_j - k,
 *   z(j, x) = (1 - a) z[j][k] + a z[j][k+1],  w(j, x) = (1 - a) w[j][k] + a w[j][k+1].
 * The statistic is Eq. 7 with the continuous frequency f = f_min + x df:
 *   S = sum_j Re[exp(2 pi i f(x_j) tau) z(j, x_j)],  W = sum_j w(j, x_j),
 *   SNR = S / sqrt(W) (weighted) or S / N (paper form).
 * At integer x_j this is the discrete statistic.  grad[0..3] receives
 * d SNR / d (f0, f1, f2, tau), by differentiating each step above (zero
 * where x_j is clamped). */
double orc_interp_score(const orc_map *m, const double f[3], double tau, double grad[4])
{
    const int n_t = m->n_t, n_f = m->n_f;
    const double M = (double)(n_t - 1), M2 = M * M;
    double S = 0, W = 0, dS[4] = {0, 0, 0, 0}, dW[3] = {0, 0, 0};
    for (int j = 0; j < n_t; ++j) {
        const double cj[3] = {(M - j) * (M - j) / M2, 2.0 * (M - j) * j / M2, (double)j * j / M2};
        double x = cj[0] * f[0] + cj[1] * f[1] + cj[2] * f[2];
        int clamped = 0;
        if (x < 0) { x = 0; clamped = 1; }
        if (x > n_f - 1) { x = n_f - 1; clamped = 1; }
        int k = (int)floor(x);
        if (k > n_f - 2) k = n_f - 2;
        if (k < 0) k = 0;
        const double a = n_f > 1 ? x - k : 0.0;
        const size_t p0 = (size_t)j * n_f + k, p1 = n_f > 1 ? p0 + 1 : p0;
        const double zr = (1 - a) * m->z[2 * p0] + a * m->z[2 * p1];
        const double zi = (1 - a) * m->z[2 * p0 + 1] + a * m->z[2 * p1 + 1];
        const double dzr = m->z[2 * p1] - m->z[2 * p0], dzi = m->z[2 * p1 + 1] - m->z[2 * p0 + 1];
        const double w = (1 - a) * m->w[p0] + a * m->w[p1], dw = m->w[p1] - m->w[p0];
        const double fr = m->f_min + x * m->df;
        const double ph = 2.0 * M_PI * fr * tau;
        const double c = cos(ph), s = sin(ph);
        const double re = c * zr - s * zi;      /* Re[e^{i ph} z] */
        const double im = s * zr + c * zi;      /* Im[e^{i ph} z] */
        S += re;
        W += w;
        /* d re / d x = -im * (2 pi df tau) + Re[e^{i ph} dz/dx]; d re / d tau = -im * 2 pi f */
        const double dre_dx = clamped ? 0.0 : (-im * 2.0 * M_PI * m->df * tau + (c * dzr - s * dzi));
        const double dw_dx = clamped ? 0.0 : dw;
        for (int q = 0; q < 3; ++q) {
            dS[q] += dre_dx * cj[q];
            dW[q] += dw_dx * cj[q];
        }
        dS[3] += -im * 2.0 * M_PI * fr;
    }
    double snr;
    if (m->paper_mode) {
        snr = S / n_t;
        if (grad) for (int q = 0; q < 4; ++q) grad[q] = dS[q] / n_t;
    } else {
        const double rw = W > 0.0 ? 1.0 / sqrt(W) : 0.0;   /* every pixel notched: no data */
        snr = S * rw;
        if (grad) {
            for (int q = 0; q < 3; ++q) grad[q] = dS[q] * rw - 0.5 * S * rw * rw * rw * dW[q];
            grad[3] = dS[3] * rw;
        }
    }
    return snr;
}

void orc_interp_explicit(const orc_map *m, const double *f3, const double *tau, uint64_t n, double *snr,
                         double *grad4)
{
    for (uint64_t i = 0; i < n; ++i) snr[i] = orc_interp_score(m, f3 + 3 * i, tau[i], grad4 ? grad4 + 4 * i : NULL);
}

/* ------------------------------------------------------ general templates */
/* Sec. III: three time-frequency control points (t_k, f_k) from six random
 * numbers, persisting at least t_min columns.  Reading: integer control times
 * t0 <= t1 <= t2 from Philox block (g, 1, 0, 0): duration d = t2 - t0 uniform on
 * [t_min, n_t - 1] (word 0), start uniform on [0, n_t - 1 - d] (word 1), t1 - t0
 * uniform on [0, d] (word 2); each as floor(word * range / 2^64). */
void orc_track_times(uint64_t seed, uint64_t g, int n_t, int t_min, uint32_t t[3])
{
    uint64_t ctr[4] = {g, 1, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t v[4];
    orc_philox4x64_10(ctr, key, v);
    uint64_t M = (uint64_t)n_t - 1;
    uint64_t d = (uint64_t)t_min + (uint64_t)(((unsigned __int128)v[0] * (M - (uint64_t)t_min + 1)) >> 64);
    uint64_t t0 = (uint64_t)(((unsigned __int128)v[1] * (M - d + 1)) >> 64);
    uint64_t t1 = t0 + (uint64_t)(((unsigned __int128)v[2] * (d + 1)) >> 64);
    t[0] = (uint32_t)t0; t[1] = (uint32_t)t1; t[2] = (uint32_t)(t0 + d);
}

/* A delay prior given by quantiles (Sec. VI: a sky patch instead of the
 * isotropic sky): the delay at probability p = (u3 >> 11) / 2^53 is the linear
 * interpolation of the table at p (n_q - 1).  Bins as orc_track_params. */
void orc_track_params_prior(uint64_t seed, uint64_t g, int n_f, const double *tq, int n_q, uint32_t f[3],
                            double *tau)
{
    uint64_t ctr[4] = {g, 0, 0, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t u[4];
    orc_philox4x64_10(ctr, key, u);
    for (int k = 0; k < 3; ++k)
        f[k] = (uint32_t)(((unsigned __int128)u[k] * (uint64_t)n_f) >> 64);
    double p = (double)(u[3] >> 11) / 9007199254740992.0;   /* 2^53 */
    double q = p * (double)(n_q - 1);
    int i = (int)floor(q);
    if (i > n_q - 2) i = n_q - 2;
    double fr = q - (double)i;
    *tau = tq[i] + fr * (tq[i + 1] - tq[i]);
}

/* The curve of a general template: t(xi) = (1-xi)^2 t0 + 2 (1-xi) xi t1 + xi^2 t2,
 * f(xi) likewise.  For column j in [t0, t2] the point xi_j in [0, 1] with
 * t(xi_j) = j, and the pixel is the nearest bin to f(xi_j), halves rounded up.
 * Test "f(xi_j) >= y" for a half-integer y exactly: write a = t0 - 2 t1 + t2,
 * b = 2 (t1 - t0), F = f0 - 2 f1 + f2, G = 2 (f1 - f0), u = 2 (j - t0),
 * Delta = b^2 + 4 a (j - t0) and s = sqrt(Delta); then xi_j = u / (s + b) and
 * (2 f(xi_j) - 2 y) (s + b)^2 = P + Q s with
 * P = 2 F u^2 + 2 G u b + e (Delta + b^2), Q = 2 G u + 2 e b, e = 2 f0 - 2 y,
 * whose sign is fixed by the signs of P, Q and, when they differ, P^2 - Q^2 Delta. */
static int orc_half_ge(const int64_t tt[3], const int64_t ff[3], int64_t j, int64_t twice_y)
{
    __int128 a = tt[0] - 2 * tt[1] + tt[2], b = 2 * (tt[1] - tt[0]);
    __int128 F = ff[0] - 2 * ff[1] + ff[2], G = 2 * (ff[1] - ff[0]);
    __int128 u = 2 * (j - tt[0]);
    __int128 Delta = b * b + 4 * a * (j - tt[0]);
    __int128 e = 2 * ff[0] - twice_y;
    __int128 P = 2 * F * u * u + 2 * G * u * b + e * (Delta + b * b);
    __int128 Q = 2 * G * u + 2 * e * b;
    if (P >= 0 && Q >= 0) return 1;
    if (P <= 0 && Q <= 0) return P == 0 && Q == 0;
    __int128 lhs = P * P, rhs = Q * Q * Delta;
    return P > 0 ? lhs >= rhs : rhs >= lhs;
}

/* Pixels of a general template: bins[j] for j in [t0, t2], -1 elsewhere.  An FP64
 * estimate of f(xi_j), then the exact test moves it to the nearest bin. */
void orc_track_bins_general(const uint32_t t[3], const uint32_t f[3], int n_t, int n_f, int32_t *bins)
{
    int64_t tt[3] = {t[0], t[1], t[2]}, ff[3] = {f[0], f[1], f[2]};
    double a = (double)(tt[0] - 2 * tt[1] + tt[2]), b = (double)(2 * (tt[1] - tt[0]));
    double F = (double)(ff[0] - 2 * ff[1] + ff[2]), G = (double)(2 * (ff[1] - ff[0]));
    for (int j = 0; j < n_t; ++j) {
        if (j < (int)t[0] || j > (int)t[2]) { bins[j] = -1; continue; }
        if (j == (int)t[0]) { bins[j] = (int32_t)f[0]; continue; }
        double Delta = b * b + 4.0 * a * (double)(j - (int64_t)t[0]);
        double xi = 2.0 * (double)(j - (int64_t)t[0]) / (sqrt(Delta > 0 ? Delta : 0) + b);
        double fx = (double)ff[0] + xi * (G + F * xi);
        int64_t k = (int64_t)floor(fx + 0.5);
        if (k < 0) k = 0;
        if (k > n_f - 1) k = n_f - 1;
        /* exact: the largest k with f >= k - 1/2 */
        while (k > 0 && !orc_half_ge(tt, ff, j, 2 * k - 1)) --k;
        while (k + 1 < n_f && orc_half_ge(tt, ff, j, 2 * (k + 1) - 1)) ++k;
        bins[j] = (int32_t)k;
    }
}

/* Eq. 7 over a general template's N = t2 - t0 + 1 pixels. */
/* Eq. 7 over a general template's pixels; *scale_out (optional) receives the
 * comparison scale sum_j |z_j| / norm. */
static double orc_score_general_scale(const orc_map *m, const uint32_t t[3], const uint32_t f[3], double tau,
                                      double *scale_out)
{
    int32_t *bins = (int32_t *)malloc(sizeof(int32_t) * (size_t)m->n_t);
    orc_track_bins_general(t, f, m->n_t, m->n_f, bins);
    double S = 0.0, W = 0.0, Z = 0.0;
    int N = 0;
    for (int j = 0; j < m->n_t; ++j) {
        if (bins[j] < 0) continue;
        size_t p = (size_t)j * m->n_f + (size_t)bins[j];
        double th = 2.0 * M_PI * (m->f_min + (double)bins[j] * m->df) * tau;
        double zr = m->z[2 * p], zi = m->z[2 * p + 1];
        S += cos(th) * zr - sin(th) * zi;
        W += m->w[p];
        Z += sqrt(zr * zr + zi * zi);
        ++N;
    }
    free(bins);
    double norm = m->paper_mode ? (double)N : sqrt(W);
    if (!(norm > 0.0)) {                                  /* every pixel notched: no data */
        if (scale_out) *scale_out = 0.0;
        return 0.0;
    }
    if (scale_out) *scale_out = Z / norm;
    return S / norm;
}

double orc_score_general(const orc_map *m, const uint32_t t[3], const uint32_t f[3], double tau)
{
    return orc_score_general_scale(m, t, f, tau, NULL);
}

void orc_score_explicit_general(const orc_map *m, const uint32_t *t3, const uint32_t *f3, const double *tau,
                                uint64_t n, double *snr)
{
    for (uint64_t i = 0; i < n; ++i) snr[i] = orc_score_general(m, t3 + 3 * i, f3 + 3 * i, tau[i]);
}

/* Templates offset .. offset + T - 1 with general times and optionally a delay
 * prior (n_q >= 2); threads take contiguous slices. */
typedef struct {
    const orc_map *m;
    uint64_t seed, g0, n;
    double tau_max;
    int general, t_min, n_q;
    const double *tq;
    double *out;
    double *scale;   /* optional: comparison scale sum_j |z_j| / norm */
} orc_gjob;

static void *orc_general_worker(void *arg)
{
    orc_gjob *jb = (orc_gjob *)arg;
    for (uint64_t i = 0; i < jb->n; ++i) {
        uint32_t f[3], t[3];
        double tau;
        uint64_t g = jb->g0 + i;
        if (jb->n_q >= 2) orc_track_params_prior(jb->seed, g, jb->m->n_f, jb->tq, jb->n_q, f, &tau);
        else orc_track_params(jb->seed, g, jb->m->n_f, jb->tau_max, f, &tau);
        if (jb->general) {
            orc_track_times(jb->seed, g, jb->m->n_t, jb->t_min, t);
            jb->out[i] = orc_score_general_scale(jb->m, t, f, tau, jb->scale ? jb->scale + i : NULL);
        } else {
            double W = 0.0, Z = 0.0;
            jb->out[i] = orc_score_track(jb->m, f, tau, NULL, &W, NULL, &Z);
            if (jb->scale) jb->scale[i] = jb->m->paper_mode ? Z / (double)jb->m->n_t : (W > 0.0 ? Z / sqrt(W) : 0.0);
        }
    }
    return NULL;
}

static int orc_range_ext_run(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max,
                             int general, int t_min, const double *tq, int n_q, int nthreads, double *snr_out,
                             double *scale_out);

int orc_score_range_ext(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max, int general,
                        int t_min, const double *tq, int n_q, int nthreads, double *snr_out)
{
    return orc_range_ext_run(m, seed, offset, T, tau_max, general, t_min, tq, n_q, nthreads, snr_out, NULL);
}

/* As orc_score_range_ext, also writing each template's comparison scale. */
int orc_score_range_ext_scale(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max,
                              int general, int t_min, const double *tq, int n_q, int nthreads, double *snr_out,
                              double *scale_out)
{
    return orc_range_ext_run(m, seed, offset, T, tau_max, general, t_min, tq, n_q, nthreads, snr_out, scale_out);
}

static int orc_range_ext_run(const orc_map *m, uint64_t seed, uint64_t offset, uint64_t T, double tau_max,
                             int general, int t_min, const double *tq, int n_q, int nthreads, double *snr_out,
                             double *scale_out)
{
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > T) nthreads = T ? (int)T : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    orc_gjob *jobs = (orc_gjob *)malloc(sizeof(orc_gjob) * (size_t)nthreads);
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    uint64_t base = T / (uint64_t)nthreads, rem = T % (uint64_t)nthreads, start = 0;
    for (int t = 0; t < nthreads; ++t) {
        uint64_t n = base + ((uint64_t)t < rem ? 1 : 0);
        orc_gjob j = {m, seed, offset + start, n, tau_max, general, t_min, n_q, tq, snr_out + start,
                      scale_out ? scale_out + start : NULL};
        jobs[t] = j;
        start += n;
    }
    int rc = 0, started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, orc_general_worker, &jobs[t]) != 0) { rc = -2; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return rc;
}
