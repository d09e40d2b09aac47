/*
 * spiir_oracle.c -- FP64 CPU oracle for SPIIR filtering (arXiv:1702.02256).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library. The product path never
 * calls it, and it shares no code, header, table or constant generator with
 * the CUDA library: everything here is written out again from the paper.
 *
 * It is deliberately plain and slow: one filter at a time, one sample at a
 * time, every product and sum in double precision, in the order the paper
 * states the method. Inputs are the exact float32 values (complex64 filter
 * coefficients, float32 strain and resampling taps) widened to double.
 *
 * What each function follows:
 *   spiir_oracle_single      Sec. 2.1, Eq. (iireq0) per filter and Eq. (iireq1)
 *                            summed over a template's filters.
 *   spiir_oracle_single_from The same recursion with the filter state zero
 *                            before a start sample while the strain before it
 *                            is real (a bank joining a running stream).
 *   spiir_oracle_decimate    Sec. 2.2, Eq. (kaiser_window_filtering), causal
 *                            T-tap form, keep every second output.
 *   spiir_oracle_upsample_add  Sec. 2.2 (Fig. 1): zero-stuff x2, Kaiser
 *                            low-pass with gain 2, add to the next rate up.
 *   spiir_oracle_multirate   Sec. 2.2: decimate in succession, filter each
 *                            rate with its own filters, upsample the lowest
 *                            rate's output and add it to the next rate up,
 *                            repeat to the input rate.
 *   spiir_oracle_kaiser_taps Sec. 2.2: Kaiser-window-tapered low-pass,
 *                            window parameter from Kaiser's published
 *                            attenuation formula, I0 by its power series.
 *   spiir_oracle_assign_level Sec. 2.2: the filter's band edge from arg(a),
 *                            its Nyquist rate rounded up to an available rate
 *                            (spiir_oracle_assign_level_margin: with an
 *                            optional passband margin).
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - filter state starts at zero and x[n] = 0 for n < 0;
 *   - x is real; a, b, y and z are complex;
 *   - d_k counts samples at the filter's own rate;
 *   - z = scale * (sum over filters), scale = 2*dt = 2/base_rate by default;
 *   - the level-i sum is delayed by D_i = R + 2*D_{i+1} (D_H = 0) so that a
 *     down/up round trip lines up with it; R = (Td-1)/2 + (Tu-1)/2 is the
 *     sum of the two linear-phase filters' group delays at the higher rate
 *     (T-1 when both have T taps; the decimator may be longer, e.g. the
 *     paper's 100 dB design, and Td + Tu must be even); align = 0 sets every
 *     D_i to 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Kaiser-window low-pass taps (Sec. 2.2)                              */
/* ------------------------------------------------------------------ */

/* Modified Bessel function of the first kind, order 0, by its power series
 * I0(x) = sum_m ((x/2)^m / m!)^2. */
double spiir_oracle_bessel_i0(double x) {
    double sum = 1.0, term = 1.0, half = 0.5 * x;
    for (int m = 1; m < 500; ++m) {
        term *= (half / m) * (half / m);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* Kaiser's empirical window parameter for stop-band attenuation A (dB). */
double spiir_oracle_kaiser_beta(double atten_db) {
    if (atten_db > 50.0) return 0.1102 * (atten_db - 8.7);
    if (atten_db >= 21.0)
        return 0.5842 * pow(atten_db - 21.0, 0.4) + 0.07886 * (atten_db - 21.0);
    return 0.0;
}

/* n_taps-tap linear-phase low-pass with cutoff at half the input Nyquist
 * frequency (pi/2 rad/sample): ideal impulse response sin(w m)/(pi m) about
 * the centre m = n - (n_taps-1)/2, times a Kaiser window, normalised to unit
 * DC gain, then rounded to float32. */
int spiir_oracle_kaiser_taps(int32_t n_taps, double atten_db, float *out) {
    if (n_taps < 2 || !out) return 1;
    double beta = spiir_oracle_kaiser_beta(atten_db);
    double i0b = spiir_oracle_bessel_i0(beta);
    double *h = (double *)malloc(sizeof(double) * (size_t)n_taps);
    if (!h) return 2;
    double total = 0.0;
    for (int n = 0; n < n_taps; ++n) {
        double m = (double)n - 0.5 * (double)(n_taps - 1);
        double wc = 0.5 * ORACLE_PI;
        double ideal = (m == 0.0) ? wc / ORACLE_PI : sin(wc * m) / (ORACLE_PI * m);
        double r = 2.0 * (double)n / (double)(n_taps - 1) - 1.0;
        double arg = 1.0 - r * r;
        if (arg < 0.0) arg = 0.0;
        double w = spiir_oracle_bessel_i0(beta * sqrt(arg)) / i0b;
        h[n] = ideal * w;
        total += h[n];
    }
    for (int n = 0; n < n_taps; ++n) out[n] = (float)(h[n] / total);
    free(h);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Rate assignment (Sec. 2.2)                                          */
/* ------------------------------------------------------------------ */

int32_t spiir_oracle_assign_level_margin(double a_re, double a_im, int32_t base_rate,
                                         int32_t n_levels, double margin);

/* a is the base-rate pole. Its band edge is f = |arg a| * base_rate / (2 pi);
 * the filter needs a rate of at least 2 f (Nyquist); the chosen level is the
 * one with the smallest available rate base_rate / 2^i that is >= 2 f. */
int32_t spiir_oracle_assign_level(double a_re, double a_im, int32_t base_rate,
                                  int32_t n_levels) {
    return spiir_oracle_assign_level_margin(a_re, a_im, base_rate, n_levels, 0.0);
}

/* The same rule with a passband margin (an optional knob; the paper's rule
 * is margin = 0): the rate must be at least 2 f (1 + margin), so that the
 * band edge stays clear of the resamplers' transition band. */
int32_t spiir_oracle_assign_level_margin(double a_re, double a_im, int32_t base_rate,
                                         int32_t n_levels, double margin) {
    double f = fabs(atan2(a_im, a_re)) * (double)base_rate / (2.0 * ORACLE_PI);
    double need = 2.0 * f * (1.0 + margin);
    for (int32_t i = n_levels - 1; i >= 0; --i) {
        double rate = (double)base_rate / (double)(1 << i);
        if (rate >= need) return i;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Single-rate SPIIR (Sec. 2.1, Eqs. iireq0 and iireq1)                 */
/* ------------------------------------------------------------------ */

/* One filter, y[n] = a*y[n-1] + b*x[n-d] for n = start..n_samples-1 with
 * y[start-1] = 0 and x[<0] = 0, its output added to acc[n] (complex,
 * interleaved re/im); acc[n] for n < start is left alone. */
static void filter_into(double a_re, double a_im, double b_re, double b_im,
                        int32_t d, const double *x, int64_t n_samples,
                        double *acc, int64_t start) {
    double y_re = 0.0, y_im = 0.0;
    for (int64_t n = start; n < n_samples; ++n) {
        double xin = (n - d >= 0) ? x[n - d] : 0.0;
        double ny_re = a_re * y_re - a_im * y_im + b_re * xin;
        double ny_im = a_re * y_im + a_im * y_re + b_im * xin;
        y_re = ny_re;
        y_im = ny_im;
        acc[2 * n] += y_re;
        acc[2 * n + 1] += y_im;
    }
}

/* Filters grouped by template through tmpl_ptr (filters tmpl_ptr[t] ..
 * tmpl_ptr[t+1]-1 belong to template t). For each selected template t
 * (tsel[j], or all when tsel is NULL) writes
 *   z[j][n] = scale * sum_k y_k[n]      (complex, interleaved)
 * summed over the template's filters in index order. */
static int single_from(int32_t n_templates, const int64_t *tmpl_ptr,
                       const float *a_re, const float *a_im,
                       const float *b_re, const float *b_im,
                       const int32_t *delay, const float *x,
                       int64_t n_samples, double scale, const int32_t *tsel,
                       int32_t n_sel, double *z, int32_t n_threads, int64_t start);

int spiir_oracle_single(int32_t n_templates, const int64_t *tmpl_ptr,
                        const float *a_re, const float *a_im,
                        const float *b_re, const float *b_im,
                        const int32_t *delay, const float *x,
                        int64_t n_samples, double scale, const int32_t *tsel,
                        int32_t n_sel, double *z, int32_t n_threads) {
    return single_from(n_templates, tmpl_ptr, a_re, a_im, b_re, b_im, delay, x, n_samples,
                       scale, tsel, n_sel, z, n_threads, 0);
}

/* As spiir_oracle_single, for filters whose state is zero before sample
 * `start` (z[n] = 0 there) and which run from `start` on with their delayed
 * inputs x[n - d_k] taken from the whole series x. */
int spiir_oracle_single_from(int32_t n_templates, const int64_t *tmpl_ptr,
                             const float *a_re, const float *a_im,
                             const float *b_re, const float *b_im,
                             const int32_t *delay, const float *x,
                             int64_t n_samples, double scale, const int32_t *tsel,
                             int32_t n_sel, double *z, int32_t n_threads, int64_t start) {
    if (start < 0 || start > n_samples) return 1;
    return single_from(n_templates, tmpl_ptr, a_re, a_im, b_re, b_im, delay, x, n_samples,
                       scale, tsel, n_sel, z, n_threads, start);
}

static int single_from(int32_t n_templates, const int64_t *tmpl_ptr,
                       const float *a_re, const float *a_im,
                       const float *b_re, const float *b_im,
                       const int32_t *delay, const float *x,
                       int64_t n_samples, double scale, const int32_t *tsel,
                       int32_t n_sel, double *z, int32_t n_threads, int64_t start) {
    if (n_samples < 0 || n_templates < 0 || !tmpl_ptr || !z) return 1;
    if (!tsel) n_sel = n_templates;
    double *xd = (double *)malloc(sizeof(double) * (size_t)(n_samples + 1));
    if (!xd) return 2;
    for (int64_t n = 0; n < n_samples; ++n) xd[n] = (double)x[n];
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t j = 0; j < n_sel; ++j) {
        int32_t t = tsel ? tsel[j] : j;
        if (t < 0 || t >= n_templates) { bad = 1; continue; }
        double *acc = z + (size_t)j * 2 * (size_t)n_samples;
        memset(acc, 0, sizeof(double) * 2 * (size_t)n_samples);
        for (int64_t k = tmpl_ptr[t]; k < tmpl_ptr[t + 1]; ++k)
            filter_into(a_re[k], a_im[k], b_re[k], b_im[k], delay[k], xd,
                        n_samples, acc, start);
        for (int64_t n = 0; n < 2 * n_samples; ++n) acc[n] *= scale;
    }
    free(xd);
    return bad ? 1 : 0;
}

/* ------------------------------------------------------------------ */
/* Resampling (Sec. 2.2, Eq. kaiser_window_filtering)                   */
/* ------------------------------------------------------------------ */

/* Causal T-tap low-pass then keep every second sample:
 *   out[m] = sum_{j=0}^{T-1} h[j] * x[2m - j],  x[<0] = 0,  m < n/2. */
int spiir_oracle_decimate(const double *x, int64_t n, const float *h,
                          int32_t n_taps, double *out) {
    for (int64_t m = 0; m < n / 2; ++m) {
        double acc = 0.0;
        for (int32_t j = 0; j < n_taps; ++j) {
            int64_t p = 2 * m - j;
            if (p >= 0) acc += (double)h[j] * x[p];
        }
        out[m] = acc;
    }
    return 0;
}

/* Zero-stuff the complex series u (length n_low) to twice the rate, filter
 * with 2*h (gain 2 restores the amplitude halved by the zeros), add to acc:
 *   acc[n] += 2 * sum_{j=0}^{T-1} h[j] * zs[n - j],
 *   zs[2m] = u[m], zs[2m+1] = 0, zs[<0] = 0,  n < 2 * n_low. */
int spiir_oracle_upsample_add(const double *u, int64_t n_low, const float *h,
                              int32_t n_taps, double *acc) {
    for (int64_t n = 0; n < 2 * n_low; ++n) {
        double s_re = 0.0, s_im = 0.0;
        for (int32_t j = 0; j < n_taps; ++j) {
            int64_t p = n - j;
            if (p < 0 || (p & 1)) continue;
            s_re += 2.0 * (double)h[j] * u[2 * (p / 2)];
            s_im += 2.0 * (double)h[j] * u[2 * (p / 2) + 1];
        }
        acc[2 * n] += s_re;
        acc[2 * n + 1] += s_im;
    }
    return 0;
}

/* Alignment delay of level i's sum, in level-i samples (reading above), for
 * a decimator of n_taps_down and an interpolator of n_taps_up taps. */
int64_t spiir_oracle_align_delay(int32_t level, int32_t n_levels,
                                 int32_t n_taps_down, int32_t n_taps_up,
                                 int32_t align) {
    if (!align) return 0;
    const int64_t R = (n_taps_down + n_taps_up) / 2 - 1; /* round trip */
    int64_t D = 0; /* D_H = 0 */
    for (int32_t i = n_levels - 2; i >= level; --i) D = R + 2 * D;
    return D;
}

/* ------------------------------------------------------------------ */
/* Multi-rate SPIIR (Sec. 2.2, Fig. 1)                                  */
/* ------------------------------------------------------------------ */

/* level[k] in [0, n_levels): the filter runs at base_rate / 2^level[k] on the
 * strain decimated level[k] times; its delay counts samples at that rate.
 * n_samples must be a multiple of 2^(n_levels-1). For each selected template:
 *   s_i[n]  = sum over the template's level-i filters of y_k[n]
 *   u_H     = s_H
 *   u_i[n]  = s_i[n - D_i] + 2 sum_j h_up[j] zs_i[n - j],  zs_i = u_{i+1}
 *             zero-stuffed
 *   z[n]    = scale * u_0[n]. */
int spiir_oracle_multirate(int32_t n_templates, const int64_t *tmpl_ptr,
                           const float *a_re, const float *a_im,
                           const float *b_re, const float *b_im,
                           const int32_t *delay, const int8_t *level,
                           int32_t n_levels, const float *h_down,
                           const float *h_up, int32_t n_taps_down,
                           int32_t n_taps_up, int32_t align,
                           const float *x, int64_t n_samples, double scale,
                           const int32_t *tsel, int32_t n_sel, double *z,
                           int32_t n_threads) {
    if (n_levels < 1 || n_levels > 16 || !tmpl_ptr || !z) return 1;
    if ((n_taps_down + n_taps_up) % 2 != 0) return 1;
    int64_t H = n_levels - 1;
    if (n_samples % ((int64_t)1 << H) != 0) return 1;
    if (!tsel) n_sel = n_templates;

    /* Strain at every rate, decimating in succession. */
    double **xl = (double **)calloc((size_t)n_levels, sizeof(double *));
    if (!xl) return 2;
    for (int32_t i = 0; i < n_levels; ++i) {
        xl[i] = (double *)malloc(sizeof(double) * (size_t)((n_samples >> i) + 1));
        if (!xl[i]) return 2;
    }
    for (int64_t n = 0; n < n_samples; ++n) xl[0][n] = (double)x[n];
    for (int32_t i = 1; i < n_levels; ++i)
        spiir_oracle_decimate(xl[i - 1], n_samples >> (i - 1), h_down,
                              n_taps_down, xl[i]);

    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int32_t j = 0; j < n_sel; ++j) {
        int32_t t = tsel ? tsel[j] : j;
        if (t < 0 || t >= n_templates) { bad = 1; continue; }
        double *u_low = NULL; /* u_{i+1}, complex interleaved */
        for (int32_t i = n_levels - 1; i >= 0; --i) {
            int64_t Ni = n_samples >> i;
            double *s = (double *)calloc((size_t)(2 * Ni), sizeof(double));
            double *u = (double *)calloc((size_t)(2 * Ni), sizeof(double));
            for (int64_t k = tmpl_ptr[t]; k < tmpl_ptr[t + 1]; ++k)
                if (level[k] == i)
                    filter_into(a_re[k], a_im[k], b_re[k], b_im[k], delay[k],
                                xl[i], Ni, s, 0);
            int64_t D = spiir_oracle_align_delay(i, n_levels, n_taps_down,
                                                 n_taps_up, align);
            for (int64_t n = 0; n < Ni; ++n) {
                if (n - D >= 0) {
                    u[2 * n] = s[2 * (n - D)];
                    u[2 * n + 1] = s[2 * (n - D) + 1];
                }
            }
            if (u_low) {
                spiir_oracle_upsample_add(u_low, Ni / 2, h_up, n_taps_up, u);
                free(u_low);
            }
            free(s);
            u_low = u;
        }
        double *out = z + (size_t)j * 2 * (size_t)n_samples;
        for (int64_t n = 0; n < 2 * n_samples; ++n) out[n] = scale * u_low[n];
        free(u_low);
    }
    for (int32_t i = 0; i < n_levels; ++i) free(xl[i]);
    free(xl);
    return bad ? 1 : 0;
}
