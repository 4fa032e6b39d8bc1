/*
 * oracle.c -- FP64 CPU reference for the discrete Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product (GPU) path may include,
 * link or call this file; it shares no code, header, table or constant with
 * the CUDA library.  Only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark load it.
 *
 * What is computed (paper Sec. III-A, "Discrete Fourier Transform Example"):
 * the DFT of a length-N complex sequence,
 *
 *     X[k] = sum_{n<N} x[n] * exp(sign * 2*pi*i * n*k / N),   sign = -1 forward,
 *                                                              sign = +1 inverse,
 *
 * unnormalised in both directions.  The paper evaluates it with the
 * Cooley-Tukey algorithm: a DFT of N = N1*N2 points is rebuilt from DFTs of
 * sizes N1 and N2; in the radix-2 form each step splits the sequence into two
 * interleaved half-length DFTs (even and odd samples).  The functions here are:
 *
 *   oracle_dft_naive   O(N^2) straight from the definition (any N).
 *   oracle_dft_bins    selected output bins, O(N) each, from the definition.
 *   oracle_fft_radix2  radix-2 decimation-in-time Cooley-Tukey (N a power of 2).
 *   oracle_fft_split_m N = m * 2^j, m in {3,5,7}: one Cooley-Tukey step with
 *                      N1 = m interleaved sub-sequences of length 2^j, each
 *                      transformed by the radix-2 routine.
 *   oracle_fft         dispatch among the three by the factorisation of N.
 *   oracle_fft_batch   oracle_fft over a batch, threads over the batch.
 *   oracle_fft2d       2-D DFT as 1-D DFTs of every row, then of every column.
 *
 * Complex data are interleaved double pairs (re, im).  Twiddle factors are
 * evaluated directly from their integer index with libm cos/sin in FP64 and
 * never by a recurrence, so their rounding is independent of the sequence
 * length walked so far.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* exp(sign * 2*pi*i * m / n) for an integer index m, reduced mod n first. */
static void unit_root(int64_t m, int64_t n, int sign, double *re, double *im)
{
    m %= n;
    if (m < 0) m += n;
    double a = 2.0 * M_PI * (double)m / (double)n;
    *re = cos(a);
    *im = (double)sign * sin(a);
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* ------------------------------------------------------------------------ */
/* Definition, evaluated term by term: X[k] = sum_n x[n] W^(n*k mod N).      */
/* ------------------------------------------------------------------------ */
int oracle_dft_naive(const double *x, double *y, int64_t n, int sign)
{
    if (n <= 0) return -1;
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!w) return -2;
    for (int64_t m = 0; m < n; ++m) unit_root(m, n, sign, &w[2 * m], &w[2 * m + 1]);
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t m = (int64_t)(((__int128)j * k) % n);
            double xr = x[2 * j], xi = x[2 * j + 1];
            double wr = w[2 * m], wi = w[2 * m + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        y[2 * k] = sr;
        y[2 * k + 1] = si;
    }
    free(w);
    return 0;
}

/* Selected bins of the definition; each twiddle is evaluated from its own
 * exact index (n*k mod N), so any single bin of any N can be checked. */
int oracle_dft_bins(const double *x, int64_t n, int sign, const int64_t *ks,
                    int64_t nk, double *out)
{
    if (n <= 0) return -1;
    for (int64_t t = 0; t < nk; ++t) {
        int64_t k = ks[t] % n;
        if (k < 0) k += n;
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double wr, wi;
            unit_root((int64_t)(((__int128)j * k) % n), n, sign, &wr, &wi);
            double xr = x[2 * j], xi = x[2 * j + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        out[2 * t] = sr;
        out[2 * t + 1] = si;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Radix-2 Cooley-Tukey, decimation in time: reorder the input by bit        */
/* reversal, then at every level merge pairs of half-length DFTs (the even   */
/* and odd interleaved sub-sequences) with the butterfly                     */
/*     X[j] = E[j] + W_len^j O[j],  X[j + len/2] = E[j] - W_len^j O[j].      */
/* ------------------------------------------------------------------------ */
int oracle_fft_radix2(const double *x, double *y, int64_t n, int sign)
{
    if (!is_pow2(n)) return -1;
    int lg = 0;
    while (((int64_t)1 << lg) < n) ++lg;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = 0;
        for (int b = 0; b < lg; ++b)
            if (i & ((int64_t)1 << b)) r |= (int64_t)1 << (lg - 1 - b);
        y[2 * r] = x[2 * i];
        y[2 * r + 1] = x[2 * i + 1];
    }
    if (n == 1) return 0;
    /* W_n^m for m < n/2, each from its own index. W_len^j = W_n^(j*n/len). */
    int64_t h = n / 2;
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)h);
    if (!w) return -2;
    for (int64_t m = 0; m < h; ++m) unit_root(m, n, sign, &w[2 * m], &w[2 * m + 1]);
    for (int64_t len = 2; len <= n; len *= 2) {
        int64_t half = len / 2, step = n / len;
        for (int64_t base = 0; base < n; base += len) {
            for (int64_t j = 0; j < half; ++j) {
                double wr = w[2 * (j * step)], wi = w[2 * (j * step) + 1];
                double *e = &y[2 * (base + j)], *o = &y[2 * (base + j + half)];
                double tr = o[0] * wr - o[1] * wi;
                double ti = o[0] * wi + o[1] * wr;
                o[0] = e[0] - tr;
                o[1] = e[1] - ti;
                e[0] = e[0] + tr;
                e[1] = e[1] + ti;
            }
        }
    }
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One Cooley-Tukey step with N1 = m, N2 = 2^j (N = N1*N2): the m interleaved */
/* sub-sequences x[r], x[r+m], x[r+2m], ... are transformed by radix 2 and   */
/* combined as X[k] = sum_{r<m} W_N^(r*k) F_r[k mod N2].                      */
/* ------------------------------------------------------------------------ */
int oracle_fft_split_m(const double *x, double *y, int64_t n, int64_t m, int sign)
{
    if (m <= 0 || n % m != 0 || !is_pow2(n / m)) return -1;
    int64_t n2 = n / m;
    double *sub = (double *)malloc(sizeof(double) * 2 * (size_t)n2);
    double *f = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!sub || !f) { free(sub); free(f); return -2; }
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t t = 0; t < n2; ++t) {
            sub[2 * t] = x[2 * (t * m + r)];
            sub[2 * t + 1] = x[2 * (t * m + r) + 1];
        }
        oracle_fft_radix2(sub, &f[2 * r * n2], n2, sign);
    }
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t r = 0; r < m; ++r) {
            double wr, wi;
            unit_root((int64_t)(((__int128)r * k) % n), n, sign, &wr, &wi);
            const double *fr = &f[2 * (r * n2 + (k % n2))];
            sr += fr[0] * wr - fr[1] * wi;
            si += fr[0] * wi + fr[1] * wr;
        }
        y[2 * k] = sr;
        y[2 * k + 1] = si;
    }
    free(sub);
    free(f);
    return 0;
}

/* Odd part m of n if m is 3, 5 or 7 and n/m a power of two; else 0. */
static int64_t small_odd_factor(int64_t n)
{
    int64_t m = n;
    while (m > 1 && (m % 2) == 0) m /= 2;
    return (m == 3 || m == 5 || m == 7) ? m : 0;
}

int oracle_fft(const double *x, double *y, int64_t n, int sign)
{
    if (n <= 0) return -1;
    if (is_pow2(n)) return oracle_fft_radix2(x, y, n, sign);
    int64_t m = small_odd_factor(n);
    if (m) return oracle_fft_split_m(x, y, n, m, sign);
    return oracle_dft_naive(x, y, n, sign);
}

/* ------------------------------------------------------------------------ */
/* Batch: independent transforms, one thread handles a contiguous share.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *x;
    double *y;
    int64_t n, b0, b1;
    int sign, rc;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    j->rc = 0;
    for (int64_t b = j->b0; b < j->b1 && j->rc == 0; ++b)
        j->rc = oracle_fft(j->x + 2 * b * j->n, j->y + 2 * b * j->n, j->n, j->sign);
    return NULL;
}

int oracle_num_cpus(void)
{
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

int oracle_fft_batch(const double *x, double *y, int64_t n, int64_t batch, int sign,
                     int nthreads)
{
    if (n <= 0 || batch < 0) return -1;
    if (nthreads <= 0) nthreads = oracle_num_cpus();
    if (nthreads > batch) nthreads = (int)(batch > 0 ? batch : 1);
    batch_job *jobs = (batch_job *)calloc((size_t)nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].x = x; jobs[t].y = y; jobs[t].n = n; jobs[t].sign = sign;
        jobs[t].b0 = batch * t / nthreads;
        jobs[t].b1 = batch * (t + 1) / nthreads;
    }
    int rc = 0;
    if (nthreads == 1) {
        batch_worker(&jobs[0]);
        rc = jobs[0].rc;
    } else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) {
            pthread_join(th[t], NULL);
            if (jobs[t].rc) rc = jobs[t].rc;
        }
    }
    free(jobs);
    free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 2-D DFT over [batch][h][w]: X[k1,k2] = sum x[n1,n2] W_h^(n1 k1) W_w^(n2 k2) */
/* is separable, so take the 1-D DFT of every row, then of every column.     */
/* ------------------------------------------------------------------------ */
int oracle_fft2d(const double *x, double *y, int64_t h, int64_t w, int64_t batch,
                 int sign, int nthreads)
{
    if (h <= 0 || w <= 0 || batch < 0) return -1;
    int rc = oracle_fft_batch(x, y, w, batch * h, sign, nthreads);
    if (rc) return rc;
    /* columns: gather into contiguous rows, transform, scatter back */
    double *col = (double *)malloc(sizeof(double) * 2 * (size_t)(h * w));
    double *fc = (double *)malloc(sizeof(double) * 2 * (size_t)(h * w));
    if (!col || !fc) { free(col); free(fc); return -2; }
    for (int64_t b = 0; b < batch && rc == 0; ++b) {
        double *img = y + 2 * b * h * w;
        for (int64_t c = 0; c < w; ++c)
            for (int64_t r = 0; r < h; ++r) {
                col[2 * (c * h + r)] = img[2 * (r * w + c)];
                col[2 * (c * h + r) + 1] = img[2 * (r * w + c) + 1];
            }
        rc = oracle_fft_batch(col, fc, h, w, sign, nthreads);
        for (int64_t c = 0; c < w; ++c)
            for (int64_t r = 0; r < h; ++r) {
                img[2 * (r * w + c)] = fc[2 * (c * h + r)];
                img[2 * (r * w + c) + 1] = fc[2 * (c * h + r) + 1];
            }
    }
    free(col);
    free(fc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Circular convolution and correlation by their definitions (the paper's   */
/* Sec. III-A names convolution among the uses of the DFT):                  */
/*   corr = 0:  y[m] = sum_j x[j] h[(m - j) mod N]                           */
/*   corr = 1:  y[m] = sum_j x[(j + m) mod N] conj(h[j])                     */
/* ------------------------------------------------------------------------ */
int oracle_circ_conv(const double *x, const double *h, double *y, int64_t n, int corr)
{
    if (n <= 0) return -1;
    for (int64_t m = 0; m < n; ++m) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double xr, xi, hr, hi;
            if (!corr) {
                int64_t q = ((m - j) % n + n) % n;
                xr = x[2 * j]; xi = x[2 * j + 1];
                hr = h[2 * q]; hi = h[2 * q + 1];
            } else {
                int64_t q = (j + m) % n;
                xr = x[2 * q]; xi = x[2 * q + 1];
                hr = h[2 * j]; hi = -h[2 * j + 1];
            }
            sr += xr * hr - xi * hi;
            si += xr * hi + xi * hr;
        }
        y[2 * m] = sr;
        y[2 * m + 1] = si;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Image example, Sec. III-B, GPU steps 1-3 (the paper names the steps but   */
/* not their formulas; readings):                                           */
/*  1. chroma + luminance: JFIF (ITU-R BT.601 full range) YCbCr of 8-bit    */
/*     RGB,  Y = .299 R + .587 G + .114 B,                                  */
/*     Cb = 128 - .168736 R - .331264 G + .5 B,                              */
/*     Cr = 128 + .5 R - .418688 G - .081312 B;                              */
/*  2. chroma downscaled to 1/4 of the pixels: mean of each 2x2 block;      */
/*  3. directional derivative of Y along the unit vector (ux, uy):          */
/*     ux dY/dx + uy dY/dy, central differences inside the image and        */
/*     one-sided first differences on its border.                           */
/* rgb: batch x h x w x 3 bytes; y, d: batch x h x w; cb, cr: batch x       */
/* (h/2) x (w/2).  h, w even and >= 2.                                      */
/* ------------------------------------------------------------------------ */
static double deriv_1d(const double *v, int64_t i, int64_t n, int64_t stride)
{
    if (i == 0) return v[stride] - v[0];
    if (i == n - 1) return v[(n - 1) * stride] - v[(n - 2) * stride];
    return 0.5 * (v[(i + 1) * stride] - v[(i - 1) * stride]);
}

int oracle_image_steps(const unsigned char *rgb, int64_t batch, int64_t h, int64_t w, double ux, double uy,
                       double *y, double *cb, double *cr, double *d)
{
    if (batch < 0 || h < 2 || w < 2 || (h & 1) || (w & 1)) return -1;
    const int64_t hw = h * w, q = (h / 2) * (w / 2);
    for (int64_t b = 0; b < batch; ++b) {
        const unsigned char *img = rgb + b * hw * 3;
        double *yb = y + b * hw, *db = d + b * hw, *cbb = cb + b * q, *crb = cr + b * q;
        for (int64_t i = 0; i < q; ++i) cbb[i] = crb[i] = 0.0;
        for (int64_t r = 0; r < h; ++r)
            for (int64_t c = 0; c < w; ++c) {
                const double R = img[3 * (r * w + c)], G = img[3 * (r * w + c) + 1], B = img[3 * (r * w + c) + 2];
                yb[r * w + c] = 0.299 * R + 0.587 * G + 0.114 * B;
                const int64_t k = (r / 2) * (w / 2) + c / 2;
                cbb[k] += 0.25 * (128.0 - 0.168736 * R - 0.331264 * G + 0.5 * B);
                crb[k] += 0.25 * (128.0 + 0.5 * R - 0.418688 * G - 0.081312 * B);
            }
        for (int64_t r = 0; r < h; ++r)
            for (int64_t c = 0; c < w; ++c)
                db[r * w + c] = ux * deriv_1d(yb + r * w, c, w, 1) + uy * deriv_1d(yb + c, r, h, w);
    }
    return 0;
}
