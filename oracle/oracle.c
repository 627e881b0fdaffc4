/*
 * FP64 CPU oracle for the segmented discrete Fourier transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * reads this file.  It is used by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py.  It shares no code, table or header with the
 * CUDA path.
 *
 * What it computes (Sec. III of the paper: a file is split into
 * <offset, FFT segment> records, each segment is transformed on its own, and
 * the outputs are concatenated in positional order; Sec. I: the transform is
 * the Cooley-Tukey FFT, which yields exactly the DFT):
 *
 *   for every segment s, with x_s[j] = signal[s*n + j], j = 0..n-1,
 *       X_s[k] = scale * sum_j x_s[j] * exp(sigma * 2*pi*i * j*k / n)
 *   sigma = -1 (forward) or +1 (inverse);
 *   scale = 1 (NONE), 1/n on the inverse only (BACKWARD), 1/sqrt(n) (ORTHO).
 *
 * Algorithm: plain recursive radix-2 decimation in time, in double precision.
 *   1. widen the single-precision input to double;
 *   2. a length-1 transform is the identity;
 *   3. transform the even-indexed and the odd-indexed samples (length n/2);
 *   4. combine: X[k] = E[k] + w^k O[k],  X[k+n/2] = E[k] - w^k O[k],
 *      w^k = cos(2*pi*k/n) + i*sigma*sin(2*pi*k/n), each twiddle evaluated
 *      directly by libm (no recurrence, no table);
 *   5. scale.
 * Segments are independent; they are spread over POSIX threads.
 *
 * Lengths that are not powers of two: oracle_dft_c64 (end of file) is the
 * definition itself, a direct sum over a table of the n roots of unity.
 *
 * Parity: pinned by the tests against a brute-force O(n^2) DFT, the impulse
 * and pure-tone closed forms, Parseval, linearity, the shift theorem,
 * conjugate symmetry and the inverse round trip (tests/test_oracle.py).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_INVALID (-1)
#define ORACLE_E_NOMEM (-2)

#define ORACLE_NORM_NONE 0
#define ORACLE_NORM_BACKWARD 1
#define ORACLE_NORM_ORTHO 2

static const double kTwoPi = 6.283185307179586476925286766559;

/*
 * One length-n transform.  x: complex128 interleaved, element j at
 * x[2*stride*j], x[2*stride*j+1].  X: contiguous complex128 output.
 */
static void fft_rec(const double *x, int64_t stride, double *X, int64_t n, int sigma)
{
    if (n == 1) {
        X[0] = x[0];
        X[1] = x[1];
        return;
    }
    const int64_t h = n / 2;
    fft_rec(x, 2 * stride, X, h, sigma);                  /* E: even samples -> X[0, h) */
    fft_rec(x + 2 * stride, 2 * stride, X + 2 * h, h, sigma); /* O: odd samples -> X[h, n) */
    for (int64_t k = 0; k < h; ++k) {
        const double a = kTwoPi * (double)k / (double)n;
        const double wr = cos(a);
        const double wi = (double)sigma * sin(a);
        const double er = X[2 * k], ei = X[2 * k + 1];
        const double orr = X[2 * (k + h)], oi = X[2 * (k + h) + 1];
        const double tr = wr * orr - wi * oi;
        const double ti = wr * oi + wi * orr;
        X[2 * k] = er + tr;
        X[2 * k + 1] = ei + ti;
        X[2 * (k + h)] = er - tr;
        X[2 * (k + h) + 1] = ei - ti;
    }
}

static double norm_scale(int64_t n, int sigma, int norm)
{
    if (norm == ORACLE_NORM_BACKWARD)
        return sigma > 0 ? 1.0 / (double)n : 1.0;
    if (norm == ORACLE_NORM_ORTHO)
        return 1.0 / sqrt((double)n);
    return 1.0;
}

static int is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

typedef struct {
    const float *in32;   /* exactly one of in32 / in64 is set */
    const double *in64;
    double *out;
    int64_t n;
    int64_t seg_begin, seg_end;
    int sigma;
    double scale;
    int status;
} job_t;

static void *run_job(void *arg)
{
    job_t *jb = (job_t *)arg;
    const int64_t n = jb->n;
    double *wide = NULL;
    if (jb->in32) {
        wide = (double *)malloc(sizeof(double) * 2 * (size_t)n);
        if (!wide) {
            jb->status = ORACLE_E_NOMEM;
            return NULL;
        }
    }
    for (int64_t s = jb->seg_begin; s < jb->seg_end; ++s) {
        const double *x;
        if (jb->in32) {
            const float *src = jb->in32 + 2 * s * n;
            for (int64_t j = 0; j < 2 * n; ++j) wide[j] = (double)src[j]; /* step 1 */
            x = wide;
        } else {
            x = jb->in64 + 2 * s * n;
        }
        double *X = jb->out + 2 * s * n;
        fft_rec(x, 1, X, n, jb->sigma);
        if (jb->scale != 1.0)
            for (int64_t j = 0; j < 2 * n; ++j) X[j] *= jb->scale;
    }
    free(wide);
    jb->status = ORACLE_OK;
    return NULL;
}

static int run(const float *in32, const double *in64, double *out, int64_t n, int64_t nseg,
               int sigma, int norm, int nthreads)
{
    if (!out || (!in32 && !in64) || !is_pow2(n) || nseg < 0 || (sigma != -1 && sigma != 1) ||
        norm < 0 || norm > 2)
        return ORACLE_E_INVALID;
    if (nseg == 0) return ORACLE_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nseg) nthreads = (int)nseg;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        return ORACLE_E_NOMEM;
    }
    const double scale = norm_scale(n, sigma, norm);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].in32 = in32;
        jobs[t].in64 = in64;
        jobs[t].out = out;
        jobs[t].n = n;
        jobs[t].seg_begin = nseg * t / nthreads;
        jobs[t].seg_end = nseg * (t + 1) / nthreads;
        jobs[t].sigma = sigma;
        jobs[t].scale = scale;
        jobs[t].status = ORACLE_E_INVALID;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tid[t], NULL, run_job, &jobs[t]) != 0) break;
        started = t;
    }
    run_job(&jobs[0]);
    /* any job whose thread could not be created runs here, serially */
    for (int t = started + 1; t < nthreads; ++t) run_job(&jobs[t]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    int status = ORACLE_OK;
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].status != ORACLE_OK) status = jobs[t].status;
    free(jobs);
    free(tid);
    return status;
}

/* complex64 input (interleaved float re, im), complex128 output. */
int oracle_fft_c64(const float *in, double *out, int64_t n, int64_t nseg, int sigma, int norm,
                   int nthreads)
{
    return run(in, NULL, out, n, nseg, sigma, norm, nthreads);
}

/* complex128 input, complex128 output (used to pin the oracle with exact inputs). */
int oracle_fft_c128(const double *in, double *out, int64_t n, int64_t nseg, int sigma, int norm,
                    int nthreads)
{
    return run(NULL, in, out, n, nseg, sigma, norm, nthreads);
}

/*
 * Direct DFT of any length n >= 1, the definition written out:
 *   X_s[k] = scale * sum_j x_s[j] * r[(j*k) mod n],  r[m] = exp(sigma*2*pi*i*m/n),
 * the exponent index reduced exactly in integers, the n roots r[m] evaluated
 * by libm once per call.  Only the bins listed in `bins` (nbins of them, each
 * in [0, n)) are computed, or all n when bins is NULL.  Complex64 input,
 * complex128 output [nseg][nbins].  It serves lengths that are not powers of
 * two, where the radix-2 recursion above does not apply, and spot checks of
 * single bins at large n.
 */
typedef struct {
    const float *in;
    double *out;
    const double *roots; /* [n][2] */
    const int64_t *bins; /* NULL: every bin */
    int64_t n, nb;
    int64_t seg_begin, seg_end;
    double scale;
} djob_t;

static void *run_djob(void *arg)
{
    djob_t *jb = (djob_t *)arg;
    const int64_t n = jb->n;
    for (int64_t s = jb->seg_begin; s < jb->seg_end; ++s) {
        const float *x = jb->in + 2 * s * n;
        double *X = jb->out + 2 * s * jb->nb;
        for (int64_t b = 0; b < jb->nb; ++b) {
            const int64_t k = jb->bins ? jb->bins[b] : b;
            double re = 0.0, im = 0.0;
            int64_t m = 0; /* (j*k) mod n, advanced by k each step */
            for (int64_t j = 0; j < n; ++j) {
                const double xr = (double)x[2 * j], xi = (double)x[2 * j + 1];
                const double wr = jb->roots[2 * m], wi = jb->roots[2 * m + 1];
                re += xr * wr - xi * wi;
                im += xr * wi + xi * wr;
                m += k;
                if (m >= n) m -= n;
            }
            X[2 * b] = re * jb->scale;
            X[2 * b + 1] = im * jb->scale;
        }
    }
    return NULL;
}

int oracle_dft_c64(const float *in, double *out, int64_t n, int64_t nseg, int sigma, int norm,
                   const int64_t *bins, int64_t nbins, int nthreads)
{
    if (!in || !out || n < 1 || nseg < 0 || (sigma != -1 && sigma != 1) || norm < 0 || norm > 2)
        return ORACLE_E_INVALID;
    if (bins)
        for (int64_t b = 0; b < nbins; ++b)
            if (bins[b] < 0 || bins[b] >= n) return ORACLE_E_INVALID;
    if (nseg == 0) return ORACLE_OK;
    double *roots = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!roots) return ORACLE_E_NOMEM;
    for (int64_t m = 0; m < n; ++m) {
        const double a = kTwoPi * ((double)m / (double)n);
        roots[2 * m] = cos(a);
        roots[2 * m + 1] = (double)sigma * sin(a);
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nseg) nthreads = (int)nseg;
    djob_t *jobs = (djob_t *)calloc((size_t)nthreads, sizeof(djob_t));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !tid) {
        free(jobs);
        free(tid);
        free(roots);
        return ORACLE_E_NOMEM;
    }
    const double scale = norm_scale(n, sigma, norm);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].in = in;
        jobs[t].out = out;
        jobs[t].roots = roots;
        jobs[t].bins = bins;
        jobs[t].n = n;
        jobs[t].nb = bins ? nbins : n;
        jobs[t].seg_begin = nseg * t / nthreads;
        jobs[t].seg_end = nseg * (t + 1) / nthreads;
        jobs[t].scale = scale;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&tid[t], NULL, run_djob, &jobs[t]) != 0) break;
        started = t;
    }
    run_djob(&jobs[0]);
    for (int t = started + 1; t < nthreads; ++t) run_djob(&jobs[t]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    free(jobs);
    free(tid);
    free(roots);
    return ORACLE_OK;
}
