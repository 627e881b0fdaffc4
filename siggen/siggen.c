/*
 * Seeded synthetic signals, readers and writers for tests and benchmarks.
 *
 * This file holds none of the transform's arithmetic.  It is the one module
 * that both the CUDA path's tests/benchmarks and the CPU oracle take their
 * inputs from: every sample is a pure function of (seed, global sample index
 * t), so any segment can be regenerated from its byte offset (8 bytes per
 * complex64 sample), as the paper's <offset, FFT segment> records require
 * (Sec. III).
 *
 * Counter-based generator: SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used as a hash of
 * a per-stream key plus the counter:  h(key, c) = mix64(key + (c+1)*GAMMA).
 *
 * Families:
 *  uniform  re, im i.i.d. uniform on [-1, 1): u = (h >> 40) * 2^-23 - 1, a
 *           24-bit grid value that float32 holds exactly.
 *  tones    sum of `ntones` complex exponentials a_k exp(2 pi i theta_k(t))
 *           plus complex Gaussian noise (sigma per component):
 *             F_k   = h(kT, 3k)          frequency, cycles/sample * 2^64
 *             a_k   = 10^(-3 u)          log-uniform on [1e-3, 1]
 *             Phi_k = h(kT, 3k+2)        initial phase * 2^64
 *             theta_k(t) = (F_k t + Phi_k) mod 2^64   (exact integer phase)
 *           In each aligned block of 64 samples starting at tb, sample
 *           tb + m takes the product of two exact phasors, both evaluated by
 *           cos and sin in double: that of the block's first sample,
 *           (F_k tb + Phi_k) mod 2^64, and that of the offset, (F_k m) mod
 *           2^64 (a table of 64 per tone).  The tones are thus independent
 *           lanes over the block's samples, with no recurrence.
 *           Noise: Box-Muller in double from two uniform counters.
 *           The double sum (noise, then the tones in order) is rounded once
 *           to float32.
 *  pool     a pre-generated host buffer read cyclically (offset mod its
 *           size), copied by several threads: a host-resident source that
 *           leaves the generator out of a streaming measurement.
 *
 * Built with floating-point contraction off so that both host architectures
 * evaluate the same expression tree.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ULL
#define BLOCK 64

static const double kTwoPi = 6.283185307179586476925286766559;

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(mix64(seed) + stream * GAMMA);
}

static inline uint64_t h(uint64_t key, uint64_t c) { return mix64(key + (c + 1) * GAMMA); }

/* [0, 1) with 53 random bits */
static inline double u01(uint64_t v) { return (double)(v >> 11) * 0x1.0p-53; }

enum { STREAM_UNIFORM = 0, STREAM_TONES = 1, STREAM_NOISE_A = 2, STREAM_NOISE_B = 3 };

/* ------------------------------------------------------------------ uniform */

static void uniform_range(uint64_t seed, int64_t t0, int64_t count, float *out)
{
    const uint64_t key = stream_key(seed, STREAM_UNIFORM);
    for (int64_t i = 0; i < count; ++i) {
        const uint64_t t = (uint64_t)(t0 + i);
        out[2 * i] = (float)((double)(h(key, 2 * t) >> 40) * 0x1.0p-23 - 1.0);
        out[2 * i + 1] = (float)((double)(h(key, 2 * t + 1) >> 40) * 0x1.0p-23 - 1.0);
    }
}

/* -------------------------------------------------------------------- tones */

#define MAX_TONES 256

typedef struct {
    int ntones;
    double sigma;
    uint64_t F[MAX_TONES], Phi[MAX_TONES];
    double a[MAX_TONES];
    double pr[MAX_TONES][BLOCK], pi[MAX_TONES][BLOCK]; /* exp(2 pi i ((F_k m) mod 2^64) 2^-64), m < BLOCK */
    uint64_t kA, kB;
} tones_t;

static void tones_init(tones_t *tp, uint64_t seed, int ntones, double sigma)
{
    const uint64_t kT = stream_key(seed, STREAM_TONES);
    tp->ntones = ntones;
    tp->sigma = sigma;
    for (int k = 0; k < ntones; ++k) {
        tp->F[k] = h(kT, 3 * (uint64_t)k);
        tp->a[k] = pow(10.0, -3.0 * u01(h(kT, 3 * (uint64_t)k + 1)));
        tp->Phi[k] = h(kT, 3 * (uint64_t)k + 2);
        for (int m = 0; m < BLOCK; ++m) {
            const double ang = kTwoPi * u01(tp->F[k] * (uint64_t)m); /* mod 2^64 */
            tp->pr[k][m] = cos(ang);
            tp->pi[k][m] = sin(ang);
        }
    }
    tp->kA = stream_key(seed, STREAM_NOISE_A);
    tp->kB = stream_key(seed, STREAM_NOISE_B);
}

/* all BLOCK samples of the aligned block starting at tb */
static void tones_block(const tones_t *tp, uint64_t tb, double *re, double *im)
{
    if (tp->sigma != 0.0) {
        for (int m = 0; m < BLOCK; ++m) {
            const uint64_t t = tb + (uint64_t)m;
            const double u1 = ((double)(h(tp->kA, t) >> 11) + 1.0) * 0x1.0p-53; /* (0, 1] */
            const double u2 = u01(h(tp->kB, t));
            const double r = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincos(kTwoPi * u2, &sn, &cs);
            re[m] = tp->sigma * r * cs;
            im[m] = tp->sigma * r * sn;
        }
    } else {
        for (int m = 0; m < BLOCK; ++m) re[m] = im[m] = 0.0;
    }
    for (int k = 0; k < tp->ntones; ++k) {
        const uint64_t theta = tp->F[k] * tb + tp->Phi[k]; /* mod 2^64 */
        double sn, cs;
        sincos(kTwoPi * u01(theta), &sn, &cs);
        const double zr = tp->a[k] * cs, zi = tp->a[k] * sn;
        const double *pr = tp->pr[k], *pi = tp->pi[k];
        for (int m = 0; m < BLOCK; ++m) {
            re[m] += zr * pr[m] - zi * pi[m];
            im[m] += zr * pi[m] + zi * pr[m];
        }
    }
}

static void tones_range(const tones_t *tp, int64_t t0, int64_t count, float *out)
{
    double re[BLOCK], im[BLOCK];
    int64_t t = t0;
    const int64_t tend = t0 + count;
    while (t < tend) {
        const int64_t tb = t - (t % BLOCK);
        tones_block(tp, (uint64_t)tb, re, im);
        int64_t stop = tb + BLOCK < tend ? tb + BLOCK : tend;
        for (; t < stop; ++t) {
            out[2 * (t - t0)] = (float)re[t - tb];
            out[2 * (t - t0) + 1] = (float)im[t - tb];
        }
    }
}

/* ------------------------------------------------------------- threading */

typedef struct {
    int kind; /* 0 uniform, 1 tones */
    uint64_t seed;
    const tones_t *tp;
    int64_t t0, count;
    float *out;
} work_t;

static void *work_run(void *arg)
{
    work_t *w = (work_t *)arg;
    if (w->kind == 0)
        uniform_range(w->seed, w->t0, w->count, w->out);
    else
        tones_range(w->tp, w->t0, w->count, w->out);
    return NULL;
}

static int run_parallel(int kind, uint64_t seed, const tones_t *tp, int64_t t0, int64_t count,
                        float *out, int nthreads)
{
    if (count <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    int64_t max_threads = count / 4096 + 1;
    if (nthreads > max_threads) nthreads = (int)max_threads;
    work_t w[256];
    pthread_t tid[256];
    if (nthreads > 256) nthreads = 256;
    for (int i = 0; i < nthreads; ++i) {
        /* split at multiples of BLOCK so no block is evaluated twice */
        int64_t b = count * i / nthreads, e = count * (i + 1) / nthreads;
        b -= (t0 + b) % BLOCK;
        if (b < 0) b = 0;
        if (i + 1 < nthreads) e -= (t0 + e) % BLOCK;
        if (i == 0) b = 0;
        w[i].kind = kind;
        w[i].seed = seed;
        w[i].tp = tp;
        w[i].t0 = t0 + b;
        w[i].count = e > b ? e - b : 0;
        w[i].out = out + 2 * b;
    }
    int started = 0;
    for (int i = 1; i < nthreads; ++i) {
        if (pthread_create(&tid[i], NULL, work_run, &w[i]) != 0) break;
        started = i;
    }
    work_run(&w[0]);
    for (int i = started + 1; i < nthreads; ++i) work_run(&w[i]);
    for (int i = 1; i <= started; ++i) pthread_join(tid[i], NULL);
    return 0;
}

/* ------------------------------------------------------------ public API */

int siggen_uniform_c64(uint64_t seed, int64_t t0, int64_t count, float *out, int nthreads)
{
    if (!out || t0 < 0 || count < 0) return -1;
    return run_parallel(0, seed, NULL, t0, count, out, nthreads);
}

int siggen_tones_c64(uint64_t seed, int64_t t0, int64_t count, float *out, int ntones,
                     double sigma, int nthreads)
{
    if (!out || t0 < 0 || count < 0 || ntones < 0 || ntones > MAX_TONES) return -1;
    tones_t *tp = (tones_t *)malloc(sizeof(tones_t));
    if (!tp) return -2;
    tones_init(tp, seed, ntones, sigma);
    int rc = run_parallel(1, seed, tp, t0, count, out, nthreads);
    free(tp);
    return rc;
}

/* Tone parameters, for tests that check the generator against its definition. */
int siggen_tone_params(uint64_t seed, int ntones, uint64_t *F, uint64_t *Phi, double *a)
{
    if (ntones < 0 || ntones > MAX_TONES) return -1;
    tones_t *tp = (tones_t *)malloc(sizeof(tones_t));
    if (!tp) return -2;
    tones_init(tp, seed, ntones, 0.0);
    for (int k = 0; k < ntones; ++k) {
        F[k] = tp->F[k];
        Phi[k] = tp->Phi[k];
        a[k] = tp->a[k];
    }
    free(tp);
    return 0;
}

/* ----------------------------------------------- reader / writer callbacks */

/*
 * Source description passed as the reader's context.  kind 0 = uniform,
 * 1 = tones.  The reader maps a byte offset into the complex64 signal to the
 * global sample index t = byte_offset / 8.  total_bytes bounds the signal.
 */
typedef struct {
    int32_t kind;
    int32_t ntones;
    uint64_t seed;
    double sigma;
    int64_t total_bytes;
    int32_t nthreads;
    int32_t fail_at_call; /* >= 0: return -1 on that call index (fault injection) */
    int64_t calls;        /* updated by the reader */
    const uint8_t *pool;  /* kind 2: the buffer read cyclically */
    int64_t pool_bytes;   /* a multiple of 8 */
} siggen_source;

typedef struct {
    uint8_t *dst;
    const uint8_t *pool;
    int64_t pool_bytes, off, bytes;
} pool_work_t;

static void *pool_copy(void *arg)
{
    pool_work_t *w = (pool_work_t *)arg;
    int64_t done = 0;
    while (done < w->bytes) {
        const int64_t o = (w->off + done) % w->pool_bytes;
        int64_t n = w->pool_bytes - o;
        if (n > w->bytes - done) n = w->bytes - done;
        memcpy(w->dst + done, w->pool + o, (size_t)n);
        done += n;
    }
    return NULL;
}

static void pool_read(const siggen_source *src, int64_t off, uint8_t *dst, int64_t bytes)
{
    int nt = src->nthreads < 1 ? 1 : src->nthreads > 64 ? 64 : src->nthreads;
    if (bytes < ((int64_t)nt << 22)) nt = (int)(bytes >> 22) + 1; /* at least 4 MiB a thread */
    pool_work_t w[64];
    pthread_t tid[64];
    int started = 0;
    for (int i = 0; i < nt; ++i) {
        int64_t b = bytes * i / nt, e = bytes * (i + 1) / nt;
        b -= b % 64;
        if (i + 1 < nt) e -= e % 64;
        w[i].dst = dst + b;
        w[i].pool = src->pool;
        w[i].pool_bytes = src->pool_bytes;
        w[i].off = off + b;
        w[i].bytes = e - b;
    }
    for (int i = 1; i < nt; ++i) {
        if (pthread_create(&tid[i], NULL, pool_copy, &w[i]) != 0) break;
        started = i;
    }
    pool_copy(&w[0]);
    for (int i = started + 1; i < nt; ++i) pool_copy(&w[i]);
    for (int i = 1; i <= started; ++i) pthread_join(tid[i], NULL);
}

int64_t siggen_read(void *ctx, int64_t byte_offset, void *dst, int64_t bytes)
{
    siggen_source *src = (siggen_source *)ctx;
    if (!src || !dst || byte_offset < 0 || bytes < 0 || (byte_offset % 8) != 0) return -1;
    const int64_t call = src->calls++;
    if (src->fail_at_call >= 0 && call == src->fail_at_call) return -1;
    if (byte_offset >= src->total_bytes) return 0;
    if (bytes > src->total_bytes - byte_offset) bytes = src->total_bytes - byte_offset;
    bytes -= bytes % 8;
    const int64_t t0 = byte_offset / 8, count = bytes / 8;
    int rc;
    if (src->kind == 2) {
        if (!src->pool || src->pool_bytes <= 0 || src->pool_bytes % 8) return -1;
        pool_read(src, byte_offset, (uint8_t *)dst, bytes);
        return bytes;
    }
    if (src->kind == 0)
        rc = siggen_uniform_c64(src->seed, t0, count, (float *)dst, src->nthreads);
    else
        rc = siggen_tones_c64(src->seed, t0, count, (float *)dst, src->ntones, src->sigma,
                              src->nthreads);
    return rc == 0 ? bytes : -1;
}

/*
 * Lending source for fftseg_stream_view (pool sources only): the address of
 * the pool's bytes for [byte_offset, byte_offset + bytes), bounded by
 * total_bytes (*got), or NULL if the range wraps past the pool's end (make the
 * pool a multiple of the chunk bytes) or on an injected failure.
 */
const void *siggen_view(void *ctx, int64_t byte_offset, int64_t bytes, int64_t *got)
{
    siggen_source *src = (siggen_source *)ctx;
    if (!src || !got || src->kind != 2 || !src->pool || src->pool_bytes <= 0 || byte_offset < 0 || bytes < 0)
        return NULL;
    const int64_t call = src->calls++;
    if (src->fail_at_call >= 0 && call == src->fail_at_call) return NULL;
    if (bytes > src->total_bytes - byte_offset) bytes = src->total_bytes - byte_offset;
    if (bytes < 0) bytes = 0;
    const int64_t o = byte_offset % src->pool_bytes;
    if (o + bytes > src->pool_bytes) return NULL;
    *got = bytes;
    return src->pool + o;
}

/*
 * Writer context: a host buffer that receives each output block at its byte
 * offset (positional order, Sec. III "getmerge" of files named by position).
 * base may be NULL: then the writer only counts bytes (a discarding sink).
 */
typedef struct {
    uint8_t *base;
    int64_t capacity;
    int32_t fail_at_call;
    int32_t pad;
    int64_t calls;
    int64_t bytes_written;
    int64_t last_offset; /* offset of the last accepted block, -1 if none */
} siggen_sink;

int siggen_write(void *ctx, int64_t byte_offset, const void *src, int64_t bytes)
{
    siggen_sink *s = (siggen_sink *)ctx;
    if (!s || !src || byte_offset < 0 || bytes < 0) return -1;
    const int64_t call = s->calls++;
    if (s->fail_at_call >= 0 && call == s->fail_at_call) return -1;
    if (s->base) {
        if (byte_offset + bytes > s->capacity) return -1;
        memcpy(s->base + byte_offset, src, (size_t)bytes);
    }
    s->bytes_written += bytes;
    s->last_offset = byte_offset;
    return 0;
}
