// Plan object and host helpers shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "fftseg.h"

namespace fftseg {

enum Path {
    PATH_BLOCK = 0,
    PATH_CLUSTER = 1,
    PATH_TWOPASS = 2,
    PATH_FOURSTEP = 4,
    PATH_REAL = 5,
    PATH_FRAMES = 6,
    PATH_BLUESTEIN = 7,
    PATH_MIXED = 8
};

}  // namespace fftseg

struct fftseg_plan_s {
    int device = 0;
    int64_t n = 0, batch = 0;
    int log_n = 0;
    int direction = FFTSEG_FORWARD, norm = FFTSEG_NORM_NONE;
    int precision = FFTSEG_PREC_FP32, out_kind = FFTSEG_OUT_COMPLEX;
    unsigned flags = 0;
    int path = 0;
    int log_n1 = 0, log_n2 = 0, log_c = 0;
    float scale = 1.f;
    // twiddle tables (device, forward values w = exp(-2 pi i m / M))
    float2 *twA = nullptr;   // stage twiddle tables of the column (block: whole) transform
    float2 *twB = nullptr;   // stage twiddle tables of the row transform
    float2 *tw4a = nullptr;  // four-step twiddles, rows k1 mod 2^tw_log_k
    float2 *tw4b = nullptr;  // rows k1 >> tw_log_k (null when one table is exact)
    int tw_log_k = 0;
    // two-pass workspace
    float2 *work = nullptr;
    int64_t work_segs = 0;
    int *d_err = nullptr;  // set by kernels whose bounded waits ran out
    // persistent four-step path
    float2 *ring = nullptr;   // ring_nr * ring_cs segments
    int ring_nr = 0, ring_cs = 0;
    int *ctr = nullptr;       // queue head + per-chunk counters
    int64_t ctr_count = 0;
    float2 *w4 = nullptr, *w4hi = nullptr;
    float2 *w4t = nullptr;  // the warp-line and lane-line kernels' factors, per column tile
    int wl_la = 0;          // lane-line kernel: chunks of lookahead of column over row passes
    // n = 2^21..2^24 (FP32, complex output): n = R * 2^16; the outer radix-R
    // pass writes the R transforms of 2^16 points interleaved into `work`, and
    // `inner`, a lane-line plan of 2^16 points over units of 32 interleaved
    // transforms (wl_ilv), finishes them
    int ilv_log_r = 0;
    bool wl_ilv = false;
    int w4_log_k = 0;
    int log_wa = 0, log_wb = 0;
    // real-signal plans (FFTSEG_FLAG_REAL): a complex plan of n/2 points
    fftseg_plan_s *inner = nullptr;
    float2 *rtw = nullptr;    // w_n^k, k = 0 .. n/4
    float2 *rwork = nullptr;  // [rchunk][n/2] complex intermediate
    int64_t rchunk = 0;  // segments (real plans) or frames (frame plans) per chunk
    // overlapping-segment plans (fftseg_plan_create_frames): rwork holds a chunk of frames
    int64_t hop = 0;
    int window = 0;
    float *fwin = nullptr;  // the window, n values (null: rectangular)
    // frame plans on the lane-line kernel (hop a multiple of N2, complex
    // output): frames go straight from the signal into its column tiles, the
    // Hann window from the factors win_row[j1] = (cos, sin)(2 pi j1 / N1),
    // win_col[j2] = (cos, sin)(2 pi j2 / n)
    bool frames_wl = false;
    float2 *win_row = nullptr, *win_col = nullptr;
    // lengths that are not powers of two: inner (forward) and inner2 (inverse)
    // M-point plans, the chirp and B = FFT_M(conjugate chirp) / M; rwork holds
    // a chunk of M-point rows
    fftseg_plan_s *inner2 = nullptr;
    // lengths 2^a 3^b 5^c 7^d <= 4096 (mixed-radix path): the radix schedule
    // (twA holds the stage twiddles, stage t at mix_twoff[t])
    int mix_nstages = 0;
    int mix_radix[16] = {}, mix_twoff[16] = {};
    float2 *bw = nullptr, *bhat = nullptr;
    int64_t bm = 0;
    // fftseg_stream phase split of the last call (ms)
    double phases[6] = {0, 0, 0, 0, 0, 0};
    // fftseg_exec_host device staging (owned; released with the plan)
    void *host_stage = nullptr;
    void (*host_stage_free)(void *) = nullptr;
};

namespace fftseg {

// error reporting (thread-local message)
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);
void count_launches(int64_t k);

// Tensor map over 8-byte (or 4-byte) elements: dims (d0 innermost, d1, d2),
// byte strides of dims 1 and 2, box (box0, box1, 1).
// swizzle128: the box lands in shared memory with the 128-byte swizzle (box0 *
// elem_bytes must be 128; the shared destination 1024-byte aligned).
int encode_tmap_3d(CUtensorMap *m, const void *base, int64_t d0, int64_t d1, int64_t d2, int64_t stride1_bytes,
                   int64_t stride2_bytes, uint32_t box0, uint32_t box1, int elem_bytes = 8, bool swizzle128 = false);
// The same with the 32-, 64- or 128-byte swizzle (swizzle_bytes; 0: none):
// box0 * elem_bytes must not exceed it, and the shared destination must be
// aligned to the swizzle pattern's repeat (8 rows of the swizzle span).
int encode_tmap_3d_swz(CUtensorMap *m, const void *base, int64_t d0, int64_t d1, int64_t d2, int64_t stride1_bytes,
                       int64_t stride2_bytes, uint32_t box0, uint32_t box1, int elem_bytes, int swizzle_bytes);
// Any rank (1..5): dims[rank] (innermost first), byte strides of dims 1..rank-1,
// box[rank], the swizzle as above.
int encode_tmap(CUtensorMap *m, const void *base, int rank, const int64_t *dims, const int64_t *strides,
                const uint32_t *box, int elem_bytes, int swizzle_bytes);

// Plan flags that select a schedule (the rest are options).
constexpr unsigned kPathFlags = FFTSEG_FLAG_FORCE_TWOPASS | FFTSEG_FLAG_FOURSTEP_L2 | FFTSEG_FLAG_FOURSTEP_PRODUCER |
                                FFTSEG_FLAG_FOURSTEP_WARP_LINES | FFTSEG_FLAG_FOURSTEP_TILES | FFTSEG_FLAG_CLUSTER_LOG2(0xF);

// Autotuner (tune.cu): the schedule flags of the fastest schedule for n on
// the current GPU, timed on min(batch, 256 MiB of input) segments.
int tune_schedule(int64_t n, int64_t batch, int prec, int out_kind, unsigned *flags_out, double *ms_out);

// Run the plan on nseg segments (arguments already validated).
int exec_plan(fftseg_plan p, const void *d_in, void *d_out, int64_t nseg, cudaStream_t st);
// Bytes of one segment's input and output in fftseg_stream (complex plans of
// any length and real-signal plans).
void segment_bytes(const fftseg_plan_s *p, int64_t *in, int64_t *out);

// Forward-direction roots of unity w_M^m for m < M, evaluated in double.
void host_roots(float2 *t, int64_t count, int64_t M, int64_t stride_exp);

// Stage twiddle tables of a length-L line in the kernels' layout.
void stage_table_host(std::vector<float2> &h, int64_t L);


}  // namespace fftseg
