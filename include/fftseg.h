/*
 * fftseg — batched forward/inverse complex FFTs over fixed-length,
 * offset-tagged segments of a very large signal, on one GB300 (sm_103a).
 *
 * The operation (paper Sec. III): a signal file is cut into <offset, FFT
 * segment> records; segment s holds samples [s*n, (s+1)*n) and starts at byte
 * offset s*n*8 of the complex64 signal; every segment is transformed on its
 * own (a batched plan partitions the segments in memory) and the outputs are
 * kept in positional order.  The transform is the Cooley-Tukey FFT (Sec. I),
 * i.e. for every segment
 *
 *     X_s[k] = scale * sum_{j<n} x_s[j] * exp(sigma * 2 pi i * j*k / n)
 *
 * sigma = -1 (FFTSEG_FORWARD) or +1 (FFTSEG_INVERSE); scale = 1 (NORM_NONE),
 * 1/n on the inverse (NORM_BACKWARD) or 1/sqrt(n) (NORM_ORTHO).  Bins are in
 * natural order k = 0..n-1.  The paper leaves the sign and the scaling open;
 * these are the conventions of the FFT library it calls.
 *
 * Data layout: complex64 = interleaved {float re, float im}, 8 bytes; a batch
 * is [batch][n] contiguous.  Power output (FFTSEG_OUT_POWER) is float32
 * |X|^2, [batch][n] contiguous.  Device buffers must be 16-byte aligned.
 *
 * Ownership: the caller owns every buffer it passes (device or host) and the
 * CUDA stream.  The library owns plans (twiddle tables, workspace) and the
 * pinned staging, streams and events it creates inside fftseg_stream and the
 * server.
 *
 * Errors: every entry point returns an fftseg_status; nothing throws or exits
 * across this boundary.  fftseg_last_error() returns a message for the last
 * failing call on the calling thread.  Asynchronous entry points report launch
 * errors; faults inside kernels surface on the caller's next synchronisation.
 *
 * There is no CPU fallback: every transform runs in this library's own
 * sm_103a kernels.
 */
#ifndef FFTSEG_H
#define FFTSEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fftseg_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    FFTSEG_OK = 0,
    FFTSEG_E_INVALID = -1,     /* bad argument (null, misaligned, out of range) */
    FFTSEG_E_NOMEM = -2,       /* device or pinned allocation failed */
    FFTSEG_E_CUDA = -3,        /* a CUDA runtime call or launch failed */
    FFTSEG_E_IO = -4,          /* a reader or writer callback failed */
    FFTSEG_E_PARTIAL = -5,     /* the signal ends inside a segment and zero padding is off */
    FFTSEG_E_TIMEOUT = -6,     /* a bounded wait ran out (server poll, device wait) */
    FFTSEG_E_UNSUPPORTED = -7  /* n outside the built lengths, or a precision/size mix not built */
} fftseg_status;

enum { FFTSEG_FORWARD = -1, FFTSEG_INVERSE = +1 };
enum { FFTSEG_NORM_NONE = 0, FFTSEG_NORM_BACKWARD = 1, FFTSEG_NORM_ORTHO = 2 };
enum { FFTSEG_PREC_FP32 = 0, FFTSEG_PREC_TC_FP16 = 1, FFTSEG_PREC_TC_BF16 = 2 };
enum { FFTSEG_OUT_COMPLEX = 0, FFTSEG_OUT_POWER = 1 };
enum { FFTSEG_WINDOW_RECT = 0, FFTSEG_WINDOW_HANN = 1 };

/* plan flags */
#define FFTSEG_FLAG_ZERO_PAD 0x1u     /* fftseg_stream: zero-pad a trailing partial segment */
#define FFTSEG_FLAG_FORCE_TWOPASS 0x2u /* use the non-persistent two-pass path (n >= 2^8) */
#define FFTSEG_FLAG_FOURSTEP_L2 0x4u   /* use the persistent four-step path with an L2-resident
                                          intermediate (n = 2^14..2^24) */
#define FFTSEG_FLAG_FOURSTEP_PRODUCER 0x8u /* four-step path, FP32: one producer warp feeds eight
                                             compute warps (TMA loads and stores) */
/* single-pass cluster path: request a cluster of 2^c CTAs (0 = the library's choice) */
#define FFTSEG_FLAG_CLUSTER_LOG2(c) (((unsigned)(c) & 0xFu) << 8)
/* time every schedule built for n on the current GPU at plan creation and use
   the fastest (replaces the schedule flags above; see fftseg_autotune) */
#define FFTSEG_FLAG_AUTOTUNE 0x10u
/* real signal (the paper's records are real single-precision samples, Sec. III):
   a forward plan of n points takes [batch][n] float32 samples and writes the
   n/2 + 1 bins X[0..n/2] of each segment's DFT, [batch][n/2 + 1] complex64 (or
   float32 |X|^2); an inverse plan takes [batch][n/2 + 1] complex64 bins and
   writes [batch][n] float32 samples of the inverse DFT of their Hermitian
   extension (the imaginary parts of X[0] and X[n/2] are ignored).  n is a power
   of two in [4, 2^24]; FP32 only; out of place only; streamed by fftseg_stream
   (4n input bytes per forward segment); not for fftseg_exec_host or the
   server.  Scaling as for complex plans, with n the
   real length.  Runs as a complex FFT of n/2 points on the samples read as
   complex values, plus the split (forward) or join (inverse) of the spectra of
   the even and odd samples: inside the transform's own kernel where it can
   (forward n <= 2^17; inverse n = 2^14, 2^15 for batches of up to 64 MiB of
   samples), else as a pass of its own over chunks of at most 512 MiB. */
#define FFTSEG_FLAG_REAL 0x20u
/* four-step path, FP32, complex output, n = 2^16: the 256 x 256 warp-line
   kernel (16 points per lane, three CTAs per SM) instead of the default
   lane-line kernel (32 points per lane, lines of 256..1024 points, the
   default for n = 2^16..2^20) */
#define FFTSEG_FLAG_FOURSTEP_WARP_LINES 0x40u
/* four-step path on the CTA-tile kernel (tiles of whole CTAs, the form that
   also runs |X|^2 output and the tensor-core stages), instead of the
   lane-line kernels */
#define FFTSEG_FLAG_FOURSTEP_TILES 0x80u
/* test only, for the lane-line kernel: the row tiles of the first segment wait
   for a counter value that is never reached, with a short spin limit, so that
   the bounded wait runs out: the kernel records it in the plan's flag and
   completes (that segment's output is not valid), and fftseg_plan_check then
   returns FFTSEG_E_TIMEOUT.  Shows that a lost dependency ends in an error
   status, not a hang. */
#define FFTSEG_FLAG_TEST_STALL 0x1000u
/* lengths that are not powers of two: Bluestein's algorithm even where the
   mixed-radix path applies (n = 2^a 3^b 5^c 7^d <= 4096) */
#define FFTSEG_FLAG_BLUESTEIN 0x2000u

#define FFTSEG_MAX_LOG2N 24

typedef struct fftseg_plan_s *fftseg_plan;

/*
 * Create a plan for `batch` segments of n points (Sec. III: one batched plan
 * over a block of segments).  Twiddle tables are evaluated in double
 * precision on the host and rounded once to float32 (split into hi+lo halves
 * for the tensor-core precisions); they stay resident on the current device.
 *   n          a power of two, 2 <= n <= 2^24; or any other length 3 <= n <= 2^23
 *              (FP32 only): n = 2^a 3^b 5^c 7^d <= 4096 by mixed-radix stages in
 *              one pass; otherwise by Bluestein's chirp-z identity as a cyclic
 *              convolution over M = 2^ceil(log2(2n - 1)) points: chirp in, M-point
 *              FFT, product with the plan's chirp spectrum, M-point inverse FFT,
 *              chirp out (one launch for M <= 4096, two per chunk for
 *              M = 2^13..2^16, five above; chunks of at most 1 GiB of M-point
 *              rows; out of place only); else FFTSEG_E_UNSUPPORTED
 *   batch      >= 1: the most segments one fftseg_exec call processes
 *   direction  FFTSEG_FORWARD or FFTSEG_INVERSE
 *   norm       FFTSEG_NORM_*
 *   precision  FFTSEG_PREC_FP32, or a tensor-core radix-16 precision
 *              (n must be a power of 16 from 16^3 to 16^6)
 *   out_kind   FFTSEG_OUT_COMPLEX or FFTSEG_OUT_POWER
 * On success *out owns device memory until fftseg_plan_destroy.
 */
int fftseg_plan_create(fftseg_plan *out, int64_t n, int64_t batch, int direction, int norm,
                       int precision, int out_kind, unsigned flags);

/*
 * Transform `batch` segments: d_in [batch][n] complex64 -> d_out [batch][n]
 * (complex64, or float32 for the power output).  d_in == d_out transforms in
 * place (complex output only).  Asynchronous on `stream`.  Device pointers,
 * 16-byte aligned.
 */
int fftseg_exec(fftseg_plan p, const void *d_in, void *d_out, fftseg_stream_t stream);

/* As fftseg_exec for the first `nseg` (0 <= nseg <= batch) segments. */
int fftseg_exec_n(fftseg_plan p, const void *d_in, void *d_out, int64_t nseg,
                  fftseg_stream_t stream);

/*
 * Overlapping segments, a short-time FFT (the paper names overlapping FFTs as
 * future work, Sec. VI): frame f of the signal holds samples [f*hop, f*hop + n),
 * multiplied point by point by the window, and is transformed like a segment
 * of a forward complex plan:
 *     X_f[k] = scale * sum_{j<n} w[j] x[f*hop + j] exp(-2 pi i j k / n)
 *   n        power of two, 2 <= n <= 2^24, else FFTSEG_E_UNSUPPORTED
 *   hop      >= 1 samples between frame starts (hop < n overlaps, hop > n skips)
 *   window   FFTSEG_WINDOW_RECT (w = 1) or FFTSEG_WINDOW_HANN
 *            (w[j] = (1 - cos(2 pi j / n)) / 2, the periodic Hann window,
 *            evaluated in double and rounded once to float32)
 *   batch    >= 1: the most frames one exec processes
 *   norm, out_kind, flags  as for fftseg_plan_create (schedule flags and
 *            FFTSEG_FLAG_AUTOTUNE apply to the n-point transform; FFTSEG_FLAG_REAL
 *            is not built for frames)
 * Run it with fftseg_exec / fftseg_exec_n: d_in is the complex64 signal and must
 * hold at least (nframes - 1)*hop + n samples (the library cannot check the
 * size of a device buffer); d_out is [nframes][n] complex64 (or float32 |X|^2);
 * out of place only.  Frames of n <= 4096 points go from the signal to their
 * bins in one pass, and so do frames of n = 2^16..2^20 whose hop is a multiple
 * of the four-step column length; other frames are windowed into an
 * intermediate of at most 512 MiB, which then goes through the n-point
 * transform.  fftseg_stream takes
 * frame plans (see there); fftseg_exec_host and the server do not.
 */
int fftseg_plan_create_frames(fftseg_plan *out, int64_t n, int64_t hop, int window, int64_t batch, int norm,
                              int out_kind, unsigned flags);

/*
 * Streaming chunker (Sec. III's split/transform/merge on one GPU; the paper's
 * per-block single allocate + copy becomes a pinned, double-buffered host
 * link): reads the signal from byte `start_offset` to `total_bytes` in chunks
 * of `chunk_segments` segments (<= the plan's batch), copies each chunk to the
 * device on one stream, transforms it on a second and copies the result back
 * on a third, and hands every result block to the writer at its output byte
 * offset (s*n*8 for complex output, s*n*4 for power output), in offset order.
 *   rd(ctx, byte_offset, dst, bytes) fills dst (pinned host memory) and
 *      returns the bytes read (a short read ends the signal) or < 0 on error.
 *   wr(ctx, byte_offset, src, bytes) consumes a result block, returns 0 or < 0.
 *   start_offset  must be a multiple of n*8 (resume point).
 *   committed_offset  receives the input byte offset up to which every output
 *      has been handed to the writer (resume from there after an error).
 * Synchronous.  Returns FFTSEG_E_IO on a callback error, FFTSEG_E_PARTIAL if
 * the signal ends inside a segment without FFTSEG_FLAG_ZERO_PAD (the complete
 * segments before it are written).
 * Real-signal plans (FFTSEG_FLAG_REAL): a segment is 4n bytes of float32
 * samples in and (n/2 + 1) bins out (forward), or the reverse (inverse);
 * offsets and start_offset count those bytes.
 * Frame plans (fftseg_plan_create_frames): the signal is complex64 samples
 * (total_bytes a multiple of 8); chunk_segments counts frames; every frame
 * that lies wholly inside the signal is transformed (trailing samples that
 * start no complete frame are not an error) and frame f's bins go to output
 * offset f*n*8 (or f*n*4).  Consecutive chunks share n - hop samples, which
 * are carried over rather than read again, so each sample is read once when
 * hop <= n.  start_offset must be f*hop*8 for a frame f, and committed_offset
 * receives f*hop*8 for the first frame whose bins were not written.  A short
 * read ends the signal after the frames that fit in it.
 */
typedef int64_t (*fftseg_read_fn)(void *ctx, int64_t byte_offset, void *dst, int64_t bytes);
typedef int (*fftseg_write_fn)(void *ctx, int64_t byte_offset, const void *src, int64_t bytes);
int fftseg_stream(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_write_fn wr, void *wctx,
                  int64_t total_bytes, int64_t start_offset, int64_t chunk_segments,
                  int64_t *committed_offset);

/* A source that lends the signal's bytes instead of copying them: returns the
 * host address of the bytes [byte_offset, byte_offset + bytes) -- all of them,
 * or fewer only where the signal ends (the count in *got) -- or NULL on
 * failure.  The memory must stay valid and unchanged until the stream call
 * returns: a signal already in host memory (a pinned buffer, a mapped file).
 * Pinned memory goes to the GPU at the host link's rate; pageable memory
 * through the driver's own staging, more slowly. */
typedef const void *(*fftseg_view_fn)(void *ctx, int64_t byte_offset, int64_t bytes, int64_t *got);

/* fftseg_stream with a lending source (fftseg_view_fn) in place of the reader:
 * each chunk is copied to the GPU straight from the lent memory, with no copy
 * into the chunker's pinned buffers (Sec. III's one copy per block).  The same
 * segmenting, positional output, partial-tail rules and resume offset as
 * fftseg_stream; the writer is called the same way.  Segment plans only (frame
 * plans: FFTSEG_E_UNSUPPORTED).  A NULL from the source ends the call with
 * FFTSEG_E_IO at that offset. */
int fftseg_stream_view(fftseg_plan p, fftseg_view_fn view, void *vctx, fftseg_write_fn wr, void *wctx,
                       int64_t total_bytes, int64_t start_offset, int64_t chunk_segments,
                       int64_t *committed_offset);

/*
 * File-backed streaming: the paper's pipeline end to end on one GPU (Sec. III,
 * a signal file cut into segments, each transformed, the results written in
 * positional order).  fftseg_stream with a reader and a writer over files:
 *   in_path     the signal (complex64; float32 samples or bins for a
 *               real-signal plan; frames for a frame plan, as fftseg_stream
 *               describes)
 *   out_path    receives the results at the output offsets of fftseg_stream
 *               (s*n*8 complex, s*n*4 power); created, and truncated when start_offset is 0
 *               unless FFTSEG_FILE_KEEP (a resumed run keeps what lies before
 *               its start)
 *   start_offset, end_offset  the input byte range [start, end) to transform;
 *               end_offset 0 (or past the end) means the end of the file;
 *               start_offset a multiple of n*8.  Several processes can each
 *               take a range of the same file and write the same output
 *               (FFTSEG_FILE_KEEP): the results land at their positions with
 *               no merge step.
 *   chunk_segments, committed_offset  as for fftseg_stream
 *   file_flags  FFTSEG_FILE_DIRECT: O_DIRECT reads and writes (the page cache
 *               bypassed) where segment sizes are multiples of 4096 bytes and
 *               the file system allows it (never for frame plans, which read
 *               at frame offsets), buffered I/O otherwise;
 *               FFTSEG_FILE_KEEP: never truncate the output
 * Synchronous.  FFTSEG_E_IO if a file cannot be opened, read or written; the
 * other results as for fftseg_stream.  The phase split of the run (file reads
 * and writes against transfers and transforms, the analog of the paper's I/O
 * versus FFT breakdown, Sec. IV) is in fftseg_stream_phases.
 */
#define FFTSEG_FILE_DIRECT 0x1u
#define FFTSEG_FILE_KEEP 0x2u
int fftseg_stream_file(fftseg_plan p, const char *in_path, const char *out_path, int64_t start_offset,
                       int64_t end_offset, int64_t chunk_segments, unsigned file_flags, int64_t *committed_offset);

/* Phase split of the last fftseg_stream call on this plan, in milliseconds
 * (the analog of the paper's I/O versus FFT breakdown, Sec. IV Figs. 4-5):
 * out[0] read callback, out[1] H2D, out[2] transform, out[3] D2H,
 * out[4] write callback, out[5] wall time. */
int fftseg_stream_phases(fftseg_plan p, double out[6]);

/*
 * Autotuner (the schedule choice that the paper leaves to its FFT library):
 * where more than one schedule is built for n (cluster sizes 2..16 CTAs, the
 * persistent four-step with or without a producer warp, the two-pass form),
 * each is timed on the current GPU over min(batch, 256 MiB of input) zero
 * segments and the fastest is returned as plan flags in *flags_out (0 where
 * one schedule exists), with its time per exec in *ms_out (may be NULL; < 0
 * when nothing was timed).  Choices are cached for the process, keyed by GPU
 * name, SM count, n, precision, output kind and the timed segment count; if
 * the environment variable FFTSEG_TUNE_CACHE names a file, choices are read
 * from it on first use and new ones appended.  Synchronous; allocates
 * scratch for the timing.  A plan created with FFTSEG_FLAG_AUTOTUNE makes
 * this call itself.
 */
int fftseg_autotune(int64_t n, int64_t batch, int precision, int out_kind, unsigned *flags_out, double *ms_out);

/*
 * A batch held in host memory through a chain of plans (Sec. III's copy in,
 * transform, copy back, as one overlapped pipeline): h_in [nseg][n] complex64
 * -> plans[0] -> plans[1] -> ... -> plans[nplans-1] -> h_out [nseg][n]
 * (complex64, or float32 when the last plan writes the power output).
 *   plans          nplans >= 1 plans of the same n on the current device;
 *                  all but the last must write complex output.
 *   h_in, h_out    host memory the caller owns (pinned runs at full link
 *                  speed; pageable works where the driver can stage it).
 *                  h_in == h_out transforms in place; other overlaps are
 *                  undefined.
 *   chunk_segments segments per chunk, 1..the smallest plan batch; 0 picks
 *                  about 256 MiB of input per chunk.
 * Chunk c+1 is copied to the device while chunk c runs through the plans and
 * chunk c-1 is copied back, on three streams the library owns.  The device
 * staging (three slots of two chunk buffers) is allocated on first use and
 * kept with plans[0] until fftseg_plan_destroy.  Synchronous: h_out is
 * complete when the call returns FFTSEG_OK.  A failing CUDA call returns
 * FFTSEG_E_CUDA (or E_NOMEM for the staging); the content of h_out is then
 * undefined.
 */
int fftseg_exec_host(const fftseg_plan *plans, int nplans, const void *h_in, void *h_out, int64_t nseg,
                     int64_t chunk_segments);

int fftseg_plan_destroy(fftseg_plan p);

/* Plan facts: info[0] path (0 block, 1 cluster, 2 two-pass, 3 tensor core,
 * 4 persistent four-step, 5 real signal over an inner complex plan,
 * 6 overlapping frames over an inner complex plan, 7 a length that is not a
 * power of two, over two inner plans of M points; info[1] is then M),
 * info[1] n1, info[2] n2, info[3] workspace bytes, info[4] segments per
 * workspace chunk, info[5] kernel launches per fftseg_exec of a full batch. */
int fftseg_plan_info(fftseg_plan p, int64_t info[6]);

/* Synchronise with the device and report whether any kernel of this plan
 * gave up a bounded wait since the last check (FFTSEG_E_TIMEOUT; the outputs
 * of that call are then not valid) -- FFTSEG_OK otherwise.  Clears the flag.
 * In the self-checking build (libfftseg_debug.so, compiled with
 * -DFFTSEG_DEBUG) a kernel that finds one of its indices outside its buffer
 * skips that access and this call returns FFTSEG_E_INVALID. */
int fftseg_plan_check(fftseg_plan p);

/* Message for the last failing call on this thread ("" if none). */
const char *fftseg_last_error(void);

/* Number of kernels this library has launched in this process. */
int64_t fftseg_launch_count(void);

/*
 * fftseg_exec_noalloc: the same batched transform as a forward/inverse plan of
 * n points, for callers that must not allocate device memory. The paper has no
 * counterpart.
 *
 * Some callers can't call cudaMalloc:
 *   - code running under a strict device-memory budget set by its host;
 *   - plugins whose host application owns all allocations;
 *   - real-time processing threads, where cudaMalloc may synchronise the device
 *     and take an unbounded time.
 * This entry point needs no plan and calls no cudaMalloc, cudaFree or other
 * allocating routine. Its scratch is one fixed array of about 25.5 MiB,
 * compiled into the library, which every GPU that loads the library holds
 * until the process exits. The scratch holds:
 *   - the L2 ring of three 8 MiB chunks;
 *   - the chunk counters;
 *   - the twiddle tables of the last length used.
 *
 *   d_in, d_out  device, 16-byte aligned, [nseg][n] complex64 (may be equal)
 *   n            a power of two from 2^17 to 2^20; anything else returns
 *                FFTSEG_E_UNSUPPORTED, since larger lengths do not fit the
 *                fixed scratch
 *   direction, norm  as for fftseg_plan_create; output is always complex
 * Asynchronous on `stream`.
 *
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address. Make that first call before any stream capture.
 * Every call shares the one array, which keeps the last call's contents. The
 * twiddle tables are recomputed on the device when n changes; the chunk
 * counters are cleared at every call. Calls that overlap on the GPU (for
 * example, on two streams) race on the array and give undefined results.
 */
int fftseg_exec_noalloc(const void *d_in, void *d_out, int64_t n, int64_t nseg, int direction, int norm,
                        fftseg_stream_t stream);

/* Error check for fftseg_exec_noalloc on the current device, the counterpart
 * of fftseg_plan_check. The kernels of fftseg_exec_noalloc record a give-up
 * (a bounded wait that ran out, or a misaligned shared buffer) in a flag kept
 * in the same fixed array; the flag is not cleared by later calls, so it
 * covers every call since the last check. This call waits for the device,
 * reads the flag and clears it: FFTSEG_E_TIMEOUT if it was set (the outputs
 * of those calls are not valid), FFTSEG_OK otherwise, and FFTSEG_OK if no
 * call has run on this device. It allocates nothing.
 * The array's device address and the record of which length's tables it
 * holds are kept per device for the life of the process: do not use these
 * two calls on a device after cudaDeviceReset. */
int fftseg_noalloc_check(void);

/* ---------------------------------------------------------------- serving
 * Continuous batching of segment-FFT jobs of different lengths.  Jobs are
 * admitted in arrival order while the bytes they touch fit the HBM budget and
 * fewer than max_inflight_jobs run (a job larger than the budget is admitted
 * in pieces of whole segments).  Each admission round runs every admitted
 * job with n <= 4096 in one persistent ragged kernel launch (a captured CUDA
 * graph replayed from one of two slots), and every piece of a longer job
 * through a resident plan of its length on one of four lane streams, so that
 * rounds and large pieces overlap on the device.  Plans and twiddles stay
 * resident.  A job's result is the same alone and in any mix.
 */
typedef struct fftsrv_s *fftsrv;
typedef struct {
    int64_t hbm_budget_bytes; /* bytes of job input+output that may be in flight (the resident
                                 plans' own scratch, made once per length, direction, norm
                                 and lane, comes on top) */
    int max_inflight_jobs;
    fftseg_stream_t stream;   /* NULL: the server creates its own streams (four lanes for
                                 large jobs); else large jobs run in order on this stream */
} fftsrv_config;
typedef struct {
    const void *d_in; /* [nseg][n] complex64, device */
    void *d_out;      /* [nseg][n] complex64, device (may equal d_in) */
    int64_t n;        /* power of two, 2^1..2^22 */
    int64_t nseg;     /* >= 1 */
    int direction;
    int norm;
} fftsrv_job;

int fftsrv_create(fftsrv *out, const fftsrv_config *cfg);
/* Queue a job (non-blocking).  *job_id identifies it for fftsrv_poll. */
int fftsrv_submit(fftsrv s, const fftsrv_job *job, uint64_t *job_id);
/* Wait up to timeout_us (0 = just check) for the job.  Returns FFTSEG_OK with
 * *job_status = the job's final status once it has completed, or
 * FFTSEG_E_TIMEOUT while it is still queued or running. */
int fftsrv_poll(fftsrv s, uint64_t job_id, int64_t timeout_us, int *job_status);
/* As fftsrv_poll; once the job has completed, also *latency_us (if not NULL)
 * = its time in the server by the host's steady clock, from fftsrv_submit
 * accepting it to the completion callback of its last piece (so a caller
 * that polls late still reads the job's own latency). */
int fftsrv_poll_latency(fftsrv s, uint64_t job_id, int64_t timeout_us, int *job_status, double *latency_us);
/* Server counters: out[0] jobs submitted, out[1] completed, out[2] launches,
 * out[3] peak admitted bytes, out[4] queue depth now. */
int fftsrv_stats(fftsrv s, int64_t out[5]);
/* Drain every queued job, then release the server. */
int fftsrv_destroy(fftsrv s);

#ifdef __cplusplus
}
#endif

#endif /* FFTSEG_H */
