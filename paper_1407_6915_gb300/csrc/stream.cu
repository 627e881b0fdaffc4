// fftseg_stream: the out-of-core chunker.
//
// The paper (Sec. III) hands each 512 MB HDFS block to the GPU with a single
// allocate + copy, runs a batched plan over the block's segments and writes
// the result under a name that keeps positional order; I/O dominates its run
// time (Sec. IV).  Here one process streams a signal of any length through a
// ring of pinned host buffers: the host reads chunk c while the GPU copies
// chunk c-1 in (copy stream), transforms it (compute stream) and copies it
// out (a second copy stream), and the writer receives each result at its
// output byte offset, in offset order.  A failed callback stops the stream
// with the offset up to which output is complete, so a later call resumes
// there.
#include <chrono>
#include <string.h>

#include "plan.h"

namespace fftseg {
namespace {

constexpr int kRing = 3;

struct Ring {
    int64_t chunk_segs = 0;
    int64_t in_bytes = 0, out_bytes = 0;  // per buffer
    void *h_in[kRing] = {}, *h_out[kRing] = {};
    void *d_in[kRing] = {}, *d_out[kRing] = {};
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    cudaEvent_t e0[kRing] = {}, e_h2d[kRing] = {}, e_comp[kRing] = {}, e_d2h[kRing] = {};

    ~Ring()
    {
        for (int i = 0; i < kRing; ++i) {
            cudaFreeHost(h_in[i]);
            cudaFreeHost(h_out[i]);
            cudaFree(d_in[i]);
            cudaFree(d_out[i]);
            if (e0[i]) cudaEventDestroy(e0[i]);
            if (e_h2d[i]) cudaEventDestroy(e_h2d[i]);
            if (e_comp[i]) cudaEventDestroy(e_comp[i]);
            if (e_d2h[i]) cudaEventDestroy(e_d2h[i]);
        }
        if (s_h2d) cudaStreamDestroy(s_h2d);
        if (s_comp) cudaStreamDestroy(s_comp);
        if (s_d2h) cudaStreamDestroy(s_d2h);
    }

    int init(int64_t segs, int64_t seg_in, int64_t seg_out) { return init_bytes(segs, segs * seg_in, segs * seg_out); }

    int init_bytes(int64_t segs, int64_t in_b, int64_t out_b)
    {
        chunk_segs = segs;
        in_bytes = in_b;
        out_bytes = out_b;
        cudaError_t e;
#define RING_CHECK(call, what)                     \
    do {                                           \
        e = (call);                                \
        if (e != cudaSuccess) return cuda_error(e, what); \
    } while (0)
        RING_CHECK(cudaStreamCreateWithFlags(&s_h2d, cudaStreamNonBlocking), "stream create");
        RING_CHECK(cudaStreamCreateWithFlags(&s_comp, cudaStreamNonBlocking), "stream create");
        RING_CHECK(cudaStreamCreateWithFlags(&s_d2h, cudaStreamNonBlocking), "stream create");
        for (int i = 0; i < kRing; ++i) {
            RING_CHECK(cudaHostAlloc(&h_in[i], (size_t)in_bytes, cudaHostAllocDefault), "pinned alloc");
            RING_CHECK(cudaHostAlloc(&h_out[i], (size_t)out_bytes, cudaHostAllocDefault), "pinned alloc");
            RING_CHECK(cudaMalloc(&d_in[i], (size_t)in_bytes), "device alloc");
            RING_CHECK(cudaMalloc(&d_out[i], (size_t)out_bytes), "device alloc");
            RING_CHECK(cudaEventCreate(&e0[i]), "event create");
            RING_CHECK(cudaEventCreate(&e_h2d[i]), "event create");
            RING_CHECK(cudaEventCreate(&e_comp[i]), "event create");
            RING_CHECK(cudaEventCreate(&e_d2h[i]), "event create");
        }
#undef RING_CHECK
        return FFTSEG_OK;
    }
};

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Pending {
    int64_t in_offset = 0;  // input byte offset of the chunk
    int64_t segs = 0;
    bool live = false;
};

int stream_frames(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_write_fn wr, void *wctx,
                  int64_t total_bytes, int64_t start_offset, int64_t chunk_frames, int64_t *committed_offset);

}  // namespace

// Bytes of one segment's input and output for the streamed plan kinds:
// complex (any length) and real-signal plans.
void segment_bytes(const fftseg_plan_s *p, int64_t *in, int64_t *out)
{
    const int64_t pw = p->out_kind == FFTSEG_OUT_POWER ? 4 : 8;
    if (p->path == PATH_REAL) {
        const int64_t bins = (p->n / 2 + 1) * 8;
        *in = p->direction == FFTSEG_FORWARD ? p->n * 4 : bins;
        *out = p->direction == FFTSEG_FORWARD ? (p->n / 2 + 1) * pw : p->n * 4;
        return;
    }
    *in = p->n * 8;
    *out = p->n * pw;
}

}  // namespace fftseg

using namespace fftseg;

namespace fftseg {
namespace {

// The segment-plan chunker, fed either by a reader that copies each chunk
// into the ring's pinned buffer (rd) or by a source that lends the chunk's
// bytes in place (view): then the copy to the GPU reads the source directly.
int stream_segments(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_view_fn view, void *vctx,
                    fftseg_write_fn wr, void *wctx, int64_t total_bytes, int64_t start_offset,
                    int64_t chunk_segments, int64_t *committed_offset);

}  // namespace
}  // namespace fftseg

extern "C" int fftseg_stream(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_write_fn wr, void *wctx,
                             int64_t total_bytes, int64_t start_offset, int64_t chunk_segments,
                             int64_t *committed_offset)
{
    if (committed_offset) *committed_offset = start_offset;
    if (!p || !rd || !wr) return set_error(FFTSEG_E_INVALID, "stream: NULL plan or callback");
    if (p->path == PATH_FRAMES)
        return stream_frames(p, rd, rctx, wr, wctx, total_bytes, start_offset, chunk_segments, committed_offset);
    return stream_segments(p, rd, rctx, nullptr, nullptr, wr, wctx, total_bytes, start_offset, chunk_segments,
                           committed_offset);
}

extern "C" int fftseg_stream_view(fftseg_plan p, fftseg_view_fn view, void *vctx, fftseg_write_fn wr, void *wctx,
                                  int64_t total_bytes, int64_t start_offset, int64_t chunk_segments,
                                  int64_t *committed_offset)
{
    if (committed_offset) *committed_offset = start_offset;
    if (!p || !view || !wr) return set_error(FFTSEG_E_INVALID, "stream_view: NULL plan or callback");
    if (p->path == PATH_FRAMES)
        return set_error(FFTSEG_E_UNSUPPORTED, "stream_view: frame plans stream through fftseg_stream");
    return stream_segments(p, nullptr, nullptr, view, vctx, wr, wctx, total_bytes, start_offset, chunk_segments,
                           committed_offset);
}

namespace fftseg {
namespace {

int stream_segments(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_view_fn view, void *vctx,
                    fftseg_write_fn wr, void *wctx, int64_t total_bytes, int64_t start_offset,
                    int64_t chunk_segments, int64_t *committed_offset)
{
    int64_t seg_in = 0, seg_out = 0;
    segment_bytes(p, &seg_in, &seg_out);
    if (total_bytes < 0 || start_offset < 0 || start_offset > total_bytes || start_offset % seg_in)
        return set_error(FFTSEG_E_INVALID, "stream: start_offset must be a segment boundary within the signal");
    if (chunk_segments == 0) chunk_segments = p->batch;
    if (chunk_segments < 1 || chunk_segments > p->batch)
        return set_error(FFTSEG_E_INVALID, "stream: chunk_segments must be in [1, plan batch]");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return set_error(FFTSEG_E_INVALID, "stream: plan belongs to another device");

    const bool zero_pad = (p->flags & FFTSEG_FLAG_ZERO_PAD) != 0;
    const double t_start = now_ms();
    double t_read = 0, t_write = 0, t_h2d = 0, t_comp = 0, t_d2h = 0;
    for (int i = 0; i < 6; ++i) p->phases[i] = 0;

    Ring ring;
    int rc = ring.init(chunk_segments, seg_in, seg_out);
    if (rc != FFTSEG_OK) return rc;

    Pending pend[kRing];
    int64_t committed = start_offset;
    int status = FFTSEG_OK;
    bool ended = false;
    bool can_write = true;  // false after a writer or CUDA failure

    // Complete chunk slot i: wait for its copy-out, account its phases, write it.
    auto retire = [&](int i) -> int {
        if (!pend[i].live) return FFTSEG_OK;
        pend[i].live = false;
        cudaError_t e = cudaEventSynchronize(ring.e_d2h[i]);
        if (e != cudaSuccess) return cuda_error(e, "stream: chunk completion");
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ring.e0[i], ring.e_h2d[i]) == cudaSuccess) t_h2d += ms;
        if (cudaEventElapsedTime(&ms, ring.e_h2d[i], ring.e_comp[i]) == cudaSuccess) t_comp += ms;
        if (cudaEventElapsedTime(&ms, ring.e_comp[i], ring.e_d2h[i]) == cudaSuccess) t_d2h += ms;
        const double t0 = now_ms();
        const int64_t out_off = (pend[i].in_offset / seg_in) * seg_out;
        const int wrc = wr(wctx, out_off, ring.h_out[i], pend[i].segs * seg_out);
        t_write += now_ms() - t0;
        if (wrc != 0) return set_error(FFTSEG_E_IO, "stream: writer failed at output offset %lld",
                                       (long long)out_off);
        committed = pend[i].in_offset + pend[i].segs * seg_in;
        return FFTSEG_OK;
    };

    int64_t offset = start_offset;
    int64_t chunk = 0;
    while (!ended && offset < total_bytes) {
        const int i = (int)(chunk % kRing);
        if ((rc = retire(i)) != FFTSEG_OK) {
            status = rc;
            can_write = false;
            break;
        }
        int64_t want = total_bytes - offset;
        if (want > ring.in_bytes) want = ring.in_bytes;
        const double t0 = now_ms();
        int64_t got = -1;
        const void *src = ring.h_in[i];  // where this chunk's bytes are
        if (view) {
            const void *lent = view(vctx, offset, want, &got);
            if (!lent) got = -1;
            src = lent;
        } else {
            got = rd(rctx, offset, ring.h_in[i], want);
        }
        t_read += now_ms() - t0;
        if (got < 0 || got > want) {
            status = set_error(FFTSEG_E_IO, "stream: reader failed at input offset %lld", (long long)offset);
            break;
        }
        if (got < want) ended = true;  // short read: the signal ends here
        int64_t segs = got / seg_in;
        const int64_t tail = got - segs * seg_in;
        if (tail) {
            if (zero_pad) {
                if (src != ring.h_in[i]) {  // a lent tail is padded in the ring's own buffer
                    memcpy(ring.h_in[i], src, (size_t)got);
                    src = ring.h_in[i];
                }
                memset(static_cast<char *>(ring.h_in[i]) + got, 0, (size_t)(seg_in - tail));
                ++segs;
            } else {
                status = set_error(FFTSEG_E_PARTIAL, "stream: the signal ends %lld bytes into a segment",
                                   (long long)tail);
            }
            ended = true;
        }
        if (segs > 0) {
            cudaError_t e;
            const int64_t bytes = segs * seg_in;
            if ((e = cudaEventRecord(ring.e0[i], ring.s_h2d)) != cudaSuccess ||
                (e = cudaMemcpyAsync(ring.d_in[i], src, (size_t)bytes, cudaMemcpyHostToDevice, ring.s_h2d)) !=
                    cudaSuccess ||
                (e = cudaEventRecord(ring.e_h2d[i], ring.s_h2d)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ring.s_comp, ring.e_h2d[i], 0)) != cudaSuccess) {
                status = cuda_error(e, "stream: copy-in");
                can_write = false;
                break;
            }
            if ((rc = exec_plan(p, ring.d_in[i], ring.d_out[i], segs, ring.s_comp)) != FFTSEG_OK) {
                status = rc;
                can_write = false;
                break;
            }
            if ((e = cudaEventRecord(ring.e_comp[i], ring.s_comp)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ring.s_d2h, ring.e_comp[i], 0)) != cudaSuccess ||
                (e = cudaMemcpyAsync(ring.h_out[i], ring.d_out[i], (size_t)(segs * seg_out),
                                     cudaMemcpyDeviceToHost, ring.s_d2h)) != cudaSuccess ||
                (e = cudaEventRecord(ring.e_d2h[i], ring.s_d2h)) != cudaSuccess) {
                status = cuda_error(e, "stream: copy-out");
                can_write = false;
                break;
            }
            pend[i].in_offset = offset;
            pend[i].segs = segs;
            pend[i].live = true;
        }
        offset += got;
        ++chunk;
    }
    // Drain in chunk order.  Chunks issued before a reader error or a short
    // signal are still written; after a writer or CUDA error nothing more is.
    for (int64_t k = chunk - kRing; k < chunk; ++k) {
        if (k < 0) continue;
        const int i = (int)(k % kRing);
        if (!can_write) {
            if (pend[i].live) cudaEventSynchronize(ring.e_d2h[i]);  // the ring is freed after this
            pend[i].live = false;
            continue;
        }
        if ((rc = retire(i)) != FFTSEG_OK) {
            if (status == FFTSEG_OK || status == FFTSEG_E_PARTIAL) status = rc;
            can_write = false;
        }
    }
    cudaStreamSynchronize(ring.s_h2d);
    cudaStreamSynchronize(ring.s_comp);
    cudaStreamSynchronize(ring.s_d2h);
    p->phases[0] = t_read;
    p->phases[1] = t_h2d;
    p->phases[2] = t_comp;
    p->phases[3] = t_d2h;
    p->phases[4] = t_write;
    p->phases[5] = now_ms() - t_start;
    if (committed_offset) *committed_offset = committed;
    return status;
}

}  // namespace
}  // namespace fftseg

namespace fftseg {
namespace {

// Frame plans: frame f holds samples [f*hop, f*hop + n).  A chunk of up to
// chunk_frames frames needs the samples [f0*hop, (f0 + cnt - 1)*hop + n); when
// hop < n, consecutive chunks share their last n - hop samples, which are
// carried over from the previous chunk's host buffer instead of being read
// again.  Frame f's bins go to output byte offset f*n*(8 or 4).  Only frames
// that lie wholly inside the signal are transformed: trailing samples that
// start no complete frame are not an error.  start_offset must be a multiple
// of hop*8 (the first sample of a frame); committed_offset receives
// f_next*hop*8 for the first frame whose output was not handed to the writer.
// The host and device input buffers hold a whole chunk's span, gaps included
// when hop > n: ((chunk_frames - 1)*hop + n)*8 bytes each.
int stream_frames(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_write_fn wr, void *wctx,
                  int64_t total_bytes, int64_t start_offset, int64_t chunk_frames, int64_t *committed_offset)
{
    const int64_t n = p->n, hop = p->hop;
    const int64_t frame_out = n * (p->out_kind == FFTSEG_OUT_POWER ? 4 : 8);
    if (total_bytes < 0 || total_bytes % 8)
        return set_error(FFTSEG_E_INVALID, "stream: a frame plan's signal is whole complex64 samples");
    if (start_offset < 0 || start_offset % (hop * 8))
        return set_error(FFTSEG_E_INVALID, "stream: start_offset must be the first sample of a frame (hop*8 bytes)");
    const int64_t samples = total_bytes / 8;
    const int64_t frames = samples >= n ? (samples - n) / hop + 1 : 0;
    const int64_t f_start = start_offset / (hop * 8);
    if (f_start > frames) return set_error(FFTSEG_E_INVALID, "stream: start_offset past the last frame");
    if (chunk_frames == 0) chunk_frames = p->batch;
    if (chunk_frames < 1 || chunk_frames > p->batch)
        return set_error(FFTSEG_E_INVALID, "stream: chunk_segments must be in [1, plan batch]");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return set_error(FFTSEG_E_INVALID, "stream: plan belongs to another device");

    const double t_start = now_ms();
    double t_read = 0, t_write = 0, t_h2d = 0, t_comp = 0, t_d2h = 0;
    for (int i = 0; i < 6; ++i) p->phases[i] = 0;
    const int64_t span_max = ((chunk_frames - 1) * hop + n) * 8;  // input bytes of a full chunk
    const int64_t halo = hop < n ? (n - hop) * 8 : 0;             // bytes shared by consecutive chunks
    Ring ring;
    int rc = ring.init_bytes(chunk_frames, span_max, chunk_frames * frame_out);
    if (rc != FFTSEG_OK) return rc;

    struct Chunk {
        int64_t f0 = 0, cnt = 0;
        bool live = false;
    } pend[kRing];
    int64_t committed_f = f_start;
    int status = FFTSEG_OK;
    bool can_write = true;

    auto retire = [&](int i) -> int {
        if (!pend[i].live) return FFTSEG_OK;
        pend[i].live = false;
        cudaError_t e = cudaEventSynchronize(ring.e_d2h[i]);
        if (e != cudaSuccess) return cuda_error(e, "stream: chunk completion");
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ring.e0[i], ring.e_h2d[i]) == cudaSuccess) t_h2d += ms;
        if (cudaEventElapsedTime(&ms, ring.e_h2d[i], ring.e_comp[i]) == cudaSuccess) t_comp += ms;
        if (cudaEventElapsedTime(&ms, ring.e_comp[i], ring.e_d2h[i]) == cudaSuccess) t_d2h += ms;
        const double t0 = now_ms();
        const int64_t out_off = pend[i].f0 * frame_out;
        const int wrc = wr(wctx, out_off, ring.h_out[i], pend[i].cnt * frame_out);
        t_write += now_ms() - t0;
        if (wrc != 0)
            return set_error(FFTSEG_E_IO, "stream: writer failed at output offset %lld", (long long)out_off);
        committed_f = pend[i].f0 + pend[i].cnt;
        return FFTSEG_OK;
    };

    int64_t chunk = 0;
    int prev = -1;  // ring slot of the previous chunk of this call (its samples supply the halo)
    for (int64_t f0 = f_start; f0 < frames; f0 += chunk_frames, ++chunk) {
        const int i = (int)(chunk % kRing);
        if ((rc = retire(i)) != FFTSEG_OK) {
            status = rc;
            can_write = false;
            break;
        }
        int64_t cnt = frames - f0 < chunk_frames ? frames - f0 : chunk_frames;
        const int64_t span = ((cnt - 1) * hop + n) * 8;
        // the halo: the previous chunk (full, so chunk_frames frames) began at
        // frame f0 - chunk_frames; its samples from frame f0 on are this
        // chunk's first n - hop samples
        int64_t have = 0;
        if (prev >= 0 && halo > 0) {
            memcpy(ring.h_in[i], static_cast<const char *>(ring.h_in[prev]) + chunk_frames * hop * 8, (size_t)halo);
            have = halo;
        }
        const double t0 = now_ms();
        const int64_t got = rd(rctx, f0 * hop * 8 + have, static_cast<char *>(ring.h_in[i]) + have, span - have);
        t_read += now_ms() - t0;
        if (got < 0 || got > span - have) {
            status = set_error(FFTSEG_E_IO, "stream: reader failed at input offset %lld",
                               (long long)(f0 * hop * 8 + have));
            break;
        }
        bool ended = false;
        if (got < span - have) {  // the signal is shorter than total_bytes: keep the frames that fit
            const int64_t s = (have + got) / 8;
            cnt = s >= n ? (s - n) / hop + 1 : 0;
            ended = true;
        }
        if (cnt > 0) {
            cudaError_t e;
            const int64_t bytes = ((cnt - 1) * hop + n) * 8;
            if ((e = cudaEventRecord(ring.e0[i], ring.s_h2d)) != cudaSuccess ||
                (e = cudaMemcpyAsync(ring.d_in[i], ring.h_in[i], (size_t)bytes, cudaMemcpyHostToDevice,
                                     ring.s_h2d)) != cudaSuccess ||
                (e = cudaEventRecord(ring.e_h2d[i], ring.s_h2d)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ring.s_comp, ring.e_h2d[i], 0)) != cudaSuccess) {
                status = cuda_error(e, "stream: copy-in");
                can_write = false;
                break;
            }
            if ((rc = exec_plan(p, ring.d_in[i], ring.d_out[i], cnt, ring.s_comp)) != FFTSEG_OK) {
                status = rc;
                can_write = false;
                break;
            }
            if ((e = cudaEventRecord(ring.e_comp[i], ring.s_comp)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ring.s_d2h, ring.e_comp[i], 0)) != cudaSuccess ||
                (e = cudaMemcpyAsync(ring.h_out[i], ring.d_out[i], (size_t)(cnt * frame_out),
                                     cudaMemcpyDeviceToHost, ring.s_d2h)) != cudaSuccess ||
                (e = cudaEventRecord(ring.e_d2h[i], ring.s_d2h)) != cudaSuccess) {
                status = cuda_error(e, "stream: copy-out");
                can_write = false;
                break;
            }
            pend[i].f0 = f0;
            pend[i].cnt = cnt;
            pend[i].live = true;
        }
        prev = i;
        if (ended) {
            ++chunk;
            break;
        }
    }
    // drain in chunk order, as for segment plans
    for (int64_t k = chunk - kRing; k < chunk; ++k) {
        if (k < 0) continue;
        const int i = (int)(k % kRing);
        if (!can_write) {
            if (pend[i].live) cudaEventSynchronize(ring.e_d2h[i]);
            pend[i].live = false;
            continue;
        }
        if ((rc = retire(i)) != FFTSEG_OK) {
            if (status == FFTSEG_OK) status = rc;
            can_write = false;
        }
    }
    cudaStreamSynchronize(ring.s_h2d);
    cudaStreamSynchronize(ring.s_comp);
    cudaStreamSynchronize(ring.s_d2h);
    p->phases[0] = t_read;
    p->phases[1] = t_h2d;
    p->phases[2] = t_comp;
    p->phases[3] = t_d2h;
    p->phases[4] = t_write;
    p->phases[5] = now_ms() - t_start;
    if (committed_offset) *committed_offset = committed_f * hop * 8;
    return status;
}

}  // namespace
}  // namespace fftseg

extern "C" int fftseg_stream_phases(fftseg_plan p, double out[6])
{
    if (!p || !out) return set_error(FFTSEG_E_INVALID, "stream_phases: NULL argument");
    for (int i = 0; i < 6; ++i) out[i] = p->phases[i];
    return FFTSEG_OK;
}
