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

    int init(int64_t segs, int64_t seg_in, int64_t seg_out)
    {
        chunk_segs = segs;
        in_bytes = segs * seg_in;
        out_bytes = segs * seg_out;
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

}  // namespace
}  // namespace fftseg

using namespace fftseg;

extern "C" int fftseg_stream(fftseg_plan p, fftseg_read_fn rd, void *rctx, fftseg_write_fn wr, void *wctx,
                             int64_t total_bytes, int64_t start_offset, int64_t chunk_segments,
                             int64_t *committed_offset)
{
    if (committed_offset) *committed_offset = start_offset;
    if (!p || !rd || !wr) return set_error(FFTSEG_E_INVALID, "stream: NULL plan or callback");
    if (p->path == PATH_REAL || p->path == PATH_FRAMES)
        return set_error(FFTSEG_E_UNSUPPORTED, "stream: real-signal and frame plans are not streamed");
    const int64_t seg_in = p->n * 8;
    const int64_t seg_out = p->n * (p->out_kind == FFTSEG_OUT_POWER ? 4 : 8);
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
        const int64_t got = rd(rctx, offset, ring.h_in[i], want);
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
                (e = cudaMemcpyAsync(ring.d_in[i], ring.h_in[i], (size_t)bytes, cudaMemcpyHostToDevice,
                                     ring.s_h2d)) != cudaSuccess ||
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

extern "C" int fftseg_stream_phases(fftseg_plan p, double out[6])
{
    if (!p || !out) return set_error(FFTSEG_E_INVALID, "stream_phases: NULL argument");
    for (int i = 0; i < 6; ++i) out[i] = p->phases[i];
    return FFTSEG_OK;
}
