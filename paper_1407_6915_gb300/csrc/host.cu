// fftseg_exec_host: a batch held in host memory, through a chain of plans.
//
// The paper (Sec. III) copies each block to the GPU, transforms it and copies
// it back, one step after the other.  Here the batch moves in chunks through
// three slots of device staging: chunk c+1 is copied in (copy stream) while
// chunk c runs through the plans (compute stream) and chunk c-1 is copied
// back (a second copy stream), so the host link carries both directions at
// once and the transforms hide behind the copies.  Host buffers are used in
// place: no pinned bounce buffer and no host-side copy.
#include "plan.h"

namespace fftseg {
namespace {

constexpr int kSlots = 3;
constexpr int64_t kDefaultChunkBytes = 256ll << 20;

// Device staging and streams, kept with the first plan of a chain.
struct HostStage {
    int64_t bytes = 0;  // per buffer
    void *d_a[kSlots] = {}, *d_b[kSlots] = {};
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    cudaEvent_t e_in[kSlots] = {}, e_comp[kSlots] = {}, e_out[kSlots] = {};

    ~HostStage()
    {
        for (int i = 0; i < kSlots; ++i) {
            cudaFree(d_a[i]);
            cudaFree(d_b[i]);
            if (e_in[i]) cudaEventDestroy(e_in[i]);
            if (e_comp[i]) cudaEventDestroy(e_comp[i]);
            if (e_out[i]) cudaEventDestroy(e_out[i]);
        }
        if (s_h2d) cudaStreamDestroy(s_h2d);
        if (s_comp) cudaStreamDestroy(s_comp);
        if (s_d2h) cudaStreamDestroy(s_d2h);
    }

    int init(int64_t b)
    {
        bytes = b;
        cudaError_t e;
#define STAGE_CHECK(call, what)                           \
    do {                                                  \
        e = (call);                                       \
        if (e != cudaSuccess) return cuda_error(e, what); \
    } while (0)
        STAGE_CHECK(cudaStreamCreateWithFlags(&s_h2d, cudaStreamNonBlocking), "exec_host: stream create");
        STAGE_CHECK(cudaStreamCreateWithFlags(&s_comp, cudaStreamNonBlocking), "exec_host: stream create");
        STAGE_CHECK(cudaStreamCreateWithFlags(&s_d2h, cudaStreamNonBlocking), "exec_host: stream create");
        for (int i = 0; i < kSlots; ++i) {
            STAGE_CHECK(cudaMalloc(&d_a[i], (size_t)bytes), "exec_host: device staging");
            STAGE_CHECK(cudaMalloc(&d_b[i], (size_t)bytes), "exec_host: device staging");
            STAGE_CHECK(cudaEventCreateWithFlags(&e_in[i], cudaEventDisableTiming), "exec_host: event create");
            STAGE_CHECK(cudaEventCreateWithFlags(&e_comp[i], cudaEventDisableTiming), "exec_host: event create");
            STAGE_CHECK(cudaEventCreateWithFlags(&e_out[i], cudaEventDisableTiming), "exec_host: event create");
        }
#undef STAGE_CHECK
        return FFTSEG_OK;
    }
};

void free_host_stage(void *s) { delete static_cast<HostStage *>(s); }

}  // namespace
}  // namespace fftseg

using namespace fftseg;

extern "C" int fftseg_exec_host(const fftseg_plan *plans, int nplans, const void *h_in, void *h_out, int64_t nseg,
                                int64_t chunk_segments)
{
    if (!plans || nplans < 1) return set_error(FFTSEG_E_INVALID, "exec_host: no plans");
    for (int k = 0; k < nplans; ++k)
        if (!plans[k]) return set_error(FFTSEG_E_INVALID, "exec_host: plan %d is NULL", k);
    const fftseg_plan p0 = plans[0], last = plans[nplans - 1];
    const int64_t n = p0->n;
    int64_t max_batch = p0->batch;
    for (int k = 0; k < nplans; ++k) {
        const fftseg_plan p = plans[k];
        if (p->n != n) return set_error(FFTSEG_E_INVALID, "exec_host: plans of different lengths");
        if (p->path == PATH_REAL || p->path == PATH_FRAMES)
            return set_error(FFTSEG_E_UNSUPPORTED, "exec_host: real-signal and frame plans are not supported here");
        if (p->device != p0->device) return set_error(FFTSEG_E_INVALID, "exec_host: plans on different devices");
        if (k + 1 < nplans && p->out_kind != FFTSEG_OUT_COMPLEX)
            return set_error(FFTSEG_E_INVALID, "exec_host: only the last plan may write the power output");
        if (p->batch < max_batch) max_batch = p->batch;
    }
    if (nseg < 0) return set_error(FFTSEG_E_INVALID, "exec_host: nseg < 0");
    if (nseg == 0) return FFTSEG_OK;
    if (!h_in || !h_out) return set_error(FFTSEG_E_INVALID, "exec_host: NULL buffer");
    if (chunk_segments == 0) {
        chunk_segments = kDefaultChunkBytes / (n * 8);
        if (chunk_segments < 1) chunk_segments = 1;
        if (chunk_segments > max_batch) chunk_segments = max_batch;
    }
    if (chunk_segments < 1 || chunk_segments > max_batch)
        return set_error(FFTSEG_E_INVALID, "exec_host: chunk_segments must be in [1, smallest plan batch]");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "exec_host: cudaGetDevice");
    if (dev != p0->device) return set_error(FFTSEG_E_INVALID, "exec_host: plans belong to another device");

    const int64_t seg_in = n * 8;
    const int64_t seg_out = n * (last->out_kind == FFTSEG_OUT_POWER ? 4 : 8);
    const int64_t bytes = chunk_segments * seg_in;
    HostStage *hs = static_cast<HostStage *>(p0->host_stage);
    if (!hs || hs->bytes < bytes) {
        if (hs) {
            e = cudaDeviceSynchronize();  // nothing of an earlier call is still in flight on the old staging
            if (e != cudaSuccess) return cuda_error(e, "exec_host: synchronize before regrowing staging");
            p0->host_stage_free(p0->host_stage);
            p0->host_stage = nullptr;
        }
        hs = new HostStage();
        const int rc = hs->init(bytes);
        if (rc != FFTSEG_OK) {
            delete hs;
            return rc;
        }
        p0->host_stage = hs;
        p0->host_stage_free = free_host_stage;
    }

    const char *src = static_cast<const char *>(h_in);
    char *dst = static_cast<char *>(h_out);
    const int64_t nchunks = (nseg + chunk_segments - 1) / chunk_segments;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int i = (int)(c % kSlots);
        const int64_t s0 = c * chunk_segments;
        const int64_t segs = nseg - s0 < chunk_segments ? nseg - s0 : chunk_segments;
        // slot i is free once its previous chunk has been copied back
        if (c >= kSlots && (e = cudaStreamWaitEvent(hs->s_h2d, hs->e_out[i], 0)) != cudaSuccess)
            return cuda_error(e, "exec_host: slot wait");
        if ((e = cudaMemcpyAsync(hs->d_a[i], src + s0 * seg_in, (size_t)(segs * seg_in), cudaMemcpyHostToDevice,
                                 hs->s_h2d)) != cudaSuccess ||
            (e = cudaEventRecord(hs->e_in[i], hs->s_h2d)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(hs->s_comp, hs->e_in[i], 0)) != cudaSuccess)
            return cuda_error(e, "exec_host: copy-in");
        void *cur = hs->d_a[i], *nxt = hs->d_b[i];
        for (int k = 0; k < nplans; ++k) {
            const int rc = exec_plan(plans[k], cur, nxt, segs, hs->s_comp);
            if (rc != FFTSEG_OK) return rc;
            void *t = cur;
            cur = nxt;
            nxt = t;
        }
        if ((e = cudaEventRecord(hs->e_comp[i], hs->s_comp)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(hs->s_d2h, hs->e_comp[i], 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dst + s0 * seg_out, cur, (size_t)(segs * seg_out), cudaMemcpyDeviceToHost,
                                 hs->s_d2h)) != cudaSuccess ||
            (e = cudaEventRecord(hs->e_out[i], hs->s_d2h)) != cudaSuccess)
            return cuda_error(e, "exec_host: copy-out");
    }
    e = cudaStreamSynchronize(hs->s_d2h);
    if (e != cudaSuccess) return cuda_error(e, "exec_host: completion");
    return FFTSEG_OK;
}
