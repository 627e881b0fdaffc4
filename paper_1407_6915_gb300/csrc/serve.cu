// Continuous-batching server for segment-FFT jobs (fftsrv_*).
//
// Jobs of any power-of-two length arrive through fftsrv_submit and wait in a
// FIFO.  A scheduler thread admits them, in arrival order, while the bytes of
// the admitted-but-unfinished work (input + output of each job) fit the HBM
// budget and fewer than max_inflight_jobs run; a job too big for the budget is
// admitted in pieces of whole segments.  Each admission round launches:
//  - every admitted job with n <= 4096 in ONE ragged persistent kernel: a
//    device work list of jobs, an atomic tile cursor, and per tile the same
//    tile code as the plain single-pass kernel (so a job's result is bit for
//    bit the same alone, in any mix, and through fftseg_exec).  The round is
//    one CUDA graph (work-list upload, cursor reset, kernel) captured once per
//    slot and replayed; two slots on two streams let consecutive rounds
//    overlap on the device;
//  - every piece of a larger job through a resident plan of its length
//    (cluster or persistent four-step kernels) on one of four more streams
//    (lanes), round-robin, each lane with plans of its own, so that pieces
//    of several large jobs overlap on the device (a caller-given stream is
//    the single lane instead).
// Completion is reported by host callbacks queued behind each launch; they
// release the job's bytes, wake the scheduler and wake fftsrv_poll.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "launch.h"
#include "plan.h"

namespace fftseg {
namespace {

constexpr int kMaxItems = 1024;  // small jobs (pieces) per ragged round
constexpr int kLanes = 4;        // streams for the pieces of large jobs
constexpr int kSmallMaxLog = 12;

struct RaggedItem {
    const float2 *in;
    float2 *out;
    int64_t nseg;
    int64_t tile0;      // first global tile of this job in the round
    const float2 *tw;   // stage tables for n
    int log_n;
    int sign;
    float scale;
    int pad;
};

struct RaggedHeader {
    int64_t njobs;
    int64_t ntiles;
};

constexpr int kRagE = 4096;  // points per tile (BlockShape: 4096 for n >= 16, 256*n below)
constexpr int kRagSlots = 4354;  // >= BlockShape<L>::SLOTS for every L <= 4096
constexpr size_t kRagSmem = (size_t)(kRagE + kRagSlots) * sizeof(float2) + 2 * sizeof(uint64_t) + 4 * sizeof(int64_t);

template <int LL>
FDEV void ragged_tile(const RaggedItem &it, const float2 *P, float2 *X, int64_t u)
{
    constexpr int64_t W = int64_t(1) << BlockShape<LL>::LOG_W;
    if (it.sign < 0)
        block_tile<LL, -1>(P, X, it.tw, u * W, it.nseg, it.out, 0, it.scale, nullptr);
    else
        block_tile<LL, 1>(P, X, it.tw, u * W, it.nseg, it.out, 0, it.scale, nullptr);
}

// Ragged persistent kernel: tiles of all jobs of a round, taken from a cursor.
__global__ void __launch_bounds__(256, 2)
    k_ragged(const RaggedHeader *hdr, const RaggedItem *items, int *cursor, int *err)
{
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;
    float2 *X = sm + kRagE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + kRagSlots);
    int64_t *info = reinterpret_cast<int64_t *>(bar + 2);  // [0] tile, [1] job
    const int tid = threadIdx.x;
    if (smem_u32(P) & 127) {
        if (tid == 0) atomicOr(err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    const int64_t ntiles = hdr->ntiles, njobs = hdr->njobs;
    for (int k = 0;; ++k) {
        __syncthreads();  // the previous tile is done with P, X and info
        if (tid == 0) {
            const int64_t t = atomicAdd(cursor, 1);
            int64_t lo = 0, hi = njobs - 1;  // last job with tile0 <= t
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (items[mid].tile0 <= t) lo = mid;
                else hi = mid - 1;
            }
            info[0] = t;
            info[1] = lo;
            if (t < ntiles) {
                const RaggedItem &it = items[lo];
                const int log_w = it.log_n >= 4 ? 12 - it.log_n : 8;
                const int64_t u = t - it.tile0;
                int64_t segs = it.nseg - (u << log_w);
                if (segs > (int64_t(1) << log_w)) segs = int64_t(1) << log_w;
                const uint32_t bytes = (uint32_t)(segs << it.log_n) * (uint32_t)sizeof(float2);
                fence_proxy_async();
                mbar_expect_tx(bar, bytes);
                tma_load_1d(P, it.in + ((u << log_w) << it.log_n), bytes, bar);
            }
        }
        __syncthreads();
        const int64_t t = info[0];
        if (t >= ntiles) break;
        const RaggedItem it = items[info[1]];
        const int64_t u = t - it.tile0;
        mbar_wait(bar, k & 1, err);
        switch (it.log_n) {
            case 1: ragged_tile<1>(it, P, X, u); break;
            case 2: ragged_tile<2>(it, P, X, u); break;
            case 3: ragged_tile<3>(it, P, X, u); break;
            case 4: ragged_tile<4>(it, P, X, u); break;
            case 5: ragged_tile<5>(it, P, X, u); break;
            case 6: ragged_tile<6>(it, P, X, u); break;
            case 7: ragged_tile<7>(it, P, X, u); break;
            case 8: ragged_tile<8>(it, P, X, u); break;
            case 9: ragged_tile<9>(it, P, X, u); break;
            case 10: ragged_tile<10>(it, P, X, u); break;
            case 11: ragged_tile<11>(it, P, X, u); break;
            case 12: ragged_tile<12>(it, P, X, u); break;
            default: break;
        }
    }
}

int ilog2i(int64_t n)
{
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

}  // namespace
}  // namespace fftseg

using namespace fftseg;

struct fftsrv_s;

namespace {

struct Job {
    fftsrv_job j{};
    int log_n = 0;
    int64_t seg_bytes = 0;   // bytes one segment adds to the budget (input + output)
    int64_t next_seg = 0;    // segments admitted so far
    int pieces_inflight = 0;
    int status = FFTSEG_OK;
    bool admitted = false;
    bool done = false;
    // host clock: fftsrv_submit accepted the job / its last piece was retired
    std::chrono::steady_clock::time_point t_submit{}, t_done{};
};

struct Done {
    fftsrv_s *srv;
    std::vector<std::pair<uint64_t, int64_t>> pieces;  // (job id, bytes)
};

struct Slot {
    RaggedHeader *h_hdr = nullptr;
    RaggedItem *h_items = nullptr;
    RaggedHeader *d_hdr = nullptr;
    RaggedItem *d_items = nullptr;
    int *d_cursor = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    cudaStream_t stream = nullptr;
    bool used = false;
};

void CUDART_CB on_done(void *arg);

}  // namespace

struct fftsrv_s {
    fftsrv_config cfg{};
    int device = 0;
    cudaStream_t s_large[kLanes] = {};
    int nlanes = 1, next_lane = 0;
    bool own_large = false;
    Slot slots[2];
    int next_slot = 0;
    float2 *d_tw = nullptr;  // small-n stage tables, log_n = 1..12
    int64_t tw_off[kSmallMaxLog + 1] = {};
    int *d_err = nullptr;
    std::map<std::pair<int, int>, fftseg_plan> plans;  // (log_n, (direction*4+norm)*kLanes+lane), n > 4096
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Job> jobs;
    int64_t inflight_bytes = 0, peak_bytes = 0;
    int inflight_jobs = 0;
    int64_t submitted = 0, completed = 0, launches = 0;
    int64_t callbacks_pending = 0;
    bool stop = false;
    int fatal = FFTSEG_OK;
    uint64_t next_id = 1;
    std::thread th;

    // Resident plan for length 2^log_n; its batch covers the largest piece any
    // job of that length can be cut into (an in-place job counts n*8 bytes a segment).
    fftseg_plan plan_for(int log_n, int direction, int norm, int lane, int *rc)
    {
        const std::pair<int, int> key(log_n, (direction * 4 + norm) * kLanes + lane);
        auto it = plans.find(key);
        if (it != plans.end()) return it->second;
        fftseg_plan p = nullptr;
        int64_t batch = cfg.hbm_budget_bytes / ((int64_t(1) << log_n) * 8);
        if (batch < 1) batch = 1;
        *rc = fftseg_plan_create(&p, int64_t(1) << log_n, batch, direction, norm, FFTSEG_PREC_FP32,
                                 FFTSEG_OUT_COMPLEX, 0);
        if (*rc == FFTSEG_OK) plans[key] = p;
        return p;
    }

    int64_t max_piece_segs(const Job &jb) const
    {
        int64_t m = cfg.hbm_budget_bytes / jb.seg_bytes;
        return m < 1 ? 1 : m;
    }

    void scheduler();
};

namespace {

void CUDART_CB on_done(void *arg)
{
    Done *d = static_cast<Done *>(arg);
    fftsrv_s *s = d->srv;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        for (auto &pc : d->pieces) {
            s->inflight_bytes -= pc.second;
            auto it = s->jobs.find(pc.first);
            if (it == s->jobs.end()) continue;
            Job &jb = it->second;
            if (--jb.pieces_inflight == 0 && jb.next_seg == jb.j.nseg) {
                jb.done = true;
                jb.t_done = std::chrono::steady_clock::now();
                s->inflight_jobs--;
                s->completed++;
            }
        }
        s->callbacks_pending--;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_all();
    delete d;
}

}  // namespace

void fftsrv_s::scheduler()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
        // admit in arrival order while the budget and the slot count allow
        std::vector<std::pair<uint64_t, std::pair<int64_t, int64_t>>> small, large;  // id, (seg0, count)
        while (!pending.empty() && (int)small.size() < kMaxItems) {
            Job &jb = jobs[pending.front()];
            if (!jb.admitted && inflight_jobs >= cfg.max_inflight_jobs) break;
            const int64_t left = jb.j.nseg - jb.next_seg;
            int64_t cnt = (cfg.hbm_budget_bytes - inflight_bytes) / jb.seg_bytes;
            if (cnt > left) cnt = left;
            if (cnt > max_piece_segs(jb)) cnt = max_piece_segs(jb);
            if (cnt < 1) break;
            if (!jb.admitted) {
                jb.admitted = true;
                inflight_jobs++;
            }
            const uint64_t id = pending.front();
            (jb.log_n <= kSmallMaxLog ? small : large).push_back({id, {jb.next_seg, cnt}});
            jb.next_seg += cnt;
            jb.pieces_inflight++;
            inflight_bytes += cnt * jb.seg_bytes;
            if (inflight_bytes > peak_bytes) peak_bytes = inflight_bytes;
            if (jb.next_seg == jb.j.nseg) pending.pop_front();
        }
        if (small.empty() && large.empty()) {
            if (stop && pending.empty() && inflight_jobs == 0 && callbacks_pending == 0) break;
            cv_sched.wait(lock);
            continue;
        }
        // copy what the launches need, then launch without holding the lock
        std::vector<Job> snap_small, snap_large;
        for (auto &x : small) snap_small.push_back(jobs[x.first]);
        for (auto &x : large) snap_large.push_back(jobs[x.first]);
        lock.unlock();

        std::vector<std::pair<uint64_t, int64_t>> failed;  // pieces never handed to the device
        int rc = FFTSEG_OK;
        auto hand_over = [&](cudaStream_t st, Done *d) {  // queue the completion callback
            {
                std::lock_guard<std::mutex> g(mu);
                callbacks_pending++;
            }
            cudaError_t e = cudaLaunchHostFunc(st, on_done, d);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> g(mu);
                callbacks_pending--;
                rc = cuda_error(e, "server: completion callback");
                failed.insert(failed.end(), d->pieces.begin(), d->pieces.end());
                delete d;
            }
        };
        if (!small.empty()) {
            Slot &sl = slots[next_slot];
            next_slot ^= 1;
            if (sl.used) cudaEventSynchronize(sl.done);  // its host buffers are free again
            sl.used = true;
            Done *d = new Done{this, {}};
            int64_t tiles = 0;
            for (size_t i = 0; i < small.size(); ++i) {
                const Job &jb = snap_small[i];
                const int64_t seg0 = small[i].second.first, cnt = small[i].second.second;
                RaggedItem &it = sl.h_items[i];
                const int64_t n = int64_t(1) << jb.log_n;
                it.in = static_cast<const float2 *>(jb.j.d_in) + seg0 * n;
                it.out = static_cast<float2 *>(jb.j.d_out) + seg0 * n;
                it.nseg = cnt;
                it.tile0 = tiles;
                it.tw = d_tw + tw_off[jb.log_n];
                it.log_n = jb.log_n;
                it.sign = jb.j.direction;
                it.scale = jb.j.norm == FFTSEG_NORM_BACKWARD ? (jb.j.direction == FFTSEG_INVERSE ? (float)(1.0 / n) : 1.f)
                           : jb.j.norm == FFTSEG_NORM_ORTHO ? (float)(1.0 / sqrt((double)n))
                                                             : 1.f;
                it.pad = 0;
                const int log_w = jb.log_n >= 4 ? 12 - jb.log_n : 8;
                tiles += (cnt + (int64_t(1) << log_w) - 1) >> log_w;
                d->pieces.push_back({small[i].first, cnt * jb.seg_bytes});
            }
            sl.h_hdr->njobs = (int64_t)small.size();
            sl.h_hdr->ntiles = tiles;
            cudaError_t e = cudaGraphLaunch(sl.exec, sl.stream);
            if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
            if (e != cudaSuccess) {
                rc = cuda_error(e, "server: ragged round launch");
                failed.insert(failed.end(), d->pieces.begin(), d->pieces.end());
                delete d;
            } else {
                count_launches(1);
                {
                    std::lock_guard<std::mutex> g(mu);
                    launches++;
                }
                hand_over(sl.stream, d);
            }
        }
        for (size_t i = 0; i < large.size(); ++i) {
            const Job &jb = snap_large[i];
            const int64_t seg0 = large[i].second.first, cnt = large[i].second.second;
            const std::pair<uint64_t, int64_t> piece(large[i].first, cnt * jb.seg_bytes);
            if (rc != FFTSEG_OK) {
                failed.push_back(piece);
                continue;
            }
            const int64_t n = int64_t(1) << jb.log_n;
            const int lane = next_lane;
            next_lane = (next_lane + 1) % nlanes;
            fftseg_plan p = plan_for(jb.log_n, jb.j.direction, jb.j.norm, lane, &rc);
            const int64_t before = fftseg_launch_count();
            if (rc == FFTSEG_OK)
                rc = exec_plan(p, static_cast<const float2 *>(jb.j.d_in) + seg0 * n,
                               static_cast<float2 *>(jb.j.d_out) + seg0 * n, cnt, s_large[lane]);
            if (rc != FFTSEG_OK) {
                failed.push_back(piece);
                continue;
            }
            {
                std::lock_guard<std::mutex> g(mu);
                launches += fftseg_launch_count() - before;
            }
            hand_over(s_large[lane], new Done{this, {piece}});
        }
        lock.lock();
        if (!failed.empty()) {  // their jobs end with the error; their bytes are released
            fatal = rc;
            for (auto &pc : failed) {
                inflight_bytes -= pc.second;
                auto it = jobs.find(pc.first);
                if (it == jobs.end()) continue;
                Job &jb = it->second;
                jb.status = rc;
                if (--jb.pieces_inflight == 0 && !jb.done) {
                    jb.done = true;
                    jb.t_done = std::chrono::steady_clock::now();
                    inflight_jobs--;
                    completed++;
                }
            }
            cv_done.notify_all();
        }
    }
}

extern "C" {

int fftsrv_create(fftsrv *out, const fftsrv_config *cfg)
{
    if (!out || !cfg) return set_error(FFTSEG_E_INVALID, "fftsrv_create: NULL argument");
    *out = nullptr;
    if (cfg->hbm_budget_bytes < (int64_t)(1 << 20) || cfg->max_inflight_jobs < 1)
        return set_error(FFTSEG_E_INVALID, "fftsrv_create: budget must be >= 1 MiB and max_inflight_jobs >= 1");
    fftsrv_s *s = new (std::nothrow) fftsrv_s();
    if (!s) return set_error(FFTSEG_E_NOMEM, "fftsrv_create: host allocation");
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    int rc = FFTSEG_OK;
#define SRV_CHECK(call, what)                          \
    do {                                               \
        if (e == cudaSuccess) e = (call);              \
        if (e != cudaSuccess && rc == FFTSEG_OK) rc = cuda_error(e, what); \
    } while (0)
    if (cfg->stream) {
        s->s_large[0] = reinterpret_cast<cudaStream_t>(cfg->stream);
        s->nlanes = 1;
    } else {
        for (int i = 0; i < kLanes; ++i)
            SRV_CHECK(cudaStreamCreateWithFlags(&s->s_large[i], cudaStreamNonBlocking), "fftsrv_create: stream");
        s->nlanes = kLanes;
        s->own_large = true;
    }
    // small-n stage tables
    std::vector<float2> all, h;
    for (int l = 1; l <= kSmallMaxLog; ++l) {
        stage_table_host(h, int64_t(1) << l);
        s->tw_off[l] = (int64_t)all.size();
        all.insert(all.end(), h.begin(), h.end());
    }
    SRV_CHECK(cudaMalloc((void **)&s->d_tw, all.size() * sizeof(float2)), "fftsrv_create: tables");
    SRV_CHECK(cudaMemcpy(s->d_tw, all.data(), all.size() * sizeof(float2), cudaMemcpyHostToDevice),
              "fftsrv_create: tables");
    SRV_CHECK(cudaMalloc((void **)&s->d_err, sizeof(int)), "fftsrv_create: flag");
    SRV_CHECK(cudaMemset(s->d_err, 0, sizeof(int)), "fftsrv_create: flag");
    SRV_CHECK(cudaFuncSetAttribute(k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRagSmem),
              "fftsrv_create: kernel attribute");
    int per_sm = 0;
    SRV_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ragged, 256, kRagSmem), "fftsrv_create: occupancy");
    const int grid = (per_sm > 0 ? per_sm : 1) * device_sm_count();
    for (int i = 0; i < 2 && rc == FFTSEG_OK; ++i) {
        Slot &sl = s->slots[i];
        SRV_CHECK(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "fftsrv_create: stream");
        SRV_CHECK(cudaHostAlloc((void **)&sl.h_hdr, sizeof(RaggedHeader), cudaHostAllocDefault), "fftsrv_create: pinned");
        SRV_CHECK(cudaHostAlloc((void **)&sl.h_items, kMaxItems * sizeof(RaggedItem), cudaHostAllocDefault),
                  "fftsrv_create: pinned");
        SRV_CHECK(cudaMalloc((void **)&sl.d_hdr, sizeof(RaggedHeader)), "fftsrv_create: work list");
        SRV_CHECK(cudaMalloc((void **)&sl.d_items, kMaxItems * sizeof(RaggedItem)), "fftsrv_create: work list");
        SRV_CHECK(cudaMalloc((void **)&sl.d_cursor, sizeof(int)), "fftsrv_create: cursor");
        SRV_CHECK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "fftsrv_create: event");
        if (rc != FFTSEG_OK) break;
        // one ragged round as a graph: upload the work list, reset the cursor, run
        SRV_CHECK(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal), "fftsrv_create: capture");
        SRV_CHECK(cudaMemcpyAsync(sl.d_hdr, sl.h_hdr, sizeof(RaggedHeader), cudaMemcpyHostToDevice, sl.stream),
                  "fftsrv_create: capture");
        SRV_CHECK(cudaMemcpyAsync(sl.d_items, sl.h_items, kMaxItems * sizeof(RaggedItem), cudaMemcpyHostToDevice,
                                  sl.stream),
                  "fftsrv_create: capture");
        SRV_CHECK(cudaMemsetAsync(sl.d_cursor, 0, sizeof(int), sl.stream), "fftsrv_create: capture");
        if (e == cudaSuccess) {
            k_ragged<<<grid, 256, kRagSmem, sl.stream>>>(sl.d_hdr, sl.d_items, sl.d_cursor, s->d_err);
            e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_error(e, "fftsrv_create: capture");
        }
        cudaError_t e2 = cudaStreamEndCapture(sl.stream, &sl.graph);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess && rc == FFTSEG_OK) rc = cuda_error(e, "fftsrv_create: capture");
        SRV_CHECK(cudaGraphInstantiate(&sl.exec, sl.graph, 0), "fftsrv_create: graph");
    }
#undef SRV_CHECK
    if (rc != FFTSEG_OK) {
        fftsrv_destroy(s);
        return rc;
    }
    s->th = std::thread([s] { s->scheduler(); });
    *out = s;
    return FFTSEG_OK;
}

int fftsrv_submit(fftsrv s, const fftsrv_job *job, uint64_t *job_id)
{
    if (!s || !job || !job_id) return set_error(FFTSEG_E_INVALID, "fftsrv_submit: NULL argument");
    const int64_t n = job->n;
    if (n < 2 || (n & (n - 1)) || n > (int64_t(1) << FFTSEG_MAX_LOG2N))
        return set_error(FFTSEG_E_UNSUPPORTED, "fftsrv_submit: n must be a power of two in [2, 2^24]");
    if (job->nseg < 1 || !job->d_in || !job->d_out) return set_error(FFTSEG_E_INVALID, "fftsrv_submit: bad job");
    if (((uintptr_t)job->d_in & 15) || ((uintptr_t)job->d_out & 15))
        return set_error(FFTSEG_E_INVALID, "fftsrv_submit: buffers must be 16-byte aligned");
    if (job->direction != FFTSEG_FORWARD && job->direction != FFTSEG_INVERSE)
        return set_error(FFTSEG_E_INVALID, "fftsrv_submit: bad direction");
    if (job->norm < FFTSEG_NORM_NONE || job->norm > FFTSEG_NORM_ORTHO)
        return set_error(FFTSEG_E_INVALID, "fftsrv_submit: bad norm");
    Job jb;
    jb.t_submit = std::chrono::steady_clock::now();
    jb.j = *job;
    jb.log_n = ilog2i(n);
    jb.seg_bytes = n * 8 * (job->d_in == job->d_out ? 1 : 2);
    if (jb.seg_bytes > s->cfg.hbm_budget_bytes)
        return set_error(FFTSEG_E_INVALID, "fftsrv_submit: one segment exceeds the HBM budget");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return set_error(FFTSEG_E_INVALID, "fftsrv_submit: server is shutting down");
        const uint64_t id = s->next_id++;
        s->jobs[id] = jb;
        s->pending.push_back(id);
        s->submitted++;
        *job_id = id;
    }
    s->cv_sched.notify_all();
    return FFTSEG_OK;
}

int fftsrv_poll(fftsrv s, uint64_t job_id, int64_t timeout_us, int *job_status)
{
    return fftsrv_poll_latency(s, job_id, timeout_us, job_status, nullptr);
}

int fftsrv_poll_latency(fftsrv s, uint64_t job_id, int64_t timeout_us, int *job_status, double *latency_us)
{
    if (!s || !job_status) return set_error(FFTSEG_E_INVALID, "fftsrv_poll: NULL argument");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(FFTSEG_E_INVALID, "fftsrv_poll: unknown job %llu", (unsigned long long)job_id);
    if (!it->second.done && timeout_us > 0) {
        s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), [&] {
            auto j = s->jobs.find(job_id);
            return j == s->jobs.end() || j->second.done;
        });
        it = s->jobs.find(job_id);
        if (it == s->jobs.end()) return set_error(FFTSEG_E_INVALID, "fftsrv_poll: unknown job");
    }
    if (!it->second.done) return set_error(FFTSEG_E_TIMEOUT, "fftsrv_poll: job %llu still queued or running",
                                           (unsigned long long)job_id);
    *job_status = it->second.status;
    if (latency_us)
        *latency_us = std::chrono::duration<double, std::micro>(it->second.t_done - it->second.t_submit).count();
    s->jobs.erase(it);  // a finished job is reported once
    return FFTSEG_OK;
}

int fftsrv_stats(fftsrv s, int64_t out[5])
{
    if (!s || !out) return set_error(FFTSEG_E_INVALID, "fftsrv_stats: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = s->submitted;
    out[1] = s->completed;
    out[2] = s->launches;
    out[3] = s->peak_bytes;
    out[4] = (int64_t)s->pending.size();
    return FFTSEG_OK;
}

int fftsrv_destroy(fftsrv s)
{
    if (!s) return set_error(FFTSEG_E_INVALID, "fftsrv_destroy: NULL server");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable()) s->th.join();  // drains every queued job first
    int rc = s->fatal;
    for (int i = 0; i < 2; ++i) {
        Slot &sl = s->slots[i];
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        if (sl.graph) cudaGraphDestroy(sl.graph);
        if (sl.done) cudaEventDestroy(sl.done);
        cudaFreeHost(sl.h_hdr);
        cudaFreeHost(sl.h_items);
        cudaFree(sl.d_hdr);
        cudaFree(sl.d_items);
        cudaFree(sl.d_cursor);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (int i = 0; i < kLanes; ++i)
        if (s->s_large[i]) cudaStreamSynchronize(s->s_large[i]);
    for (auto &kv : s->plans) fftseg_plan_destroy(kv.second);
    for (int i = 0; i < kLanes; ++i)
        if (s->own_large && s->s_large[i]) cudaStreamDestroy(s->s_large[i]);
    cudaFree(s->d_tw);
    cudaFree(s->d_err);
    delete s;
    return rc;
}

}  // extern "C"
