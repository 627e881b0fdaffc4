// Autotuner: where more than one schedule is built for a length (cluster
// sizes, the persistent four-step with or without a producer warp, the
// two-pass form), time each on the current GPU and keep the fastest.
//
// A choice is keyed by (GPU name, SM count, log2 n, precision, output kind,
// tuning batch) and kept for the life of the process; if FFTSEG_TUNE_CACHE
// names a file, choices are read from it on first use and new ones appended,
// one line each:
//   <gpu name, spaces as '_'> <SMs> <log2 n> <precision> <out kind> <segments> <flags, hex> <ms>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace fftseg {
namespace {

constexpr int64_t kTuneBytes = 256ll << 20;  // input bytes of one timed exec, at most
constexpr int kTuneWarm = 2, kTuneReps = 5;

std::mutex g_tune_mu;
std::map<std::string, std::pair<unsigned, double>> g_tune;
bool g_tune_loaded = false;

std::string gpu_tag(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown 0";
    std::string name = prop.name;
    for (char &c : name)
        if (c == ' ' || c == '\t') c = '_';
    return name + " " + std::to_string(prop.multiProcessorCount);
}

std::string tune_key(const std::string &gpu, int log_n, int prec, int out_kind, int64_t segs)
{
    return gpu + " " + std::to_string(log_n) + " " + std::to_string(prec) + " " + std::to_string(out_kind) + " " +
           std::to_string((long long)segs);
}

void load_cache_file()  // with g_tune_mu held
{
    g_tune_loaded = true;
    const char *path = getenv("FFTSEG_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char name[256];
    int sms, log_n, prec, out;
    long long segs;
    unsigned flags;
    double ms;
    while (fscanf(f, "%255s %d %d %d %d %lld %x %lf", name, &sms, &log_n, &prec, &out, &segs, &flags, &ms) == 8) {
        const std::string gpu = std::string(name) + " " + std::to_string(sms);
        g_tune[tune_key(gpu, log_n, prec, out, segs)] = {flags & kPathFlags, ms};
    }
    fclose(f);
}

void append_cache_file(const std::string &key, unsigned flags, double ms)  // with g_tune_mu held
{
    const char *path = getenv("FFTSEG_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %x %.6f\n", key.c_str(), flags, ms);
    fclose(f);
}

// The schedules built for this length and precision, as plan flags.
std::vector<unsigned> candidates(int log_n, int prec)
{
    std::vector<unsigned> c;
    if (prec != FFTSEG_PREC_FP32 || log_n <= 12) {  // one schedule per size
        c.push_back(0);
        return c;
    }
    for (int lc = 1; lc <= 4; ++lc) {
        int l1, l2, got;
        if (log_n <= 17 && cluster_shape(log_n, lc, &l1, &l2, &got) && got == lc)
            c.push_back(FFTSEG_FLAG_CLUSTER_LOG2(lc));
    }
    if (log_n >= 14) {
        c.push_back(FFTSEG_FLAG_FOURSTEP_L2);  // the lane- or warp-line kernel where one applies
        c.push_back(FFTSEG_FLAG_FOURSTEP_L2 | FFTSEG_FLAG_FOURSTEP_PRODUCER);
        c.push_back(FFTSEG_FLAG_FOURSTEP_L2 | FFTSEG_FLAG_FOURSTEP_TILES);
        if (log_n == 16) c.push_back(FFTSEG_FLAG_FOURSTEP_L2 | FFTSEG_FLAG_FOURSTEP_WARP_LINES);
    }
    c.push_back(FFTSEG_FLAG_FORCE_TWOPASS);
    return c;
}

// Mean time of one exec of `segs` segments with these flags, or < 0 if the
// schedule is not built or did not run cleanly.
double time_schedule(int64_t n, int64_t segs, int prec, int out_kind, unsigned flags, void *din, void *dout,
                     cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    fftseg_plan p = nullptr;
    if (fftseg_plan_create(&p, n, segs, FFTSEG_FORWARD, FFTSEG_NORM_NONE, prec, out_kind, flags) != FFTSEG_OK)
        return -1.0;
    double ms = -1.0;
    bool ok = true;
    for (int i = 0; i < kTuneWarm && ok; ++i) ok = exec_plan(p, din, dout, segs, st) == FFTSEG_OK;
    ok = ok && cudaEventRecord(e0, st) == cudaSuccess;
    for (int i = 0; i < kTuneReps && ok; ++i) ok = exec_plan(p, din, dout, segs, st) == FFTSEG_OK;
    ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
    float t = 0.f;
    if (ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && fftseg_plan_check(p) == FFTSEG_OK)
        ms = (double)t / kTuneReps;
    fftseg_plan_destroy(p);
    return ms;
}

}  // namespace

int tune_schedule(int64_t n, int64_t batch, int prec, int out_kind, unsigned *flags_out, double *ms_out)
{
    int log_n = 0;
    while ((int64_t(1) << log_n) < n) ++log_n;
    int64_t segs = kTuneBytes / (n * 8);
    if (segs < 1) segs = 1;
    if (segs > batch) segs = batch;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "autotune: cudaGetDevice");
    const std::string key = tune_key(gpu_tag(dev), log_n, prec, out_kind, segs);
    std::lock_guard<std::mutex> lock(g_tune_mu);  // one tuning at a time: timings must not overlap
    if (!g_tune_loaded) load_cache_file();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
        *flags_out = it->second.first;
        if (ms_out) *ms_out = it->second.second;
        return FFTSEG_OK;
    }
    const std::vector<unsigned> cand = candidates(log_n, prec);
    unsigned best = cand[0];
    double best_ms = -1.0;
    if (cand.size() > 1) {
        void *din = nullptr, *dout = nullptr;
        cudaStream_t st = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        const size_t bytes = (size_t)(segs * n * 8);
        e = cudaMalloc(&din, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&dout, bytes);
        if (e == cudaSuccess) e = cudaMemset(din, 0, bytes);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) {
            for (unsigned f : cand) {
                const double ms = time_schedule(n, segs, prec, out_kind, f, din, dout, st, e0, e1);
                if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
                    best_ms = ms;
                    best = f;
                }
            }
        }
        if (e1) cudaEventDestroy(e1);
        if (e0) cudaEventDestroy(e0);
        if (st) cudaStreamDestroy(st);
        cudaFree(dout);
        cudaFree(din);
        if (e != cudaSuccess) return cuda_error(e, "autotune: scratch");
        if (best_ms < 0) return set_error(FFTSEG_E_CUDA, "autotune: no schedule ran for n=%lld", (long long)n);
    }
    g_tune[key] = {best, best_ms};
    if (best_ms >= 0) append_cache_file(key, best, best_ms);
    *flags_out = best;
    if (ms_out) *ms_out = best_ms;
    return FFTSEG_OK;
}

}  // namespace fftseg

using namespace fftseg;

extern "C" int fftseg_autotune(int64_t n, int64_t batch, int precision, int out_kind, unsigned *flags_out,
                               double *ms_out)
{
    if (!flags_out) return set_error(FFTSEG_E_INVALID, "autotune: flags_out is NULL");
    if (n < 2 || n > (int64_t(1) << FFTSEG_MAX_LOG2N) || (n & (n - 1)))
        return set_error(FFTSEG_E_UNSUPPORTED, "autotune: n=%lld is not a power of two in [2, 2^24]", (long long)n);
    if (batch < 1) return set_error(FFTSEG_E_INVALID, "autotune: batch must be >= 1");
    if (precision < FFTSEG_PREC_FP32 || precision > FFTSEG_PREC_TC_BF16)
        return set_error(FFTSEG_E_INVALID, "autotune: bad precision %d", precision);
    if (out_kind != FFTSEG_OUT_COMPLEX && out_kind != FFTSEG_OUT_POWER)
        return set_error(FFTSEG_E_INVALID, "autotune: bad out_kind %d", out_kind);
    return tune_schedule(n, batch, precision, out_kind, flags_out, ms_out);
}
