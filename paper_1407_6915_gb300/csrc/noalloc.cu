// fftseg_exec_noalloc: the persistent four-step transform without any device
// allocation.  Its scratch (the L2 ring, the chunk counters and the twiddle
// tables) lives in one file-scope __device__ array that exists on every GPU
// that loads this library, for as long as the process runs.
#include <math.h>

#include <mutex>

#include "fourstep.cuh"
#include "launch.h"
#include "plan.h"

namespace fftseg {
namespace {

constexpr int kNaMinLogN = 17, kNaMaxLogN = 20;
constexpr int64_t kNaChunkBytes = 8ll << 20;                      // one ring chunk
constexpr int kNaRing = 3;                                         // chunks in the ring
constexpr int64_t kNaRingElems = kNaRing * kNaChunkBytes / 8;      // float2 elements
constexpr int64_t kNaW4Elems = int64_t(1) << 16;                   // [j2][k1 mod K] (2^15 used at n = 2^20)
constexpr int64_t kNaW4hiElems = int64_t(1) << 16;                 // [j2][k1 div K] (2^15 used at n = 2^20)
constexpr int64_t kNaStageElems = 1024;                            // stage tables of one line (< 1024 entries)
constexpr int kNaMaxChunks = 65536;                                // chunks per launch
constexpr int64_t kNaCtrElems = (1 + 2 * (int64_t)kNaMaxChunks + 1 + 1) / 2;  // counters + flag, as float2 slots

constexpr int64_t kNaOffRing = 0;
constexpr int64_t kNaOffW4 = kNaOffRing + kNaRingElems;
constexpr int64_t kNaOffW4hi = kNaOffW4 + kNaW4Elems;
constexpr int64_t kNaOffStageA = kNaOffW4hi + kNaW4hiElems;
constexpr int64_t kNaOffStageB = kNaOffStageA + kNaStageElems;
constexpr int64_t kNaOffCtr = kNaOffStageB + kNaStageElems;
constexpr int64_t kNaElems = kNaOffCtr + kNaCtrElems;

}  // namespace
}  // namespace fftseg

// 8 B * (3 Mi + 128 Ki + 2 Ki + 64 Ki) elements = about 25.5 MiB per GPU.
static __device__ __align__(256) float2 g_noalloc_scratch[fftseg::kNaElems];

namespace fftseg {
namespace {

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 64;
float2 *g_na_base[kNaMaxDevices] = {};  // device address of g_noalloc_scratch, per device
int g_na_table_logn[kNaMaxDevices] = {};  // n whose tables the array holds (0: none)

// w_M^e = exp(-2 pi i e / M), evaluated in double and rounded once to float
__device__ float2 root_fwd(int64_t e, int64_t M)
{
    double s, c;
    sincospi(2.0 * (double)(e % M) / (double)M, &s, &c);
    return make_float2((float)c, (float)-s);
}

// Stage tables of a length-L line in the layout the kernels read (see
// stage_table_offset): stage s >= 1, radix R, Ns = 16^s: [r-1][m] = w_{Ns R}^{m r}.
__device__ void stage_entry(float2 *tab, int log_l, int idx)
{
    int off = 0;
    for (int s = 1;; ++s) {
        const int lr = s < log_l / 4 ? 4 : log_l % 4;
        if (lr == 0 || 4 * s >= log_l) return;
        const int ns = 1 << (4 * s), size = ((1 << lr) - 1) * ns;
        if (idx < off + size) {
            const int k = idx - off, r = 1 + k / ns, m = k % ns;
            tab[idx] = root_fwd((int64_t)m * r, (int64_t)ns << lr);
            return;
        }
        off += size;
    }
}

// Four-step factor tables (w_n^{j2 k1} = lo[j2][k1 mod K] * hi[j2][k1 div K])
// and the stage tables of both line lengths.
__global__ void k_noalloc_tables(float2 *scratch, int log_n1, int log_n2)
{
    const int log_k = fourstep_log_k(log_n1);
    const int64_t n1 = int64_t(1) << log_n1, n2 = int64_t(1) << log_n2, n = n1 * n2;
    const int64_t K = int64_t(1) << log_k, nhi = n1 >> log_k;
    float2 *lo = scratch + kNaOffW4, *hi = scratch + kNaOffW4hi;
    const int64_t count = n2 * (K > nhi ? K : nhi);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count || e < kNaStageElems;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < n2 * K) lo[e] = root_fwd((e >> log_k) * (e & (K - 1)), n);
        if (e < n2 * nhi) hi[e] = root_fwd((e / nhi) * K * (e % nhi), n);
        if (e < kNaStageElems) {
            stage_entry(scratch + kNaOffStageA, log_n1, (int)e);
            stage_entry(scratch + kNaOffStageB, log_n2, (int)e);
        }
    }
}

}  // namespace
}  // namespace fftseg

using namespace fftseg;

extern "C" int fftseg_exec_noalloc(const void *d_in, void *d_out, int64_t n, int64_t nseg, int direction, int norm,
                                   fftseg_stream_t stream)
{
    int log_n = 0;
    while (log_n < 62 && (int64_t(1) << log_n) < n) ++log_n;
    if (n <= 0 || (int64_t(1) << log_n) != n || log_n < kNaMinLogN || log_n > kNaMaxLogN)
        return set_error(FFTSEG_E_UNSUPPORTED,
                         "exec_noalloc: n=%lld is outside what its fixed scratch holds (powers of two 2^17..2^20)",
                         (long long)n);
    if (nseg < 0) return set_error(FFTSEG_E_INVALID, "exec_noalloc: nseg < 0");
    if (direction != FFTSEG_FORWARD && direction != FFTSEG_INVERSE)
        return set_error(FFTSEG_E_INVALID, "exec_noalloc: direction must be -1 or +1");
    if (norm < FFTSEG_NORM_NONE || norm > FFTSEG_NORM_ORTHO)
        return set_error(FFTSEG_E_INVALID, "exec_noalloc: bad norm %d", norm);
    if (nseg == 0) return FFTSEG_OK;
    if (!d_in || !d_out) return set_error(FFTSEG_E_INVALID, "exec_noalloc: NULL buffer");
    if (((uintptr_t)d_in & 15) || ((uintptr_t)d_out & 15))
        return set_error(FFTSEG_E_INVALID, "exec_noalloc: buffers must be 16-byte aligned");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "exec_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(FFTSEG_E_INVALID, "exec_noalloc: device %d", dev);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    int l1, l2, lwa, lwb;
    fourstep_shape(log_n, &l1, &l2, &lwa, &lwb);
    float2 *base;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_base[dev]) {  // first call on this device (it is current): find the array
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) return cuda_error(e, "exec_noalloc: cudaGetSymbolAddress");
            g_na_base[dev] = static_cast<float2 *>(ptr);
        }
        base = g_na_base[dev];
        if (g_na_table_logn[dev] != log_n) {  // tables of another length: recompute them on the device
            k_noalloc_tables<<<1024, 256, 0, st>>>(base, l1, l2);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_error(e, "exec_noalloc: table kernel launch");
            count_launches(1);
            g_na_table_logn[dev] = log_n;
        }
    }

    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    int64_t cs = kNaChunkBytes / (n * 8);
    if (cs < 1) cs = 1;
    const int64_t per_launch = (int64_t)kNaMaxChunks * cs;
    float scale = 1.f;
    if (norm == FFTSEG_NORM_BACKWARD) scale = direction == FFTSEG_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    else if (norm == FFTSEG_NORM_ORTHO) scale = (float)(1.0 / sqrt((double)n));
    int *ctr = reinterpret_cast<int *>(base + kNaOffCtr);
    for (int64_t s0 = 0; s0 < nseg; s0 += per_launch) {
        const int64_t cnt = nseg - s0 < per_launch ? nseg - s0 : per_launch;
        const int64_t nc = (cnt + cs - 1) / cs;
        FourStepArgs a{};
        const float2 *in = static_cast<const float2 *>(d_in) + s0 * n;
        const uint32_t boxa = (uint32_t)(n1 < 256 ? n1 : 256), boxb = (uint32_t)(n2 < 256 ? n2 : 256);
        int rc = encode_tmap_3d(&a.tmA, in, n2, n1, cnt, n2 * 8, n * 8, 1u << lwa, boxa);
        if (rc != FFTSEG_OK) return rc;
        rc = encode_tmap_3d(&a.tmB, base + kNaOffRing, n1, n2, kNaRing * cs, n1 * 8, n * 8, 1u << lwb, boxb);
        if (rc != FFTSEG_OK) return rc;
        a.out = static_cast<float2 *>(d_out) + s0 * n;
        a.ring = base + kNaOffRing;
        a.twA = base + kNaOffStageA;
        a.twB = base + kNaOffStageB;
        a.w4 = base + kNaOffW4;
        a.w4hi = base + kNaOffW4hi;
        a.ctr = ctr;
        a.err = ctr + 1 + 2 * kNaMaxChunks;
        a.nseg = cnt;
        a.nchunks = (int)nc;
        a.cs = (int)cs;
        a.nr = kNaRing;
        a.log_k = fourstep_log_k(l1);
        a.out_power = 0;
        a.scale = scale;
        e = cudaMemsetAsync(ctr, 0, (size_t)(1 + 2 * nc) * sizeof(int), st);  // queue head and chunk counters
        if (e != cudaSuccess) return cuda_error(e, "exec_noalloc: counter reset");
        e = launch_fourstep(log_n, direction, PREC_FP32, a, st);
        if (e != cudaSuccess) return cuda_error(e, "exec_noalloc: kernel launch");
        count_launches(1);
    }
    return FFTSEG_OK;
}

// Reads and clears the give-up flag that fftseg_exec_noalloc's kernels set on
// the current device (a slot of the same fixed array): FFTSEG_E_TIMEOUT if any
// call since the last check gave up a bounded wait, FFTSEG_OK otherwise.
extern "C" int fftseg_noalloc_check(void)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "noalloc_check: cudaGetDevice");
    if (dev < 0 || dev >= kNaMaxDevices) return set_error(FFTSEG_E_INVALID, "noalloc_check: device %d", dev);
    float2 *base;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        base = g_na_base[dev];
    }
    if (!base) return FFTSEG_OK;  // no call has run on this device
    int *flag = reinterpret_cast<int *>(base + kNaOffCtr) + 1 + 2 * kNaMaxChunks;
    int v = 0;
    e = cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost);  // waits for the device
    if (e != cudaSuccess) return cuda_error(e, "noalloc_check: read flag");
    if (v) {
        e = cudaMemset(flag, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_error(e, "noalloc_check: clear flag");
        return set_error(FFTSEG_E_TIMEOUT,
                         "exec_noalloc: a kernel gave up (flag %d): a bounded wait ran out or a shared buffer was "
                         "misaligned; the outputs of the calls since the last check are not valid",
                         v);
    }
    return FFTSEG_OK;
}
