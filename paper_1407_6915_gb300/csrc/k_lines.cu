// Instantiations and launchers of k_lines: the single-pass block kernel
// (n <= 4096) and the column/row passes of the two-pass path.
#include "launch.h"
#include "programmatic.h"

namespace fftseg {

namespace {

int g_sm_count[kMaxDevices] = {};

int sm_count()
{
    int &c = g_sm_count[current_device_slot()];
    if (c == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        c = v > 0 ? v : 1;
    }
    return c;
}

template <int LOG_L, int S, int PREC = PREC_FP32>
cudaError_t block_t(const BlockArgs &a, cudaStream_t st)
{
    using B = BlockShape<LOG_L>;
    auto k = k_block<LOG_L, S, PREC>;
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, B::T, B::SMEM);
        if (e != cudaSuccess) return e;
        per_sm = occ > 0 ? occ : 1;
    }
    if (a.ntiles == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * sm_count();
    if (grid > a.ntiles) grid = a.ntiles;
    // the blocks of back-to-back batches take the SMs as the previous grid
    // leaves them (the kernel waits for the previous kernel's writes before it
    // touches global memory)
    return launch_programmatic(k, (unsigned)grid, B::T, B::SMEM, st, a);
}

template <int LOG_L>
struct PassShape {
    // up to 16 lines of up to 1024 points (16 KB..128 KB per tile)
    static constexpr int LOG_W = (14 - LOG_L) < 4 ? (14 - LOG_L) : 4;
    static constexpr int T = (1 << (LOG_L + LOG_W)) / 16;
    static constexpr int SLOTS = smem_slots<LOG_L, LOG_W, 4>();
};

template <int LOG_L, int S>
cudaError_t pass_t(const LinesArgs &a, int64_t units, cudaStream_t st)
{
    using P = PassShape<LOG_L>;
    auto k = k_lines<LOG_L, P::LOG_W, true, S, P::T>;
    const size_t smem = (size_t)P::SLOTS * sizeof(float2);
    static bool configured_dev[kMaxDevices] = {};  // per instantiation and device
    bool &configured = configured_dev[current_device_slot()];
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (units == 0) return cudaSuccess;
    k<<<(unsigned)units, P::T, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int block_segments_per_cta(int log_n)
{
    return log_n >= 4 ? 1 << (12 - log_n) : 256;
}

int device_sm_count() { return sm_count(); }

int pass_log_w(int log_l)
{
    return (14 - log_l) < 4 ? (14 - log_l) : 4;
}

#define FFTSEG_BLOCK_CASE(LL) \
    case LL: return sign < 0 ? block_t<LL, -1>(a, st) : block_t<LL, 1>(a, st);

cudaError_t launch_block(int log_n, int sign, int prec, const BlockArgs &a, cudaStream_t st)
{
    if (prec != PREC_FP32) {  // tensor-core radix-16 stages: n a power of 16
#define FFTSEG_BLOCK_TC(LL)                                                                                   \
    case LL:                                                                                                  \
        if (prec == PREC_FP16) return sign < 0 ? block_t<LL, -1, PREC_FP16>(a, st) : block_t<LL, 1, PREC_FP16>(a, st); \
        return sign < 0 ? block_t<LL, -1, PREC_BF16>(a, st) : block_t<LL, 1, PREC_BF16>(a, st);
        switch (log_n) {
            FFTSEG_BLOCK_TC(4)
            FFTSEG_BLOCK_TC(8)
            FFTSEG_BLOCK_TC(12)
            default: return cudaErrorInvalidValue;
        }
    }
    switch (log_n) {
        FFTSEG_BLOCK_CASE(1)
        FFTSEG_BLOCK_CASE(2)
        FFTSEG_BLOCK_CASE(3)
        FFTSEG_BLOCK_CASE(4)
        FFTSEG_BLOCK_CASE(5)
        FFTSEG_BLOCK_CASE(6)
        FFTSEG_BLOCK_CASE(7)
        FFTSEG_BLOCK_CASE(8)
        FFTSEG_BLOCK_CASE(9)
        FFTSEG_BLOCK_CASE(10)
        FFTSEG_BLOCK_CASE(11)
        FFTSEG_BLOCK_CASE(12)
        default: return cudaErrorInvalidValue;
    }
}

#define FFTSEG_PASS_CASE(LL) \
    case LL: return sign < 0 ? pass_t<LL, -1>(a, units, st) : pass_t<LL, 1>(a, units, st);

cudaError_t launch_pass(int log_l, int sign, const LinesArgs &a, int64_t units, cudaStream_t st)
{
    switch (log_l) {
        FFTSEG_PASS_CASE(4)
        FFTSEG_PASS_CASE(5)
        FFTSEG_PASS_CASE(6)
        FFTSEG_PASS_CASE(7)
        FFTSEG_PASS_CASE(8)
        FFTSEG_PASS_CASE(9)
        FFTSEG_PASS_CASE(10)
        FFTSEG_PASS_CASE(11)
        FFTSEG_PASS_CASE(12)
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
