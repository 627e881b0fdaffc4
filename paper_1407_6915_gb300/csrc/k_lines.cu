// Instantiations and launchers of k_lines: the single-pass block kernel
// (n <= 4096) and the column/row passes of the two-pass path.
#include "launch.h"

namespace fftseg {

namespace {

template <int LOG_L>
struct BlockShape {
    // 16 points per thread, 256 threads, 4096 points per CTA; lines shorter
    // than 16 points put L points in a thread and 256 lines in a CTA.
    static constexpr int LOG_W = LOG_L >= 4 ? 12 - LOG_L : 8;
    static constexpr int T = 256;
    static constexpr int SLOTS = smem_slots<LOG_L, LOG_W, 4>();
};

template <int LOG_L, int S>
cudaError_t block_t(const LinesArgs &a, int64_t nseg, cudaStream_t st)
{
    using B = BlockShape<LOG_L>;
    auto k = k_lines<LOG_L, B::LOG_W, false, S, B::T>;
    const size_t smem = (size_t)B::SLOTS * sizeof(float2);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t per = 1 << B::LOG_W;
    const int64_t grid = (nseg + per - 1) / per;
    if (grid == 0) return cudaSuccess;
    k<<<(unsigned)grid, B::T, smem, st>>>(a);
    return cudaGetLastError();
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
    static bool configured = false;
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

int pass_log_w(int log_l)
{
    return (14 - log_l) < 4 ? (14 - log_l) : 4;
}

#define FFTSEG_BLOCK_CASE(LL) \
    case LL: return sign < 0 ? block_t<LL, -1>(a, nseg, st) : block_t<LL, 1>(a, nseg, st);

cudaError_t launch_block(int log_n, int sign, const LinesArgs &a, int64_t nseg, cudaStream_t st)
{
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
