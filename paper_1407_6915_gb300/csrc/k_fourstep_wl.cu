// Instantiations and launcher of the lane-line persistent four-step kernel
// (n = 2^16 .. 2^20, FP32, complex output).
#include "fourstep_wl.cuh"
#include "launch.h"

namespace fftseg {

namespace {

// 8192-point tiles, three buffers, one CTA per SM (eight compute warps of
// 32 points per lane, a loader warp and a retirer warp).  Measured on GB300:
// two buffers were 5-9 % slower.
// (4096-point tiles at two CTAs per SM measured no faster at 2^16 and
// 4-27 % slower at 2^17..2^20.)
constexpr int kWlLogE = 13, kWlNb = 3, kWlMinB = 1;

template <int LOG_N1, int LOG_N2, int S, bool ILV = false>
cudaError_t wl_t(const FourStepWlArgs &a, cudaStream_t st)
{
    using Sh = FourStepWlShape<LOG_N1, LOG_N2, kWlLogE, kWlNb, kWlMinB, ILV>;
    auto k = k_fourstep_wl<LOG_N1, LOG_N2, kWlLogE, kWlNb, kWlMinB, S, ILV>;
    // per device: the occupancy of this instantiation (the grid is the
    // resident CTAs of the GPU the launch goes to)
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, Sh::TT, Sh::SMEM);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorLaunchOutOfResources;
        per_sm = occ;
    }
    const int64_t items = (int64_t)a.nchunks * a.cs * (Sh::TSEG_A + Sh::TSEG_B);
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, Sh::TT, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2>
cudaError_t wl_s(int sign, const FourStepWlArgs &a, cudaStream_t st)
{
    return sign < 0 ? wl_t<LOG_N1, LOG_N2, -1>(a, st) : wl_t<LOG_N1, LOG_N2, 1>(a, st);
}

}  // namespace

bool fourstep_wl_shape(int log_n, int *log_n1, int *log_n2, int *log_e)
{
    if (log_n < 16 || log_n > 20) return false;
    *log_n1 = (log_n + 1) / 2;
    *log_n2 = log_n / 2;
    *log_e = kWlLogE;
    return true;
}

cudaError_t launch_fourstep_wl_ilv(int sign, const FourStepWlArgs &a, cudaStream_t st)
{
    return sign < 0 ? wl_t<8, 8, -1, true>(a, st) : wl_t<8, 8, 1, true>(a, st);
}

cudaError_t launch_fourstep_wl(int log_n, int sign, const FourStepWlArgs &a, cudaStream_t st)
{
    switch (log_n) {
        case 16: return wl_s<8, 8>(sign, a, st);
        case 17: return wl_s<9, 8>(sign, a, st);
        case 18: return wl_s<9, 9>(sign, a, st);
        case 19: return wl_s<10, 9>(sign, a, st);
        case 20: return wl_s<10, 10>(sign, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
