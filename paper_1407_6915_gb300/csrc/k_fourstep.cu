// Instantiations and launcher of the persistent L2 four-step kernel (n = 2^14..2^24).
#include "fourstep.cuh"
#include "fourstep_ws.cuh"
#include "fourstep_hw.cuh"
#include "launch.h"

namespace fftseg {

namespace {

template <int LOG_N1, int LOG_N2, int LOG_E, int S, int PREC = PREC_FP32>
cudaError_t fourstep_t(const FourStepArgs &a, cudaStream_t st)
{
    using Sh = FourStepShape<LOG_N1, LOG_N2, LOG_E>;
    auto k = k_fourstep<LOG_N1, LOG_N2, LOG_E, S, PREC>;
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, Sh::T, Sh::SMEM);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorLaunchOutOfResources;
        per_sm = occ;
    }
    const int64_t items = (int64_t)a.nchunks * a.cs * (Sh::N2 / (1 << Sh::LOG_WA) + Sh::N1 / (1 << Sh::LOG_WB));
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, Sh::T, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2, int LOG_E>
cudaError_t fourstep_s(int sign, const FourStepArgs &a, cudaStream_t st)
{
    return sign < 0 ? fourstep_t<LOG_N1, LOG_N2, LOG_E, -1>(a, st) : fourstep_t<LOG_N1, LOG_N2, LOG_E, 1>(a, st);
}

template <int LOG_N1, int LOG_N2, int LOG_E>
cudaError_t fourstep_tc(int sign, int prec, const FourStepArgs &a, cudaStream_t st)
{
    if (prec == PREC_FP16)
        return sign < 0 ? fourstep_t<LOG_N1, LOG_N2, LOG_E, -1, PREC_FP16>(a, st)
                        : fourstep_t<LOG_N1, LOG_N2, LOG_E, 1, PREC_FP16>(a, st);
    return sign < 0 ? fourstep_t<LOG_N1, LOG_N2, LOG_E, -1, PREC_BF16>(a, st)
                    : fourstep_t<LOG_N1, LOG_N2, LOG_E, 1, PREC_BF16>(a, st);
}

template <int S>
cudaError_t fourstep_hw_t(const FourStepHwArgs &a, cudaStream_t st)
{
    using Sh = FourStepHwShape;
    auto k = k_fourstep_hw<S>;
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
    const int64_t items = (int64_t)a.nchunks * a.cs * 2 * Sh::TILES_SEG;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, Sh::TT, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2, int LOG_E, int S>
cudaError_t fourstep_ws_t(const FourStepWsArgs &a, cudaStream_t st)
{
    using Sh = FourStepWsShape<LOG_N1, LOG_N2, LOG_E>;
    auto k = k_fourstep_ws<LOG_N1, LOG_N2, LOG_E, S>;
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
    const int64_t items = (int64_t)a.nchunks * a.cs * (Sh::N2 / (1 << Sh::LOG_WA) + Sh::N1 / (1 << Sh::LOG_WB));
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    k<<<(unsigned)grid, Sh::TT, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2, int LOG_E>
cudaError_t fourstep_ws_s(int sign, const FourStepWsArgs &a, cudaStream_t st)
{
    return sign < 0 ? fourstep_ws_t<LOG_N1, LOG_N2, LOG_E, -1>(a, st) : fourstep_ws_t<LOG_N1, LOG_N2, LOG_E, 1>(a, st);
}

}  // namespace

cudaError_t launch_fourstep_ws(int log_n, int sign, const FourStepWsArgs &a, cudaStream_t st)
{
    switch (log_n) {
        case 14: return fourstep_ws_s<7, 7, 12>(sign, a, st);
        case 15: return fourstep_ws_s<8, 7, 12>(sign, a, st);
        case 16: return fourstep_ws_s<8, 8, 12>(sign, a, st);
        case 17: return fourstep_ws_s<9, 8, 12>(sign, a, st);
        case 18: return fourstep_ws_s<9, 9, 12>(sign, a, st);
        case 19: return fourstep_ws_s<10, 9, 13>(sign, a, st);
        case 20: return fourstep_ws_s<10, 10, 13>(sign, a, st);
        case 21: return fourstep_ws_s<11, 10, 13>(sign, a, st);
        case 22: return fourstep_ws_s<11, 11, 13>(sign, a, st);
        case 23: return fourstep_ws_s<12, 11, 13>(sign, a, st);
        case 24: return fourstep_ws_s<12, 12, 13>(sign, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fourstep_hw(int sign, const FourStepHwArgs &a, cudaStream_t st)
{
    return sign < 0 ? fourstep_hw_t<-1>(a, st) : fourstep_hw_t<1>(a, st);
}

bool fourstep_shape(int log_n, int *log_n1, int *log_n2, int *log_wa, int *log_wb)
{
    if (log_n < 14 || log_n > 24) return false;
    *log_n1 = (log_n + 1) / 2;
    *log_n2 = log_n / 2;
    const int log_e = *log_n1 <= 9 ? 12 : 13;  // 4096-point tiles (two CTAs per SM) up to N1 = 512
    *log_wa = log_e - *log_n1;
    *log_wb = log_e - *log_n2;
    return true;
}

cudaError_t launch_fourstep(int log_n, int sign, int prec, const FourStepArgs &a, cudaStream_t st)
{
    if (prec != PREC_FP32) {  // tensor-core radix-16 stages: n a power of 16
        switch (log_n) {
            case 16: return fourstep_tc<8, 8, 12>(sign, prec, a, st);
            case 20: return fourstep_tc<10, 10, 13>(sign, prec, a, st);
            case 24: return fourstep_tc<12, 12, 13>(sign, prec, a, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (log_n) {
        case 14: return fourstep_s<7, 7, 12>(sign, a, st);
        case 15: return fourstep_s<8, 7, 12>(sign, a, st);
        case 16: return fourstep_s<8, 8, 12>(sign, a, st);
        case 17: return fourstep_s<9, 8, 12>(sign, a, st);
        case 18: return fourstep_s<9, 9, 12>(sign, a, st);
        case 19: return fourstep_s<10, 9, 13>(sign, a, st);
        case 20: return fourstep_s<10, 10, 13>(sign, a, st);
        case 21: return fourstep_s<11, 10, 13>(sign, a, st);
        case 22: return fourstep_s<11, 11, 13>(sign, a, st);
        case 23: return fourstep_s<12, 11, 13>(sign, a, st);
        case 24: return fourstep_s<12, 12, 13>(sign, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
