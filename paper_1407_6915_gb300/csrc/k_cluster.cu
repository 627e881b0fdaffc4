// Instantiations and launcher of the single-pass cluster kernel (n = 2^13..2^17).
#include "launch.h"

namespace fftseg {

namespace {

template <int LOG_N1, int LOG_N2, int LOG_C, int S>
cudaError_t cluster_t(const ClusterArgs &a, int64_t nseg, cudaStream_t st)
{
    using Sh = ClusterShape<LOG_N1, LOG_N2, LOG_C>;
    auto k = k_cluster<LOG_N1, LOG_N2, LOG_C, S>;
    const size_t smem = (size_t)Sh::SLOTS * sizeof(float2);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (Sh::C > 8) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        configured = true;
    }
    if (nseg == 0) return cudaSuccess;
    k<<<(unsigned)(nseg * Sh::C), Sh::T, smem, st>>>(a);
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2, int LOG_C>
cudaError_t cluster_s(int sign, const ClusterArgs &a, int64_t nseg, cudaStream_t st)
{
    return sign < 0 ? cluster_t<LOG_N1, LOG_N2, LOG_C, -1>(a, nseg, st)
                    : cluster_t<LOG_N1, LOG_N2, LOG_C, 1>(a, nseg, st);
}

}  // namespace

bool cluster_shape(int log_n, int log_c_req, int *log_n1, int *log_n2, int *log_c)
{
    switch (log_n) {
        case 13: *log_n1 = 6; *log_n2 = 7; *log_c = 1; return log_c_req == 0 || log_c_req == 1;
        case 14: *log_n1 = 7; *log_n2 = 7; *log_c = 2; return log_c_req == 0 || log_c_req == 2;
        case 15: *log_n1 = 7; *log_n2 = 8; *log_c = 3; return log_c_req == 0 || log_c_req == 3;
        case 16:
            *log_n1 = 8; *log_n2 = 8;
            *log_c = log_c_req == 4 ? 4 : 3;
            return log_c_req == 0 || log_c_req == 3 || log_c_req == 4;
        case 17: *log_n1 = 8; *log_n2 = 9; *log_c = 4; return log_c_req == 0 || log_c_req == 4;
        default: return false;
    }
}

cudaError_t launch_cluster(int log_n, int log_c, int sign, const ClusterArgs &a, int64_t nseg,
                           cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_n, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_n) {
        case 13: return cluster_s<6, 7, 1>(sign, a, nseg, st);
        case 14: return cluster_s<7, 7, 2>(sign, a, nseg, st);
        case 15: return cluster_s<7, 8, 3>(sign, a, nseg, st);
        case 16: return lc == 4 ? cluster_s<8, 8, 4>(sign, a, nseg, st) : cluster_s<8, 8, 3>(sign, a, nseg, st);
        case 17: return cluster_s<8, 9, 4>(sign, a, nseg, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
