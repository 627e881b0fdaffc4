// Instantiations and launchers of the single-pass cluster kernel (n = 2^13..2^17),
// complex segments, real-signal segments of 2n samples (forward and inverse)
// and the two passes of Bluestein rows (M = 2^13..2^16).
#include "launch.h"

namespace fftseg {

namespace {

template <int LOG_N1, int LOG_N2, int LOG_C, int S, bool RF = false, bool RI = false, bool BL = false,
          bool BF = false>
cudaError_t cluster_t(const ClusterArgs &a, cudaStream_t st)
{
    using Sh = ClusterShape<LOG_N1, LOG_N2, LOG_C>;
    auto k = k_cluster<LOG_N1, LOG_N2, LOG_C, S, RF, RI, BL, BF>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Sh::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(Sh::T);
    cfg.dynamicSmemBytes = Sh::SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters_dev[kMaxDevices] = {};  // per instantiation and device
    int &max_clusters = max_clusters_dev[current_device_slot()];
    if (max_clusters == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
        if (e != cudaSuccess) return e;
        if (Sh::C > 8) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        int m = 0;
        cfg.gridDim = dim3(Sh::C * 1024);
        e = cudaOccupancyMaxActiveClusters(&m, k, &cfg);
        if (e != cudaSuccess) return e;
        if (m < 1) return cudaErrorLaunchOutOfResources;
        max_clusters = m;
    }
    if (a.nseg == 0) return cudaSuccess;
    const int64_t ncl = a.nseg < max_clusters ? a.nseg : max_clusters;
    cfg.gridDim = dim3((unsigned)(ncl * Sh::C));
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int LOG_N1, int LOG_N2, int LOG_C>
cudaError_t cluster_s(int sign, const ClusterArgs &a, cudaStream_t st)
{
    return sign < 0 ? cluster_t<LOG_N1, LOG_N2, LOG_C, -1>(a, st) : cluster_t<LOG_N1, LOG_N2, LOG_C, 1>(a, st);
}

}  // namespace

bool cluster_shape(int log_n, int log_c_req, int *log_n1, int *log_n2, int *log_c)
{
    switch (log_n) {
        case 13: *log_n1 = 6; *log_n2 = 7; *log_c = 1; return log_c_req == 0 || log_c_req == 1;
        case 14: *log_n1 = 7; *log_n2 = 7; *log_c = 2; return log_c_req == 0 || log_c_req == 2;
        // (256 x 128 at 2^15: 32 rows of 256-byte output runs per CTA; measured 1 %
        // faster than 128 x 256 for complex segments and 4 % for the real split)
        case 15: *log_n1 = 8; *log_n2 = 7; *log_c = 3; return log_c_req == 0 || log_c_req == 3;
        case 16:
            *log_n1 = 8; *log_n2 = 8;
            *log_c = log_c_req == 3 ? 3 : 4;
            return log_c_req == 0 || log_c_req == 3 || log_c_req == 4;
        case 17: *log_n1 = 8; *log_n2 = 9; *log_c = 4; return log_c_req == 0 || log_c_req == 4;
        default: return false;
    }
}

cudaError_t launch_cluster(int log_n, int log_c, int sign, const ClusterArgs &a, cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_n, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_n) {
        case 13: return cluster_s<6, 7, 1>(sign, a, st);
        case 14: return cluster_s<7, 7, 2>(sign, a, st);
        case 15: return cluster_s<8, 7, 3>(sign, a, st);
        case 16: return lc == 4 ? cluster_s<8, 8, 4>(sign, a, st) : cluster_s<8, 8, 3>(sign, a, st);
        case 17: return cluster_s<8, 9, 4>(sign, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster_r2c(int log_n, int log_c, const ClusterArgs &a, cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_n, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_n) {
        case 13: return cluster_t<6, 7, 1, -1, true>(a, st);
        case 14: return cluster_t<7, 7, 2, -1, true>(a, st);
        case 15: return cluster_t<8, 7, 3, -1, true>(a, st);
        case 16: return lc == 4 ? cluster_t<8, 8, 4, -1, true>(a, st) : cluster_t<8, 8, 3, -1, true>(a, st);
        case 17: return cluster_t<8, 9, 4, -1, true>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster_c2r(int log_n, int log_c, const ClusterArgs &a, cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_n, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_n) {
        // (n/2 = 2^13 and 2^14: larger inverse plans are faster chunked)
        case 13: return cluster_t<6, 7, 1, 1, false, true>(a, st);
        case 14: return cluster_t<7, 7, 2, 1, false, true>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster_blue_inv(int log_m, int log_c, const ClusterArgs &a, cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_m, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_m) {
        case 13: return cluster_t<6, 7, 1, 1, false, false, true>(a, st);
        case 14: return cluster_t<7, 7, 2, 1, false, false, true>(a, st);
        case 15: return cluster_t<8, 7, 3, 1, false, false, true>(a, st);
        case 16: return lc == 4 ? cluster_t<8, 8, 4, 1, false, false, true>(a, st)
                                : cluster_t<8, 8, 3, 1, false, false, true>(a, st);
        case 17: return cluster_t<8, 9, 4, 1, false, false, true>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_cluster_blue_fwd(int log_m, int log_c, const ClusterArgs &a, cudaStream_t st)
{
    int l1, l2, lc;
    if (!cluster_shape(log_m, log_c, &l1, &l2, &lc)) return cudaErrorInvalidValue;
    switch (log_m) {
        case 13: return cluster_t<6, 7, 1, -1, false, false, false, true>(a, st);
        case 14: return cluster_t<7, 7, 2, -1, false, false, false, true>(a, st);
        case 15: return cluster_t<8, 7, 3, -1, false, false, false, true>(a, st);
        case 16: return lc == 4 ? cluster_t<8, 8, 4, -1, false, false, false, true>(a, st)
                                : cluster_t<8, 8, 3, -1, false, false, false, true>(a, st);
        case 17: return cluster_t<8, 9, 4, -1, false, false, false, true>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
