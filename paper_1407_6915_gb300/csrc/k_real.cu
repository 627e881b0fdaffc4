// Real-signal segments (FFTSEG_FLAG_REAL): the split between a length-n real
// DFT and a length-M = n/2 complex DFT.
//
// Forward.  The n real samples of a segment, read as M complex values
// z[m] = x[2m] + i x[2m+1], go through the complex FFT: Z = DFT_M(z).  With
// A = Z[k], B = conj(Z[(M - k) mod M]) and w = w_n^k = exp(-2 pi i k / n):
//   Fe = (A + B) / 2        (the DFT of the even samples)
//   Fo = -i (A - B) / 2     (the DFT of the odd samples)
//   X[k]     = Fe + w Fo
//   X[M - k] = conj(Fe - w Fo)
// for k = 0 .. M/2, which gives the n/2 + 1 bins X[0..M] of the real DFT
// (X[0] and X[M] are real).  k_real_post does this per pair (k, M - k).
//
// Inverse.  From the bins X[0..M] (the imaginary parts of X[0] and X[M] are
// ignored, as for the real part of the Hermitian extension), with A = X[k],
// B = conj(X[M - k]):
//   Z[k] = (A + B) + i conj(w_n^k) (A - B)
// so that the inverse complex FFT of length M gives z[m] = x[2m] + i x[2m+1]
// with x[j] = sum over all n bins of the Hermitian extension times
// exp(+2 pi i j k / n) (unnormalised, the library's NORM_NONE).
// k_real_pre does this per pair (k, M - k).
//
// Both passes apply the real transform's scale.  The twiddle table holds the
// forward values w_n^k for k = 0 .. M/2, evaluated in double, rounded once.
#include "launch.h"
#include "programmatic.h"

namespace fftseg {

namespace {

constexpr int kRealThreads = 256;

FDEV float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
FDEV float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
FDEV float2 scalef2(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// One block covers kRealThreads pairs of one segment: block b -> segment
// b / bps, pairs (b % bps) * kRealThreads + threadIdx.x.
template <bool POWER>
__global__ void __launch_bounds__(kRealThreads) k_real_post(const RealArgs a)
{
    const int64_t bps = a.blocks_per_seg;
    const int64_t s = blockIdx.x / bps;
    const int k = (int)(blockIdx.x - s * bps) * kRealThreads + threadIdx.x;
    const int M = a.m;
    if (k > M / 2) return;
    const float2 *Z = a.zin + s * M;
    const float2 A = Z[k];
    const float2 B = conjf2(Z[(M - k) & (M - 1)]);
    const float2 fe = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
    const float2 fo = make_float2(0.5f * (A.y - B.y), -0.5f * (A.x - B.x));  // -i (A - B) / 2
    const float2 wfo = cmul(__ldg(a.tw + k), fo);
    const float2 xk = scalef2(make_float2(fe.x + wfo.x, fe.y + wfo.y), a.scale);
    const float2 xm = scalef2(make_float2(fe.x - wfo.x, -(fe.y - wfo.y)), a.scale);  // conj(Fe - w Fo)
    const int64_t o = s * (M + 1);
    if (POWER) {
        float *P = static_cast<float *>(a.out) + o;
        P[k] = xk.x * xk.x + xk.y * xk.y;
        if (2 * k != M) P[M - k] = xm.x * xm.x + xm.y * xm.y;
    } else {
        float2 *X = static_cast<float2 *>(a.out) + o;
        X[k] = xk;
        if (2 * k != M) X[M - k] = xm;
    }
}

__global__ void __launch_bounds__(kRealThreads) k_real_pre(const RealArgs a)
{
    const int64_t bps = a.blocks_per_seg;
    const int64_t s = blockIdx.x / bps;
    const int k = (int)(blockIdx.x - s * bps) * kRealThreads + threadIdx.x;
    const int M = a.m;
    if (k > M / 2) return;
    const float2 *X = a.xin + s * (M + 1);
    float2 A = X[k], C = X[M - k];
    if (k == 0) {  // the imaginary parts of the real bins X[0] and X[M] do not enter
        A.y = 0.f;
        C.y = 0.f;
    }
    const float2 w = __ldg(a.tw + k);  // w_n^k (forward value); conj(w) = exp(+2 pi i k / n)
    float2 *Z = static_cast<float2 *>(a.out) + s * M;
    {  // Z[k] = (A + conj(C)) + i conj(w) (A - conj(C))
        const float2 B = conjf2(C);
        const float2 d = cmul(conjf2(w), make_float2(A.x - B.x, A.y - B.y));
        Z[k] = scalef2(make_float2(A.x + B.x - d.y, A.y + B.y + d.x), a.scale);
    }
    if (k != 0 && 2 * k != M) {  // Z[M - k] from the same pair: conj(w_n^{M-k}) = -w_n^k
        const float2 B = conjf2(A);
        const float2 d = cmul(make_float2(-w.x, -w.y), make_float2(C.x - B.x, C.y - B.y));
        Z[M - k] = scalef2(make_float2(C.x + B.x - d.y, C.y + B.y + d.x), a.scale);
    }
}

// Forward real segments of n = 2L <= 8192 points in one pass: the block
// kernel's persistent CTAs and bulk-copied tiles of whole segments (the L
// complex values of each), the L-point Stockham FFT, then the split above
// inside the tile: Z goes to the tile buffer in natural order and every
// thread forms bin pairs (k, L - k) of one segment, written as n/2 + 1 bins.
template <int LOG_L>
__global__ void __launch_bounds__(256, 2) k_block_r2c(const RealBlockArgs a)
{
    using Sh = BlockShape<LOG_L>;
    constexpr int L = 1 << LOG_L, W = 1 << Sh::LOG_W, E = Sh::E, T = Sh::T, V = E / T;
    constexpr int PAIRS = L / 2 + 1;
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;
    float2 *X = sm + 2 * E;
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    const int tid = threadIdx.x;
    if (smem_u32(P) & 127) {
        if (tid == 0) atomicOr(a.err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto tile_bytes = [&](int64_t u) {
        int64_t segs = a.nseg - u * W;
        if (segs > W) segs = W;
        return (uint32_t)(segs * L * (int64_t)sizeof(float2));
    };
    // (launched with programmatic stream serialization, as k_block: the L2
    // fetch of the first two tiles starts before the wait for the previous
    // kernel)
    grid_launch_dependents();
    if (tid == 0)
        for (int64_t u = blockIdx.x, q = 0; q < 2 && u < a.ntiles; ++q, u += gridDim.x)
            prefetch_l2_bulk(a.in + u * E, tile_bytes(u));
    grid_dependency_wait();
    auto issue = [&](int64_t u, int b) {
        if (tid == 0) {
            const uint32_t bytes = tile_bytes(u);
            fence_proxy_async();
            mbar_expect_tx(&bar[b], bytes);
            tma_load_1d(P + b * E, a.in + u * E, bytes, &bar[b]);
        }
    };
    int64_t u = blockIdx.x;
    if (u < a.ntiles) issue(u, 0);
    for (int k = 0; u < a.ntiles; u += gridDim.x, ++k) {
        const int b = k & 1;
        if (u + gridDim.x < a.ntiles) issue(u + gridDim.x, b ^ 1);
        mbar_wait(&bar[b], (k >> 1) & 1, a.err);
        float2 *Pb = P + b * E;
        float2 v[V];
        gather<LOG_L, Sh::LOG_W, false, T, 0>(v, [&](int c, int i) { return Pb[(c << LOG_L) + i]; });
        run_stages<LOG_L, Sh::LOG_W, false, -1, T, Sh::PS, 0, false>(v, X, a.twL);
        // Z of every segment of the tile, natural order, into the tile buffer
        // (its last reads were the gather, ordered by the stages' barriers)
        scatter_last<LOG_L, Sh::LOG_W, false, T>(v, [&](int c, int i, float2 x) { Pb[(c << LOG_L) + i] = x; });
        __syncthreads();
        const int64_t line0 = u * W;
        for (int p = tid; p < W * PAIRS; p += T) {
            const int c = p / PAIRS, kk = p - c * PAIRS;
            const int64_t seg = line0 + c;
            if (seg >= a.nseg) continue;
            const float2 A = Pb[(c << LOG_L) + kk];
            const float2 B = conjf2(Pb[(c << LOG_L) + ((L - kk) & (L - 1))]);
            const float2 fe = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y + B.y));
            const float2 fo = make_float2(0.5f * (A.y - B.y), -0.5f * (A.x - B.x));
            const float2 wfo = cmul(__ldg(a.tw + kk), fo);
            const float2 xk = scalef2(make_float2(fe.x + wfo.x, fe.y + wfo.y), a.scale);
            const float2 xm = scalef2(make_float2(fe.x - wfo.x, -(fe.y - wfo.y)), a.scale);
            const int64_t o = seg * (L + 1);
            if (a.out_power) {
                float *Q = static_cast<float *>(a.out) + o;
                Q[kk] = xk.x * xk.x + xk.y * xk.y;
                if (2 * kk != L) Q[L - kk] = xm.x * xm.x + xm.y * xm.y;
            } else {
                float2 *Q = static_cast<float2 *>(a.out) + o;
                Q[kk] = xk;
                if (2 * kk != L) Q[L - kk] = xm;
            }
        }
        __syncthreads();  // P[b] and X read in full before they are reused
    }
}

template <int LOG_L>
cudaError_t block_r2c_t(const RealBlockArgs &a, cudaStream_t st)
{
    using B = BlockShape<LOG_L>;
    auto k = k_block_r2c<LOG_L>;
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
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > a.ntiles) grid = a.ntiles;
    return launch_programmatic(k, (unsigned)grid, B::T, B::SMEM, st, a);
}

}  // namespace

cudaError_t launch_block_r2c(int log_l, const RealBlockArgs &a, cudaStream_t st)
{
    switch (log_l) {
        case 1: return block_r2c_t<1>(a, st);
        case 2: return block_r2c_t<2>(a, st);
        case 3: return block_r2c_t<3>(a, st);
        case 4: return block_r2c_t<4>(a, st);
        case 5: return block_r2c_t<5>(a, st);
        case 6: return block_r2c_t<6>(a, st);
        case 7: return block_r2c_t<7>(a, st);
        case 8: return block_r2c_t<8>(a, st);
        case 9: return block_r2c_t<9>(a, st);
        case 10: return block_r2c_t<10>(a, st);
        case 11: return block_r2c_t<11>(a, st);
        case 12: return block_r2c_t<12>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_real(bool post, bool power, RealArgs a, int64_t nseg, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    a.blocks_per_seg = (a.m / 2 + 1 + kRealThreads - 1) / kRealThreads;
    const int64_t blocks = nseg * a.blocks_per_seg;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    if (post) {
        if (power) k_real_post<true><<<(unsigned)blocks, kRealThreads, 0, st>>>(a);
        else k_real_post<false><<<(unsigned)blocks, kRealThreads, 0, st>>>(a);
    } else {
        k_real_pre<<<(unsigned)blocks, kRealThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace fftseg
