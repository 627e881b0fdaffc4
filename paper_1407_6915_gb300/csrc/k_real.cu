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

}  // namespace

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
