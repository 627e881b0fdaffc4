// Lengths that are not powers of two: Bluestein's chirp-z identity on top of
// the power-of-two kernels.  With j k = (j^2 + k^2 - (k - j)^2) / 2,
//   X[k] = sum_j x[j] exp(sigma 2 pi i j k / n)
//        = w[k] sum_j (x[j] w[j]) conj(w[k - j]),   w[m] = exp(sigma pi i m^2 / n),
// a convolution, done as a cyclic one of length M = 2^ceil(log2(2n - 1)):
//   a[m] = x[m] w[m] (m < n), 0 up to M;  b[m] = conj(w[m]) for |m| < n (cyclic)
//   X[k] = w[k] * IFFT_M(FFT_M(a) * FFT_M(b) / M)[k],  k < n.
// The plan keeps w and B = FFT_M(b) / M; these kernels do the chirp in, the
// pointwise product and the chirp out, around two M-point plans.  The phase of
// w[m] is reduced exactly in integers (m^2 mod 2n) and evaluated in double.
#include "launch.h"

namespace fftseg {

namespace {

constexpr int kBlueThreads = 256;

FDEV float2 cmulb(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// a[s][m] = m < n ? x[s][m] w[m] : 0, m < M
__global__ void __launch_bounds__(kBlueThreads) k_blue_in(const BlueArgs a)
{
    const int64_t s = blockIdx.y;
    const int64_t m = (int64_t)blockIdx.x * kBlueThreads + threadIdx.x;
    if (m >= a.m) return;
    float2 v = make_float2(0.f, 0.f);
    if (m < a.n) v = cmulb(__ldg(a.x + s * a.n + m), __ldg(a.w + m));
    a.work[s * a.m + m] = v;
}

// a[s][m] *= B[m]
__global__ void __launch_bounds__(kBlueThreads) k_blue_mul(const BlueArgs a)
{
    const int64_t s = blockIdx.y;
    const int64_t m = (int64_t)blockIdx.x * kBlueThreads + threadIdx.x;
    if (m >= a.m) return;
    float2 *p = a.work + s * a.m + m;
    *p = cmulb(*p, __ldg(a.bhat + m));
}

// X[s][k] = scale * w[k] * c[s][k], k < n (complex64, or float32 |X|^2)
template <bool POWER>
__global__ void __launch_bounds__(kBlueThreads) k_blue_out(const BlueArgs a)
{
    const int64_t s = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * kBlueThreads + threadIdx.x;
    if (k >= a.n) return;
    float2 v = cmulb(a.work[s * a.m + k], __ldg(a.w + k));
    v = make_float2(v.x * a.scale, v.y * a.scale);
    if (POWER) static_cast<float *>(a.out)[s * a.n + k] = v.x * v.x + v.y * v.y;
    else static_cast<float2 *>(a.out)[s * a.n + k] = v;
}

}  // namespace

cudaError_t launch_blue(int step, bool power, const BlueArgs &a, int64_t nseg, cudaStream_t st)
{
    if (nseg <= 0) return cudaSuccess;
    if (nseg > 65535) return cudaErrorInvalidValue;
    const int64_t len = step == 2 ? a.n : a.m;
    const dim3 grid((unsigned)((len + kBlueThreads - 1) / kBlueThreads), (unsigned)nseg);
    if (step == 0) k_blue_in<<<grid, kBlueThreads, 0, st>>>(a);
    else if (step == 1) k_blue_mul<<<grid, kBlueThreads, 0, st>>>(a);
    else if (power) k_blue_out<true><<<grid, kBlueThreads, 0, st>>>(a);
    else k_blue_out<false><<<grid, kBlueThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fftseg
