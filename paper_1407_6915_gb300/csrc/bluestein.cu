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

// Rows with M <= 4096 in one pass.  A CTA takes tiles of W = 4096 / M rows
// (the block kernel's tile shape) and keeps each row on chip from the chirp-in
// to the chirp-out.  The next tile's samples are copied asynchronously into
// one of two staging tiles, zero beyond n, while the current tile is
// transformed (BULK, for 16-byte aligned rows and M >= 256: one bulk copy
// per row on an mbarrier; otherwise 8-byte cp.async by every thread, any n);
// the samples are multiplied by w in place, the M-point forward FFT runs in
// registers and the exchange buffer, its output goes back to the buffer in
// natural order and is multiplied by B there, the inverse FFT follows, and a
// coalesced store applies w and the scale to the first n points.  Each row
// crosses HBM once each way: 8n bytes in, 8n (complex) or 4n (|X|^2) out.
template <int LOG_M, bool BULK>
__global__ void __launch_bounds__(256, 2) k_blue_block(const BlueBlockArgs a)
{
    using Sh = BlockShape<LOG_M>;
    constexpr int M = 1 << LOG_M, W = 1 << Sh::LOG_W, T = Sh::T, E = Sh::E, V = E / T;
    extern __shared__ __align__(1024) float2 sm[];
    float2 *S = sm;          // staging tiles [2][W][M]
    float2 *X = sm + 2 * E;  // exchange buffer of the stages
    [[maybe_unused]] uint64_t *bar = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    const int tid = threadIdx.x;
    const int64_t n = a.n;
    auto slot = [](int c, int i) { return smem_slot<LOG_M, Sh::LOG_W, false, Sh::PS>(c, i); };
    if constexpr (BULK) {
        // the bulk copies fill points 0..n-1 of each row; points n..M-1 of
        // both staging tiles are zeroed once and never written again
        for (int e = tid; e < 2 * E; e += T)
            if ((e & (M - 1)) >= n) S[e] = make_float2(0.f, 0.f);
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    // copies of tile u's rows into staging tile b.  BULK: one bulk copy per
    // row by one thread, on an mbarrier (rows past the last stay stale and are
    // never stored); otherwise 8-byte cp.async by every thread, zero past n
    // and past the last row, one commit group per call (empty past the end).
    auto issue = [&](int64_t u, int b) {
        if (u < a.ntiles) {
            const int64_t line0 = u * W;
            const int64_t rows = a.nseg - line0 < W ? a.nseg - line0 : W;
            const float2 *src = a.x + line0 * n;
            if constexpr (BULK) {
                if (tid == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar[b], (uint32_t)(rows * n * (int64_t)sizeof(float2)));
                    for (int c = 0; c < rows; ++c)
                        tma_load_1d(S + b * E + c * M, src + c * n, (uint32_t)(n * sizeof(float2)), &bar[b]);
                }
            } else {
#pragma unroll 4
                for (int q = 0; q < V; ++q) {
                    const int e = tid + T * q;
                    const int c = e >> LOG_M, i = e & (M - 1);
                    const bool ok = c < rows && i < n;
                    cp_async8(S + b * E + e, ok ? src + c * n + i : a.x, ok ? 8u : 0u);
                }
            }
        }
        if constexpr (!BULK) cp_async_commit();
    };
    int64_t u = blockIdx.x;
    issue(u, 0);
    for (int k = 0; u < a.ntiles; u += gridDim.x, ++k) {
        const int b = k & 1;
        float2 *Sb = S + b * E;
        issue(u + gridDim.x, b ^ 1);
        if constexpr (BULK) mbar_wait(&bar[b], (k >> 1) & 1, a.err);  // tile u has landed
        else cp_async_wait<1>();  // this thread's copies of tile u have landed
#pragma unroll 4
        for (int q = 0; q < V; ++q) {  // chirp-in (without BULK: on the samples this thread copied)
            const int e = tid + T * q;
            const int i = e & (M - 1);
            if (i < n) Sb[e] = cmulb(Sb[e], __ldg(a.w + i));
        }
        __syncthreads();
        const int64_t line0 = u * W;
        float2 v[V];
        gather<LOG_M, Sh::LOG_W, false, T, 0>(v, [&](int c, int i) { return Sb[(c << LOG_M) + i]; });
        run_stages<LOG_M, Sh::LOG_W, false, -1, T, Sh::PS, 0, false>(v, X, a.twL);
        __syncthreads();  // the last stage's inputs were read from X
        scatter_last<LOG_M, Sh::LOG_W, false, T>(v, [&](int c, int i, float2 x) { X[slot(c, i)] = x; });
        __syncthreads();
#pragma unroll 4
        for (int q = 0; q < V; ++q) {  // the product with B, along the rows
            const int e = tid + T * q;
            const int c = e >> LOG_M, i = e & (M - 1);
            X[slot(c, i)] = cmulb(X[slot(c, i)], __ldg(a.bhat + i));
        }
        __syncthreads();
        gather<LOG_M, Sh::LOG_W, false, T, 0>(v, [&](int c, int i) { return X[slot(c, i)]; });
        run_stages<LOG_M, Sh::LOG_W, false, 1, T, Sh::PS, 0, true>(v, X, a.twL);
        __syncthreads();
        scatter_last<LOG_M, Sh::LOG_W, false, T>(v, [&](int c, int i, float2 x) {
            if (i < n) X[slot(c, i)] = x;
        });
        __syncthreads();
        // chirp-out, coalesced along the rows
        {
            const int64_t rows = a.nseg - line0 < W ? a.nseg - line0 : W;
            const float scale = a.scale;
#pragma unroll 4
            for (int q = 0; q < V; ++q) {
                const int e = tid + T * q;
                const int c = e >> LOG_M, i = e & (M - 1);
                if (c >= rows || i >= n) continue;
                float2 x = cmulb(X[slot(c, i)], __ldg(a.w + i));
                x = make_float2(x.x * scale, x.y * scale);
                const int64_t o = (line0 + c) * n + i;
                if (a.out_power) static_cast<float *>(a.out)[o] = x.x * x.x + x.y * x.y;
                else static_cast<float2 *>(a.out)[o] = x;
            }
        }
        __syncthreads();  // S[b] and X read in full before they are rewritten
    }
    if constexpr (!BULK) cp_async_wait<0>();
}

template <int LOG_M, bool BULK>
cudaError_t blue_block_launch(const BlueBlockArgs &a, cudaStream_t st)
{
    using B = BlockShape<LOG_M>;
    constexpr size_t smem = (size_t)(B::SLOTS + 2 * B::E) * sizeof(float2) + 2 * sizeof(uint64_t);
    auto k = k_blue_block<LOG_M, BULK>;
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, B::T, smem);
        if (e != cudaSuccess) return e;
        per_sm = occ > 0 ? occ : 1;
    }
    if (a.ntiles == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > a.ntiles) grid = a.ntiles;
    k<<<(unsigned)grid, B::T, smem, st>>>(a);
    return cudaGetLastError();
}

// Bulk copies want 16-byte aligned rows (an even n on an aligned input);
// below M = 256 a tile has too many rows for one issuing thread.
template <int LOG_M>
cudaError_t blue_block_t(const BlueBlockArgs &a, cudaStream_t st)
{
    if constexpr (LOG_M >= 8) {
        if ((a.n & 1) == 0 && (reinterpret_cast<uintptr_t>(a.x) & 15) == 0)
            return blue_block_launch<LOG_M, true>(a, st);
    }
    return blue_block_launch<LOG_M, false>(a, st);
}

}  // namespace

cudaError_t launch_blue_block(int log_m, const BlueBlockArgs &a, cudaStream_t st)
{
    switch (log_m) {
        case 3: return blue_block_t<3>(a, st);
        case 4: return blue_block_t<4>(a, st);
        case 5: return blue_block_t<5>(a, st);
        case 6: return blue_block_t<6>(a, st);
        case 7: return blue_block_t<7>(a, st);
        case 8: return blue_block_t<8>(a, st);
        case 9: return blue_block_t<9>(a, st);
        case 10: return blue_block_t<10>(a, st);
        case 11: return blue_block_t<11>(a, st);
        case 12: return blue_block_t<12>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

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
