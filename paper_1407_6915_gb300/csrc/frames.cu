// Overlapping segments (frames): frame f of a signal holds samples
// [f*hop, f*hop + n), multiplied point by point by a real window w[j]
// (rectangular or periodic Hann, evaluated in double and rounded once).
// Frames of n <= 4096 points run in one fused pass (k_block_frames).  Longer
// frames go in chunks: k_frames copies a chunk of windowed frames into an
// intermediate that the batched complex plan of n points then transforms; the
// chunk is sized so that the intermediate stays in L2 between the two passes,
// and overlapping frames re-read their shared samples from L2.
#include "launch.h"

namespace fftseg {

namespace {

constexpr int kFrameThreads = 256;

// Block b covers kFrameThreads * 2 points of frame b / bpf: two consecutive
// points per thread, read and written as one 16-byte access when aligned.
__global__ void __launch_bounds__(kFrameThreads) k_frames(const FramesArgs a)
{
    const int64_t bpf = a.blocks_per_frame;
    const int64_t f = blockIdx.x / bpf;
    const int64_t j = ((blockIdx.x - f * bpf) * kFrameThreads + threadIdx.x) * 2;
    if (j >= a.n) return;
    const float2 *src = a.signal + f * a.hop + j;
    float2 *dst = a.frames + f * a.n + j;
    const float w0 = a.window ? __ldg(a.window + j) : 1.f;
    const float w1 = a.window ? __ldg(a.window + j + 1) : 1.f;
    float2 x0, x1;
    if ((a.hop & 1) == 0) {  // the frame starts on a 16-byte boundary
        const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
        x0 = make_float2(v.x, v.y);
        x1 = make_float2(v.z, v.w);
    } else {
        x0 = __ldg(src);
        x1 = __ldg(src + 1);
    }
    *reinterpret_cast<float4 *>(dst) = make_float4(x0.x * w0, x0.y * w0, x1.x * w1, x1.y * w1);
}

// Frames of n <= 4096 points in one pass: a CTA takes tiles of W = 4096 / n
// frames (the block kernel's tile shape).  The samples of the next tile are
// copied asynchronously into one of two staging tiles while the current tile
// is transformed: with BULK (16-byte aligned frames, n >= 256) one thread
// issues a bulk copy per frame, completed on an mbarrier; otherwise every
// thread issues 8-byte cp.async copies (any hop).  The window is applied as
// the first stage gathers its inputs, the n-point forward FFT runs, and the
// bins are stored from the last stage.  The samples that neighbouring frames
// share are re-read from L2; each bin crosses HBM once.
template <int LOG_L, bool BULK>
__global__ void __launch_bounds__(256, 2) k_block_frames(const FramesBlockArgs a)
{
    using Sh = BlockShape<LOG_L>;
    constexpr int L = 1 << LOG_L, W = 1 << Sh::LOG_W, T = Sh::T, E = Sh::E, V = E / T;
    extern __shared__ __align__(1024) float2 sm[];
    float2 *S = sm;          // staging tiles [2][W][L]
    float2 *X = sm + 2 * E;  // exchange buffer of the stages
    [[maybe_unused]] uint64_t *bar = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    const int tid = threadIdx.x;
    if constexpr (BULK) {
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    // copies of tile u's samples into staging tile b.  cp.async zero-fills
    // the rows past the last frame and makes one commit group per call (empty
    // past the end); bulk copies leave those rows stale (never stored).
    auto issue = [&](int64_t u, int b) {
        if (u < a.ntiles) {
            const int64_t f0 = u * W;
            const int64_t rows = a.nframes - f0 < W ? a.nframes - f0 : W;
            const float2 *src = a.signal + f0 * a.hop;
            if constexpr (BULK) {
                if (tid == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar[b], (uint32_t)(rows * L * (int64_t)sizeof(float2)));
                    for (int c = 0; c < rows; ++c)
                        tma_load_1d(S + b * E + c * L, src + c * a.hop, L * (uint32_t)sizeof(float2), &bar[b]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    const int e = tid + T * q;
                    const int c = e >> LOG_L, i = e & (L - 1);
                    const bool ok = c < rows;
                    cp_async8(S + b * E + e, ok ? src + c * a.hop + i : a.signal, ok ? 8u : 0u);
                }
            }
        }
        if constexpr (!BULK) cp_async_commit();
    };
    int64_t u = blockIdx.x;
    issue(u, 0);
    for (int k = 0; u < a.ntiles; u += gridDim.x, ++k) {
        const int b = k & 1;
        const float2 *Sb = S + b * E;
        issue(u + gridDim.x, b ^ 1);
        if constexpr (BULK) {
            mbar_wait(&bar[b], (k >> 1) & 1, a.err);
        } else {
            cp_async_wait<1>();  // this thread's copies of tile u have landed
            __syncthreads();     // and every other thread's
        }
        const int64_t f0 = u * W;
        const int64_t rows = a.nframes - f0 < W ? a.nframes - f0 : W;
        float2 v[V];
        gather<LOG_L, Sh::LOG_W, false, T, 0>(v, [&](int c, int i) {
            const float2 x = Sb[(c << LOG_L) + i];
            if (!a.window) return x;
            const float w = __ldg(a.window + i);
            return make_float2(x.x * w, x.y * w);
        });
        run_stages<LOG_L, Sh::LOG_W, false, -1, T, Sh::PS, 0, false>(v, X, a.twL);
        const float scale = a.scale;
        scatter_last<LOG_L, Sh::LOG_W, false, T>(v, [&](int c, int i, float2 x) {
            if (c >= rows) return;
            if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
            const int64_t o = (f0 + c) * L + i;
            if (a.out_power) static_cast<float *>(a.out)[o] = x.x * x.x + x.y * x.y;
            else static_cast<float2 *>(a.out)[o] = x;
        });
        __syncthreads();  // S[b] and X read in full before they are rewritten
    }
    if constexpr (!BULK) cp_async_wait<0>();
}

template <int LOG_L, bool BULK>
cudaError_t block_frames_launch(const FramesBlockArgs &a, cudaStream_t st)
{
    using B = BlockShape<LOG_L>;
    constexpr size_t smem = (size_t)(B::SLOTS + 2 * B::E) * sizeof(float2) + 2 * sizeof(uint64_t);
    auto k = k_block_frames<LOG_L, BULK>;
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

// Bulk copies want 16-byte aligned frames (an even hop on an aligned signal);
// below 256 points a tile has too many frames for one issuing thread.
template <int LOG_L>
cudaError_t block_frames_t(const FramesBlockArgs &a, cudaStream_t st)
{
    if constexpr (LOG_L >= 8) {
        if ((a.hop & 1) == 0 && (reinterpret_cast<uintptr_t>(a.signal) & 15) == 0)
            return block_frames_launch<LOG_L, true>(a, st);
    }
    return block_frames_launch<LOG_L, false>(a, st);
}

}  // namespace

cudaError_t launch_block_frames(int log_l, const FramesBlockArgs &a, cudaStream_t st)
{
    switch (log_l) {
        case 1: return block_frames_t<1>(a, st);
        case 2: return block_frames_t<2>(a, st);
        case 3: return block_frames_t<3>(a, st);
        case 4: return block_frames_t<4>(a, st);
        case 5: return block_frames_t<5>(a, st);
        case 6: return block_frames_t<6>(a, st);
        case 7: return block_frames_t<7>(a, st);
        case 8: return block_frames_t<8>(a, st);
        case 9: return block_frames_t<9>(a, st);
        case 10: return block_frames_t<10>(a, st);
        case 11: return block_frames_t<11>(a, st);
        case 12: return block_frames_t<12>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_frames(FramesArgs a, int64_t nframes, cudaStream_t st)
{
    if (nframes <= 0) return cudaSuccess;
    a.blocks_per_frame = (a.n / 2 + kFrameThreads - 1) / kFrameThreads;
    const int64_t blocks = nframes * a.blocks_per_frame;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    k_frames<<<(unsigned)blocks, kFrameThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fftseg
