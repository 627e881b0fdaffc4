// Overlapping segments (frames): frame f of a signal holds samples
// [f*hop, f*hop + n), multiplied point by point by a real window w[j]
// (rectangular or periodic Hann, evaluated in double and rounded once).
// k_frames copies a chunk of windowed frames into an intermediate that the
// batched complex plan of n points then transforms; the chunk is sized so that
// the intermediate stays in L2 between the two passes, and overlapping frames
// re-read their shared samples from L2.
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

}  // namespace

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
