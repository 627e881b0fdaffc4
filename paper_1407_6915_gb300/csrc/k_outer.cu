// The outer pass of the interleaved four-step (n = R * M, M = 2^16,
// R = 32..256), persistent and fed by TMA.
//
// For every column j < M of a segment viewed as [R][M] (x[j + M t']), the
// R-point DFT over t' times w_n^{j t} gives Y_t[j] (decimation in frequency
// over the outer index).  A tile is W = 4096 / R consecutive columns (one
// row j1 of the 256 x 256 inner matrix, columns j2 .. j2 + W - 1); it
// arrives as one 2-D TMA box of W x R points (rows at stride M) into a
// double buffer while the previous tile is transformed, so the tile lands
// point-major ([t'][c], the line-interleaved layout) and the first stage
// reads it conflict-free.  The stages run in registers with a padded
// exchange buffer; the result, times w_n^{j t} from two exact factors
// [t mod 16][j] and [t div 16][j], is staged line-major in that buffer and
// stored unit by unit (32 transforms per unit, point j1 256 + j2 of
// transform 32 b + c at ((b 256 + j2) 256 + j1) 32 + c of the segment) in
// 256-byte runs.
#include "launch.h"

namespace fftseg {

namespace {

template <int LOG_R>
struct OuterShape {
    static constexpr int LOG_W = 12 - LOG_R;
    static constexpr int R = 1 << LOG_R, W = 1 << LOG_W, E = 4096, T = 256, V = 16, PS = 4;
    static constexpr int SLOTS = (smem_slots<LOG_R, LOG_W, PS>() + 1) & ~1;
    static constexpr size_t SMEM = (size_t)(2 * E + SLOTS) * sizeof(float2) + 2 * sizeof(uint64_t);
    static_assert(W * (R + 1) <= SLOTS, "line-major output tile in the exchange buffer");
};

template <int LOG_R, int S>
__global__ void __launch_bounds__(256, 2) k_outer(const __grid_constant__ OuterArgs a)
{
    using Sh = OuterShape<LOG_R>;
    constexpr int R = Sh::R, W = Sh::W, E = Sh::E, T = Sh::T, V = Sh::V, LOG_W = Sh::LOG_W;
    constexpr int64_t M = 1 << 16, N1 = 256, N2 = 256;
    constexpr int64_t TPS = M / W;  // tiles per segment
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;           // [2][R][W] TMA destinations
    float2 *X = sm + 2 * E;   // exchange buffer, then the line-major output tile
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
    auto issue = [&](int64_t u, int b) {
        if (tid == 0) {
            const int64_t s = u / TPS, t = u - s * TPS;
            fence_proxy_async();
            mbar_expect_tx(&bar[b], (uint32_t)(E * sizeof(float2)));
            tma_load_2d_hint(P + b * E, &a.tm, (int)(t * W), (int)(s * R), &bar[b], policy_evict_first());
        }
    };
    int64_t u = blockIdx.x;
    if (u < a.ntiles) issue(u, 0);
    for (int k = 0; u < a.ntiles; u += gridDim.x, ++k) {
        const int b = k & 1;
        if (u + gridDim.x < a.ntiles) issue(u + gridDim.x, b ^ 1);
        mbar_wait(&bar[b], (k >> 1) & 1, a.err);
        const float2 *Pb = P + b * E;
        float2 v[V];
        gather<LOG_R, LOG_W, true, T, 0>(v, [&](int c, int i) { return Pb[(i << LOG_W) + c]; });
        run_stages<LOG_R, LOG_W, true, S, T, Sh::PS, 0, false>(v, X, a.twL);
        const int64_t s = u / TPS, jt = (u - s * TPS) * W;
        __syncthreads();  // the last stage's reads of X are done: it takes the output tile
        scatter_last<LOG_R, LOG_W, true, T>(v, [&](int c, int i, float2 x) {
            // w_n^{j t}, j = jt + c, t = i
            const int64_t j = jt + c;
            float2 w = __ldg(a.tw4a + (int64_t)(i & 15) * M + j);
            if constexpr (R > 16) {
                const float2 w2 = __ldg(a.tw4b + (int64_t)(i >> 4) * M + j);
                w = make_float2(w.x * w2.x - w.y * w2.y, w.x * w2.y + w.y * w2.x);
            }
            X[c * (R + 1) + i] = twmul<S>(x, w);
        });
        __syncthreads();
        const int64_t j1 = jt / N2, j20 = jt - j1 * N2;
        float2 *o = a.out + s * (R * M) + (j20 * N1 + j1) * 32;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int e = tid + T * q;  // e = (unit W + c) 32 + tl
            const int tl = e & 31, c = (e >> 5) & (W - 1), blk = e >> (5 + LOG_W);
            o[blk * (32 * M) + (int64_t)c * N1 * 32 + tl] = X[c * (R + 1) + blk * 32 + tl];
        }
        __syncthreads();  // P[b] and X fully read before they are refilled
    }
}

template <int LOG_R, int S>
cudaError_t outer_t(const OuterArgs &a, cudaStream_t st)
{
    using Sh = OuterShape<LOG_R>;
    auto k = k_outer<LOG_R, S>;
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, Sh::T, Sh::SMEM);
        if (e != cudaSuccess) return e;
        per_sm = occ > 0 ? occ : 1;
    }
    if (a.ntiles == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > a.ntiles) grid = a.ntiles;
    k<<<(unsigned)grid, Sh::T, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_outer(int log_r, int sign, const OuterArgs &a, cudaStream_t st)
{
    switch (log_r) {
        case 5: return sign < 0 ? outer_t<5, -1>(a, st) : outer_t<5, 1>(a, st);
        case 6: return sign < 0 ? outer_t<6, -1>(a, st) : outer_t<6, 1>(a, st);
        case 7: return sign < 0 ? outer_t<7, -1>(a, st) : outer_t<7, 1>(a, st);
        case 8: return sign < 0 ? outer_t<8, -1>(a, st) : outer_t<8, 1>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fftseg
