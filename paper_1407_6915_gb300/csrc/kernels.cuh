// FP32 segment-FFT kernels for sm_103a.
//
//  k_lines    one CTA transforms a tile of W lines of L <= 4096 points.
//             Segment-major tiles (CFAST = false) are whole segments (the
//             single-pass path for n <= 4096); line-interleaved tiles
//             (CFAST = true) are the column and row passes of the two-pass
//             four-step path for n >= 2^18.
//  k_cluster  one thread-block cluster of C CTAs transforms one whole
//             segment of n = N1*N2 points (2^13..2^17) in a single HBM pass:
//             column DFTs, four-step twiddle, an all-to-all exchange through
//             distributed shared memory, row DFTs.
//
// Four-step factorisation (n = N1*N2, input j = j1*N2 + j2, output k = k1 + N1*k2):
//   X[k1 + N1 k2] = sum_{j2} w_{N2}^{j2 k2} [ w_n^{j2 k1} sum_{j1} x[j1 N2 + j2] w_{N1}^{j1 k1} ].
#pragma once
#include <cooperative_groups.h>

#include "engine.cuh"

namespace fftseg {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------- stage runner

template <int LOG_L, int LOG_W, bool CFAST, int T, int STAGE, class Get>
FDEV void gather(float2 *v, Get &&get)
{
    using I = StageInfo<LOG_L, STAGE>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        butterfly_coords<LOG_L, LOG_W, CFAST, I::LOG_R>(threadIdx.x + T * b, c, j);
#pragma unroll
        for (int r = 0; r < I::R; ++r) v[b * I::R + r] = get(c, j + (r << (LOG_L - I::LOG_R)));
    }
}

// Hand every output of the last stage, (line c, index i), to put().
template <int LOG_L, int LOG_W, bool CFAST, int T, class Put>
FDEV void scatter_last(const float2 *v, Put &&put)
{
    using I = StageInfo<LOG_L, StageInfo<LOG_L, 0>::NSTAGES - 1>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        butterfly_coords<LOG_L, LOG_W, CFAST, I::LOG_R>(threadIdx.x + T * b, c, j);
#pragma unroll
        for (int r = 0; r < I::R; ++r) put(c, j + (r << (LOG_L - I::LOG_R)), v[b * I::R + r]);
    }
}

// Run stages STAGE..last on the values in v (this stage's inputs).  Between
// stages the tile goes through shared memory `sm` (layout smem_slot<..., PS>).
// After the last butterflies the outputs stay in v for the caller.
template <int LOG_L, int LOG_W, bool CFAST, int S, int T, int PS, int STAGE>
FDEV void run_stages(float2 *v, float2 *sm, const float2 *__restrict__ twL)
{
    using I = StageInfo<LOG_L, STAGE>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        butterfly_coords<LOG_L, LOG_W, CFAST, I::LOG_R>(threadIdx.x + T * b, c, j);
        butterfly<LOG_L, STAGE, S>(v + b * I::R, j, twL);
    }
    if constexpr (!I::LAST) {
        __syncthreads();  // every thread has read this stage's inputs from sm
#pragma unroll
        for (int b = 0; b < B; ++b) {
            int c, j;
            butterfly_coords<LOG_L, LOG_W, CFAST, I::LOG_R>(threadIdx.x + T * b, c, j);
#pragma unroll
            for (int r = 0; r < I::R; ++r)
                sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, stockham_out_index<LOG_L, STAGE>(j, r))] =
                    v[b * I::R + r];
        }
        __syncthreads();
        gather<LOG_L, LOG_W, CFAST, T, STAGE + 1>(
            v, [&](int c, int i) { return sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, i)]; });
        run_stages<LOG_L, LOG_W, CFAST, S, T, PS, STAGE + 1>(v, sm, twL);
    }
}

FDEV float power_of(float2 x) { return x.x * x.x + x.y * x.y; }

// --------------------------------------------------------------------- k_lines

struct LinesArgs {
    const float2 *in;
    void *out;
    int64_t tiles_per_seg;      // tiles in one segment (CFAST); 1 for segment-major tiles
    int64_t nseg;               // segment-major: segments in the batch (masks the ragged last tile)
    int64_t in_seg, out_seg;    // element stride between segments (segment-major: between tiles)
    int64_t in_tile, out_tile;  // element stride between tiles of one segment
    int64_t in_cs, in_is;       // input: stride between lines, between points of a line
    int64_t out_cs, out_is;     // output: same
    const float2 *twL;          // w_L^m, m < L
    const float2 *tw4a;         // four-step twiddle rows k1 mod 2^tw_log_k, [2^tw_log_k][tw_ncols], or null
    const float2 *tw4b;         // rows k1 >> tw_log_k, [n1 >> tw_log_k][tw_ncols], or null
    int64_t tw_ncols;
    int tw_log_k;
    int in_staged;              // 1: load through shared memory, coalesced along the line (in_is == 1)
    int out_power;              // 1: store |X|^2 as float
    float scale;
};

template <int LOG_L, int LOG_W, bool CFAST, int S, int T>
__global__ void __launch_bounds__(T) k_lines(const LinesArgs a)
{
    constexpr int L = 1 << LOG_L, W = 1 << LOG_W, E = L * W, V = E / T;
    constexpr int PS = 4;
    static_assert(V == 16 || (L < 16 && V == L), "16 points per thread");
    extern __shared__ float2 sm[];
    const int64_t u = blockIdx.x;
    const int64_t seg = u / a.tiles_per_seg, tile = u - seg * a.tiles_per_seg;
    const float2 *__restrict__ in = a.in + seg * a.in_seg + tile * a.in_tile;
    const int64_t line0 = CFAST ? 0 : u * W;
    const int64_t out_base = seg * a.out_seg + tile * a.out_tile;
    float2 v[V];

    if (a.in_staged) {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int e = threadIdx.x + T * q;
            const int c = e >> LOG_L, i = e & (L - 1);
            float2 x = make_float2(0.f, 0.f);
            if (CFAST || line0 + c < a.nseg) x = in[c * a.in_cs + i];
            sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, i)] = x;
        }
        __syncthreads();
        gather<LOG_L, LOG_W, CFAST, T, 0>(v, [&](int c, int i) { return sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, i)]; });
    } else {
        gather<LOG_L, LOG_W, CFAST, T, 0>(v, [&](int c, int i) {
            if (CFAST || line0 + c < a.nseg) return in[c * a.in_cs + i * a.in_is];
            return make_float2(0.f, 0.f);
        });
    }
    run_stages<LOG_L, LOG_W, CFAST, S, T, PS, 0>(v, sm, a.twL);

    const float scale = a.scale;
    scatter_last<LOG_L, LOG_W, CFAST, T>(v, [&](int c, int i, float2 x) {
        if (!CFAST && line0 + c >= a.nseg) return;
        if (a.tw4a) {  // four-step twiddle w_n^{col * k1}, k1 = i
            const int64_t col = tile * W + c;
            float2 w = __ldg(a.tw4a + (int64_t)(i & ((1 << a.tw_log_k) - 1)) * a.tw_ncols + col);
            if (a.tw4b) {
                const float2 w2 = __ldg(a.tw4b + (int64_t)(i >> a.tw_log_k) * a.tw_ncols + col);
                w = make_float2(w.x * w2.x - w.y * w2.y, w.x * w2.y + w.y * w2.x);
            }
            x = twmul<S>(x, w);
        }
        if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
        const int64_t o = out_base + c * a.out_cs + i * a.out_is;
        if (a.out_power) static_cast<float *>(a.out)[o] = power_of(x);
        else static_cast<float2 *>(a.out)[o] = x;
    });
}

// ------------------------------------------------------------------- k_cluster

struct ClusterArgs {
    const float2 *in;
    void *out;
    const float2 *twA;  // w_{N1}^m
    const float2 *twB;  // w_{N2}^m
    const float2 *tw4;  // w_n^{k1 j2}, [N1][N2]
    int out_power;
    float scale;
};

template <int LOG_N1, int LOG_N2, int LOG_C>
struct ClusterShape {
    static constexpr int C = 1 << LOG_C;
    static constexpr int LOG_WA = LOG_N2 - LOG_C;  // columns per CTA in the column pass
    static constexpr int LOG_WB = LOG_N1 - LOG_C;  // rows per CTA in the row pass
    static constexpr int E = 1 << (LOG_N1 + LOG_N2 - LOG_C);
    static constexpr int T = E / 16;
    static constexpr int PSA = 4;
    static constexpr int PSB = LOG_WB < 4 ? 4 : LOG_WB;
    static constexpr int SLOTS_A = smem_slots<LOG_N1, LOG_WA, PSA>();
    static constexpr int SLOTS_B = smem_slots<LOG_N2, LOG_WB, PSB>();
    static constexpr int SLOTS = SLOTS_A > SLOTS_B ? SLOTS_A : SLOTS_B;
};

template <int LOG_N1, int LOG_N2, int LOG_C, int S>
__global__ void __cluster_dims__(1 << LOG_C, 1, 1)
    __launch_bounds__(ClusterShape<LOG_N1, LOG_N2, LOG_C>::T) k_cluster(const ClusterArgs a)
{
    using Sh = ClusterShape<LOG_N1, LOG_N2, LOG_C>;
    constexpr int N1 = 1 << LOG_N1, N2 = 1 << LOG_N2, T = Sh::T;
    constexpr int WA = 1 << Sh::LOG_WA, WB = 1 << Sh::LOG_WB;
    extern __shared__ float2 sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int64_t seg = blockIdx.x >> LOG_C;
    const float2 *__restrict__ in = a.in + seg * ((int64_t)N1 * N2);
    float2 v[16];

    // column pass: line c is column j2 = rank*WA + c, points at j1*N2 + j2
    gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int c, int i) { return in[i * N2 + rank * WA + c]; });
    run_stages<LOG_N1, Sh::LOG_WA, true, S, T, Sh::PSA, 0>(v, sm, a.twA);

    cl.sync();  // every CTA of the cluster is done with its own buffer
    scatter_last<LOG_N1, Sh::LOG_WA, true, T>(v, [&](int c, int k1, float2 x) {
        const int j2 = rank * WA + c;
        x = twmul<S>(x, __ldg(a.tw4 + k1 * N2 + j2));
        float2 *dst = cl.map_shared_rank(sm, k1 >> Sh::LOG_WB);
        dst[smem_slot<LOG_N2, Sh::LOG_WB, true, Sh::PSB>(k1 & (WB - 1), j2)] = x;
    });
    cl.sync();  // every row this CTA owns has arrived

    // row pass: line c is row k1 = rank*WB + c, points over j2
    gather<LOG_N2, Sh::LOG_WB, true, T, 0>(
        v, [&](int c, int i) { return sm[smem_slot<LOG_N2, Sh::LOG_WB, true, Sh::PSB>(c, i)]; });
    run_stages<LOG_N2, Sh::LOG_WB, true, S, T, Sh::PSB, 0>(v, sm, a.twB);

    const float scale = a.scale;
    const int64_t obase = seg * ((int64_t)N1 * N2) + rank * WB;
    scatter_last<LOG_N2, Sh::LOG_WB, true, T>(v, [&](int c, int k2, float2 x) {
        if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
        const int64_t o = obase + (int64_t)k2 * N1 + c;
        if (a.out_power) static_cast<float *>(a.out)[o] = power_of(x);
        else static_cast<float2 *>(a.out)[o] = x;
    });
}

}  // namespace fftseg
