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

#include <type_traits>

#include "engine.cuh"
#include "tc.cuh"

namespace fftseg {

namespace cg = cooperative_groups;

// f(std::integral_constant<int, i>()) for i = I .. N-1 (indices usable as
// template arguments inside f).
template <int N, int I = 0, class F>
FDEV void unroll_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>());
        unroll_for<N, I + 1>(f);
    }
}

// ---------------------------------------------------------------- stage runner

// Thread -> butterfly coordinates of stage STAGE.  CFAST tiles put lanes
// along the lines; with JLAST the last stage instead puts lanes along the
// points of a line (the shared-memory layout does not change).
template <int LOG_L, int LOG_W, bool CFAST, bool JLAST, int STAGE>
FDEV void stage_coords(int g, int &c, int &j)
{
    using I = StageInfo<LOG_L, STAGE>;
    butterfly_coords<LOG_L, LOG_W, CFAST && !(JLAST && I::LAST), I::LOG_R>(g, c, j);
}

template <int LOG_L, int LOG_W, bool CFAST, int T, int STAGE, bool JLAST = false, class Get>
FDEV void gather(float2 *v, Get &&get)
{
    using I = StageInfo<LOG_L, STAGE>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        stage_coords<LOG_L, LOG_W, CFAST, JLAST, STAGE>(threadIdx.x + T * b, c, j);
#pragma unroll
        for (int r = 0; r < I::R; ++r) v[b * I::R + r] = get(c, j + (r << (LOG_L - I::LOG_R)));
    }
}

// Hand every output of the last stage, (line c, index i), to put().
template <int LOG_L, int LOG_W, bool CFAST, int T, bool JLAST = false, class Put>
FDEV void scatter_last(const float2 *v, Put &&put)
{
    constexpr int LASTS = StageInfo<LOG_L, 0>::NSTAGES - 1;
    using I = StageInfo<LOG_L, LASTS>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        stage_coords<LOG_L, LOG_W, CFAST, JLAST, LASTS>(threadIdx.x + T * b, c, j);
#pragma unroll
        for (int r = 0; r < I::R; ++r) put(c, j + (r << (LOG_L - I::LOG_R)), v[b * I::R + r]);
    }
}

// As scatter_last, also passing the butterfly slot b of the calling thread.
template <int LOG_L, int LOG_W, bool CFAST, int T, class Put>
FDEV void scatter_last_b(const float2 *v, Put &&put)
{
    using I = StageInfo<LOG_L, StageInfo<LOG_L, 0>::NSTAGES - 1>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        int c, j;
        butterfly_coords<LOG_L, LOG_W, CFAST, I::LOG_R>(threadIdx.x + T * b, c, j);
#pragma unroll
        for (int r = 0; r < I::R; ++r) put(b, c, j + (r << (LOG_L - I::LOG_R)), v[b * I::R + r]);
    }
}

// Run stages STAGE..last on the values in v (this stage's inputs).  Between
// stages the tile goes through shared memory `sm` (layout smem_slot<..., PS>).
// After the last butterflies the outputs stay in v for the caller.  IN_SM:
// this stage's inputs were read from `sm` (so a barrier must separate those
// reads from the writes below).
// Barrier among the T threads that run the stages: the whole CTA, or (when
// other warps of the CTA do other work) named barrier 1 over threads 0..T-1.
template <int T, bool NAMED>
FDEV void stage_sync()
{
    if constexpr (NAMED) asm volatile("bar.sync 1, %0;" ::"n"(T) : "memory");
    else __syncthreads();
}

// Stage twiddles of stage STAGE for this thread's butterflies, loaded ahead
// of use (they depend only on the thread's coordinates): tw[b*(R-1) + r-1].
template <int LOG_L, int LOG_W, bool CFAST, int T, int STAGE, bool JLAST>
struct StageTw {
    using I = StageInfo<LOG_L, STAGE>;
    static constexpr int B = ((1 << (LOG_L + LOG_W)) / T) / I::R;
    static constexpr int COUNT = I::FIRST ? 1 : B * (I::R - 1);
    float2 w[COUNT];
    // TW_SM: twL points into shared memory (plain loads), else global (read-only path)
    template <bool TW_SM = false>
    FDEV void load(const float2 *__restrict__ twL)
    {
        if constexpr (!I::FIRST) {
            constexpr int OFF = stage_table_offset<LOG_L>(STAGE);
#pragma unroll
            for (int b = 0; b < B; ++b) {
                int c, j;
                stage_coords<LOG_L, LOG_W, CFAST, JLAST, STAGE>(threadIdx.x + T * b, c, j);
                const float2 *t = twL + OFF + (j & (I::NS - 1));
#pragma unroll
                for (int r = 1; r < I::R; ++r) {
                    if constexpr (TW_SM) w[b * (I::R - 1) + r - 1] = t[(r - 1) * I::NS];
                    else w[b * (I::R - 1) + r - 1] = __ldg(t + (r - 1) * I::NS);
                }
            }
        }
    }
};

template <int LOG_L, int LOG_W, bool CFAST, int S, int T, int PS, int STAGE, bool IN_SM = true, bool JLAST = false,
          int PREC = PREC_FP32, bool NAMED = false, bool TW_SM = false>
FDEV void run_stages(float2 *v, float2 *sm, const float2 *__restrict__ twL, const TcCtx *tc = nullptr,
                     const StageTw<LOG_L, LOG_W, CFAST, T, STAGE, JLAST> *pre = nullptr)
{
    using I = StageInfo<LOG_L, STAGE>;
    constexpr int V = (1 << (LOG_L + LOG_W)) / T, B = V / I::R;
    // the next stage's twiddles are requested now (global tables); their
    // latency hides behind this stage's butterflies and the exchange.  Tables
    // in shared memory are read at use.
    StageTw<LOG_L, LOG_W, CFAST, T, (I::LAST ? STAGE : STAGE + 1), JLAST> next;
    if constexpr (!I::LAST && !TW_SM) next.load(twL);
    StageTw<LOG_L, LOG_W, CFAST, T, STAGE, JLAST> mine;
    if constexpr (!I::FIRST) {
        if (pre) mine = *pre;
        else mine.template load<TW_SM>(twL);
    }
#pragma unroll
    for (int b = 0; b < B; ++b) {
        float2 *x = v + b * I::R;
        if constexpr (!I::FIRST) {
#pragma unroll
            for (int r = 1; r < I::R; ++r) x[r] = twmul<S>(x[r], mine.w[b * (I::R - 1) + r - 1]);
        }
        if constexpr (PREC != PREC_FP32 && I::R == 16) {
            // radix-16 stages on the tensor cores (warp-collective; every
            // lane of every warp takes this branch together)
            dft16_tc<S, PREC>(x, *tc);
        } else {
            dft<I::R, S>(x);
        }
    }
    if constexpr (!I::LAST) {
        if constexpr (IN_SM) stage_sync<T, NAMED>();  // every thread has read this stage's inputs from sm
#pragma unroll
        for (int b = 0; b < B; ++b) {
            int c, j;
            stage_coords<LOG_L, LOG_W, CFAST, JLAST, STAGE>(threadIdx.x + T * b, c, j);
#pragma unroll
            for (int r = 0; r < I::R; ++r)
                sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, stockham_out_index<LOG_L, STAGE>(j, r))] =
                    v[b * I::R + r];
        }
        stage_sync<T, NAMED>();
        gather<LOG_L, LOG_W, CFAST, T, STAGE + 1, JLAST>(
            v, [&](int c, int i) { return sm[smem_slot<LOG_L, LOG_W, CFAST, PS>(c, i)]; });
        run_stages<LOG_L, LOG_W, CFAST, S, T, PS, STAGE + 1, true, JLAST, PREC, NAMED, TW_SM>(v, sm, twL, tc,
                                                                                          TW_SM ? nullptr : &next);
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
    const float2 *twL;          // stage twiddle tables of a length-L line
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

// --------------------------------------------------------------------- k_block

// Single-pass segment-major tiles (n <= 4096).  Persistent: each CTA walks
// tiles u, u + gridDim.x, ...; tile u (W whole segments, contiguous in memory)
// arrives by one TMA bulk copy into a double buffer while the previous tile
// is being transformed.
struct BlockArgs {
    const float2 *in;
    void *out;
    int64_t nseg;
    int64_t ntiles;
    const float2 *twL;  // stage twiddle tables of a length-n line
    int *err;           // set to 1 if a copy never completed
    int out_power;
    float scale;
};

template <int LOG_L>
struct BlockShape {
    // 16 points per thread, 256 threads, 4096 points per tile; lines shorter
    // than 16 points put L points in a thread and 256 lines in a tile.
    static constexpr int LOG_W = LOG_L >= 4 ? 12 - LOG_L : 8;
    static constexpr int T = 256;
    static constexpr int E = 1 << (LOG_L + LOG_W);
    static constexpr int PS = 4;
    static constexpr int SLOTS = (smem_slots<LOG_L, LOG_W, PS>() + 1) & ~1;  // keeps the barriers 8-byte aligned
    static constexpr size_t SMEM = (size_t)(SLOTS + 2 * E) * sizeof(float2) + 2 * sizeof(uint64_t);
};

// One tile of whole segments, already in shared memory (Pb, dense [c][i]):
// W segments from segment line0 on (those at or past nseg are not stored).
// With tensor-core stages tc->stage must point into Pb (this warp's 4 KB).
template <int LOG_L, int S, int PREC = PREC_FP32>
FDEV void block_tile(const float2 *Pb, float2 *X, const float2 *__restrict__ twL, int64_t line0, int64_t nseg,
                     void *out, int out_power, float scale, const TcCtx *tc)
{
    using Sh = BlockShape<LOG_L>;
    constexpr int L = 1 << LOG_L, T = Sh::T, V = Sh::E / T;
    float2 v[V];
    gather<LOG_L, Sh::LOG_W, false, T, 0>(v, [&](int c, int i) { return Pb[(c << LOG_L) + i]; });
    if constexpr (PREC == PREC_FP32) {
        run_stages<LOG_L, Sh::LOG_W, false, S, T, Sh::PS, 0, false>(v, X, twL);
    } else {
        __syncthreads();  // the tensor-core stages stage their operands in the tile just read
        run_stages<LOG_L, Sh::LOG_W, false, S, T, Sh::PS, 0, false, false, PREC>(v, X, twL, tc);
    }
    scatter_last<LOG_L, Sh::LOG_W, false, T>(v, [&](int c, int i, float2 x) {
        if (line0 + c >= nseg) return;
        if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
        const int64_t o = (line0 + c) * L + i;
        if (out_power) static_cast<float *>(out)[o] = power_of(x);
        else static_cast<float2 *>(out)[o] = x;
    });
}

template <int LOG_L, int S, int PREC = PREC_FP32>
__global__ void __launch_bounds__(256, PREC == PREC_FP32 ? 2 : 1) k_block(const BlockArgs a)
{
    using Sh = BlockShape<LOG_L>;
    constexpr int L = 1 << LOG_L, W = 1 << Sh::LOG_W, E = Sh::E, T = Sh::T, V = E / T;
    // TMA destinations first: the dynamic shared base is 1024-byte aligned and
    // each prefetch buffer is a multiple of 1024 bytes
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;
    float2 *X = sm + 2 * E;
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    const int tid = threadIdx.x;
    if (smem_u32(P) & 127) {  // never expected; refuse rather than issue a misaligned copy
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
    // (launched with programmatic stream serialization: the next launch's
    // blocks may take the SMs this grid leaves; this grid's blocks start the
    // L2 fetch of their first two tiles, then wait here for the previous
    // kernel's writes)
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
    const float scale = a.scale;
    [[maybe_unused]] TcCtx tc;
    if constexpr (PREC != PREC_FP32) tc_init<S, PREC>(tc, P);
    for (int k = 0; u < a.ntiles; u += gridDim.x, ++k) {
        const int b = k & 1;
        if (u + gridDim.x < a.ntiles) issue(u + gridDim.x, b ^ 1);
        mbar_wait(&bar[b], (k >> 1) & 1, a.err);
        if constexpr (PREC != PREC_FP32) tc.stage = P + b * E + (threadIdx.x >> 5) * 512;
        block_tile<LOG_L, S, PREC>(P + b * E, X, a.twL, u * W, a.nseg, a.out, a.out_power, scale, &tc);
        __syncthreads();  // P[b] fully read before it is refilled two tiles on
    }
}

// ------------------------------------------------------------------- k_cluster

struct ClusterArgs {
    CUtensorMap tmap;  // the input as [nseg][N1][N2] 8-byte elements, box [1][N1][WA]
    const float2 *in;
    void *out;
    int64_t nseg;
    const float2 *twA;  // stage twiddle tables, length N1
    const float2 *twB;  // stage twiddle tables, length N2
    const float2 *tw4;  // w_n^{k1 j2}, [N1][N2]
    const float2 *rtw;  // real-signal segments: w_{2n}^k for k = 0 .. n/2
    // Bluestein rows (BL kernels, the inverse M-point transform of a row of
    // n < M): the input times bl_bhat[m] as it is read; bin k < bl_n of the
    // result times scale * bl_w[k] to out[row * bl_n + k]; bins k >= bl_n dropped.
    // (BF kernels, the forward transform: point m of row s is
    // in[s * bl_n + m] * bl_w[m] for m < bl_n and 0 above, read straight from
    // global memory.)
    const float2 *bl_bhat;
    const float2 *bl_w;
    int64_t bl_n;
    int *err;
    int out_power;
    float scale;
};

#ifndef FFTSEG_CLUSTER_MINB
#define FFTSEG_CLUSTER_MINB 3
#endif

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
    // one source CTA's part of a receiver's row-pass buffer: WA*WB points plus pads
    static constexpr int Q = 1 << (LOG_WA + LOG_WB);
    static constexpr int SLICE = Q + (Q >> PSB);
    static constexpr int SEND = C * SLICE;
    static constexpr int U0 = SLOTS_A > SEND ? SLOTS_A : SEND;
    static constexpr int SLOTS_U = ((U0 > E ? U0 : E) + 1) & ~1;
    static constexpr int SLOTS_X = (SLOTS_B + 1) & ~1;
    static constexpr int R_LAST = StageInfo<LOG_N1, StageInfo<LOG_N1, 0>::NSTAGES - 1>::R;
    // stage twiddle tables of the column and row lines (one copy when N1 == N2)
    static constexpr int TWA = stage_table_offset<LOG_N1>(StageInfo<LOG_N1, 0>::NSTAGES);
    static constexpr int TWB = LOG_N1 == LOG_N2 ? 0 : stage_table_offset<LOG_N2>(StageInfo<LOG_N2, 0>::NSTAGES);
    // U (input tile, column-pass scratch, send staging) | X (row pass) | TR | stage tables | barriers
    static constexpr size_t SMEM =
        (size_t)(SLOTS_U + SLOTS_X + R_LAST * (1 << LOG_WA) + TWA + TWB) * sizeof(float2) + 2 * sizeof(uint64_t);
    static constexpr int MINB = T <= 256 ? FFTSEG_CLUSTER_MINB : 1;  // CTAs per SM the registers must allow
};

// One cluster of C CTAs per segment, persistent over segments
// s = cluster, cluster + nclusters, ...  CTA r of the cluster owns the column
// slab j2 in [r*WA, (r+1)*WA) (N1 rows of WA points) in the column pass and
// the rows k1 in [r*WB, (r+1)*WB) in the row pass.  Two shared buffers:
//  - U receives the slab (one tiled TMA copy), serves as the column pass's
//    exchange buffer, and finally stages the column-pass results times the
//    four-step twiddle exactly as each receiver's row-pass buffer wants them
//    (one slice per receiver); C bulk shared-to-shared copies send the slices,
//    completing on the receivers' barriers `rbar`.  Once those copies have
//    read U, the next segment's slab is requested into it, so the load
//    overlaps the row pass.
//  - X receives the slices and serves as the row pass's exchange buffer.  A
//    relaxed cluster barrier makes sure no receiver still reads it before the
//    copies are sent: each CTA arrives once its row pass has consumed X (end
//    of an iteration) and waits just before it sends (after the next column
//    pass), so the barrier's latency hides behind a column pass.
//  - The stage twiddle tables are copied into shared memory once.
//  - Four-step twiddle w_n^{j2 k1} with k1 = j + (N1/R)*q (j = butterfly
//    index of the last column stage): w_n^{j2 j} (per thread, kept in
//    registers) times w_n^{j2 (N1/R) q} (table TR in shared memory), both
//    exact table entries.
// RF (forward real-signal segments, S = -1): a segment is 2n real samples
// read as n complex values z[m] = x[2m] + i x[2m+1], and the output is the
// n + 1 bins of their real DFT.  Bin k = k1 + N1 k2 needs A = Z[k] and
// B = conj(Z[(n - k) mod n]), which sits in row (N1 - k1) mod N1 (column
// N2 - 1 - k2 for k1 > 0, column -k2 mod N2 for k1 = 0).  So the row pass
// deals rows out in mirror pairs (rf_row): CTA d takes rows d H + c and
// their mirrors N1 - (d H + c), c < H = WB/2 (CTA 0: rows 0 and N1/2 are
// their own mirrors), and the split is local to the CTA:
//   X[k] = (A + B) / 2 + w_{2n}^k (-i) (A - B) / 2,   X[n] = Re Z[0] - Im Z[0].
// Mirror-pair rows of the RF row pass: local row c of CTA d -> row k1, and back.
template <int N1, int WB>
FDEV int rf_row(int d, int c)
{
    constexpr int H = WB / 2;
    if (c < H) return d * H + c;
    const int m = d * H + c - H;
    return m == 0 ? N1 / 2 : N1 - m;
}
template <int N1, int WB>
FDEV void rf_place(int k1, int &d, int &c)
{
    // k1 < N1/2: m = k1, first half; k1 > N1/2: m = N1 - k1, second half;
    // k1 = N1/2: m = 0, second half of CTA 0
    constexpr int H = WB / 2;
    const int hb = k1 >= N1 / 2;
    const int m = (hb ? N1 - k1 : k1) & (N1 / 2 - 1);
    d = m / H;
    c = hb * H + (m & (H - 1));
}

// RI (inverse real-signal segments, S = +1): the input is the n + 1 bins
// X[0..n] of each segment's real DFT (stride n + 1), and the column pass
// reads them straight from global memory, each point m taking
//   Z[m] = (A + B) + i conj(w_{2n}^m) (A - B),  A = X[m], B = conj(X[n - m])
// (the imaginary parts of X[0] and X[n] ignored), so that the inverse
// n-point transform of Z gives x[2j] + i x[2j + 1] (no slab copy, no
// intermediate; the mirror point's load is another CTA's, mostly from L2).
// BL (Bluestein rows, S = +1): the inverse transform of the product with
// B, its input multiplied by B as the column pass reads the slab, and the
// chirp-out and the crop to n bins in the row pass's epilogue (the pointwise
// product and chirp-out passes of the chunked form folded in).
// BF (Bluestein rows, S = -1): the forward transform of the chirped row,
// read from the n input samples directly (zero past n, no slab copy).
template <int LOG_N1, int LOG_N2, int LOG_C, int S, bool RF = false, bool RI = false, bool BL = false,
          bool BF = false>
__global__ void __launch_bounds__(ClusterShape<LOG_N1, LOG_N2, LOG_C>::T, ClusterShape<LOG_N1, LOG_N2, LOG_C>::MINB)
    k_cluster(const __grid_constant__ ClusterArgs a)
{
    constexpr bool DIRECT = RI || BF;  // the column pass reads global memory itself (no slab copy)
    using Sh = ClusterShape<LOG_N1, LOG_N2, LOG_C>;
    constexpr int N1 = 1 << LOG_N1, N2 = 1 << LOG_N2, T = Sh::T, E = Sh::E, C = Sh::C;
    constexpr int WA = 1 << Sh::LOG_WA, WB = 1 << Sh::LOG_WB;
    constexpr int64_t N = (int64_t)N1 * N2;
    constexpr int LOG_STEP = LOG_N1 - StageInfo<LOG_N1, StageInfo<LOG_N1, 0>::NSTAGES - 1>::LOG_R;  // log2(N1/R)
    // the tiled TMA write needs a 128-byte aligned destination: U comes first
    extern __shared__ __align__(1024) float2 sm[];
    float2 *U = sm;
    float2 *X = U + Sh::SLOTS_U;
    float2 *TR = X + Sh::SLOTS_X;
    float2 *TWA = TR + Sh::R_LAST * WA;
    float2 *TWB = LOG_N1 == LOG_N2 ? TWA : TWA + Sh::TWA;
    uint64_t *bar = reinterpret_cast<uint64_t *>(TWA + Sh::TWA + Sh::TWB);  // slab arrived
    uint64_t *rbar = bar + 1;                                            // row-pass slices arrived
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x;
    if (smem_u32(U) & 127) {  // same layout in every CTA: the whole cluster leaves together
        if (tid == 0) atomicOr(a.err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(rbar, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < Sh::R_LAST * WA; e += T)  // TR[q][c] = w_n^{(rank*WA + c) (N1/R) q}
        TR[e] = __ldg(a.tw4 + (int64_t)((e >> Sh::LOG_WA) << LOG_STEP) * N2 + rank * WA + (e & (WA - 1)));
    for (int e = tid; e < Sh::TWA; e += T) TWA[e] = __ldg(a.twA + e);
    if constexpr (Sh::TWB > 0)
        for (int e = tid; e < Sh::TWB; e += T) TWB[e] = __ldg(a.twB + e);
    // w_n^{j2 j} for this thread's butterflies of the last column stage
    float2 wbase[(E / T) / Sh::R_LAST];
    {
        using IL = StageInfo<LOG_N1, StageInfo<LOG_N1, 0>::NSTAGES - 1>;
#pragma unroll
        for (int b = 0; b < (E / T) / IL::R; ++b) {
            int c, j;
            butterfly_coords<LOG_N1, Sh::LOG_WA, true, IL::LOG_R>(tid + T * b, c, j);
            wbase[b] = __ldg(a.tw4 + (int64_t)j * N2 + rank * WA + c);
        }
    }
    // RF: this thread's local row of the row pass (fixed: T is a multiple of
    // WB), its row k1 and its mirror's local row, and the split's factors
    // -i (scale/2) w_{2n}^{k1 + N1 j} for the butterflies j of the last row
    // stage (bin k = k1 + N1 (j + r N2/R) then takes that times w_{2R}^r)
    static_assert(!RF || WB >= 2, "mirror pairs of rows per CTA");
    using IRL = StageInfo<LOG_N2, StageInfo<LOG_N2, 0>::NSTAGES - 1>;
    constexpr int RB = (E / T) / IRL::R;
    const int rcl = tid & (WB - 1);
    const int rk1 = RF ? rf_row<N1, WB>(rank, rcl) : 0;
    const int rcm = (rk1 == 0 || rk1 == N1 / 2) ? rcl : rcl ^ (WB / 2);
    float2 rpw[RF ? RB : 1];
    if constexpr (RF) {
        const float2 w1 = __ldg(a.rtw + rk1);  // k1 < N1 <= n/2
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            int c, j;
            butterfly_coords<LOG_N2, Sh::LOG_WB, true, IRL::LOG_R>(tid + T * b, c, j);
            const float2 w2 = __ldg(a.rtw + N1 * j);  // N1 j < n / R <= n/2
            const float h = 0.5f * a.scale;
            const float2 w = make_float2(h * (w1.x * w2.x - w1.y * w2.y), h * (w1.x * w2.y + w1.y * w2.x));
            rpw[b] = make_float2(w.y, -w.x);  // times -i
        }
    }
    cl.sync();  // every peer's barriers are initialised before any copy reaches them
    const uint32_t x_remote0 = smem_u32(X) + (uint32_t)(rank * Sh::SLICE * sizeof(float2));

    auto issue = [&](int64_t s) {  // thread 0
        fence_proxy_async();
        mbar_expect_tx(bar, (uint32_t)(E * sizeof(float2)));
        tma_load_3d(U, &a.tmap, rank * WA, 0, (int)s, bar);
    };

    const int64_t cid = blockIdx.x >> LOG_C, ncl = gridDim.x >> LOG_C;
    int64_t s = cid;
    if (!DIRECT && s < a.nseg && tid == 0) issue(s);
    const float scale = a.scale;
    cluster_arrive_relaxed();  // X is free
    for (int k = 0; s < a.nseg; s += ncl, ++k) {
        if (tid == 0) mbar_expect_tx(rbar, (uint32_t)(C * Sh::SLICE * sizeof(float2)));  // this segment's rows
        if constexpr (!DIRECT) mbar_wait(bar, k & 1, a.err);
        float2 v[16];

        // column pass: line c is column j2 = rank*WA + c, points j1 = i
        if constexpr (RI) {
            static_assert(!RI || (S == 1 && !RF), "real-signal bins in: inverse only");
            const float2 *Xs = a.in + s * (N + 1);
            gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int c, int i) {
                const int m = i * N2 + rank * WA + c;
                float2 A = __ldg(Xs + m), Cm = __ldg(Xs + ((int)N - m));  // X[m], X[n - m] (X[n] at m = 0)
                if (m == 0) {
                    A.y = 0.f;
                    Cm.y = 0.f;
                }
                // conj(w_{2n}^m) from the table of m <= n/2 (w_{2n}^m = -conj(w_{2n}^{n-m}) above)
                const bool lo = 2 * m <= (int)N;
                const float2 t = __ldg(a.rtw + (lo ? m : (int)N - m));
                const float2 cw = lo ? make_float2(t.x, -t.y) : make_float2(-t.x, -t.y);
                const float sx = A.x + Cm.x, sy = A.y - Cm.y;  // A + B, B = conj(X[n - m])
                const float dx = A.x - Cm.x, dy = A.y + Cm.y;  // A - B
                const float ex = cw.x * dx - cw.y * dy, ey = cw.x * dy + cw.y * dx;
                return make_float2(sx - ey, sy + ex);  // (A + B) + i conj(w) (A - B)
            });
        } else if constexpr (BF) {
            static_assert(!BF || (S == -1 && !RF && !BL), "Bluestein rows in: the forward transform only");
            const int64_t nb = a.bl_n;
            const float2 *xs = a.in + s * nb;
            gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int c, int i) {
                const int64_t m = (int64_t)i * N2 + rank * WA + c;
                if (m >= nb) return make_float2(0.f, 0.f);
                const float2 x = __ldg(xs + m), w = __ldg(a.bl_w + m);
                return make_float2(x.x * w.x - x.y * w.y, x.x * w.y + x.y * w.x);
            });
        } else if constexpr (BL) {
            static_assert(!BL || (S == 1 && !RF && !RI), "Bluestein rows: the inverse transform only");
            gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int c, int i) {
                const float2 x = U[i * WA + c], b = __ldg(a.bl_bhat + i * N2 + rank * WA + c);
                return make_float2(x.x * b.x - x.y * b.y, x.x * b.y + x.y * b.x);
            });
        } else {
            gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int c, int i) { return U[i * WA + c]; });
        }
        run_stages<LOG_N1, Sh::LOG_WA, true, S, T, Sh::PSA, 0, true, false, PREC_FP32, false, true>(v, U, TWA);
        __syncthreads();  // U no longer read as column-pass scratch

        // send staging: slice d of U holds, for receiver d, element
        // (k1, j2) at q' = (j2 - rank*WA)*WB + (k1 mod WB), padded as in X
        scatter_last_b<LOG_N1, Sh::LOG_WA, true, T>(v, [&](int b, int c, int k1, float2 x) {
            const float2 w = TR[(k1 >> LOG_STEP) * WA + c];  // k1 = j + (N1/R) q
            const float2 wb = wbase[b];
            x = twmul<S>(x, make_float2(w.x * wb.x - w.y * wb.y, w.x * wb.y + w.y * wb.x));
            int d = k1 >> Sh::LOG_WB, cl = k1 & (WB - 1);
            if constexpr (RF) rf_place<N1, WB>(k1, d, cl);
            const int qq = c * WB + cl;
            U[d * Sh::SLICE + qq + (qq >> Sh::PSB)] = x;
        });
        fence_proxy_async();      // these generic writes are read by the async-proxy copies below
        __syncthreads();          // U complete
        cluster_wait();           // no receiver still reads its X
        if (tid == 0) {
#pragma unroll 1
            for (int d = 0; d < C; ++d)
                dsmem_bulk_copy(mapa_u32(x_remote0, d), U + d * Sh::SLICE, Sh::SLICE * sizeof(float2),
                                mapa_u32(smem_u32(rbar), d));
            bulk_commit();
        }
        mbar_wait(rbar, k & 1, a.err);  // every slice of this CTA's rows has arrived
        if (tid == 0) {
            bulk_wait_read_all();  // the outgoing copies have read U: refill it
            if (!DIRECT && s + ncl < a.nseg) issue(s + ncl);
        }

        // row pass: line c is row k1 = rank*WB + c, points j2 = i
        gather<LOG_N2, Sh::LOG_WB, true, T, 0>(
            v, [&](int c, int i) { return X[smem_slot<LOG_N2, Sh::LOG_WB, true, Sh::PSB>(c, i)]; });
        run_stages<LOG_N2, Sh::LOG_WB, true, S, T, Sh::PSB, 0, true, false, PREC_FP32, false, true>(v, X, TWB);

        if constexpr (BL) {
            // bin k = k1 + N1 k2 of the row: the chirp-out and the crop to n bins
            const int64_t nb = a.bl_n;
            scatter_last<LOG_N2, Sh::LOG_WB, true, T>(v, [&](int c, int k2, float2 x) {
                const int64_t k = rank * WB + c + (int64_t)k2 * N1;
                if (k >= nb) return;
                const float2 w = __ldg(a.bl_w + k);
                x = make_float2(scale * (x.x * w.x - x.y * w.y), scale * (x.x * w.y + x.y * w.x));
                if (a.out_power) static_cast<float *>(a.out)[s * nb + k] = power_of(x);
                else static_cast<float2 *>(a.out)[s * nb + k] = x;
            });
        } else if constexpr (!RF) {
            const int64_t obase = s * N + rank * WB;
            scatter_last<LOG_N2, Sh::LOG_WB, true, T>(v, [&](int c, int k2, float2 x) {
                if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
                const int64_t o = obase + (int64_t)k2 * N1 + c;
                if (a.out_power) static_cast<float *>(a.out)[o] = power_of(x);
                else static_cast<float2 *>(a.out)[o] = x;
            });
        } else {
            static_assert(!RF || S == -1, "real-signal segments: forward only");
            // Bins pair up: k (column k2 < N2/2, i.e. r < R/2) with n - k (its
            // mirror row's column N2 - 1 - k2, or -k2 mod N2 in row 0).  With
            // A = Z[k], B = conj(Z[n - k]), P = (scale/2)(A + B) and
            // Q = -i (scale/2) w_{2n}^k (A - B):  X[k] = P + Q, X[n - k] = conj(P - Q)
            // (w_{2n}^{n-k} = -conj(w_{2n}^k)).  k = 0 gives X[0] and X[n];
            // k = n/2 (row 0, column N2/2) pairs with itself.
            // Element u = (b, r) of this thread is column k2 = j0 + dk2(u) of its
            // row, dk2 = b T/WB + r N2/R; its slot and its partner's step with
            // dk2 by whole multiples of 2^PSB (WB is one), so the padded slot
            // index is linear in dk2.
            static_assert(!RF || WB % (1 << Sh::PSB) == 0, "linear slots");
            constexpr int SLOT_STEP = WB + (WB >> Sh::PSB);
            auto dk2 = [](int b, int r) { return b * (T / WB) + (r << (LOG_N2 - IRL::LOG_R)); };
            const int j0 = tid >> Sh::LOG_WB;
            const int koff = rk1 == 0 ? N2 : N2 - 1;  // partner column koff - k2 (row 0: N2 at k2 = 0, unused)
            const int wslot = smem_slot<LOG_N2, Sh::LOG_WB, true, Sh::PSB>(rcl, j0);
            const int rslot = smem_slot<LOG_N2, Sh::LOG_WB, true, Sh::PSB>(rcm, koff - j0);
            __syncthreads();  // the last row stage has read X: it now takes the partners' halves of Z
            unroll_for<E / T>([&](auto uc) {
                constexpr int u = decltype(uc)::value, b = u / IRL::R, r = u % IRL::R;
                if constexpr (r >= IRL::R / 2) X[wslot + dk2(b, r) * SLOT_STEP] = v[u];
            });
            __syncthreads();  // every partner is in X
            const int64_t ob = s * (N + 1);
            const float h = 0.5f * scale;
            const int kbase = rk1 + N1 * j0;
            auto put = [&](int k, int km, float2 za, float2 zb, float2 w) {
                const float2 P = make_float2(h * (za.x + zb.x), h * (za.y - zb.y));
                const float dx = za.x - zb.x, dy = za.y + zb.y;
                const float2 Q = make_float2(w.x * dx - w.y * dy, w.x * dy + w.y * dx);
                const float2 xk = make_float2(P.x + Q.x, P.y + Q.y), xm = make_float2(P.x - Q.x, Q.y - P.y);
                if (a.out_power) {
                    float *Po = static_cast<float *>(a.out) + ob;
                    Po[k] = power_of(xk);
                    Po[km] = power_of(xm);
                } else {
                    float2 *Xo = static_cast<float2 *>(a.out) + ob;
                    Xo[k] = xk;
                    Xo[km] = xm;
                }
            };
            unroll_for<E / T>([&](auto uc) {
                constexpr int u = decltype(uc)::value, b = u / IRL::R, r = u % IRL::R;
                if constexpr (r < IRL::R / 2) {
                    float2 zb = X[rslot - dk2(b, r) * SLOT_STEP];
                    const bool z0 = u == 0 && rk1 == 0 && j0 == 0;  // k = 0: its own partner, in v[0]
                    if (z0) zb = v[0];
                    const int k = kbase + N1 * dk2(b, r);
                    put(k, (int)N - k, v[u], zb, rot32<(r * (16 / IRL::R)) & 15, -1>(rpw[b]));
                    if constexpr (u == 0) {
                        if (z0) {  // k = n/2 (column N2/2 of row 0): v[R/2], its own partner
                            const int kh = (int)N / 2;
                            put(kh, kh, v[IRL::R / 2], v[IRL::R / 2],
                                rot32<(IRL::R / 2) * (16 / IRL::R) & 15, -1>(rpw[0]));
                        }
                    }
                }
            });
        }
        cluster_arrive_relaxed();  // this thread's reads of X were consumed above
    }
    cluster_wait();
    if (tid == 0) bulk_wait_read_all();
    cl.sync();  // no CTA leaves while a peer could still copy into its X
}

}  // namespace fftseg
