// Persistent two-pass four-step kernel with an L2-resident intermediate.
//
// n = N1*N2, input x[j1*N2 + j2], output X[k1 + N1*k2]:
//   pass A (column DFTs): Y[k1][j2] = w_n^{j2 k1} sum_{j1} x[j1 N2 + j2] w_{N1}^{j1 k1}
//   pass B (row DFTs):    X[k1 + N1 k2] = sum_{j2} Y[k1][j2] w_{N2}^{j2 k2}
// Pass A stores Y transposed, as Yt[j2][k1], into a ring of NR chunk buffers
// of CS segments each, small enough to stay in L2; pass B reads Yt tiles with
// the same kind of tiled TMA copy that pass A uses on the input.
//
// Work items are A and B tiles of chunks, taken from a global queue in the
// order A(0), A(1) B(0), A(2) B(1), ..., B(NC-1).  B(c) waits until every
// A(c) tile has stored its part of Yt (a per-chunk counter); A(c) waits until
// B(c-NR) no longer reads the ring buffer it overwrites.  A tile only waits on
// tiles that were taken from the queue before it, and a CTA never blocks while
// it holds a started tile, so the persistent grid cannot deadlock.  Every spin
// is bounded; a spin that runs out records a flag in *err and goes on.
//
// Each CTA double-buffers its input tiles: the next tile's TMA copy is issued
// while the current tile is transformed whenever the next tile's dependency is
// already met.
//
// Shared memory also holds the stage twiddle tables (lines up to 2048
// points) and, per A tile, the two factor tables of the four-step twiddle for
// the tile's columns, so that the only global loads of a tile are its TMA
// copy and those few table entries.
#pragma once
#include "kernels.cuh"
#include "launch.h"

namespace fftseg {

struct FourStepArgs {
    CUtensorMap tmA;        // input  [nseg][N1][N2] (8-byte elements), box [1][BOXA][WA]
    CUtensorMap tmB;        // ring   [NR*CS][N2][N1], box [1][BOXB][WB]
    void *out;              // [nseg][n] complex64, or float32 |X|^2
    float2 *ring;           // NR*CS segments of n points, [slot*CS + sl][j2][k1]
    const float2 *twA;      // stage tables, length N1
    const float2 *twB;      // stage tables, length N2
    const float2 *w4;       // [j2][k1 mod K] = w_n^{j2 (k1 mod K)}, K = 2^fourstep_log_k(log2 N1)
    const float2 *w4hi;     // [j2][k1 div K] = w_n^{j2 K (k1 div K)}
    int *ctr;               // [0] queue head, [1 + c] A tiles done, [1 + NC + c] B tiles done
    int *err;
    int64_t nseg;
    int nchunks;            // NC
    int cs;                 // segments per chunk
    int nr;                 // ring buffers
    int log_k;              // log2 K (checked against the kernel's own choice by the host)
    int out_power;
    float scale;
};

template <int LOG_N1, int LOG_N2, int LOG_E>
struct FourStepShape {
    static constexpr int N1 = 1 << LOG_N1, N2 = 1 << LOG_N2, E = 1 << LOG_E;
    static constexpr int LOG_WA = LOG_E - LOG_N1;  // columns per A tile
    static constexpr int LOG_WB = LOG_E - LOG_N2;  // rows per B tile
    static constexpr int T = E / 16;
    static constexpr int PS = 4;
    static constexpr int BOXA = N1 < 256 ? N1 : 256;
    static constexpr int BOXB = N2 < 256 ? N2 : 256;
    static constexpr int SLOTS_A = smem_slots<LOG_N1, LOG_WA, PS>();
    static constexpr int SLOTS_B = smem_slots<LOG_N2, LOG_WB, PS>();
    static constexpr int SLOTS = ((SLOTS_A > SLOTS_B ? SLOTS_A : SLOTS_B) + 1) & ~1;
    // stage twiddle tables in shared memory for lines up to 2048 points (one
    // copy when N1 == N2); longer lines read them from global memory
    static constexpr bool TW_SM = LOG_N1 <= 11 && LOG_N2 <= 11;
    static constexpr int TWA = TW_SM ? stage_table_offset<LOG_N1>(StageInfo<LOG_N1, 0>::NSTAGES) : 0;
    static constexpr int TWB =
        TW_SM && LOG_N1 != LOG_N2 ? stage_table_offset<LOG_N2>(StageInfo<LOG_N2, 0>::NSTAGES) : 0;
    // four-step twiddle factors of an A tile's columns: per column K + N1/K entries
    static constexpr int LOG_K = fourstep_log_k(LOG_N1);
    static constexpr int FK = (1 << LOG_K) + (N1 >> LOG_K);
    static constexpr int FA = FK << LOG_WA;
    // P[2] (input tiles) | X (stage scratch) | stage tables | factors | 2 barriers | 2 item slots
    static constexpr size_t SMEM = (size_t)(2 * E + SLOTS + TWA + TWB + FA) * sizeof(float2) +
                                   2 * sizeof(uint64_t) + 10 * sizeof(int64_t);
    static constexpr int MINB = T <= 256 ? 2 : 1;
    static_assert(LOG_WA >= 1 && LOG_WB >= 1, "a tile row must hold at least 16 bytes");
    // the stage exchange's barrier also orders the tile reads before the refill
    static_assert(StageInfo<LOG_N1, 0>::NSTAGES >= 2 && StageInfo<LOG_N2, 0>::NSTAGES >= 2, "two stages per pass");
};

// bounded spin until *p >= target (acquire); false (and bit 4 of *err set)
// if it never got there within `limit` polls
FDEV bool spin_until(const int *p, int target, int *err, uint32_t limit = 1u << 22)
{
    for (uint32_t it = 0; it < limit; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return true;
        __nanosleep(64);
    }
    atomicOr(err, 4);
    return false;
}

FDEV bool probe(const int *p, int target)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v >= target;
}

template <int LOG_N1, int LOG_N2, int LOG_E, int S, int PREC = PREC_FP32>
__global__ void __launch_bounds__(FourStepShape<LOG_N1, LOG_N2, LOG_E>::T,
                                  PREC == PREC_FP32 ? FourStepShape<LOG_N1, LOG_N2, LOG_E>::MINB : 1)
    k_fourstep(const __grid_constant__ FourStepArgs a)
{
    using Sh = FourStepShape<LOG_N1, LOG_N2, LOG_E>;
    constexpr int K = 1 << Sh::LOG_K;
    constexpr int N1 = Sh::N1, N2 = Sh::N2, E = Sh::E, T = Sh::T;
    constexpr int WA = 1 << Sh::LOG_WA, WB = 1 << Sh::LOG_WB;
    constexpr int64_t N = (int64_t)N1 * N2;
    constexpr int TA_SEG = N2 / WA, TB_SEG = N1 / WB;  // tiles per segment
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;  // two input tiles
    float2 *X = sm + 2 * E;
    float2 *TWA = X + Sh::SLOTS;  // stage tables (TW_SM)
    float2 *TWB = LOG_N1 == LOG_N2 ? TWA : TWA + Sh::TWA;
    float2 *F = TWA + Sh::TWA + Sh::TWB;  // [c][K + N1/K] four-step factors of the current A tile
    uint64_t *bar = reinterpret_cast<uint64_t *>(F + Sh::FA);
    int64_t *item = reinterpret_cast<int64_t *>(bar + 2);  // [2]: the queue item held in P[b]
    int64_t *info = item + 2;                               // [2][4]: is_b, chunk, tile, segment
    const int tid = threadIdx.x;
    if (smem_u32(P) & 127) {
        if (tid == 0) atomicOr(a.err, 2);
        return;
    }
    const int TA = a.cs * TA_SEG, TB = a.cs * TB_SEG;
    const int64_t total = (int64_t)a.nchunks * (TA + TB);
    int *doneA = a.ctr + 1, *doneB = a.ctr + 1 + a.nchunks;

    // item -> (is_b, chunk, tile within chunk)
    auto decode = [&](int64_t t, int &isb, int &c, int &w) {
        if (t < TA) {
            isb = 0;
            c = 0;
            w = (int)t;
            return;
        }
        const int64_t t2 = t - TA;
        const int r = 1 + (int)(t2 / (TA + TB));
        const int x = (int)(t2 % (TA + TB));
        if (r < a.nchunks && x < TA) {
            isb = 0;
            c = r;
            w = x;
        } else {
            isb = 1;
            c = r - 1;
            w = r < a.nchunks ? x - TA : x;
        }
    };
    auto seg_of = [&](int isb, int c, int w) -> int64_t {
        return (int64_t)c * a.cs + (isb ? w / TB_SEG : w / TA_SEG);
    };
    // dependency of a tile: (counter, target), or none
    // (the counters count warps: every warp of a tile adds one when done)
    auto dep = [&](int isb, int c, const int *&p, int &target) {
        if (isb) {
            p = doneA + c;
            target = TA * (T / 32);
        } else if (c >= a.nr) {
            p = doneB + (c - a.nr);
            target = TB * (T / 32);
        } else {
            p = nullptr;
            target = 0;
        }
    };
    // thread 0: issue the tile's input copy into P[b] (valid tiles only)
    auto issue = [&](int64_t t, int b) {
        int isb, c, w;
        decode(t, isb, c, w);
        const int64_t s = seg_of(isb, c, w);
        if (s >= a.nseg) return;
        fence_proxy_async();
        mbar_expect_tx(&bar[b], (uint32_t)(E * sizeof(float2)));
        if (!isb) {
            const int ct = w % TA_SEG;
#pragma unroll
            for (int q = 0; q < N1 / Sh::BOXA; ++q)
                tma_load_3d(P + b * E + q * Sh::BOXA * WA, &a.tmA, ct * WA, q * Sh::BOXA, (int)s, &bar[b]);
        } else {
            const int rt = w % TB_SEG;
            const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);
#pragma unroll
            for (int q = 0; q < N2 / Sh::BOXB; ++q)
                tma_load_3d(P + b * E + q * Sh::BOXB * WB, &a.tmB, rt * WB, q * Sh::BOXB, slab, &bar[b]);
        }
    };
    // thread 0: take the next item; issue its copy now if its dependency is met
    // (returns whether the copy still has to be issued later)
    auto take = [&](int b) -> bool {
        const int64_t t = atomicAdd(a.ctr, 1);
        item[b] = t;
        if (t >= total) return false;
        int isb, c, w;
        decode(t, isb, c, w);
        info[4 * b] = isb;
        info[4 * b + 1] = c;
        info[4 * b + 2] = w;
        info[4 * b + 3] = seg_of(isb, c, w);
        const int *p;
        int target;
        dep(isb, c, p, target);
        if (p && !probe(p, target)) return true;  // deferred
        fence_proxy_async_global();
        issue(t, b);
        return false;
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if constexpr (Sh::TW_SM) {
        for (int e = tid; e < Sh::TWA; e += T) TWA[e] = __ldg(a.twA + e);
        for (int e = tid; e < Sh::TWB; e += T) TWB[e] = __ldg(a.twB + e);
    }
    const float2 *twA = Sh::TW_SM ? TWA : a.twA;
    const float2 *twB = Sh::TW_SM ? TWB : a.twB;
    __syncthreads();
    bool deferred[2] = {false, false};  // meaningful in thread 0 only
    if (tid == 0) {
        deferred[0] = take(0);
        if (deferred[0]) {  // nothing is held yet: wait here
            int isb, c, w;
            decode(item[0], isb, c, w);
            const int *p;
            int target;
            dep(isb, c, p, target);
            spin_until(p, target, a.err);
            fence_proxy_async_global();
            issue(item[0], 0);
            deferred[0] = false;
        }
        deferred[1] = take(1);
    }
    uint32_t phase = 0;  // bit b: parity of the next completion of bar[b]
    const float scale = a.scale;
    const int warp = tid >> 5, lane = tid & 31;
    [[maybe_unused]] TcCtx tc;
    if constexpr (PREC != PREC_FP32) tc_init<S, PREC>(tc, P);

    for (int k = 0;; ++k) {
        const int b = k & 1;
        __syncthreads();  // item[b] (and its copy) published by thread 0
        const int64_t t = item[b];
        if (t >= total) break;
        const int isb = (int)info[4 * b], c = (int)info[4 * b + 1], w = (int)info[4 * b + 2];
        const int64_t s = info[4 * b + 3];
        const bool valid = s < a.nseg;
        const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);  // ring slab of segment s
        const float2 *Pb = P + b * E;
        float2 v[16];
        if (valid) {
            mbar_wait(&bar[b], (phase >> b) & 1, a.err);
            phase ^= 1u << b;
        }
        if (!isb) {
            // ---- A tile: columns j2 = ct*WA + cc of segment s, points j1 over N1
            const int ct = w % TA_SEG;
            if (valid) {
                // the tile's four-step factors (read after the stage exchange's barrier)
                for (int e = tid; e < Sh::FA; e += T) {
                    const int cc = e / Sh::FK, q = e - cc * Sh::FK;
                    const int64_t j2 = ct * WA + cc;
                    F[e] = q < K ? __ldg(a.w4 + (j2 << Sh::LOG_K) + q)
                                 : __ldg(a.w4hi + j2 * (N1 >> Sh::LOG_K) + (q - K));
                }
                gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WA + cc]; });
                if constexpr (PREC != PREC_FP32) {
                    __syncthreads();  // P[b] is about to hold tensor-core operands
                    tc.stage = P + b * E + warp * 512;
                }
                // (FP32: the stage exchange's barrier orders every read of P[b]
                // before thread 0 refills it at the end of the iteration)
                run_stages<LOG_N1, Sh::LOG_WA, true, S, T, Sh::PS, 0, false, true, PREC, false, Sh::TW_SM>(v, X, twA,
                                                                                                     &tc);
                // last stage in line-major order: this thread's outputs are
                // k1 = j + (N1/R) r of column j2 = ct*WA + cc
                using IL = StageInfo<LOG_N1, StageInfo<LOG_N1, 0>::NSTAGES - 1>;
                constexpr int BL = 16 / IL::R;
#pragma unroll
                for (int bb = 0; bb < BL; ++bb) {
                    int cc, j;
                    stage_coords<LOG_N1, Sh::LOG_WA, true, true, IL::NSTAGES - 1>(tid + T * bb, cc, j);
                    const int j2 = ct * WA + cc;
                    float2 *dst = a.ring + (int64_t)slab * N + (int64_t)j2 * N1 + j;
                    const float2 *Fc = F + cc * Sh::FK;
#pragma unroll
                    for (int r = 0; r < IL::R; ++r) {
                        const int k1 = j + r * (N1 / IL::R);
                        const float2 w1 = Fc[k1 & (K - 1)], w2 = Fc[K + (k1 >> Sh::LOG_K)];
                        const float2 wv = make_float2(w1.x * w2.x - w1.y * w2.y, w1.x * w2.y + w1.y * w2.x);
                        dst[r * (N1 / IL::R)] = twmul<S>(v[bb * IL::R + r], wv);
                    }
                }
            }
            // each warp publishes its part of the tile once its stores are out
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicAdd(doneA + c, 1);
            }
        } else {
            // ---- B tile: rows k1 = rt*WB + cc of segment s, points j2 over N2
            const int rt = w % TB_SEG;
            if (valid) {
                // the tile's ring lines are in shared memory now: drop them from
                // L2 so the consumed intermediate is never written back to HBM
                constexpr int LINES_PER_ROW = WB * 8 / 128 > 0 ? WB * 8 / 128 : 1;
                const float2 *tile = a.ring + (int64_t)slab * N + rt * WB;
                if (WB * 8 % 128 == 0)
                    for (int l = tid; l < N2 * LINES_PER_ROW; l += T)
                        discard_l2_line(tile + (int64_t)(l / LINES_PER_ROW) * N1 + (l % LINES_PER_ROW) * 16);
            }
            // each warp releases its part of the ring buffer (its lines dropped)
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                atomicAdd(doneB + c, 1);
            }
            if (valid) {
                gather<LOG_N2, Sh::LOG_WB, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WB + cc]; });
                if constexpr (PREC != PREC_FP32) {
                    __syncthreads();  // P[b] is about to hold tensor-core operands
                    tc.stage = P + b * E + warp * 512;
                }
                run_stages<LOG_N2, Sh::LOG_WB, true, S, T, Sh::PS, 0, false, false, PREC, false, Sh::TW_SM>(v, X, twB,
                                                                                                      &tc);
                using IL = StageInfo<LOG_N2, StageInfo<LOG_N2, 0>::NSTAGES - 1>;
                constexpr int BL = 16 / IL::R;
#pragma unroll
                for (int bb = 0; bb < BL; ++bb) {
                    int cc, j;
                    stage_coords<LOG_N2, Sh::LOG_WB, true, false, IL::NSTAGES - 1>(tid + T * bb, cc, j);
                    const int64_t o = s * N + rt * WB + cc + (int64_t)j * N1;  // k2 = j + (N2/R) r
                    if (a.out_power) {
                        float *op = static_cast<float *>(a.out) + o;
#pragma unroll
                        for (int r = 0; r < IL::R; ++r) {
                            float2 x = v[bb * IL::R + r];
                            x = make_float2(x.x * scale, x.y * scale);
                            op[(int64_t)r * (N2 / IL::R) * N1] = power_of(x);
                        }
                    } else if (scale != 1.f) {
                        float2 *op = static_cast<float2 *>(a.out) + o;
#pragma unroll
                        for (int r = 0; r < IL::R; ++r)
                            op[(int64_t)r * (N2 / IL::R) * N1] =
                                make_float2(v[bb * IL::R + r].x * scale, v[bb * IL::R + r].y * scale);
                    } else {
                        float2 *op = static_cast<float2 *>(a.out) + o;
#pragma unroll
                        for (int r = 0; r < IL::R; ++r) op[(int64_t)r * (N2 / IL::R) * N1] = v[bb * IL::R + r];
                    }
                }
            }
        }
        // P[b] (tensor-core operand staging) is refilled below
        if constexpr (PREC != PREC_FP32) __syncthreads();
        // thread 0: make sure the next tile's copy is under way, then take one more
        if (tid == 0) {
            const int nb = b ^ 1;
            if (deferred[nb]) {  // the current tile is finished: waiting cannot deadlock
                const int *p;
                int target;
                dep((int)info[4 * nb], (int)info[4 * nb + 1], p, target);
                spin_until(p, target, a.err);
                fence_proxy_async_global();
                issue(item[nb], nb);
                deferred[nb] = false;
            }
            deferred[b] = take(b);
        }
    }
}

}  // namespace fftseg
