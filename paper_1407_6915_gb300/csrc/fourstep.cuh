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
#pragma once
#include "kernels.cuh"

namespace fftseg {

struct FourStepArgs {
    CUtensorMap tmA;        // input  [nseg][N1][N2] (8-byte elements), box [1][BOXA][WA]
    CUtensorMap tmB;        // ring   [NR*CS][N2][N1], box [1][BOXB][WB]
    void *out;              // [nseg][n] complex64, or float32 |X|^2
    float2 *ring;           // NR*CS segments of n points, [slot*CS + sl][j2][k1]
    const float2 *twA;      // stage tables, length N1
    const float2 *twB;      // stage tables, length N2
    const float2 *w4;       // [j2][k1 mod K] = w_n^{j2 (k1 mod K)}, K = 2^log_k
    const float2 *w4hi;     // [j2][k1 >> log_k] = w_n^{j2 K (k1 >> log_k)}, or null when K = N1
    int *ctr;               // [0] queue head, [1 + c] A tiles done, [1 + NC + c] B tiles done
    int *err;
    int64_t nseg;
    int nchunks;            // NC
    int cs;                 // segments per chunk
    int nr;                 // ring buffers
    int log_k;
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
    // P[2] (input tiles) | X (stage scratch) | 2 barriers | 2 item slots
    static constexpr size_t SMEM = (size_t)(2 * E + SLOTS) * sizeof(float2) + 2 * sizeof(uint64_t) + 2 * sizeof(int64_t);
    static constexpr int MINB = T <= 256 ? 2 : 1;
    static_assert(LOG_WA >= 1 && LOG_WB >= 1, "a tile row must hold at least 16 bytes");
};

// bounded spin until *p >= target (acquire); false if it never got there
FDEV bool spin_until(const int *p, int target, int *err)
{
    for (uint32_t it = 0; it < (1u << 22); ++it) {
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
    constexpr int N1 = Sh::N1, N2 = Sh::N2, E = Sh::E, T = Sh::T;
    constexpr int WA = 1 << Sh::LOG_WA, WB = 1 << Sh::LOG_WB;
    constexpr int64_t N = (int64_t)N1 * N2;
    constexpr int TA_SEG = N2 / WA, TB_SEG = N1 / WB;  // tiles per segment
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;  // two input tiles
    float2 *X = sm + 2 * E;
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    int64_t *item = reinterpret_cast<int64_t *>(bar + 2);
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
    auto dep = [&](int isb, int c, const int *&p, int &target) {
        if (isb) {
            p = doneA + c;
            target = TA;
        } else if (c >= a.nr) {
            p = doneB + (c - a.nr);
            target = TB;
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
    [[maybe_unused]] TcCtx tc;
    if constexpr (PREC != PREC_FP32) tc_init<S, PREC>(tc, P);

    for (int k = 0;; ++k) {
        const int b = k & 1;
        __syncthreads();  // item[b] (and its copy) published by thread 0
        const int64_t t = item[b];
        if (t >= total) break;
        int isb, c, w;
        decode(t, isb, c, w);
        const int64_t s = seg_of(isb, c, w);
        const bool valid = s < a.nseg;
        float2 v[16];
        if (valid) {
            mbar_wait(&bar[b], (phase >> b) & 1, a.err);
            phase ^= 1u << b;
        }
        if (!isb) {
            // ---- A tile: columns j2 = ct*WA + cc of segment s, points j1 over N1
            const int ct = w % TA_SEG;
            const float2 *Pb = P + b * E;
            if (valid) gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WA + cc]; });
            __syncthreads();  // P[b] read
            if constexpr (PREC != PREC_FP32) tc.stage = P + b * E + (tid >> 5) * 512;  // operand staging
            if (valid) {
                run_stages<LOG_N1, Sh::LOG_WA, true, S, T, Sh::PS, 0, false, true, PREC>(v, X, a.twA, &tc);
                float2 *dst = a.ring + ((int64_t)(c % a.nr) * a.cs + (s - (int64_t)c * a.cs)) * N;
                scatter_last<LOG_N1, Sh::LOG_WA, true, T, true>(v, [&](int cc, int k1, float2 x) {
                    const int j2 = ct * WA + cc;
                    float2 wv = __ldg(a.w4 + ((int64_t)j2 << a.log_k) + (k1 & ((1 << a.log_k) - 1)));
                    if (a.w4hi) {
                        const float2 w2 = __ldg(a.w4hi + (int64_t)j2 * (N1 >> a.log_k) + (k1 >> a.log_k));
                        wv = make_float2(wv.x * w2.x - wv.y * w2.y, wv.x * w2.y + wv.y * w2.x);
                    }
                    dst[(int64_t)j2 * N1 + k1] = twmul<S>(x, wv);
                });
            }
            __syncthreads();  // every store of this tile issued
            if (tid == 0) {
                __threadfence();
                atomicAdd(doneA + c, 1);
            }
        } else {
            // ---- B tile: rows k1 = rt*WB + cc of segment s, points j2 over N2
            const int rt = w % TB_SEG;
            const float2 *Pb = P + b * E;
            if (valid) {
                // the tile's ring lines are in shared memory now: drop them from
                // L2 so the consumed intermediate is never written back to HBM
                constexpr int LINES_PER_ROW = WB * 8 / 128 > 0 ? WB * 8 / 128 : 1;
                const float2 *tile = a.ring + ((int64_t)(c % a.nr) * a.cs + (s - (int64_t)c * a.cs)) * N + rt * WB;
                if (WB * 8 % 128 == 0)
                    for (int l = tid; l < N2 * LINES_PER_ROW; l += T)
                        discard_l2_line(tile + (int64_t)(l / LINES_PER_ROW) * N1 + (l % LINES_PER_ROW) * 16);
                gather<LOG_N2, Sh::LOG_WB, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WB + cc]; });
            }
            __syncthreads();  // P[b] read: the ring buffer part is no longer needed
            if (tid == 0) atomicAdd(doneB + c, 1);
            if constexpr (PREC != PREC_FP32) tc.stage = P + b * E + (tid >> 5) * 512;  // operand staging
            if (valid) {
                run_stages<LOG_N2, Sh::LOG_WB, true, S, T, Sh::PS, 0, false, false, PREC>(v, X, a.twB, &tc);
                const int64_t obase = s * N + rt * WB;
                scatter_last<LOG_N2, Sh::LOG_WB, true, T>(v, [&](int cc, int k2, float2 x) {
                    if (scale != 1.f) x = make_float2(x.x * scale, x.y * scale);
                    const int64_t o = obase + (int64_t)k2 * N1 + cc;
                    if (a.out_power) static_cast<float *>(a.out)[o] = power_of(x);
                    else static_cast<float2 *>(a.out)[o] = x;
                });
            }
        }
        // P[b] (tensor-core operand staging) is refilled below
        if constexpr (PREC != PREC_FP32) __syncthreads();
        // thread 0: make sure the next tile's copy is under way, then take one more
        if (tid == 0) {
            const int nb = b ^ 1;
            if (deferred[nb]) {  // the current tile is finished: waiting cannot deadlock
                int isb2, c2, w2;
                decode(item[nb], isb2, c2, w2);
                const int *p;
                int target;
                dep(isb2, c2, p, target);
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
