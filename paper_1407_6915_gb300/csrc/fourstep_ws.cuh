// Warp-specialised persistent four-step kernel (FP32), selected with
// FFTSEG_FLAG_FOURSTEP_PRODUCER.  Measured on GB300 it is slower than the
// all-compute k_fourstep (the compute warps then wait on latencies that the
// barrier-synchronised form overlaps), so it is not the default.
//
// Same factorisation, work queue, L2 ring and chunk counters as k_fourstep
// (fourstep.cuh), with the roles split inside each CTA:
//  - eight compute warps only transform: they wait for a tile on its `full`
//    barrier, run the stages (synchronising among themselves on named barrier
//    1), stage the tile's results in the tile's own shared buffer and arrive
//    on its `ready` barrier;
//  - one producer warp runs a non-blocking event loop: it takes items from
//    the global queue, probes their dependencies, loads tiles with tiled TMA
//    copies, stores finished tiles with tiled TMA stores (column-pass tiles to
//    the ring, row-pass tiles to the output), waits for those stores and
//    publishes the per-chunk counters, and drops consumed ring lines from L2.
// The queue's atomics, the counters' fences and the stores' completion never
// stall the compute warps.  The producer never blocks on another CTA (only
// on its own bulk stores), so the persistent grid cannot deadlock; its idle
// polling is bounded, and on running out it records a flag and lets the
// compute warps finish with whatever they hold.
#pragma once
#include "fourstep.cuh"

namespace fftseg {

struct FourStepWsArgs {
    CUtensorMap tmA;  // input  [nseg][N1][N2], box [1][BOXA][WA]          (column-pass loads)
    CUtensorMap tmB;  // ring   [NR*CS][N2][N1], box [1][BOXB][WB]         (row-pass loads)
    CUtensorMap tmY;  // ring   [NR*CS][N2][N1], box [1][WA][BOXY]         (column-pass stores)
    CUtensorMap tmO;  // output [nseg][N2][N1] (8-byte or 4-byte), box [1][BOXB][WB]  (row-pass stores)
    float2 *ring;
    const float2 *twA, *twB;
    const float2 *w4, *w4hi;  // four-step tables as in FourStepArgs
    int *ctr;
    int *err;
    int64_t nseg;
    int nchunks, cs, nr;
    int out_power;
    float scale;
};

template <int LOG_N1, int LOG_N2, int LOG_E>
struct FourStepWsShape : FourStepShape<LOG_N1, LOG_N2, LOG_E> {
    using B = FourStepShape<LOG_N1, LOG_N2, LOG_E>;
    static constexpr int TC = B::T;       // compute threads
    static constexpr int TT = B::T + 32;  // plus the producer warp
    static constexpr int BOXY = B::N1 < 256 ? B::N1 : 256;
    // P[2] | X | full[2], ready[2] | info[2][6]
    static constexpr size_t SMEM = (size_t)(2 * B::E + B::SLOTS) * sizeof(float2) + 4 * sizeof(uint64_t) +
                                   12 * sizeof(int64_t);
};

template <int LOG_N1, int LOG_N2, int LOG_E, int S>
__global__ void __launch_bounds__(FourStepWsShape<LOG_N1, LOG_N2, LOG_E>::TT, FourStepWsShape<LOG_N1, LOG_N2, LOG_E>::TC <= 256 ? 2 : 1)
    k_fourstep_ws(const __grid_constant__ FourStepWsArgs a)
{
    using Sh = FourStepWsShape<LOG_N1, LOG_N2, LOG_E>;
    constexpr int N1 = Sh::N1, N2 = Sh::N2, E = Sh::E, T = Sh::TC;
    constexpr int WA = 1 << Sh::LOG_WA, WB = 1 << Sh::LOG_WB;
    constexpr int64_t N = (int64_t)N1 * N2;
    constexpr int TA_SEG = N2 / WA, TB_SEG = N1 / WB;
    constexpr int TW_LOG_K = Sh::LOG_K;  // four-step twiddle from two table factors
    extern __shared__ __align__(1024) float2 sm[];
    float2 *P = sm;
    float2 *X = sm + 2 * E;
    uint64_t *full = reinterpret_cast<uint64_t *>(X + Sh::SLOTS);
    uint64_t *ready = full + 2;
    int64_t *info = reinterpret_cast<int64_t *>(ready + 2);  // [b][6]: stop, is_b, chunk, tile, segment, valid
    const int tid = threadIdx.x;
    if (smem_u32(P) & 127) {
        if (tid == 0) atomicOr(a.err, 2);
        return;
    }
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&ready[0], T / 32);
        mbar_init(&ready[1], T / 32);
        fence_mbar_init();
    }
    __syncthreads();

    const int TA = a.cs * TA_SEG, TB = a.cs * TB_SEG;
    int *doneA = a.ctr + 1, *doneB = a.ctr + 1 + a.nchunks;

    if (tid >= T) {
        // =================================================== producer warp
        const int lane = tid - T;
        const int64_t total = (int64_t)a.nchunks * (TA + TB);
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
        // per buffer: 0 idle, 1 loading/computing, 2 store reading the buffer
        int st[2] = {0, 0}, uses[2] = {0, 0}, released[2] = {0, 0};
        int isb_[2] = {0, 0}, c_[2] = {0, 0}, w_[2] = {0, 0};
        int64_t s_[2] = {0, 0};
        int64_t issued = 0, held = -1;
        int hisb = 0, hc = 0, hw = 0;  // the held item, decoded
        bool stop_sent = false, exhausted = false;
        // column-pass tiles stored but not yet published (their stores may still be writing)
        int unpub[4] = {0, 0, 0, 0}, nunpub = 0;
        uint32_t idle = 0;
        auto publish = [&]() {  // every store has completed: publish the stored column tiles
            if (lane == 0) {
                bulk_wait_all();
                if (nunpub) __threadfence();
                for (int i = 0; i < nunpub; ++i) atomicAdd(doneA + unpub[i], 1);
            }
            __syncwarp();
            nunpub = 0;
        };
        for (;;) {
            bool progress = false;
            // ---- take the next item early, so its dependency can be probed ahead
            if (held < 0 && !exhausted) {
                int64_t t = 0;
                if (lane == 0) t = atomicAdd(a.ctr, 1);
                t = __shfl_sync(0xffffffffu, t, 0);
                if (t >= total) {
                    exhausted = true;
                } else {
                    held = t;
                    decode(held, hisb, hc, hw);
                }
                progress = true;
            }
            // ---- completions
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (st[b] != 1) continue;
                const bool valid = s_[b] < a.nseg;
                const uint32_t u = (uint32_t)(uses[b] - 1) & 1;
                // (every decision is taken by lane 0 and broadcast: the warp moves as one)
                const bool loaded = __shfl_sync(0xffffffffu, (int)mbar_try_wait(&full[b], u), 0) != 0;
                const bool finished = __shfl_sync(0xffffffffu, (int)mbar_try_wait(&ready[b], u), 0) != 0;
                // a finished tile was loaded too (the compute warps waited for it),
                // even if `loaded` was polled just before the load landed
                if (isb_[b] && valid && !released[b] && (loaded || finished)) {
                    // row-pass tile loaded: drop its ring lines and release them
                    constexpr int LPR = WB * 8 / 128 > 0 ? WB * 8 / 128 : 1;
                    if (WB * 8 % 128 == 0) {
                        const int slab = (c_[b] % a.nr) * a.cs + (int)(s_[b] - (int64_t)c_[b] * a.cs);
                        const float2 *tile = a.ring + (int64_t)slab * N + (w_[b] % TB_SEG) * WB;
                        for (int l = lane; l < N2 * LPR; l += 32)
                            discard_l2_line(tile + (int64_t)(l / LPR) * N1 + (l % LPR) * 16);
                    }
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence();
                        atomicAdd(doneB + c_[b], 1);
                    }
                    released[b] = 1;
                    progress = true;
                }
                if (finished) {  // the compute warps are done with it
                    if (valid) {
                        if (nunpub == 4) publish();
                        if (lane == 0) {
                            fence_proxy_async();
                            const float2 *Pb = P + b * E;
                            if (!isb_[b]) {
                                const int slab = (c_[b] % a.nr) * a.cs + (int)(s_[b] - (int64_t)c_[b] * a.cs);
#pragma unroll
                                for (int q = 0; q < N1 / Sh::BOXY; ++q)
                                    tma_store_3d(&a.tmY, q * Sh::BOXY, (w_[b] % TA_SEG) * WA, slab,
                                                 Pb + q * Sh::BOXY * WA);
                            } else {
                                const int esz = a.out_power ? 4 : 8;
                                const char *base = reinterpret_cast<const char *>(Pb);
#pragma unroll
                                for (int q = 0; q < N2 / Sh::BOXB; ++q)
                                    tma_store_3d(&a.tmO, (w_[b] % TB_SEG) * WB, q * Sh::BOXB, (int)s_[b],
                                                 base + (size_t)q * Sh::BOXB * WB * esz);
                            }
                            bulk_commit();
                        }
                        if (!isb_[b]) unpub[nunpub++] = c_[b];
                        st[b] = 2;
                    } else {
                        if (lane == 0) atomicAdd((isb_[b] ? doneB : doneA) + c_[b], 1);
                        st[b] = 0;
                    }
                    progress = true;
                }
            }
            // ---- the next buffer in sequence: free it once its store has read it
            const int nb = (int)(issued & 1);
            if (st[nb] == 2) {
                if (lane == 0) bulk_wait_read();
                __syncwarp();
                st[0] = st[0] == 2 ? 0 : st[0];
                st[1] = st[1] == 2 ? 0 : st[1];
                progress = true;
            }
            // ---- issue the held item into it
            if (st[nb] == 0 && !stop_sent) {
                if (held >= 0) {
                    bool ok = true;
                    if (lane == 0) {
                        const int *p = hisb ? doneA + hc : (hc >= a.nr ? doneB + (hc - a.nr) : nullptr);
                        ok = p == nullptr || probe(p, hisb ? TA : TB) || idle > (1u << 22);
                        if (idle > (1u << 22)) atomicOr(a.err, 4);  // never met: go on rather than hang
                    }
                    ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
                    if (ok) {
                        const int isb = hisb, c = hc, w = hw;
                        const int64_t s = (int64_t)c * a.cs + (isb ? w / TB_SEG : w / TA_SEG);
                        isb_[nb] = isb;
                        c_[nb] = c;
                        w_[nb] = w;
                        s_[nb] = s;
                        released[nb] = 0;
                        if (lane == 0) {
                            int64_t *in = info + 6 * nb;
                            in[0] = 0;
                            in[1] = isb;
                            in[2] = c;
                            in[3] = w;
                            in[4] = s;
                            in[5] = s < a.nseg;
                            if (s < a.nseg) {
                                fence_proxy_async_global();
                                fence_proxy_async();
                                mbar_expect_tx(&full[nb], (uint32_t)(E * sizeof(float2)));
                                float2 *dst = P + nb * E;
                                if (!isb) {
#pragma unroll
                                    for (int q = 0; q < N1 / Sh::BOXA; ++q)
                                        tma_load_3d(dst + q * Sh::BOXA * WA, &a.tmA, (w % TA_SEG) * WA, q * Sh::BOXA,
                                                    (int)s, &full[nb]);
                                } else {
                                    const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);
#pragma unroll
                                    for (int q = 0; q < N2 / Sh::BOXB; ++q)
                                        tma_load_3d(dst + q * Sh::BOXB * WB, &a.tmB, (w % TB_SEG) * WB, q * Sh::BOXB,
                                                    slab, &full[nb]);
                                }
                            } else {
                                mbar_arrive(&full[nb]);  // nothing to load: the compute warps skip it
                            }
                        }
                        uses[nb]++;
                        st[nb] = 1;
                        issued++;
                        held = -1;
                        progress = true;
                    }
                } else if (exhausted) {  // no more work: tell the compute warps to stop
                    if (lane == 0) {
                        info[6 * nb] = 1;
                        mbar_arrive(&full[nb]);
                    }
                    uses[nb]++;
                    stop_sent = true;
                    progress = true;
                }
            }
            if (stop_sent && st[0] != 1 && st[1] != 1) {  // the last stores are waited for in publish()
                publish();
                break;
            }
            if (progress) {
                idle = 0;
            } else if (nunpub) {
                publish();  // nothing else to do: let the row passes that wait on these start
            } else {
                ++idle;
                __nanosleep(32);
                if (idle > (1u << 24)) {  // nothing moves any more: give up
                    if (lane == 0) atomicOr(a.err, 4);
                    if (!stop_sent) {
                        if (lane == 0) {
                            info[6 * nb] = 1;
                            mbar_arrive(&full[nb]);
                        }
                        stop_sent = true;
                    }
                    publish();
                    break;
                }
            }
        }
        if (lane == 0) bulk_wait_all();  // no store may outlive the CTA
        return;
    }

    // ======================================================= compute warps
    const int warp = tid >> 5, lane = tid & 31;
    const float scale = a.scale;
    for (int k = 0;; ++k) {
        const int b = k & 1;
        mbar_wait(&full[b], (uint32_t)(k >> 1) & 1, a.err);
        const int64_t *in = info + 6 * b;
        if (in[0]) break;
        const int isb = (int)in[1], w = (int)in[3];
        const bool valid = in[5] != 0;
        float2 *Pb = P + b * E;
        float2 v[16];
        if (valid && !isb) {
            // ---- column pass: columns j2 = ct*WA + cc, points j1 over N1
            const int ct = w % TA_SEG;
            gather<LOG_N1, Sh::LOG_WA, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WA + cc]; });
            run_stages<LOG_N1, Sh::LOG_WA, true, S, T, Sh::PS, 0, true, true, PREC_FP32, true>(v, X, a.twA);
            // results times w_n^{j2 k1}, staged as the ring's box layout
            // [k1 / BOXY][j2 - ct*WA][k1 mod BOXY]
            using IL = StageInfo<LOG_N1, StageInfo<LOG_N1, 0>::NSTAGES - 1>;
#pragma unroll
            for (int bb = 0; bb < 16 / IL::R; ++bb) {
                int cc, j;
                stage_coords<LOG_N1, Sh::LOG_WA, true, true, IL::NSTAGES - 1>(tid + T * bb, cc, j);
                const int j2 = ct * WA + cc;
#pragma unroll
                for (int r = 0; r < IL::R; ++r) {
                    const int k1 = j + r * (N1 / IL::R);
                    const float2 w1 = __ldg(a.w4 + ((int64_t)j2 << TW_LOG_K) + (k1 & ((1 << TW_LOG_K) - 1)));
                    const float2 w2 = __ldg(a.w4hi + (int64_t)j2 * (N1 >> TW_LOG_K) + (k1 >> TW_LOG_K));
                    const float2 wv = make_float2(w1.x * w2.x - w1.y * w2.y, w1.x * w2.y + w1.y * w2.x);
                    Pb[(k1 / Sh::BOXY) * (Sh::BOXY * WA) + cc * Sh::BOXY + (k1 % Sh::BOXY)] =
                        twmul<S>(v[bb * IL::R + r], wv);
                }
            }
        } else if (valid) {
            // ---- row pass: rows k1 = rt*WB + cc, points j2 over N2; results
            // staged as the output's box layout [k2][cc]
            gather<LOG_N2, Sh::LOG_WB, true, T, 0>(v, [&](int cc, int i) { return Pb[i * WB + cc]; });
            run_stages<LOG_N2, Sh::LOG_WB, true, S, T, Sh::PS, 0, true, false, PREC_FP32, true>(v, X, a.twB);
            using IL = StageInfo<LOG_N2, StageInfo<LOG_N2, 0>::NSTAGES - 1>;
            if (a.out_power) {
                float *Pf = reinterpret_cast<float *>(Pb);
#pragma unroll
                for (int bb = 0; bb < 16 / IL::R; ++bb) {
                    int cc, j;
                    stage_coords<LOG_N2, Sh::LOG_WB, true, false, IL::NSTAGES - 1>(tid + T * bb, cc, j);
#pragma unroll
                    for (int r = 0; r < IL::R; ++r) {
                        const float2 x = v[bb * IL::R + r];
                        Pf[(j + r * (N2 / IL::R)) * WB + cc] = power_of(make_float2(x.x * scale, x.y * scale));
                    }
                }
            } else {
#pragma unroll
                for (int bb = 0; bb < 16 / IL::R; ++bb) {
                    int cc, j;
                    stage_coords<LOG_N2, Sh::LOG_WB, true, false, IL::NSTAGES - 1>(tid + T * bb, cc, j);
#pragma unroll
                    for (int r = 0; r < IL::R; ++r) {
                        const float2 x = v[bb * IL::R + r];
                        Pb[(j + r * (N2 / IL::R)) * WB + cc] = make_float2(x.x * scale, x.y * scale);
                    }
                }
            }
        }
        fence_proxy_async();  // the staged results are read by the producer's TMA store
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[b]);
        (void)warp;
    }
}

}  // namespace fftseg
