// Persistent four-step kernel with lane-local lines for n = N1 x N2,
// N1, N2 in {256, 512, 1024} (n = 2^16 .. 2^20).
//
// The factorisation is the one of k_fourstep and k_fourstep_hw:
//   pass A (column DFTs): Yt[j2][k1] = w_n^{j2 k1} sum_{j1} x[j1 N2 + j2] w_{N1}^{j1 k1}
//   pass B (row DFTs):    X[k1 + N1 k2] = sum_{j2} Yt[j2][k1] w_{N2}^{j2 k2}
// with Yt in an L2-resident ring of chunk buffers, stored in blocks of the
// row tiles' W_B rows, [k1 / W_B][j2][k1 mod W_B], so that every row tile is
// one contiguous block (its TMA load is one region, and once it is consumed
// its L2 lines are dropped whole); a row tile of segment s
// waits for the column tiles of s, a column tile for the row tiles of the
// segment that last used its ring slot (per-segment counters).
//
// A tile is W = E / L lines of L points.  Each lane holds 32 points of one
// line, so a line has P = L / 32 lanes and its DFT is two Stockham stages:
//   stage 1, radix 32: butterfly b < P reads line[b + P r], r < 32, and its
//     outputs go to positions 32 b + r;
//   stage 2, radix P (8, 16 or 32): butterfly b < 32 reads line[b + 32 r],
//     r < P, times w_L^{b r}, and its outputs are the bins b + 32 r.
// Lane j of a line runs stage-1 butterfly j and the stage-2 butterflies
// b = j + P e, e < 32 / P, so it ends with the bins k = j + P m, m < 32.
// The one exchange between the stages goes through the line's own column of
// the tile buffer, in place, so a line needs no shared memory beyond its
// tile.  Two lines are interleaved over each half-warp (8 lanes of each), so
// that every shared access of a half-warp touches 16 distinct 8-byte bank
// pairs; with the TMA swizzle of the tile rows and the exchange's row
// permutation phi(m) = m ^ ((m >> 5) & 7), every access is conflict-free.  The
// lanes of a pair of lines (2P threads: half a warp, a warp, or two warps)
// synchronise with __syncwarp or a named barrier only.
//
// Tile layout: columns are grouped in panels of PW = min(W, 16) columns (one
// TMA box row of PW * 8 <= 128 bytes); element (row i, column c) of panel
// c / PW sits at i * ROWB + 16 ((c mod PW) / 2 ^ ((i >> s) & M)) + 8 (c mod 2),
// ROWB = PW * 8, the 128-, 64- or 32-byte TMA swizzle (s = 0, 1, 2; M =
// ROWB / 16 - 1).
//
// Work: column and row tiles in the global order of k_fourstep_hw (column
// passes `la` chunks ahead of row passes), taken from a queue (one atomic
// add per tile by the loader warp), so that a tile only ever waits on tiles
// taken before it by CTAs that are running: no co-residency is assumed.
// Per CTA: NB tile buffers, compute warps that run a tile at a time, a loader
// warp (takes tiles, probes their dependency, issues the TMA loads and, for
// column tiles, the tile's four-step factors) and a retirer warp (stores row
// tiles with TMA, drops consumed ring lines from L2, frees buffers, publishes
// finished tiles on the segment counters in batches).  Every wait is bounded
// and records a flag in *err when it runs out.
#pragma once
#include "fourstep.cuh"

namespace fftseg {

struct FourStepWlArgs {
    CUtensorMap tmA;     // input  [nseg][N1][N2], box [PW_A][256][1], swizzled
    CUtensorMap tmB;     // ring   [slabs][N1/W_B][N2][W_B], box [PW_B][256][1][1], swizzled
    CUtensorMap tmO;     // output [nseg][N2][N1], box [PW_B][256][1], swizzled
    float2 *ring;        // nr*cs segments, [slot*cs + sl][k1 / W_B][j2][k1 mod W_B]
    const float2 *twA;   // stage-2 twiddles of an N1-point line: [r-1][b] = w_{N1}^{b r}, r < P1, b < 32
    const float2 *twB;   // the same for N2
    const float2 *w4t;   // per column tile ct, columns in pairs (c / 2, c mod 2 fastest):
                         // [W_A/2][P1][2] w_n^{j2 j}, then [W_A/2][32][2] scale * w_n^{j2 P1 m}
    int *ctr;            // [0] queue head, [1 + s] column tiles of s done, [1 + nc*cs + s] row tiles of s done
    int *err;
    int64_t nseg;
    int nchunks;         // NC
    int cs;              // segments per chunk
    int nr;              // ring chunks (>= la + 2)
    int la;              // column passes run this many chunks ahead of row passes (>= 1)
    // overlapping frames (a frame plan whose hop is a multiple of N2): frame s
    // starts frame_rows rows of N2 samples after frame s - 1, and tmA is then
    // the 2-D map of the signal's rows, box [PW_A][256]; 0 for segments
    int frame_rows;
    // periodic Hann window on the frames, w[j1 N2 + j2] = (1 - cos(2 pi (j1/N1 + j2/n))) / 2,
    // from win_row[j1] = (cos, sin)(2 pi j1 / N1) and win_col[j2] = (cos, sin)(2 pi j2 / n);
    // null: no window
    const float2 *win_row;
    const float2 *win_col;
    int stall;           // test only: segment 0's row tiles wait for one column tile more than
                         // exists, with a short spin limit, so that the bounded wait runs out
    // interleaved units (ILV kernels): R transforms of n = N1 N2 points per
    // segment of R n points, G = R / 32 = 2^ilv_log_g units of 32 each.  The
    // input holds unit u = s G + b contiguously, column after column:
    // point j1 N2 + j2 of transform 32 b + c at ((u N2 + j2) N1 + j1) 32 + c
    // (tmA is that array as [u N2 + j2][j1][c]); bin k1 + N1 k2 of transform
    // t goes to X[t + R (k1 + N1 k2)] of segment s
    int ilv_r;
    int ilv_log_g;
    // 1: the output is |X|^2, float32, in the same places (tmO over 4-byte
    // elements, box [W_B][256], the W_B * 4-byte swizzle)
    int out_power;
};

// One pass over lines of L = 2^LOG_L points in tiles of E = 2^LOG_E points.
template <int LOG_L, int LOG_E>
struct WlPass {
    static constexpr int L = 1 << LOG_L;
    static constexpr int LOG_P = LOG_L - 5;
    static constexpr int P = 1 << LOG_P;       // lanes per line (32 points each)
    static constexpr int Q = 32 / P;           // stage-2 butterflies per lane
    static constexpr int W = 1 << (LOG_E - LOG_L);  // lines per tile
    static constexpr int PW = W < 16 ? W : 16;      // columns per panel
    static constexpr int ROWB = PW * 8;             // bytes per panel row
    static constexpr int NPANEL = W / PW;
    static constexpr int PANEL_BYTES = L * ROWB;
    static constexpr int NBOXY = L / 256;           // TMA boxes of 256 rows per panel
    static constexpr int SWZ_S = ROWB == 128 ? 0 : ROWB == 64 ? 1 : 2;
    static constexpr int SWZ_M = ROWB / 16 - 1;
    static constexpr int GROUP = 2 * P;             // threads of a pair of lines
    static constexpr int TW = (P - 1) * 32;         // stage-2 twiddles
    static constexpr int FT = W * (P + 32);         // a column tile's four-step factors
    static_assert(LOG_L >= 8 && LOG_L <= 10, "lines of 256 .. 1024 points");
    static_assert(ROWB >= 32, "tile rows of at least 32 bytes");
    // the XOR constant that applies the exchange permutation and the swizzle
    // to a row offset whose low three row bits are x
    __host__ __device__ static constexpr uint32_t K(int x) { return (uint32_t)(ROWB * x + 16 * ((x >> SWZ_S) & SWZ_M)); }
};

// ILV: the kernel's unit is 32 interleaved transforms (see FourStepWlArgs):
// a column tile is column j2 of all 32 of them and a row tile row k1 of all
// 32, so that every tile's lines are the 32 transforms and its loads and
// stores stay 256-byte runs.
template <int LOG_N1, int LOG_N2, int LOG_E, int NB, int MINB, bool ILV = false>
struct FourStepWlShape {
    using PA = WlPass<LOG_N1, LOG_E>;
    using PB = WlPass<LOG_N2, LOG_E>;
    static constexpr int N1 = 1 << LOG_N1, N2 = 1 << LOG_N2;
    static constexpr int64_t N = (int64_t)N1 * N2;
    static constexpr int64_t NS = ILV ? 32 * N : N;  // points of one unit (one ring slab)
    static constexpr int E = 1 << LOG_E;
    static constexpr int TC = E / 32;        // compute threads: 32 points each
    static constexpr int TT = TC + 64;       // plus a loader warp and a retirer warp
    static constexpr int TSEG_A = ILV ? N2 : N2 / PA::W;  // column tiles per unit
    static constexpr int TSEG_B = ILV ? N1 : N1 / PB::W;  // row tiles per unit
    static_assert(!ILV || (PA::W == 32 && PB::W == 32), "interleaved units: tiles of 32 lines");
    static constexpr uint32_t TILE_BYTES = E * sizeof(float2);
    static constexpr uint32_t F_BYTES = PA::FT * sizeof(float2);
    static constexpr int TWA = PA::TW, TWB = LOG_N1 == LOG_N2 ? 0 : PB::TW;
    // P[NB] (1024-byte aligned) | F[NB] | stage-2 tables | full, done, empty [NB] | item [NB][4]
    static constexpr size_t SMEM = (size_t)NB * E * sizeof(float2) + (size_t)NB * PA::FT * sizeof(float2) +
                                   (size_t)(TWA + TWB) * sizeof(float2) + 3 * NB * sizeof(uint64_t) +
                                   NB * 4 * sizeof(int);
    static_assert(TC % 32 == 0 && TC >= 64, "whole compute warps");
    static_assert((PA::FT * sizeof(float2)) % 16 == 0, "bulk copy of the factors");
};

// Execution barrier over the 2P threads of a pair of lines.
template <int GROUP>
FDEV void wl_group_sync(int group)
{
    if constexpr (GROUP <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "n"(GROUP) : "memory");
    }
}

// The lane's stage-2 twiddles of an L-point line, w_L^{(j + P e) r} for
// e < 32 / P, 1 <= r < P, at [e (P - 1) + r - 1] (held in registers when both
// passes have the same line length).
template <class PS>
struct WlTw {
    float2 w[PS::Q * (PS::P - 1)];
    FDEV void load(const float2 *tab, int j)
    {
#pragma unroll
        for (int e = 0; e < PS::Q; ++e)
#pragma unroll
            for (int r = 1; r < PS::P; ++r) w[e * (PS::P - 1) + r - 1] = tab[(r - 1) * 32 + j + PS::P * e];
    }
};

// The DFT of the calling lane's line of a pass, in place in the tile buffer
// at byte offset tb.  On return v[e * P + r] holds bin j + P e + 32 r.
// tw: stage-2 twiddles in shared memory, or (treg) the lane's own in registers.
template <class PS, int S>
FDEV void wl_line(float2 (&v)[32], char *Pc, uint32_t tb, int c, int j, int group, const float2 *tw,
                  const WlTw<PS> *treg = nullptr, const float2 *wrow = nullptr, float2 wcol = float2{},
                  [[maybe_unused]] int *err = nullptr)
{
    constexpr int P = PS::P, Q = PS::Q, ROWB = PS::ROWB;
    const int j7 = j & 7, ch = (c % PS::PW) >> 1, h = c & 1;
    const uint32_t pb = tb + (uint32_t)((c / PS::PW) * PS::PANEL_BYTES);
    const uint32_t sw = (uint32_t)(16 * (ch ^ ((j7 >> PS::SWZ_S) & PS::SWZ_M)) + 8 * h);
    // rows j + P r (stage 1 reads, stage 2 reads with x = 0, bins): ROWB (j + P r) + sw
    const uint32_t rb = pb + (uint32_t)(ROWB * j) + sw;
    // exchange rows phi(32 j + r) = 32 j + (r ^ j7)
    const uint32_t wb = pb + (uint32_t)(32 * ROWB * j + ROWB * j7) + sw;
    // (self-checking build: every slot within this tile's buffer, 8-byte aligned)
    auto at = [&](uint32_t off) -> float2 & {
        if (!FFTSEG_CHECK(off - tb < (uint32_t)(PS::L * PS::W * 8) && (off & 7) == 0, err)) off = tb;
        return *reinterpret_cast<float2 *>(Pc + off);
    };
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = at(rb + ROWB * P * r);
    if (wrow) {  // the frame's window on rows j + P r of this column
        // row factor of row j + P r: (cos, sin)(2 pi j / N1) times exp(2 pi i r / 32)
        // (P r / N1 = r / 32), an exact constant rotation: one table entry per lane
        const float2 r0 = __ldg(wrow + j);
        unroll_for<32>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            float2 rr = rot32<r & 15, 1>(r0);
            if constexpr (r >= 16) rr = make_float2(-rr.x, -rr.y);  // exp(i pi) = -1
            const float wv = 0.5f - 0.5f * (rr.x * wcol.x - rr.y * wcol.y);
            v[r] = make_float2(v[r].x * wv, v[r].y * wv);
        });
    }
    dft32<S>(v);
    wl_group_sync<PS::GROUP>(group);  // every lane of the line has read its rows
#pragma unroll
    for (int r = 0; r < 32; ++r) at((wb ^ PS::K(r & 7)) + 8 * ROWB * (r >> 3)) = v[r];
    wl_group_sync<PS::GROUP>(group);
#pragma unroll
    for (int e = 0; e < Q; ++e)
#pragma unroll
        for (int r = 0; r < P; ++r) v[e * P + r] = at((rb ^ PS::K(r & 7)) + ROWB * (P * e + 32 * r));
#pragma unroll
    for (int e = 0; e < Q; ++e) {
#pragma unroll
        for (int r = 1; r < P; ++r)
            v[e * P + r] = twmul<S>(v[e * P + r], treg ? treg->w[e * (P - 1) + r - 1] : tw[(r - 1) * 32 + j + P * e]);
        dft<P, S>(v + e * P);
    }
}

template <int LOG_N1, int LOG_N2, int LOG_E, int NB, int MINB, int S, bool ILV = false>
__global__ void __launch_bounds__(FourStepWlShape<LOG_N1, LOG_N2, LOG_E, NB, MINB, ILV>::TT, MINB)
    k_fourstep_wl(const __grid_constant__ FourStepWlArgs a)
{
    using Sh = FourStepWlShape<LOG_N1, LOG_N2, LOG_E, NB, MINB, ILV>;
    using PA = typename Sh::PA;
    using PB = typename Sh::PB;
    constexpr int E = Sh::E, TC = Sh::TC, N1 = Sh::N1;
    constexpr int64_t NS = Sh::NS;
    extern __shared__ __align__(1024) float2 sm[];
    float2 *const P = sm;
    float2 *const F = P + NB * E;
    float2 *const TWA = F + NB * PA::FT;
    float2 *const TWB = LOG_N1 == LOG_N2 ? TWA : TWA + Sh::TWA;
    uint64_t *const full = reinterpret_cast<uint64_t *>(TWA + Sh::TWA + Sh::TWB);
    uint64_t *const done = full + NB;
    uint64_t *const empty = done + NB;
    int *const item = reinterpret_cast<int *>(empty + NB);  // [b]: kind, segment, tile, slab
    const int tid = threadIdx.x;
    if (smem_u32(P) & 1023) {  // the swizzle arithmetic assumes 1024-byte aligned tiles
        if (tid == 0) atomicOr(a.err, 2);
        return;
    }
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&done[b], TC / 32);
            mbar_init(&empty[b], 1);
        }
        fence_mbar_init();
    }
    for (int e = tid; e < Sh::TWA; e += Sh::TT) TWA[e] = __ldg(a.twA + e);
    for (int e = tid; e < Sh::TWB; e += Sh::TT) TWB[e] = __ldg(a.twB + e);
    __syncthreads();

    constexpr int KIND_A = 0, KIND_B = 1, KIND_SKIP = 2, KIND_END = 3;

    if (tid >= TC + 32) {
        // ============================================================= retirer
        // Retires the CTA's tiles in buffer order as the compute warps finish
        // them: frees a column tile's buffer at once (its ring stores came from
        // registers); stores a row tile with TMA and frees its buffer once the
        // store has read it; drops consumed ring lines from L2.  Segment
        // counters are published in batches (one GPU-scope fence, then one add
        // per tile) whenever no finished tile is waiting.  It waits only on this
        // CTA's own warps and bulk stores.
        const int lane = tid & 31;
        const uint64_t stream_policy = policy_evict_first();  // the output is written once
        int *const doneA = a.ctr + 1;
        int *const doneB = a.ctr + 1 + (int64_t)a.nchunks * a.cs;
        int *pend[4];
        int npend = 0;
        auto publish = [&]() {
            if (lane == 0 && npend) {
                fence_acq_rel_gpu();  // every write of the tiles (observed through `done`) first
                for (int i = 0; i < 4; ++i)
                    if (i < npend) atomicAdd(pend[i], 1);
            }
            npend = 0;
        };
        for (int64_t m = 0;; ++m) {
            const int b = (int)(m % NB);
            const uint32_t par = (uint32_t)(m / NB) & 1;
            for (;;) {
                const bool fin = __shfl_sync(0xffffffffu, (int)mbar_test_wait(&done[b], par), 0) != 0;
                if (fin) break;
                if (npend) {
                    publish();
                } else {
                    mbar_wait(&done[b], par, a.err);
                    break;
                }
            }
            const int kind = item[4 * b], s = item[4 * b + 1], w = item[4 * b + 2], slab = item[4 * b + 3];
            if (kind == KIND_END) break;
            if (kind == KIND_A || (kind == KIND_SKIP && w >= 0)) {
                if (lane == 0) mbar_arrive(&empty[b]);
                pend[npend++] = doneA + s;
            } else {
                const bool valid = kind == KIND_B;
                const int rt = valid ? w : -w - 1;
                if (lane == 0) {
                    if (valid && a.out_power) {
                        // one float box per 256 rows: [W_B floats][256 k2]
                        constexpr int RBP = PB::W * 4;
#pragma unroll
                        for (int q = 0; q < PB::NBOXY; ++q)
                            tma_store_3d_hint(&a.tmO,
                                              ILV ? rt * a.ilv_r + (s & ((1 << a.ilv_log_g) - 1)) * 32 : rt * PB::W,
                                              q * 256, ILV ? s >> a.ilv_log_g : s,
                                              reinterpret_cast<char *>(P + b * E) + q * 256 * RBP, stream_policy);
                        bulk_commit();
                        bulk_wait_read();  // the store has read the buffer
                    } else if (valid) {
#pragma unroll
                        for (int p = 0; p < PB::NPANEL; ++p)
#pragma unroll
                            for (int q = 0; q < PB::NBOXY; ++q)
                                tma_store_3d_hint(&a.tmO,
                                                  (ILV ? rt * a.ilv_r + (s & ((1 << a.ilv_log_g) - 1)) * 32
                                                       : rt * PB::W) + p * PB::PW,
                                                  q * 256, ILV ? s >> a.ilv_log_g : s,
                                                  reinterpret_cast<char *>(P + b * E) + p * PB::PANEL_BYTES +
                                                      q * 256 * PB::ROWB,
                                                  stream_policy);
                        bulk_commit();
                        bulk_wait_read();  // the store has read the buffer
                    }
                    mbar_arrive(&empty[b]);
                }
                if (valid) {
                    // the tile's ring block was consumed: drop its lines from L2
                    constexpr int LINES = Sh::N2 * PB::W * 8 / 128;
                    const float2 *tile = a.ring + (int64_t)slab * NS + (int64_t)rt * Sh::N2 * PB::W;
                    // (self-checking build: the block lies inside the ring)
                    if (FFTSEG_CHECK(slab < a.nr * a.cs && rt < Sh::TSEG_B, a.err))
                        for (int l = lane; l < LINES; l += 32) discard_l2_line(tile + (int64_t)l * 16);
                    __syncwarp();
                }
                pend[npend++] = doneB + s;
            }
            if (npend == 4) publish();
        }
        publish();
        if (lane == 0) bulk_wait_all();  // no store may outlive the CTA
        return;
    }
    if (tid >= TC) {
        // ============================================================== loader
        // Takes tiles from the queue, in order, one ahead; probes a tile's
        // dependency, waits for a free buffer and issues the tile's TMA loads.
        const int lane = tid & 31;
        const int TA = a.cs * Sh::TSEG_A, TB = a.cs * Sh::TSEG_B;
        const int total = a.nchunks * (TA + TB);  // < 2^31 (checked by the host)
        int *const doneA = a.ctr + 1;
        int *const doneB = a.ctr + 1 + (int64_t)a.nchunks * a.cs;
        const int64_t ring_segs = (int64_t)a.nr * a.cs;
        const int LA = a.la;
        const int lead = a.nchunks < LA ? a.nchunks : LA;
        const int full_groups = a.nchunks - lead;
        // Global order: A(0) .. A(LA-1), then for g = 0, 1, ...: A(g+LA) (while
        // it exists), B(g).  B(c) needs A(c); A(c) needs B(c - nr), nr >= LA + 2.
        // (32-bit arithmetic: the decode is on the loader's critical path)
        auto decode = [&](int t, int &isb, int &c, int &w) {
            if (t < lead * TA) {
                isb = 0;
                c = t / TA;
                w = t - c * TA;
                return;
            }
            const int t2 = t - lead * TA;
            if (t2 < full_groups * (TA + TB)) {
                const int g = t2 / (TA + TB);
                const int x = t2 - g * (TA + TB);
                if (x < TA) {
                    isb = 0;
                    c = g + LA;
                    w = x;
                } else {
                    isb = 1;
                    c = g;
                    w = x - TA;
                }
                return;
            }
            const int t3 = t2 - full_groups * (TA + TB);
            isb = 1;
            c = full_groups + t3 / TB;
            w = t3 - (t3 / TB) * TB;
        };
        int64_t a_seen = -1, b_seen = -1;  // highest segment whose column / row tiles were seen complete
        // the input is read once (evicted first), except where consecutive
        // frames overlap: then the overlap is read again by the next frame
        const bool overlap = a.frame_rows > 0 && (int64_t)a.frame_rows * Sh::N2 < Sh::N;
        const uint64_t stream_policy = overlap ? policy_evict_unchanged() : policy_evict_first();
        int t = 0;
        if (lane == 0) t = atomicAdd(a.ctr, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        for (int64_t m = 0;; ++m) {
            const int b = (int)(m % NB);
            int isb = 0, c = 0, w = 0;
            int64_t s = 0;
            const bool end = t >= total;
            // the next tile is taken now: the atomic's latency overlaps this
            // tile's dependency probe, buffer wait and copies
            int t_next = 0;
            if (lane == 0 && !end) t_next = atomicAdd(a.ctr, 1);
            if (lane == 0 && !end) {
                decode(t, isb, c, w);
                s = (int64_t)c * a.cs + (isb ? w / Sh::TSEG_B : w / Sh::TSEG_A);
                // the dependency first (its probe's latency overlaps the wait for a buffer)
                if (s < a.nseg) {
                    if (isb && s > a_seen) {
                        const bool stall = a.stall && s == 0;
                        if (spin_until(doneA + s, Sh::TSEG_A + (stall ? 1 : 0), a.err, stall ? 4096u : 1u << 22))
                            a_seen = s;
                    } else if (!isb && s >= ring_segs && s - ring_segs > b_seen) {
                        if (spin_until(doneB + (s - ring_segs), Sh::TSEG_B, a.err)) b_seen = s - ring_segs;
                    }
                }
            }
            if (m >= NB) mbar_wait(&empty[b], (uint32_t)(m / NB - 1) & 1, a.err);
            if (lane == 0) {
                if (end) {
                    item[4 * b] = KIND_END;
                    mbar_arrive(&full[b]);
                } else {
                    const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);
                    const int tile = isb ? w % Sh::TSEG_B : w % Sh::TSEG_A;
                    item[4 * b + 1] = (int)s;
                    item[4 * b + 3] = slab;
                    if (s < a.nseg) {
                        item[4 * b] = isb ? KIND_B : KIND_A;
                        item[4 * b + 2] = tile;
                        if (isb) fence_proxy_async_global();  // ring data written by other CTAs' generic stores
                        fence_proxy_async();
                        char *dst = reinterpret_cast<char *>(P + b * E);
                        if (!isb) {
                            mbar_expect_tx(&full[b], Sh::TILE_BYTES + Sh::F_BYTES);
#pragma unroll
                            for (int p = 0; p < PA::NPANEL; ++p)
#pragma unroll
                                for (int q = 0; q < PA::NBOXY; ++q) {
                                    char *box = dst + p * PA::PANEL_BYTES + q * 256 * PA::ROWB;
                                    // (ILV: column j2 = tile of the unit's 32 transforms, one
                                    // contiguous 256 x 32 block)
                                    const int x = (ILV ? 0 : tile * PA::W) + p * PA::PW;
                                    if (a.frame_rows)  // rows of the signal from the frame's start
                                        tma_load_2d_hint(box, &a.tmA, x, (int)s * a.frame_rows + q * 256, &full[b],
                                                         stream_policy);
                                    else
                                        tma_load_3d_hint(box, &a.tmA, x, q * 256, ILV ? (int)s * Sh::N2 + tile : (int)s,
                                                         &full[b], stream_policy);
                                }
                            tma_load_1d(F + b * PA::FT, a.w4t + (int64_t)tile * PA::FT, Sh::F_BYTES, &full[b]);
                        } else {
                            mbar_expect_tx(&full[b], Sh::TILE_BYTES);
#pragma unroll
                            for (int p = 0; p < PB::NPANEL; ++p)
#pragma unroll
                                for (int q = 0; q < PB::NBOXY; ++q)
                                    tma_load_4d(dst + p * PB::PANEL_BYTES + q * 256 * PB::ROWB, &a.tmB,
                                                p * PB::PW, q * 256, tile, slab, &full[b]);
                        }
                    } else {
                        // an absent segment of the last chunk: nothing to load, but its
                        // tiles are published like the others (w >= 0: a column tile)
                        item[4 * b] = KIND_SKIP;
                        item[4 * b + 2] = isb ? -tile - 1 : tile;
                        mbar_arrive(&full[b]);
                    }
                }
            }
            t = __shfl_sync(0xffffffffu, t_next, 0);
            if (end) break;
        }
        return;
    }

    // ================================================================ compute
    // with one line length for both passes a lane keeps the same j, so its
    // stage-2 twiddles live in registers for the whole launch
    constexpr bool TW_REG = LOG_N1 == LOG_N2;
    WlTw<PA> treg;
    if constexpr (TW_REG) {
        const int u = tid % PA::GROUP;
        treg.load(TWA, (u & 7) | ((u >> 4) << 3));
    }
    int bb = 0;
    uint32_t par = 0;
    char *const Pc = reinterpret_cast<char *>(P);
    for (;;) {
        mbar_wait(&full[bb], par, a.err);
        const int kind = item[4 * bb];
        if (kind == KIND_END) {  // the retirer reads the end after this buffer's `done`
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&done[bb]);
            break;
        }
        const uint32_t tb = (uint32_t)bb * Sh::TILE_BYTES;
        if (kind == KIND_A) {
            // column tile: lines are the columns j2 = W ct + c over j1
            using PS = PA;
            const int s = item[4 * bb + 1], ct = item[4 * bb + 2], slab = item[4 * bb + 3];
            const int group = tid / PS::GROUP, u = tid % PS::GROUP;
            const int c = 2 * group + ((u >> 3) & 1), j = (u & 7) | ((u >> 4) << 3);
            float2 v[32];
            const float2 wcol = a.win_row ? __ldg(a.win_col + ct * PS::W + c) : float2{};
            wl_line<PS, S>(v, Pc, tb, c, j, group, TWA, TW_REG ? &treg : nullptr, a.win_row, wcol, a.err);
            // times w_n^{j2 k1}, k1 = j + P m: w_n^{j2 j} w_n^{j2 P m} (scale folded in), into the ring
            const float2 *Fb = F + bb * PS::FT;
            const float2 f1 = Fb[((c >> 1) * PS::P + j) * 2 + (c & 1)];
            const float2 *f2p = Fb + PS::W * PS::P + (c >> 1) * 64 + (c & 1);
            // ring block layout [k1 / W_B][j2][k1 mod W_B], k1 = j + P m
            // (ILV: [k1][j2][transform c of the unit])
            constexpr int WB = PB::W;
            constexpr int64_t BLK = (int64_t)Sh::N2 * WB;
            const int j2 = ct * PS::W + c;
            float2 *row = a.ring + (int64_t)slab * NS + (int64_t)j2 * WB;
            float2 *dst = ILV ? a.ring + (int64_t)slab * NS + ct * WB + c + (int64_t)j * BLK
                          : PS::P >= WB ? row + (int64_t)(j / WB) * BLK + (j % WB)
                                        : row + j;
#pragma unroll
            for (int e = 0; e < PS::Q; ++e)
#pragma unroll
                for (int r = 0; r < PS::P; ++r) {
                    const int mm = e + PS::Q * r;
                    const float2 f2 = f2p[2 * mm];
                    const float2 wv = make_float2(f1.x * f2.x - f1.y * f2.y, f1.x * f2.y + f1.y * f2.x);
                    // P >= W_B: k1 / W_B = j / W_B + m P / W_B, k1 mod W_B = j mod W_B;
                    // else (W_B a multiple of P, j < P): k1 / W_B = m P / W_B, k1 mod W_B = j + m P mod W_B
                    const int64_t off = ILV ? (int64_t)mm * PS::P * BLK
                                        : PS::P >= WB ? (int64_t)mm * (PS::P / WB) * BLK
                                                      : (int64_t)(mm * PS::P / WB) * BLK + (mm * PS::P) % WB;
                    // (self-checking build: inside this segment's ring slab)
                    if (FFTSEG_CHECK(dst + off - (a.ring + (int64_t)slab * NS) < NS &&
                                         dst + off >= a.ring + (int64_t)slab * NS && slab < a.nr * a.cs,
                                     a.err))
                        dst[off] = twmul<S>(v[e * PS::P + r], wv);
                }
            (void)s;
        } else if (kind == KIND_B) {
            // row tile: lines are the rows k1 = W rt + c over j2; the bins
            // X[k1 + N1 k2] are staged as the output box [k2][k1 - W rt] in the
            // line's own column (the plan's scale is in the column pass's factors)
            using PS = PB;
            const int group = tid / PS::GROUP, u = tid % PS::GROUP;
            const int c = 2 * group + ((u >> 3) & 1), j = (u & 7) | ((u >> 4) << 3);
            float2 v[32];
            if constexpr (TW_REG)
                wl_line<PS, S>(v, Pc, tb, c, j, group, TWB, reinterpret_cast<const WlTw<PS> *>(&treg), nullptr,
                               float2{}, a.err);
            else
                wl_line<PS, S>(v, Pc, tb, c, j, group, TWB, nullptr, nullptr, float2{}, a.err);
            if (a.out_power) {
                // |X|^2 staged as the float output box: row k2 holds the tile's
                // W_B lines in RBP = 4 W_B bytes, 16-byte chunks swizzled by the
                // row like the complex panels.  Rows span every line's column, so
                // all compute warps must have read their exchange rows first.
                constexpr int RBP = PS::W * 4, SP = RBP == 128 ? 0 : RBP == 64 ? 1 : 2, MP = RBP / 16 - 1;
                static_assert(RBP >= 32 && RBP <= 128, "float output rows of 32..128 bytes");
                asm volatile("bar.sync 15, %0;" ::"n"(TC) : "memory");
#pragma unroll
                for (int e = 0; e < PS::Q; ++e)
#pragma unroll
                    for (int r = 0; r < PS::P; ++r) {
                        const int k2 = j + PS::P * e + 32 * r;
                        const uint32_t off = tb + (uint32_t)(k2 * RBP) +
                                             (uint32_t)((((c >> 2) ^ ((k2 >> SP) & MP)) << 4) + (c & 3) * 4);
                        if (FFTSEG_CHECK(off - tb < Sh::TILE_BYTES, a.err))
                            *reinterpret_cast<float *>(Pc + off) = power_of(v[e * PS::P + r]);
                    }
            } else {
                const int j7 = j & 7, ch = (c % PS::PW) >> 1, h = c & 1;
                const uint32_t rb = tb + (uint32_t)((c / PS::PW) * PS::PANEL_BYTES) + (uint32_t)(PS::ROWB * j) +
                                    (uint32_t)(16 * (ch ^ ((j7 >> PS::SWZ_S) & PS::SWZ_M)) + 8 * h);
                wl_group_sync<PS::GROUP>(group);  // every lane of the line has read its exchange rows
#pragma unroll
                for (int e = 0; e < PS::Q; ++e)
#pragma unroll
                    for (int r = 0; r < PS::P; ++r) {
                        const uint32_t off = rb + PS::ROWB * (PS::P * e + 32 * r);
                        if (FFTSEG_CHECK(off - tb < Sh::TILE_BYTES, a.err))
                            *reinterpret_cast<float2 *>(Pc + off) = v[e * PS::P + r];
                    }
            }
            fence_proxy_async();  // read by the retirer's TMA store
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&done[bb]);
        if (++bb == NB) {
            bb = 0;
            par ^= 1;
        }
    }
}

}  // namespace fftseg
