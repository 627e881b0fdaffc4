// Persistent four-step kernel for n = 256 x 256 with warp-local lines.
//
// Same factorisation as k_fourstep (n = N1*N2, N1 = N2 = 256):
//   pass A (column DFTs): Yt[j2][k1] = w_n^{j2 k1} sum_{j1} x[j1 N2 + j2] w_{N1}^{j1 k1}
//   pass B (row DFTs):    X[k1 + N1 k2] = sum_{j2} Yt[j2][k1] w_{N2}^{j2 k2}
// with the intermediate Yt in an L2-resident ring of chunk buffers, and the
// same global order of work (A(0), A(1) B(0), A(2) B(1), ...: column passes
// one 16 MiB chunk of segments ahead of row passes).  Dependencies are per
// segment: a row tile of segment s waits for the 16 column tiles of s, a
// column tile for the 16 row tiles of the segment that last used its ring
// slot.
//
// What differs is how a CTA runs a tile (16 lines of 256 points):
//  - Each 256-point line belongs to 16 lanes of one warp (16 points each; a
//    warp holds two lines).  Both radix-16 stages and the Stockham exchange
//    between them stay inside the warp: the exchange goes through the line's
//    own slots of the tile buffer, so the compute warps synchronise with
//    __syncwarp only.
//  - Tiles arrive by TMA with the 128-byte swizzle (the 16-byte chunk index of
//    each 128-byte row XORed with the row index mod 8).  Reading a line's
//    points j + 16r (lane j) is conflict-free as it lands.  For the exchange,
//    logical slot m of a line is kept in row phi(m) = m ^ ((m >> 4) & 7),
//    which makes both the writes (m = 16j + q) and the reads (m = j + 16r)
//    conflict-free; with that choice every exchange address is a per-thread
//    base XORed with a compile-time constant, plus an immediate.
//  - Two more warps per CTA do everything else over the CTA's static share of
//    the work (items blockIdx.x, blockIdx.x + gridDim.x, ...), in order.  The
//    loader waits for a free buffer (of two) and for the item's dependency,
//    then loads the tile (and, for column tiles, the tile's four-step twiddle
//    factors) with TMA.  The retirer waits for the compute warps to finish an
//    item, publishes finished tiles on their segment counters (a GPU-scope
//    fence, then adds), stores a row tile with a TMA store (the row pass stages its output in its
//    own tile buffer, again within the line's own column), drops and
//    releases the consumed ring lines, and frees the buffer.  The input and
//    output are streamed with an L2 evict-first policy, so that they do not
//    push the ring out of L2.
// Deadlock freedom: all CTAs are resident; each CTA takes its items in global
// order; an item only depends on earlier items; the retirer never waits on
// another CTA, so every finished tile is published.  Hence the smallest
// unfinished item can always proceed.  Every wait is bounded and records a
// flag in *err when it runs out.
#pragma once
#include "fourstep.cuh"

namespace fftseg {

struct FourStepHwArgs {
    CUtensorMap tmA;     // input  [nseg][256][256], box [1][256][16], 128-byte swizzle
    CUtensorMap tmB;     // ring   [slabs][256][256], box [1][256][16], 128-byte swizzle
    CUtensorMap tmO;     // output [nseg][256][256], box [1][256][16], 128-byte swizzle
    float2 *ring;        // nr*cs segments, [slot*cs + sl][j2][k1]
    const float2 *twL;   // stage tables of a 256-point line (stage 1: [r-1][m], 240 entries)
    const float2 *w4t;   // per column tile ct: [16 cols][16] w_n^{j2 (k1 mod 16)}, then
                         // [16 cols][16] scale * w_n^{j2 16 (k1 div 16)}
    int *ctr;            // per segment s < NC*cs: [1 + s] column tiles done, [1 + NC*cs + s] row tiles done
    int *err;
    int64_t nseg;
    int nchunks;         // NC
    int cs;              // segments per chunk
    int nr;              // ring buffers (at least FourStepHwShape::MIN_RING)
};

struct FourStepHwShape {
    static constexpr int L = 256, W = 16;  // line length, lines per tile
    static constexpr int E = L * W;        // 4096 points per tile
    static constexpr int TC = 256;         // compute threads (8 warps, two lines each)
    static constexpr int TT = TC + 64;     // plus a loader warp and a retirer warp
    // two tile buffers per CTA and three CTAs per SM (measured faster than
    // three buffers and two CTAs: more compute warps for the same buffering)
    static constexpr int NB = 2;           // tile buffers
    static constexpr int MINB = 3;         // CTAs per SM (the registers must allow it)
    static constexpr int LOOKAHEAD = 1;    // column passes run this many chunks ahead of row passes
    static constexpr int MIN_RING = LOOKAHEAD + 2;
    static constexpr int TW = 240;         // stage-1 twiddles of a 256-point line
    static constexpr int FT = 2 * W * 16;  // a column tile's four-step factors: [16 cols][16], twice
    static constexpr int TILES_SEG = L / W;
    static constexpr uint32_t TILE_BYTES = E * sizeof(float2);
    static constexpr uint32_t F_BYTES = FT * sizeof(float2);  // a column tile's factor tables
    // P[NB] (1024-byte aligned) | F[NB] | stage table | full[NB], done[NB], empty[NB] | item[NB][4]
    static constexpr size_t SMEM =
        (size_t)(NB * E + NB * FT + TW) * sizeof(float2) + 3 * NB * sizeof(uint64_t) + NB * 4 * sizeof(int);
};

template <int S>
__global__ void __launch_bounds__(FourStepHwShape::TT, FourStepHwShape::MINB) k_fourstep_hw(const __grid_constant__ FourStepHwArgs a)
{
    using Sh = FourStepHwShape;
    constexpr int E = Sh::E, NB = Sh::NB, TC = Sh::TC, TSEG = Sh::TILES_SEG;
    constexpr int64_t N = 65536;
    extern __shared__ __align__(1024) float2 sm[];
    float2 *const P = sm;
    float2 *const F = P + NB * E;
    float2 *const TWS = F + NB * Sh::FT;
    uint64_t *const full = reinterpret_cast<uint64_t *>(TWS + Sh::TW);
    uint64_t *const done = full + NB;
    uint64_t *const empty = done + NB;
    int *const item = reinterpret_cast<int *>(empty + NB);  // [b]: row pass?, chunk, tile, segment (-1: none)
    const int tid = threadIdx.x;
    if (smem_u32(P) & 1023) {  // the swizzle pattern assumes 1024-byte aligned tiles
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
    for (int e = tid; e < Sh::TW; e += Sh::TT) TWS[e] = __ldg(a.twL + e);
    __syncthreads();

    const int TA = a.cs * TSEG, TB = a.cs * TSEG;
    const int64_t total = (int64_t)a.nchunks * (TA + TB);
    // dependencies are per segment: a row tile of segment s needs the 16
    // column tiles of s; a column tile of s needs the 16 row tiles of the
    // segment that last used its ring slot, s - nr*cs
    int *const doneA = a.ctr + 1;
    int *const doneB = a.ctr + 1 + (int64_t)a.nchunks * a.cs;
    const int64_t ring_segs = (int64_t)a.nr * a.cs;
    const int64_t first = blockIdx.x, stride = gridDim.x;
    const int64_t items = first < total ? (total - first + stride - 1) / stride : 0;

    // Global order of the work, with column passes LA chunks ahead of row
    // passes: A(0) .. A(LA-1), then for g = 0, 1, ...: A(g+LA) (while it
    // exists), B(g).  B(g) needs A(g); A(c) needs B(c - nr) (its ring
    // buffer), and nr >= LA + 2 puts both two chunk groups back.
    // item t -> (row pass?, chunk, tile within the chunk's pass)
    constexpr int LA = Sh::LOOKAHEAD;
    const int lead = a.nchunks < LA ? a.nchunks : LA;  // chunks of the leading column passes
    const int full_groups = a.nchunks - lead;           // groups with both an A and a B part
    auto decode = [&](int64_t t, int &isb, int &c, int &w) {
        if (t < (int64_t)lead * TA) {
            isb = 0;
            c = (int)(t / TA);
            w = (int)(t % TA);
            return;
        }
        const int64_t t2 = t - (int64_t)lead * TA;
        if (t2 < (int64_t)full_groups * (TA + TB)) {
            const int g = (int)(t2 / (TA + TB));
            const int x = (int)(t2 % (TA + TB));
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
        const int64_t t3 = t2 - (int64_t)full_groups * (TA + TB);
        isb = 1;
        c = full_groups + (int)(t3 / TB);
        w = (int)(t3 % TB);
    };

    if (tid >= TC + 32) {
        // ============================================================= retirer
        // Retires this CTA's items in order as the compute warps finish them:
        // frees a column tile's buffer at once (its ring stores come from
        // registers), stores a row tile with a TMA store and frees its buffer
        // once the store has read it, drops consumed ring lines from L2.  The
        // segment counters are published in batches (one GPU-scope fence, then
        // one add per tile) whenever no finished item is waiting, so the
        // fence's latency never holds a buffer.  It only ever waits on this
        // CTA's own compute warps and bulk stores.
        const int lane = tid & 31;
        const uint64_t stream_policy = policy_evict_first();  // the output is written once
        int *pend[4];  // counters of finished, unpublished tiles
        int npend = 0;
        auto publish = [&]() {
            if (lane == 0 && npend) {
                fence_acq_rel_gpu();  // every write of the tiles (observed through `done`) first
                for (int i = 0; i < 4; ++i)
                    if (i < npend) atomicAdd(pend[i], 1);
            }
            npend = 0;
        };
        for (int64_t m = 0; m < items; ++m) {
            const int b = (int)(m % NB);
            const uint32_t par = (uint32_t)(m / NB) & 1;
            // wait for the item; publish what is pending meanwhile
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
            int isb, c, w;
            decode(first + m * stride, isb, c, w);
            const int64_t s = (int64_t)c * a.cs + w / TSEG;
            if (!isb) {
                if (lane == 0) mbar_arrive(&empty[b]);
                pend[npend++] = doneA + s;
            } else {
                const bool valid = s < a.nseg;
                const int rt = w % TSEG;
                if (lane == 0) {
                    if (valid) {
                        tma_store_3d_hint(&a.tmO, rt * Sh::W, 0, (int)s, P + b * E, stream_policy);
                        bulk_commit();
                        bulk_wait_read();  // the store has read the buffer
                    }
                    mbar_arrive(&empty[b]);
                }
                if (valid) {
                    // the tile's ring lines were consumed: drop them from L2
                    const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);
                    const float2 *tile = a.ring + (int64_t)slab * N + rt * Sh::W;
                    for (int l = lane; l < Sh::L; l += 32) discard_l2_line(tile + (int64_t)l * Sh::L);
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
        // Loads this CTA's items in order into the tile buffers once a buffer
        // is free and the item's dependency is met (probed before the wait
        // for the buffer, so that the probe's latency overlaps it).
        const int lane = tid & 31;
        int64_t a_seen = -1, b_seen = -1;  // highest segment whose column / row tiles were seen complete
        const uint64_t stream_policy = policy_evict_first();  // the input is read once
        for (int64_t m = 0; m < items; ++m) {
            const int b = (int)(m % NB);
            int isb, c, w;
            decode(first + m * stride, isb, c, w);
            const int64_t s = (int64_t)c * a.cs + w / TSEG;
            // the dependency first (its probe's latency overlaps the wait for a buffer)
            if (lane == 0) {
                if (isb && s > a_seen) {
                    if (spin_until(doneA + s, TSEG, a.err)) a_seen = s;
                } else if (!isb && s >= ring_segs && s - ring_segs > b_seen) {
                    if (spin_until(doneB + (s - ring_segs), TSEG, a.err)) b_seen = s - ring_segs;
                }
            }
            if (m >= NB) mbar_wait(&empty[b], (uint32_t)(m / NB - 1) & 1, a.err);
            if (lane == 0) {
                // the decoded item, for the compute warps (released by the arrive below)
                item[4 * b] = isb;
                item[4 * b + 1] = c;
                item[4 * b + 2] = w;
                item[4 * b + 3] = s < a.nseg ? (int)s : -1;
                if (s < a.nseg) {
                    if (isb) fence_proxy_async_global();  // ring data written by other CTAs' generic stores
                    fence_proxy_async();
                    float2 *dst = P + b * E;
                    if (!isb) {
                        const int ct = w % TSEG;
                        mbar_expect_tx(&full[b], Sh::TILE_BYTES + Sh::F_BYTES);
                        tma_load_3d_hint(dst, &a.tmA, ct * Sh::W, 0, (int)s, &full[b], stream_policy);
                        tma_load_1d(F + b * Sh::FT, a.w4t + (int64_t)ct * Sh::FT, Sh::F_BYTES, &full[b]);
                    } else {
                        const int slab = (c % a.nr) * a.cs + (int)(s - (int64_t)c * a.cs);
                        mbar_expect_tx(&full[b], Sh::TILE_BYTES);
                        tma_load_3d(dst, &a.tmB, (w % TSEG) * Sh::W, 0, slab, &full[b]);
                    }
                } else {
                    mbar_arrive(&full[b]);  // nothing to load: the compute warps skip it
                }
            }
            __syncwarp();
        }
        return;
    }

    // ================================================================ compute
    const int lane = tid & 31;
    // Warp w holds lines 2w and 2w+1, interleaved over its half-warps (lanes
    // 0-7 and 16-23: line 2w; 8-15 and 24-31: line 2w+1), so that the eight
    // lanes of each line in a half-warp fill the banks the other line's eight
    // leave free (a 64-bit shared access is served per half-warp).
    const int h = ((tid >> 5) << 1) | ((lane >> 3) & 1);  // line of the tile (column of the tile buffer)
    const int j = (lane & 7) | ((lane >> 4) << 3);        // butterfly index within the line
    const int hc = (h >> 1) & 7, j7 = j & 7;
    char *const Pc = reinterpret_cast<char *>(P);
    // byte offsets within a tile (see the file comment):
    //   row i, column h  ->  128 i + 16 ((h/2 ^ i) mod 8) + 8 (h mod 2)
    const uint32_t Mj = (uint32_t)(128 * j7 + 16 * (hc ^ j7));
    const uint32_t lin = (uint32_t)(128 * j + 16 * ((hc ^ j) & 7) + 8 * (h & 1));  // rows j + 16r: + 2048 r
    const uint32_t wr = (uint32_t)(2048 * j + 8 * (h & 1)) + Mj;  // slot 16j + q: (wr ^ 144 (q mod 8)) + 1024 (q / 8)
    const uint32_t rd = (uint32_t)(1024 * (j >> 3) + 8 * (h & 1)) + Mj;  // slot j + 16r: (rd ^ 144 (r mod 8)) + 2048 r
    auto at = [&](uint32_t off) -> float2 & { return *reinterpret_cast<float2 *>(Pc + off); };

    int b = 0;
    uint32_t par = 0;
    for (int64_t m = 0; m < items; ++m) {
        mbar_wait(&full[b], par, a.err);
        const int isb = item[4 * b], c = item[4 * b + 1], w = item[4 * b + 2], s = item[4 * b + 3];
        if (s >= 0) {
            const uint32_t tb = (uint32_t)b * Sh::TILE_BYTES;
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = at(tb + lin + 2048 * r);
            dft16<S>(v);
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 16; ++q) at(((tb + wr) ^ (144u * (q & 7))) + 1024 * (q >> 3)) = v[q];
            __syncwarp();
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = at(((tb + rd) ^ (144u * (r & 7))) + 2048 * r);
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = twmul<S>(v[r], TWS[(r - 1) * 16 + j]);
            dft16<S>(v);  // outputs k = j + 16 q in v[q]
            if (!isb) {
                // column j2 = 16 ct + h: times w_n^{j2 k1} = w_n^{j2 j} w_n^{j2 16 q}, into the ring
                const int ct = w % TSEG;
                const int slab = (c % a.nr) * a.cs + (s - c * a.cs);
                const float2 *Fb = F + b * Sh::FT;
                const float2 f1 = Fb[h * 16 + j];
                float2 *dst = a.ring + (int64_t)slab * N + (int64_t)(ct * Sh::W + h) * Sh::L + j;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float2 f2 = Fb[Sh::W * 16 + h * 16 + q];
                    const float2 wv = make_float2(f1.x * f2.x - f1.y * f2.y, f1.x * f2.y + f1.y * f2.x);
                    dst[16 * q] = twmul<S>(v[q], wv);
                }
            } else {
                // row k1 = 16 rt + h: X[k1 + 256 k2], k2 = j + 16 q, staged as the
                // output box [k2][k1 - 16 rt] in this line's own column of the tile
                // (the plan's scale is already in the column pass's factors)
                __syncwarp();  // every lane has read its exchange slots
#pragma unroll
                for (int q = 0; q < 16; ++q) at(tb + lin + 2048 * q) = v[q];
                fence_proxy_async();  // read by the producer's TMA store
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&done[b]);
        if (++b == NB) {
            b = 0;
            par ^= 1;
        }
    }
}

}  // namespace fftseg
