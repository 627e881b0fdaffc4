// Radix-16 DFT on the tensor cores with split hi+lo operands.
//
// A radix-16 butterfly is the row-vector product y = x F16 with the 16x16
// DFT matrix; in real arithmetic a row of 32 reals (re, im interleaved) times
// the 32x32 real matrix F:
//   F[2j][2m] = c, F[2j+1][2m] = -s, F[2j][2m+1] = s, F[2j+1][2m+1] = c,
//   c + i s = w_16^{jm} = exp(sigma 2 pi i jm / 16).
// A warp stacks its 32 butterflies (one per thread) into a 32 x 32 matrix X and
// computes Y = X F on mma.sync.m16n8k16 with FP32 accumulation.  To win back
// precision each operand is split into a high and a low 16-bit part,
// X = Xh + Xl and F = Fh + Fl, and Y ~ Xh Fh + Xh Fl + Xl Fh (the dropped
// Xl Fl term is about 2^-22 (FP16) or 2^-16 (BF16) relative).  For FP16 each
// row is first scaled by a power of two so that its largest entry lies in
// [2^13, 2^14) (FP16 range), and its outputs are scaled back exactly.
//
// Rows go through a per-warp 4 KB shared staging area: the hi and lo halves
// of the 32 rows (64 B each, 16-byte chunks XOR-swizzled against bank
// conflicts) feed ldmatrix; the FP32 results come back through the same area
// (8-byte slots rotated per row) so that every thread again holds its own
// butterfly's 16 outputs, in natural order.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "engine.cuh"

namespace fftseg {

enum { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2 };

struct TcCtx {
    uint32_t bh[16];  // F hi fragments: [(ks * 4 + nt) * 2 + q]
    uint32_t bl[16];  // F lo fragments
    float2 *stage;    // this warp's 4 KB staging area (shared memory)
};

template <int PREC>
FDEV uint32_t pack_hi(float a, float b, float &ra, float &rb)
{
    uint32_t u;
    if (PREC == PREC_FP16) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        ra = a - f.x;
        rb = b - f.y;
        u = *reinterpret_cast<const uint32_t *>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 f = __bfloat1622float2(h);
        ra = a - f.x;
        rb = b - f.y;
        u = *reinterpret_cast<const uint32_t *>(&h);
    }
    return u;
}

template <int PREC>
FDEV uint32_t pack_lo(float a, float b)
{
    if (PREC == PREC_FP16) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// F fragments for this lane (B operand of m16n8k16: k pairs (2t, 2t+1) and
// (2t+8, 2t+9) of the k-step, column n = 8 nt + g), split into hi and lo.
template <int S, int PREC>
FDEV void tc_init(TcCtx &tc, float2 *stage)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    tc.stage = stage;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int n = 8 * nt + g;
                const int m = n >> 1, im_out = n & 1;
                float f[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int k = 16 * ks + 2 * t + 8 * q + e;
                    const int j = k >> 1, im_in = k & 1;
                    double sd, cd;
                    sincospi(2.0 * (double)((j * m) & 15) / 16.0, &sd, &cd);
                    const float c = (float)cd, s = (float)(S * sd);
                    f[e] = im_in == 0 ? (im_out == 0 ? c : s) : (im_out == 0 ? -s : c);
                }
                float la, lb;
                tc.bh[(ks * 4 + nt) * 2 + q] = pack_hi<PREC>(f[0], f[1], la, lb);
                tc.bl[(ks * 4 + nt) * 2 + q] = pack_lo<PREC>(la, lb);
            }
}

FDEV void ldsm_x4(uint32_t *r, uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

template <int PREC>
FDEV void mma16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1)
{
    if (PREC == PREC_FP16)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    else
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

FDEV int tc_out_slot(int row, int m) { return (m + 4 * (row & 3) + (row >> 2)) & 15; }

// In place: v[0..15] (this thread's butterfly) <- its 16-point DFT.  Every
// lane of the warp must call this together.
template <int S, int PREC>
FDEV void dft16_tc(float2 *v, const TcCtx &tc)
{
    const int lane = threadIdx.x & 31;
    const uint32_t base = smem_u32(tc.stage);

    // ---- scale (FP16 only) and split this lane's row into hi and lo halves
    float sc = 1.f, inv = 1.f;
    if (PREC == PREC_FP16) {
        float mx = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) mx = fmaxf(mx, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
        int e = (int)((__float_as_uint(mx) >> 23) & 0xFF) - 127;  // floor(log2 mx) for normal mx
        e = e < -100 ? -100 : (e > 100 ? 100 : e);
        sc = __uint_as_float((uint32_t)(127 + 13 - e) << 23);  // 2^(13 - e)
        inv = __uint_as_float((uint32_t)(127 - 13 + e) << 23);
    }
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float la, lb;
            h[u] = pack_hi<PREC>(v[4 * q + u].x * sc, v[4 * q + u].y * sc, la, lb);
            l[u] = pack_lo<PREC>(la, lb);
        }
        const uint32_t off = (uint32_t)(lane * 64 + 16 * (q ^ sw));
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + off), "r"(h[0]), "r"(h[1]), "r"(h[2]),
                     "r"(h[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + 2048 + off), "r"(l[0]), "r"(l[1]),
                     "r"(l[2]), "r"(l[3])
                     : "memory");
    }
    __syncwarp();

    // ---- Y = Xh Fh + Xh Fl + Xl Fh for the warp's two 16-row tiles
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int mi = lane >> 3;
            const int row = mt * 16 + (mi & 1) * 8 + (lane & 7);
            const int q = 2 * ks + (mi >> 1);
            const uint32_t off = (uint32_t)(row * 64 + 16 * (q ^ ((row >> 1) & 3)));
            ldsm_x4(ah[ks], base + off);
            ldsm_x4(al[ks], base + 2048 + off);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            float *d = acc[mt][nt];
            d[0] = d[1] = d[2] = d[3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int fi = (ks * 4 + nt) * 2;
                mma16816<PREC>(d, al[ks], tc.bh[fi], tc.bh[fi + 1]);
                mma16816<PREC>(d, ah[ks], tc.bl[fi], tc.bl[fi + 1]);
                mma16816<PREC>(d, ah[ks], tc.bh[fi], tc.bh[fi + 1]);
            }
        }
    }
    __syncwarp();  // every lane has its fragments: the staging area is free

    // ---- results back to one row per lane (scaled back exactly)
    const int g = lane >> 2, t = lane & 3;
    float2 *stg = tc.stage;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int ra = mt * 16 + g, rb = ra + 8;
        const float ia = PREC == PREC_FP16 ? __shfl_sync(0xffffffffu, inv, ra) : 1.f;
        const float ib = PREC == PREC_FP16 ? __shfl_sync(0xffffffffu, inv, rb) : 1.f;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int m = 4 * nt + t;
            const float *d = acc[mt][nt];
            stg[ra * 16 + tc_out_slot(ra, m)] = make_float2(d[0] * ia, d[1] * ia);
            stg[rb * 16 + tc_out_slot(rb, m)] = make_float2(d[2] * ib, d[3] * ib);
        }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = stg[lane * 16 + tc_out_slot(lane, m)];
    __syncwarp();  // the area may be reused by the next call
}

}  // namespace fftseg
