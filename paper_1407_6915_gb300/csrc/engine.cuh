// Register/shared-memory FFT engine shared by the sm_103a kernels.
//
// A "tile" is W lines of L points each (L, W powers of two).  Each of the T
// threads of a CTA holds V = W*L/T points in registers.  A length-L DFT runs
// as Stockham autosort stages of radix 16 (then one radix 2/4/8 stage for the
// remainder).  Stage with radix R after Ns points have been combined:
//   butterfly (c, j), j < L/R, reads  a_r = line_c[j + r*L/R],
//   multiplies a_r by w_{Ns*R}^{(j mod Ns)*r}, takes the R-point DFT, and
//   writes  line_c[(j/Ns)*Ns*R + (j mod Ns) + r*Ns] = A_r.
// The first stage reads global memory and the last writes it, both in the
// coalesced "j + r*L/R" order; stages in between exchange through shared
// memory.  This is the Cooley-Tukey FFT (Sec. I of the paper) in the
// self-sorting Stockham arrangement, so the output is in natural order.
//
// w_M^m = exp(sigma * 2 pi i m / M); tables hold the forward value
// (cos, -sin), evaluated in double on the host and rounded once to float.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define FDEV __device__ __forceinline__
#define HDEV __host__ __device__ __forceinline__

// Self-checking build (compiled with -DFFTSEG_DEBUG): FFTSEG_CHECK(cond, err)
// is cond, and when cond is false it also sets bit 8 of *err, which
// fftseg_plan_check reports.  The caller then keeps the access inside its
// buffer (it is skipped or redirected), so a bad index is recorded, never
// performed: nothing traps.  In the normal build it is `true` and costs
// nothing.
#ifdef FFTSEG_DEBUG
#define FFTSEG_CHECK(cond, err) ((cond) ? true : (atomicOr((err), 8), false))
#else
#define FFTSEG_CHECK(cond, err) true
#endif

namespace fftseg {

HDEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
HDEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// a * w for the forward table entry w; the inverse uses conj(w).
template <int S>
HDEV float2 twmul(float2 a, float2 w)
{
    if (S < 0) return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
    return make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}

// a * (sigma i)
template <int S>
HDEV float2 mul_si(float2 a)
{
    return S < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16a = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kC16b = 0.38268343236508977173f;  // sin(pi/8)

// a * w_16^M, w_16 = exp(sigma 2 pi i / 16), for the exponents a radix-16 butterfly needs
template <int M, int S>
HDEV float2 rot16(float2 a)
{
    constexpr float s = (float)S;
    if (M == 0) return a;
    if (M == 4) return mul_si<S>(a);
    if (M == 2) return make_float2(kC8 * (a.x - s * a.y), kC8 * (a.y + s * a.x));
    if (M == 6) return make_float2(kC8 * (-a.x - s * a.y), kC8 * (-a.y + s * a.x));
    if (M == 1) return make_float2(a.x * kC16a - s * a.y * kC16b, a.y * kC16a + s * a.x * kC16b);
    if (M == 3) return make_float2(a.x * kC16b - s * a.y * kC16a, a.y * kC16b + s * a.x * kC16a);
    if (M == 9) return make_float2(-a.x * kC16a + s * a.y * kC16b, -a.y * kC16a - s * a.x * kC16b);
    return a;  // not reached for the exponents used below
}

template <int S>
HDEV void dft2(float2 &a, float2 &b)
{
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// X_k = sum_j v_j w_4^{jk}, in place, natural order.
template <int S>
HDEV void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3)
{
    const float2 a0 = cadd(v0, v2), a1 = csub(v0, v2);
    const float2 a2 = cadd(v1, v3), a3 = mul_si<S>(csub(v1, v3));
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = cadd(a1, a3);
    v3 = csub(a1, a3);
}

// 8 = 2 x 4: X_k = E_k + w_8^k O_k, X_{k+4} = E_k - w_8^k O_k.
template <int S>
HDEV void dft8(float2 *v)
{
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    o1 = rot16<2, S>(o1);
    o2 = rot16<4, S>(o2);
    o3 = rot16<6, S>(o3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// 16 = 4 x 4 with j = 4 j1 + j2 and k = k1 + 4 k2:
//   Y[j2][k1] = w_16^{j2 k1} sum_{j1} v[4 j1 + j2] w_4^{j1 k1};
//   X[k1 + 4 k2] = sum_{j2} Y[j2][k1] w_4^{j2 k2}.
template <int S>
HDEV void dft16(float2 *v)
{
#pragma unroll
    for (int j2 = 0; j2 < 4; ++j2) dft4<S>(v[j2], v[4 + j2], v[8 + j2], v[12 + j2]);
    // v[j2 + 4 k1] = Y[j2][k1] before the twiddle
    v[5] = rot16<1, S>(v[5]);
    v[6] = rot16<2, S>(v[6]);
    v[7] = rot16<3, S>(v[7]);
    v[9] = rot16<2, S>(v[9]);
    v[10] = rot16<4, S>(v[10]);
    v[11] = rot16<6, S>(v[11]);
    v[13] = rot16<3, S>(v[13]);
    v[14] = rot16<6, S>(v[14]);
    v[15] = rot16<9, S>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<S>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] = X[k1 + 4 k2]; restore natural order
    float2 t[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) t[k] = v[4 * (k & 3) + (k >> 2)];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = t[k];
}

// a * w_32^M, w_32 = exp(sigma 2 pi i / 32), M = 0..15, from cos(M pi/16)
// and sin(M pi/16) (first-octant values c1 = cos(pi/16), s1 = sin(pi/16),
// c3 = cos(3 pi/16), s3 = sin(3 pi/16), and those of rot16)
template <int M, int S>
HDEV float2 rot32(float2 a)
{
    static_assert(M >= 0 && M < 16, "rot32 exponent");
    if constexpr (M == 0) return a;
    else if constexpr (M == 8) return mul_si<S>(a);
    else {
        constexpr float c1 = 0.98078528040323044913f, s1 = 0.19509032201612826785f;
        constexpr float c3 = 0.83146961230254523708f, s3 = 0.55557023301960222474f;
        constexpr float CS[16][2] = {{1.f, 0.f},      {c1, s1},        {kC16a, kC16b},  {c3, s3},
                                     {kC8, kC8},      {s3, c3},        {kC16b, kC16a},  {s1, c1},
                                     {0.f, 1.f},      {-s1, c1},       {-kC16b, kC16a}, {-s3, c3},
                                     {-kC8, kC8},     {-c3, s3},       {-kC16a, kC16b}, {-c1, s1}};
        constexpr float C = CS[M][0], Sn = CS[M][1];
        constexpr float s = (float)S;
        return make_float2(a.x * C - s * a.y * Sn, a.y * C + s * a.x * Sn);
    }
}

// 32 = 2 x 16: X_k = E_k + w_32^k O_k, X_{k+16} = E_k - w_32^k O_k, with E, O
// the 16-point DFTs of the even and odd samples.
template <int S>
HDEV void dft32(float2 *v)
{
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft16<S>(e);
    dft16<S>(o);
    o[1] = rot32<1, S>(o[1]);
    o[2] = rot32<2, S>(o[2]);
    o[3] = rot32<3, S>(o[3]);
    o[4] = rot32<4, S>(o[4]);
    o[5] = rot32<5, S>(o[5]);
    o[6] = rot32<6, S>(o[6]);
    o[7] = rot32<7, S>(o[7]);
    o[8] = rot32<8, S>(o[8]);
    o[9] = rot32<9, S>(o[9]);
    o[10] = rot32<10, S>(o[10]);
    o[11] = rot32<11, S>(o[11]);
    o[12] = rot32<12, S>(o[12]);
    o[13] = rot32<13, S>(o[13]);
    o[14] = rot32<14, S>(o[14]);
    o[15] = rot32<15, S>(o[15]);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 16] = csub(e[k], o[k]);
    }
}

// Odd prime radix R = 3, 5, 7 by the pair sums and differences of the
// inputs: with A_k = v_k + v_{R-k}, B_k = v_k - v_{R-k} (k = 1..(R-1)/2),
//   X_0 = v_0 + sum_k A_k,
//   X_m, X_{R-m} = v_0 + sum_k cos(2 pi m k / R) A_k  +/-  sigma i sum_k sin(2 pi m k / R) B_k.
// odd_cos / odd_sin give cos and sin(2 pi q / R) for q = m k mod R (cos is
// even and sin odd in q, so q in 1..R-1 is enough).
template <int R>
HDEV constexpr float odd_cos(int q)
{
    // R = 3: cos(2 pi / 3); R = 5: cos(2 pi / 5), cos(4 pi / 5); R = 7: cos(2 pi k / 7), k = 1, 2, 3
    const int r = q <= R / 2 ? q : R - q;
    return R == 3 ? -0.5f
           : R == 5 ? (r == 1 ? 0.30901699437494742410f : -0.80901699437494742410f)
                    : (r == 1 ? 0.62348980185873353053f : r == 2 ? -0.22252093395631440429f : -0.90096886790241912624f);
}
template <int R>
HDEV constexpr float odd_sin(int q)
{
    const int r = q <= R / 2 ? q : R - q;
    const float v = R == 3 ? 0.86602540378443864676f
                    : R == 5 ? (r == 1 ? 0.95105651629515357212f : 0.58778525229247312917f)
                             : (r == 1 ? 0.78183148246802980871f : r == 2 ? 0.97492791218182360702f
                                                                          : 0.43388373911755812048f);
    return q <= R / 2 ? v : -v;
}

template <int R, int S>
HDEV void dft_odd(float2 *v)
{
    constexpr int H = (R - 1) / 2;
    float2 A[H], B[H];
    float2 x0 = v[0];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        A[k] = cadd(v[k + 1], v[R - 1 - k]);
        B[k] = csub(v[k + 1], v[R - 1 - k]);
    }
    float2 X0 = x0;
#pragma unroll
    for (int k = 0; k < H; ++k) X0 = cadd(X0, A[k]);
#pragma unroll
    for (int m = 0; m < H; ++m) {
        float2 P = x0, Q = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float c = odd_cos<R>(((m + 1) * (k + 1)) % R), sn = odd_sin<R>(((m + 1) * (k + 1)) % R);
            P = make_float2(P.x + c * A[k].x, P.y + c * A[k].y);
            Q = make_float2(Q.x + sn * B[k].x, Q.y + sn * B[k].y);
        }
        const float2 iQ = mul_si<S>(Q);  // sigma i Q
        v[m + 1] = cadd(P, iQ);
        v[R - 1 - m] = csub(P, iQ);
    }
    v[0] = X0;
}

template <int R, int S>
HDEV void dft(float2 *v)
{
    if constexpr (R == 2) dft2<S>(v[0], v[1]);
    else if constexpr (R == 3 || R == 5 || R == 7) dft_odd<R, S>(v);
    else if constexpr (R == 4) dft4<S>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<S>(v);
    else if constexpr (R == 16) dft16<S>(v);
    else if constexpr (R == 32) dft32<S>(v);
}

// Radix schedule of a length-2^LOG_L line: radix 16 while possible, then one
// 2/4/8 stage.
template <int LOG_L, int STAGE>
struct StageInfo {
    static constexpr int NFULL = LOG_L / 4;
    static constexpr int REM = LOG_L % 4;
    static constexpr int NSTAGES = NFULL + (REM ? 1 : 0);
    static constexpr int LOG_R = (STAGE < NFULL) ? 4 : REM;
    static constexpr int R = 1 << LOG_R;
    static constexpr int LOG_NS = 4 * STAGE;
    static constexpr int NS = 1 << LOG_NS;
    static constexpr bool FIRST = STAGE == 0;
    static constexpr bool LAST = STAGE == NSTAGES - 1;
};

// Shared-memory slot of (line c, index i).  CFAST: lines interleaved
// (q = i*W + c); else line-major (q = c*L + i).  One pad slot every 2^PS
// slots keeps the strided accesses of the first stage conflict-free.
template <int LOG_L, int LOG_W, bool CFAST, int PS>
FDEV int smem_slot(int c, int i)
{
    const int q = CFAST ? ((i << LOG_W) + c) : ((c << LOG_L) + i);
    return q + (q >> PS);
}

template <int LOG_L, int LOG_W, int PS>
constexpr int smem_slots()
{
    return (1 << (LOG_L + LOG_W)) + ((1 << (LOG_L + LOG_W)) >> PS) + 1;
}

// Butterfly g of a stage with radix 2^LOG_R -> (line c, butterfly index j).
template <int LOG_L, int LOG_W, bool CFAST, int LOG_R>
FDEV void butterfly_coords(int g, int &c, int &j)
{
    if (CFAST) {
        c = g & ((1 << LOG_W) - 1);
        j = g >> LOG_W;
    } else {
        c = g >> (LOG_L - LOG_R);
        j = g & ((1 << (LOG_L - LOG_R)) - 1);
    }
}

// Stage twiddle tables.  Stage s > 0 (radix R, Ns = 16^s) multiplies element
// r of butterfly j by w_{Ns R}^{m r}, m = j mod Ns.  Its table holds these
// values r-major, [r-1][m], so that lanes with consecutive m read consecutive
// entries (or one broadcast entry); tables of stages 1, 2, ... follow each
// other.  stage_table_offset gives where stage s starts.
template <int LOG_L>
__host__ __device__ constexpr int stage_table_offset(int stage)
{
    int off = 0;
    for (int s = 1; s < stage; ++s) {
        const int lr = s < LOG_L / 4 ? 4 : LOG_L % 4;
        off += ((1 << lr) - 1) << (4 * s);
    }
    return off;
}

// Twiddle + DFT of one butterfly held in x[0..R).  tw: the stage tables of
// a length-L line (laid out as stage_table_offset gives).
template <int LOG_L, int STAGE, int S>
FDEV void apply_twiddles(float2 *x, int j, const float2 *__restrict__ tw)
{
    using I = StageInfo<LOG_L, STAGE>;
    if constexpr (!I::FIRST) {
        constexpr int OFF = stage_table_offset<LOG_L>(STAGE);
        const float2 *t = tw + OFF + (j & (I::NS - 1));
#pragma unroll
        for (int r = 1; r < I::R; ++r) x[r] = twmul<S>(x[r], __ldg(t + (r - 1) * I::NS));
    }
}

template <int LOG_L, int STAGE, int S>
FDEV void butterfly(float2 *x, int j, const float2 *__restrict__ tw)
{
    apply_twiddles<LOG_L, STAGE, S>(x, j, tw);
    dft<StageInfo<LOG_L, STAGE>::R, S>(x);
}

// Output index of element r of butterfly j.
template <int LOG_L, int STAGE>
FDEV int stockham_out_index(int j, int r)
{
    using I = StageInfo<LOG_L, STAGE>;
    return ((j >> I::LOG_NS) << (I::LOG_NS + I::LOG_R)) + (j & (I::NS - 1)) + (r << I::LOG_NS);
}

}  // namespace fftseg

// ------------------------------------------------------------------ TMA bulk
// 1-D bulk copies global -> shared (cp.async.bulk), completed on an mbarrier
// with transaction-byte accounting.  Every wait is bounded: after
// kSpinLimit polls the waiter records a timeout in *err and carries on, so a
// lost copy can never hang the GPU.
namespace fftseg {

constexpr uint32_t kSpinLimit = 1u << 24;

FDEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 8-byte asynchronous copy global -> shared (cp.async; any 8-byte-aligned
// source).  src_bytes = 0 writes zeros and reads nothing.  Copies are grouped
// by cp_async_commit; cp_async_wait<N> returns once at most N of the calling
// thread's groups are pending, and the thread then sees its own copies
// (other threads' copies need a barrier after their waits).
FDEV void cp_async8(void *smem_dst, const void *gsrc, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
FDEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
FDEV void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel in its stream is still
// running; grid_dependency_wait returns once that kernel has completed and
// its memory operations are visible (no global access of the data path may
// come before it), and launch_dependents lets the next such kernel start its
// own blocks as this one's leave.
FDEV void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
FDEV void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bulk prefetch of global memory into L2 (16-byte aligned, bytes % 16 == 0).
// A hint only: lines fetched before a producer's writes to them are updated
// in L2 by those writes, so it may precede grid_dependency_wait.
FDEV void prefetch_l2_bulk(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

FDEV void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

FDEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses
FDEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// order this thread's generic-proxy view of global memory (e.g. data another
// CTA published with a release) before its later async-proxy (TMA) reads
FDEV void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Tiled 3-D TMA store of one box from shared memory (16-byte aligned, dense
// box layout) to `tmap` at (x, y, z); tracked by bulk groups of this thread.
FDEV void tma_store_3d(const CUtensorMap *tmap, int x, int y, int z, const void *src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}

// wait until every committed bulk copy of this thread has completed its writes
FDEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// wait until every committed bulk store of this thread has read its source
FDEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// plain arrive (count 1) on an mbarrier
FDEV void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Release add at GPU scope: this thread's earlier memory operations, and those
// it has observed through synchronisation, are visible before the add.
FDEV void red_release_add(int *p, int v)
{
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Drop a 128-byte line from L2 without writing it back (its contents become
// undefined): for intermediate data that has been consumed.
FDEV void discard_l2_line(const void *p) { asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory"); }

FDEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// dst (shared, 16-byte aligned) <- src (global, 16-byte aligned), bytes % 16 == 0
FDEV void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Tiled 3-D TMA load of one box of `tmap` at element coordinates (x, y, z)
// into shared memory (16-byte aligned), completed on *bar.  x * 8 bytes must
// be a multiple of 16 (8-byte elements: x even).
FDEV void tma_load_3d(void *dst, const CUtensorMap *tmap, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Tiled 2-D TMA load of one box of `tmap` at (x, y) into shared memory with
// an L2 cache policy, completed on *bar (x * element size a multiple of 16).
FDEV void tma_load_2d_hint(void *dst, const CUtensorMap *tmap, int x, int y, uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// Tiled 4-D TMA load of one box of `tmap` at element coordinates (x, y, z, w)
// into shared memory, completed on *bar (x * element size a multiple of 16).
FDEV void tma_load_4d(void *dst, const CUtensorMap *tmap, int x, int y, int z, int w, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// L2 cache policy that leaves a line's eviction priority as it is (for data
// that is read twice, such as the overlap of consecutive frames).
FDEV uint64_t policy_evict_unchanged()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_unchanged.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// L2 cache policy: lines fetched or written under it are evicted first (for
// data streamed once, so that it does not displace data kept in L2).
FDEV uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// tma_load_3d with an L2 cache policy
FDEV void tma_load_3d_hint(void *dst, const CUtensorMap *tmap, int x, int y, int z, uint64_t *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

// tma_store_3d with an L2 cache policy
FDEV void tma_store_3d_hint(const CUtensorMap *tmap, int x, int y, int z, const void *src, uint64_t policy)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint [%0, {%1, %2, %3}], [%4], %5;" ::"l"(
                     reinterpret_cast<uint64_t>(tmap)),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src)), "l"(policy)
                 : "memory");
}

// address of the same shared-memory variable in CTA `rank` of the cluster
FDEV uint32_t mapa_u32(uint32_t smem_addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr), "r"(rank));
    return r;
}

FDEV void st_cluster_v2(uint32_t addr, float2 v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// Remote store into CTA-shared memory of a cluster peer that also credits 8
// bytes to the peer's mbarrier (st.async): the receiver learns of the data by
// waiting on its own barrier; no release fence is needed on the sender side.
FDEV void st_async_v2(uint32_t remote_addr, float2 v, uint32_t remote_bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
                     remote_addr),
                 "f"(v.x), "f"(v.y), "r"(remote_bar)
                 : "memory");
}

// Bulk copy from this CTA's shared memory to a cluster peer's shared memory
// (both addresses 16-byte aligned, bytes % 16 == 0), completing on the peer's
// mbarrier.  dst and bar are shared::cluster addresses (mapa).
FDEV void dsmem_bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "r"(smem_u32(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

FDEV void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// wait until every committed bulk copy of this thread has finished reading its source
FDEV void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Cluster-wide execution barrier without memory ordering (arrive.relaxed):
// used where every thread has already consumed what it read.
FDEV void cluster_sync_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// The two halves of cluster_sync_relaxed, for an arrive early and a wait late.
FDEV void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
FDEV void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

FDEV bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity` of *bar.
FDEV bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// GPU-scope acquire-release fence.
FDEV void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Wait for phase `parity` of *bar; false (and *err set) if it never completes.
FDEV bool mbar_wait(uint64_t *bar, uint32_t parity, int *err)
{
    for (uint32_t it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, 1);
    return false;
}

}  // namespace fftseg
