// Plans, twiddle tables, dispatch and the plain C-ABI entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <cudaTypedefs.h>

#include "fourstep.cuh"
#include "fourstep_ws.cuh"
#include "launch.h"
#include "fourstep_hw.cuh"
#include "fourstep_wl.cuh"
#include "plan.h"

namespace fftseg {

namespace {
thread_local char g_msg[512] = "";
std::atomic<int64_t> g_launches{0};

constexpr int64_t kWorkTargetBytes = 32ll << 20;  // two-pass chunk: stays resident in L2
constexpr int kTwoLevelAbove = 20;                 // n > 2^20: four-step table split in two
constexpr int kTwLogK = 6;
constexpr int64_t kChunkBytes = 16ll << 20;  // four-step chunk; the ring holds kRingNr of them
constexpr int kRingNr = 3;

bool is_pow2(int64_t n) { return n >= 1 && (n & (n - 1)) == 0; }

// FP32 complex output on the persistent four-step path, not asked for the
// producer or CTA-tile kernels: the lane-local-line kernels can run it.
bool lane_kernels_apply(const fftseg_plan_s *p)
{
    return p->precision == FFTSEG_PREC_FP32 &&
           !(p->flags & (FFTSEG_FLAG_FOURSTEP_PRODUCER | FFTSEG_FLAG_FOURSTEP_TILES));
}
// n = 2^16..2^20: the lane-line kernel (fourstep_wl.cuh), measured faster
// than the warp-line kernel at 2^16 (0.60 against 0.59 of the copy peak).
bool uses_fourstep_wl(const fftseg_plan_s *p)
{
    return lane_kernels_apply(p) && p->log_n >= 16 && p->log_n <= 20 &&
           !(p->flags & FFTSEG_FLAG_FOURSTEP_WARP_LINES);
}
// n = 2^21..2^24: the outer radix-R pass and the lane-line kernel over
// interleaved transforms of 2^16 points (two HBM passes).
bool uses_fourstep_ilv(const fftseg_plan_s *p)
{
    return lane_kernels_apply(p) && p->log_n >= 21 && p->log_n <= 24 &&
           !(p->flags & FFTSEG_FLAG_FOURSTEP_WARP_LINES);
}
// n = 256 x 256 on request: the warp-line kernel (fourstep_hw.cuh).
bool uses_fourstep_hw(const fftseg_plan_s *p)
{
    return p->log_n == 16 && lane_kernels_apply(p) && p->out_kind == FFTSEG_OUT_COMPLEX &&
           (p->flags & FFTSEG_FLAG_FOURSTEP_WARP_LINES);
}
// Bluestein plans whose M-point rows fit one block tile (M <= 4096, the
// inner forward plan on the block path) run as one fused kernel.
bool blue_fused(const fftseg_plan_s *p)
{
    return p->bm <= 4096 && p->inner && p->inner->path == PATH_BLOCK && p->inner->precision == FFTSEG_PREC_FP32;
}
// Bluestein plans whose inverse M-point plan runs on the cluster kernel
// (M = 2^13..2^17) fold the product with B and the chirp-out into it.
bool blue_inv_fused(const fftseg_plan_s *p)
{
    return p->path == PATH_BLUESTEIN && p->inner2 && p->inner2->path == PATH_CLUSTER &&
           p->inner2->precision == FFTSEG_PREC_FP32;
}
// Frame plans of n <= 4096 points (the inner plan on the block path) run as
// one fused kernel.
bool frames_fused(const fftseg_plan_s *p)
{
    return p->path == PATH_FRAMES && p->inner && p->inner->path == PATH_BLOCK &&
           p->inner->precision == FFTSEG_PREC_FP32;
}

// Forward real-signal plans whose n/2-point complex transform runs on the
// block or the cluster kernel split the spectrum inside that kernel (one
// pass, no intermediate); inverse ones join the bins inside the cluster
// kernel up to n/2 = 2^14 for batches of at most 64 MiB of samples.  (The
// fused join reads its bins with plain loads, a point and its mirror:
// measured on GB300 at n = 2^14 and 2^15 over 4 GiB, 0.37 and 0.35 of the
// copy peak against 0.39 and 0.37 in 512 MiB chunks, at 256 MiB 0.35 / 0.34
// against 0.37 / 0.36, and for 37 segments 9.1 / 12.4 us against
// 12.7 / 14.5 us; from n = 2^16 on it fell to 0.29..0.22, and copying the
// bins and their mirrors in ahead by 8-byte cp.async, at two CTAs per SM,
// measured slower still: 0.33..0.21 at n = 2^14..2^17.)
bool real_fused(const fftseg_plan_s *p)
{
    if (p->path != PATH_REAL || !p->inner) return false;
    if (p->direction == FFTSEG_INVERSE)
        return p->inner->path == PATH_CLUSTER && p->inner->log_n <= 14 && p->batch * p->n * 4 <= (int64_t(64) << 20);
    return p->inner->path == PATH_BLOCK || p->inner->path == PATH_CLUSTER;
}
int ilog2(int64_t n)
{
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}
}  // namespace

int set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char *what)
{
    return set_error(e == cudaErrorMemoryAllocation ? FFTSEG_E_NOMEM : FFTSEG_E_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void host_roots(float2 *t, int64_t count, int64_t M, int64_t stride_exp)
{
    // t[m] = exp(-2 pi i (m * stride_exp mod M) / M), the exponent reduced exactly in integers
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t m = 0; m < count; ++m) {
        const int64_t e = (int64_t)(((unsigned __int128)m * (unsigned __int128)stride_exp) % (unsigned __int128)M);
        const double a = two_pi * ((double)e / (double)M);
        t[m] = make_float2((float)cos(a), (float)-sin(a));
    }
}

namespace {

int upload(float2 **dst, const std::vector<float2> &h)
{
    cudaError_t e = cudaMalloc((void **)dst, h.size() * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(twiddles)");
    e = cudaMemcpy(*dst, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(twiddles)");
    return FFTSEG_OK;
}

}  // namespace

// Stage twiddle tables of a length-L line, in the order the kernels read them:
// for every stage s >= 1 (radix R_s, Ns = 16^s combined points before it),
// entries [r-1][m] = w_{Ns R_s}^{m r}, r = 1..R_s-1, m = 0..Ns-1.  The radix
// schedule is 16, 16, ..., then one 2/4/8 stage for the remainder.
void stage_table_host(std::vector<float2> &h, int64_t L)
{
    int log_l = ilog2(L);
    h.clear();
    int64_t ns = 1;
    for (int left = log_l; left > 0;) {
        const int lr = left >= 4 ? 4 : left;
        const int64_t R = int64_t(1) << lr;
        if (ns > 1) {
            const size_t base = h.size();
            h.resize(base + (size_t)((R - 1) * ns));
            for (int64_t r = 1; r < R; ++r) host_roots(h.data() + base + (r - 1) * ns, ns, ns * R, r);
        }
        ns *= R;
        left -= lr;
    }
    if (h.empty()) h.push_back(make_float2(1.f, 0.f));
}

namespace {

int stage_table(float2 **dst, int64_t L)
{
    std::vector<float2> h;
    stage_table_host(h, L);
    return upload(dst, h);
}

// Four-step table rows k1 < rows of w_n^{(k1 * row_mult) * j2}, [rows][n2]
int fourstep_table(float2 **dst, int64_t n, int64_t rows, int64_t row_mult, int64_t n2)
{
    std::vector<float2> h((size_t)(rows * n2));
    for (int64_t k1 = 0; k1 < rows; ++k1) host_roots(h.data() + k1 * n2, n2, n, k1 * row_mult);
    return upload(dst, h);
}

void free_plan(fftseg_plan p)
{
    if (!p) return;
    free_plan(p->inner);
    free_plan(p->inner2);
    cudaFree(p->bw);
    cudaFree(p->bhat);
    cudaFree(p->rtw);
    cudaFree(p->rwork);
    cudaFree(p->fwin);
    cudaFree(p->win_row);
    cudaFree(p->win_col);
    if (p->host_stage && p->host_stage_free) p->host_stage_free(p->host_stage);
    cudaFree(p->twA);
    cudaFree(p->twB);
    cudaFree(p->tw4a);
    cudaFree(p->tw4b);
    cudaFree(p->work);
    cudaFree(p->d_err);
    cudaFree(p->ring);
    cudaFree(p->ctr);
    cudaFree(p->w4);
    cudaFree(p->w4hi);
    cudaFree(p->w4t);
    delete p;
}

int env_int(const char *name, int dflt, int lo, int hi)
{
    const char *v = getenv(name);
    if (!v || !*v) return dflt;
    const int x = atoi(v);
    return x < lo ? lo : x > hi ? hi : x;
}

// Lane-line four-step kernel: its stage-2 tables, per-column-tile factors,
// ring and per-segment counters.  Ring chunks of FFTSEG_WL_CHUNK_MB MiB
// (default 24) and FFTSEG_WL_LOOKAHEAD chunks (default 1) of lead of the
// column passes are tuning knobs read at plan creation.
int build_fourstep_wl(fftseg_plan p)
{
    int l1, l2, le;
    if (!fourstep_wl_shape(p->log_n, &l1, &l2, &le)) return set_error(FFTSEG_E_UNSUPPORTED, "lane-line shape");
    p->path = PATH_FOURSTEP;
    p->log_n1 = l1;
    p->log_n2 = l2;
    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    const int64_t p1 = n1 / 32, p2 = n2 / 32;
    const int64_t wa = (int64_t(1) << le) / n1;  // columns per column tile
    p->log_wa = le - l1;
    p->log_wb = le - l2;
    int rc;
    // stage 2 of an L-point line: [r-1][b] = w_L^{b r}, r = 1 .. L/32 - 1, b < 32
    auto stage2 = [&](float2 **dst, int64_t L) -> int {
        const int64_t P = L / 32;
        std::vector<float2> h((size_t)((P - 1) * 32));
        for (int64_t r = 1; r < P; ++r) host_roots(h.data() + (r - 1) * 32, 32, L, r);
        return upload(dst, h);
    };
    if ((rc = stage2(&p->twA, n1))) return rc;
    if (l2 != l1 && (rc = stage2(&p->twB, n2))) return rc;
    {
        // per column tile ct, its columns col (j2 = ct wa + col) in pairs, the
        // pair's two columns side by side (so that the two lines a half-warp
        // holds read adjacent entries): [wa/2][P1][2] w_n^{j2 j}, then
        // [wa/2][32][2] scale * w_n^{j2 P1 m}
        // (interleaved units: column tile j2 holds column j2 of 32 transforms,
        // so every column of tile j2 takes the factors of j2)
        const int64_t ft = wa * (p1 + 32);
        const int64_t ntile = p->wl_ilv ? n2 : n2 / wa;
        std::vector<float2> h((size_t)(ntile * ft));
        std::vector<float2> t1((size_t)p1), t2(32);
        for (int64_t tc = 0; tc < ntile * wa; ++tc) {
            const int64_t j2 = p->wl_ilv ? tc / wa : tc;
            float2 *t = h.data() + (tc / wa) * ft;
            const int64_t col = tc % wa, pr = col >> 1, hc = col & 1;
            host_roots(t1.data(), p1, p->n, j2);
            host_roots(t2.data(), 32, p->n, j2 * p1);
            for (int64_t j = 0; j < p1; ++j) t[(pr * p1 + j) * 2 + hc] = t1[(size_t)j];
            for (int m = 0; m < 32; ++m)
                t[wa * p1 + (pr * 32 + m) * 2 + hc] = make_float2(t2[m].x * p->scale, t2[m].y * p->scale);
        }
        if ((rc = upload(&p->w4t, h))) return rc;
    }
    // (interleaved units of 16 MiB: two per chunk measured 6 % faster than one)
    const int64_t chunk = (int64_t)env_int("FFTSEG_WL_CHUNK_MB", p->wl_ilv ? 32 : 24, 1, 64) << 20;
    const int64_t slab = p->n * (p->wl_ilv ? 32 : 1);  // points of one unit
    int64_t cs = chunk / (slab * 8);
    if (cs < 1) cs = 1;
    if (cs > p->batch) cs = p->batch;
    p->ring_cs = (int)cs;
    p->wl_la = env_int("FFTSEG_WL_LOOKAHEAD", 1, 1, 4);
    p->ring_nr = p->wl_la + 2;
    cudaError_t e = cudaMalloc((void **)&p->ring, (size_t)(p->ring_nr * cs * slab) * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(ring)");
    const int64_t nc = (p->batch + cs - 1) / cs;
    p->ctr_count = 1 + 2 * nc * cs;
    e = cudaMalloc((void **)&p->ctr, (size_t)p->ctr_count * sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(counters)");
    return FFTSEG_OK;
}

// n = R * M, M = 2^16, R = 2^(log2 n - 16) = 32..256 (decimation in
// frequency over the outer index): the outer pass forms, for every j < M,
//   Y_t[j] = w_n^{j t} sum_{t'} x[j + M t'] w_R^{t' t},   t < R,
// written interleaved (Y_t[j] at R j + t); the lane-line plan of M points
// then transforms each Y_t, 32 at a time, and writes bin k of Y_t to
// X[t + R k].  Both passes stream the segment once: 32 bytes of HBM traffic
// per point.  Work in chunks of segments through a 1 GiB workspace.
int build_fourstep_ilv(fftseg_plan p)
{
    constexpr int kLogM = 16;
    // (1 GiB: 1.5-2 % faster than 512 MiB over 4 GiB batches at 2^21..2^24,
    // 2 GiB another 1 %; 128..32 MiB, the intermediate kept in L2, 9-33 %
    // slower: launches and per-launch ramps then dominate)
    const int64_t kIlvWorkBytes = (int64_t)env_int("FFTSEG_ILV_WORK_MB", 1024, 1, 4096) << 20;
    const int log_r = p->log_n - kLogM;
    const int64_t R = int64_t(1) << log_r, M = int64_t(1) << kLogM;
    p->path = PATH_FOURSTEP;
    p->ilv_log_r = log_r;
    p->log_n1 = log_r;
    p->log_n2 = kLogM;
    int rc;
    if ((rc = stage_table(&p->twA, R))) return rc;
    // w_n^{j t} = [t mod 16][j] x [t div 16][j]
    if ((rc = fourstep_table(&p->tw4a, p->n, 16, 1, M))) return rc;
    if ((rc = fourstep_table(&p->tw4b, p->n, R / 16, 16, M))) return rc;
    int64_t segs = kIlvWorkBytes / (p->n * 8);
    if (segs < 1) segs = 1;
    if (segs > p->batch) segs = p->batch;
    p->work_segs = segs;
    cudaError_t e = cudaMalloc((void **)&p->work, (size_t)(segs * p->n) * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(workspace)");
    fftseg_plan q = new (std::nothrow) fftseg_plan_s();
    if (!q) return set_error(FFTSEG_E_NOMEM, "plan_create: host allocation failed");
    p->inner = q;
    q->device = p->device;
    q->n = M;
    q->log_n = kLogM;
    q->batch = segs * (R / 32);  // units of 32 interleaved transforms
    q->direction = p->direction;
    q->norm = p->norm;
    q->precision = p->precision;
    q->out_kind = p->out_kind;
    q->scale = p->scale;  // the whole transform's scale, folded into the column factors
    q->wl_ilv = true;
    e = cudaMalloc((void **)&q->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(q->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(status flag)");
    return build_fourstep_wl(q);
}

// Persistent four-step: ring, counters, stage tables and the two factor
// tables of the four-step twiddle, [j2][k1 mod K] and [j2][k1 div K].
int build_fourstep(fftseg_plan p)
{
    if ((p->flags & FFTSEG_FLAG_FOURSTEP_WARP_LINES) && !uses_fourstep_hw(p))
        return set_error(FFTSEG_E_UNSUPPORTED,
                         "plan_create: the warp-line four-step kernel runs FP32 complex output at n = 2^16");
    if (uses_fourstep_wl(p)) return build_fourstep_wl(p);
    if (uses_fourstep_ilv(p)) return build_fourstep_ilv(p);
    int l1, l2, lwa, lwb;
    if (!fourstep_shape(p->log_n, &l1, &l2, &lwa, &lwb))
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: the four-step path needs n in [2^14, 2^24]");
    p->path = PATH_FOURSTEP;
    p->log_n1 = l1;
    p->log_n2 = l2;
    p->log_wa = lwa;
    p->log_wb = lwb;
    const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
    int rc;
    if ((rc = stage_table(&p->twA, n1))) return rc;
    if ((rc = stage_table(&p->twB, n2))) return rc;
    p->w4_log_k = fourstep_log_k(l1);
    const int64_t K = int64_t(1) << p->w4_log_k;
    {
        std::vector<float2> h((size_t)(n2 * K));
        for (int64_t j2 = 0; j2 < n2; ++j2) host_roots(h.data() + j2 * K, K, p->n, j2);
        if ((rc = upload(&p->w4, h))) return rc;
    }
    if (K < n1) {
        std::vector<float2> h((size_t)(n2 * (n1 / K)));
        for (int64_t j2 = 0; j2 < n2; ++j2) host_roots(h.data() + j2 * (n1 / K), n1 / K, p->n, j2 * K);
        if ((rc = upload(&p->w4hi, h))) return rc;
    }
    if (uses_fourstep_hw(p)) {
        // the same two factors grouped per column tile of 16 columns j2, the
        // plan's scale (a power of two at n = 2^16, so exact) folded into the
        // second: [ct][w_n^{j2 m}: 16 cols x 16][scale * w_n^{j2 16 q}: 16 cols x 16]
        std::vector<float2> h((size_t)(n2 * 32));
        for (int64_t j2 = 0; j2 < n2; ++j2) {
            float2 *t = h.data() + (j2 >> 4) * 512 + (j2 & 15) * 16;
            host_roots(t, 16, p->n, j2);
            host_roots(t + 256, 16, p->n, j2 * 16);
            for (int q = 0; q < 16; ++q) t[256 + q] = make_float2(t[256 + q].x * p->scale, t[256 + q].y * p->scale);
        }
        if ((rc = upload(&p->w4t, h))) return rc;
    }
    int64_t cs = kChunkBytes / (p->n * 8);
    if (cs < 1) cs = 1;
    if (cs > p->batch) cs = p->batch;
    p->ring_cs = (int)cs;
    p->ring_nr = uses_fourstep_hw(p) ? FourStepHwShape::MIN_RING : kRingNr;
    cudaError_t e = cudaMalloc((void **)&p->ring, (size_t)(p->ring_nr * cs * p->n) * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(ring)");
    const int64_t nc = (p->batch + cs - 1) / cs;
    // counters per chunk, or per segment for the warp-local-line kernel
    p->ctr_count = 1 + 2 * (uses_fourstep_hw(p) ? nc * cs : nc);
    e = cudaMalloc((void **)&p->ctr, (size_t)p->ctr_count * sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(counters)");
    return FFTSEG_OK;
}

int kernel_prec(fftseg_plan p)
{
    return p->precision == FFTSEG_PREC_TC_FP16 ? PREC_FP16 : p->precision == FFTSEG_PREC_TC_BF16 ? PREC_BF16 : PREC_FP32;
}

// Tensor-core precisions: radix-16 stages as split hi+lo GEMMs (n a power of
// 16): n <= 4096 on the block kernel, larger n on the persistent four-step.
int build_tc(fftseg_plan p)
{
    const int ln = p->log_n;
    if (ln % 4 != 0 || ln < 4)
        return set_error(FFTSEG_E_UNSUPPORTED,
                         "plan_create: the tensor-core precisions need n to be a power of 16 (16 .. 2^24)");
    if (p->flags & FFTSEG_FLAG_FORCE_TWOPASS)
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: the tensor-core precisions have no two-pass form");
    if (ln <= 12) {
        p->path = PATH_BLOCK;
        p->log_n1 = ln;
        return stage_table(&p->twA, p->n);
    }
    return build_fourstep(p);
}

int build_fp32(fftseg_plan p)
{
    const int ln = p->log_n;
    if (p->flags & (FFTSEG_FLAG_FOURSTEP_L2 | FFTSEG_FLAG_FOURSTEP_WARP_LINES | FFTSEG_FLAG_FOURSTEP_TILES))
        return build_fourstep(p);
    const bool force2 = (p->flags & FFTSEG_FLAG_FORCE_TWOPASS) && ln >= 8;
    int rc;
    if (ln <= 12 && !force2) {
        p->path = PATH_BLOCK;
        p->log_n1 = ln;
        p->log_n2 = 0;
        return stage_table(&p->twA, p->n);
    }
    int l1, l2, lc;
    const int want_c = (int)((p->flags >> 8) & 0xFu);
    // measured on GB300: the cluster path wins up to 2^15, the persistent
    // four-step above: at 2^16 its lane-line kernel (16384 segments: 4.14 ms
    // against 5.5 ms for 16-CTA clusters, whose all-to-all exchange is bound
    // by the SM-to-SM network; |X|^2 of 4 GiB: 1.97 ms against 2.75 ms), from
    // 2^17 on because a 16-CTA cluster per segment leaves SMs idle
    // (at 2^24 with complex output the two-pass path measured 8 % faster than
    // the persistent four-step: a segment's 128 MiB intermediate cannot stay
    // in L2, so both make two HBM passes)
    // (complex FP32 output at 2^21..2^24 runs the interleaved four-step instead)
    const bool twopass_24 = ln == 24 && p->out_kind == FFTSEG_OUT_COMPLEX && !uses_fourstep_ilv(p);
    if (!force2 && want_c == 0 && !twopass_24 && ln >= 16) return build_fourstep(p);
    if (!force2 && ln >= 13 && ln <= 17 && !cluster_shape(ln, want_c, &l1, &l2, &lc))
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: no cluster of 2^%d CTAs is built for n=2^%d",
                         want_c, ln);
    if (!force2 && cluster_shape(ln, want_c, &l1, &l2, &lc)) {
        p->path = PATH_CLUSTER;
        p->log_n1 = l1;
        p->log_n2 = l2;
        p->log_c = lc;
        if ((rc = stage_table(&p->twA, int64_t(1) << l1))) return rc;
        if ((rc = stage_table(&p->twB, int64_t(1) << l2))) return rc;
        return fourstep_table(&p->tw4a, p->n, int64_t(1) << l1, 1, int64_t(1) << l2);
    }
    p->path = PATH_TWOPASS;
    p->log_n1 = (ln + 1) / 2;  // column length (pass A)
    p->log_n2 = ln / 2;        // row length (pass B)
    const int64_t n1 = int64_t(1) << p->log_n1, n2 = int64_t(1) << p->log_n2;
    if ((rc = stage_table(&p->twA, n1))) return rc;
    if ((rc = stage_table(&p->twB, n2))) return rc;
    if (ln > kTwoLevelAbove) {
        p->tw_log_k = kTwLogK;
        const int64_t K = int64_t(1) << kTwLogK;
        if ((rc = fourstep_table(&p->tw4a, p->n, K, 1, n2))) return rc;
        if ((rc = fourstep_table(&p->tw4b, p->n, n1 / K, K, n2))) return rc;
    } else {
        p->tw_log_k = p->log_n1;
        if ((rc = fourstep_table(&p->tw4a, p->n, n1, 1, n2))) return rc;
    }
    int64_t segs = kWorkTargetBytes / (p->n * 8);
    if (segs < 1) segs = 1;
    if (segs > p->batch) segs = p->batch;
    p->work_segs = segs;
    cudaError_t e = cudaMalloc((void **)&p->work, (size_t)(segs * p->n) * sizeof(float2));
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(workspace)");
    return FFTSEG_OK;
}

int64_t launches_per_exec(fftseg_plan p, int64_t nseg)
{
    if (nseg <= 0) return 0;
    switch (p->path) {
        case PATH_BLOCK:
        case PATH_CLUSTER: return 1;
        case PATH_TWOPASS: return 2 * ((nseg + p->work_segs - 1) / p->work_segs);
        case PATH_FOURSTEP: return p->ilv_log_r ? 2 * ((nseg + p->work_segs - 1) / p->work_segs) : 1;
        case PATH_MIXED: return 1;
        case PATH_BLUESTEIN: {
            if (blue_fused(p)) return 1;
            int64_t k = 0;
            for (int64_t s0 = 0; s0 < nseg; s0 += p->rchunk) {
                const int64_t c = nseg - s0 < p->rchunk ? nseg - s0 : p->rchunk;
                k += blue_inv_fused(p) ? (p->inner->path == PATH_CLUSTER ? 2 : 2 + launches_per_exec(p->inner, c))
                                       : 3 + launches_per_exec(p->inner, c) + launches_per_exec(p->inner2, c);
            }
            return k;
        }
        case PATH_REAL:
        case PATH_FRAMES: {
            if (real_fused(p)) return 1;
            if (frames_fused(p) || p->frames_wl) return 1;
            int64_t k = 0;
            for (int64_t s0 = 0; s0 < nseg; s0 += p->rchunk)
                k += 1 + launches_per_exec(p->inner, nseg - s0 < p->rchunk ? nseg - s0 : p->rchunk);
            return k;
        }
        default: return 0;
    }
}

}  // namespace

int encode_tmap_3d(CUtensorMap *m, const void *base, int64_t d0, int64_t d1, int64_t d2, int64_t stride1_bytes,
                   int64_t stride2_bytes, uint32_t box0, uint32_t box1, int elem_bytes, bool swizzle128)
{
    return encode_tmap_3d_swz(m, base, d0, d1, d2, stride1_bytes, stride2_bytes, box0, box1, elem_bytes,
                              swizzle128 ? 128 : 0);
}

int encode_tmap_3d_swz(CUtensorMap *m, const void *base, int64_t d0, int64_t d1, int64_t d2, int64_t stride1_bytes,
                       int64_t stride2_bytes, uint32_t box0, uint32_t box1, int elem_bytes, int swizzle_bytes)
{
    const int64_t dims[3] = {d0, d1, d2};
    const int64_t strides[2] = {stride1_bytes, stride2_bytes};
    const uint32_t box[3] = {box0, box1, 1};
    return encode_tmap(m, base, 3, dims, strides, box, elem_bytes, swizzle_bytes);
}

int encode_tmap(CUtensorMap *m, const void *base, int rank, const int64_t *dims_in, const int64_t *strides_in,
                const uint32_t *box_in, int elem_bytes, int swizzle_bytes)
{
    if (rank < 1 || rank > 5) return set_error(FFTSEG_E_INVALID, "tensor map rank %d", rank);
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5];
    for (int i = 0; i < rank; ++i) {
        dims[i] = (cuuint64_t)dims_in[i];
        box[i] = (cuuint32_t)box_in[i];
        estr[i] = 1;
        if (i + 1 < rank) strides[i] = (cuuint64_t)strides_in[i];
    }
    const CUtensorMapSwizzle swz = swizzle_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                   : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                   : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                         : CU_TENSOR_MAP_SWIZZLE_NONE;
    // the driver entry point is looked up through the runtime, so the library
    // does not link libcuda and loads on machines without a GPU driver
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return set_error(FFTSEG_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    CUresult r = encode(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT64,
                        (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FFTSEG_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FFTSEG_OK;
}

// The lane-line four-step kernel over nseg segments, or (fr) over the nseg
// frames of a frame plan whose hop is a multiple of N2 (the frames' column
// tiles come straight from the signal, windowed as they are read).
struct WlFrames {
    int64_t hop;
    const float2 *win_row, *win_col;  // null: rectangular window
};

int exec_fourstep_wl(fftseg_plan p, const void *in, void *d_out, int64_t nseg, cudaStream_t st, const WlFrames *fr)
{
    const int64_t n = p->n;
    const int cs = (int)(nseg < p->ring_cs ? nseg : p->ring_cs);
    FourStepWlArgs a{};
    const int64_t n1 = int64_t(1) << p->log_n1, n2 = int64_t(1) << p->log_n2;
    const int64_t wa = int64_t(1) << p->log_wa, wb = int64_t(1) << p->log_wb;
    const int64_t pwa = wa < 16 ? wa : 16, pwb = wb < 16 ? wb : 16;
    const int64_t slabs = (int64_t)p->ring_nr * cs;
    int rc;
    if (fr) {
        // the signal as rows of N2 samples: frame s starts at row s * hop / N2
        const int64_t rows = ((nseg - 1) * fr->hop + n) / n2;
        if (rows >= (int64_t(1) << 31)) return set_error(FFTSEG_E_INVALID, "exec: signal too long for one launch");
        const int64_t dims[2] = {n2, rows};
        const int64_t strides[1] = {n2 * 8};
        const uint32_t box[2] = {(uint32_t)pwa, 256};
        rc = encode_tmap(&a.tmA, in, 2, dims, strides, box, 8, (int)(pwa * 8));
        a.frame_rows = (int)(fr->hop / n2);
        a.win_row = fr->win_row;
        a.win_col = fr->win_col;
    } else {
        rc = encode_tmap_3d_swz(&a.tmA, in, n2, n1, nseg, n2 * 8, n * 8, (uint32_t)pwa, 256, 8, (int)(pwa * 8));
    }
    if (rc == FFTSEG_OK) {
        // ring blocks [slab][k1 / wb][j2][k1 mod wb]
        const int64_t dims[4] = {wb, n2, n1 / wb, slabs};
        const int64_t strides[3] = {wb * 8, n2 * wb * 8, n * 8};
        const uint32_t box[4] = {(uint32_t)pwb, 256, 1, 1};
        rc = encode_tmap(&a.tmB, p->ring, 4, dims, strides, box, 8, (int)(pwb * 8));
    }
    if (rc == FFTSEG_OK) {
        if (p->out_kind == FFTSEG_OUT_POWER)  // |X|^2: float rows of the row tile's wb lines
            rc = encode_tmap_3d_swz(&a.tmO, d_out, n1, n2, nseg, n1 * 4, n * 4, (uint32_t)wb, 256, 4, (int)(wb * 4));
        else
            rc = encode_tmap_3d_swz(&a.tmO, d_out, n1, n2, nseg, n1 * 8, n * 8, (uint32_t)pwb, 256, 8, (int)(pwb * 8));
    }
    if (rc != FFTSEG_OK) return rc;
    a.out_power = p->out_kind == FFTSEG_OUT_POWER;
    const int64_t nc = (nseg + cs - 1) / cs;
    if (nc * cs * ((n2 / wa) + (n1 / wb)) >= (int64_t(1) << 31))
        return set_error(FFTSEG_E_INVALID, "exec: too many tiles for one launch of the lane-line kernel");
    a.ring = p->ring;
    a.twA = p->twA;
    a.twB = p->twB ? p->twB : p->twA;
    a.w4t = p->w4t;
    a.ctr = p->ctr;
    a.err = p->d_err;
    a.nseg = nseg;
    a.nchunks = (int)nc;
    a.cs = cs;
    a.nr = p->ring_nr;
    a.la = p->wl_la;
    a.stall = (p->flags & FFTSEG_FLAG_TEST_STALL) ? 1 : 0;
    cudaError_t e = cudaMemsetAsync(p->ctr, 0, (size_t)(1 + 2 * nc * cs) * sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "four-step counter reset");
    e = launch_fourstep_wl(p->log_n, p->direction, a, st);
    if (e != cudaSuccess) return cuda_error(e, "four-step kernel launch");
    count_launches(1);
    return FFTSEG_OK;
}

// The interleaved four-step (build_fourstep_ilv) on nseg segments, chunk by
// chunk: the outer pass into the workspace, then the lane-line kernel.
int exec_fourstep_ilv(fftseg_plan p, const void *d_in, void *d_out, int64_t nseg, cudaStream_t st)
{
    const int log_r = p->ilv_log_r;
    const int64_t n = p->n, R = int64_t(1) << log_r, M = n >> log_r;
    const int64_t W = int64_t(4096) >> log_r;  // columns per outer tile
    const fftseg_plan_s *q = p->inner;
    const int64_t n1 = 256, n2 = 256;
    for (int64_t s0 = 0; s0 < nseg; s0 += p->work_segs) {
        const int64_t cnt = nseg - s0 < p->work_segs ? nseg - s0 : p->work_segs;
        // Y_t[j] = w_n^{j t} DFT_R over t' of x[j + M t'], stored unit by unit
        OuterArgs O{};
        const int64_t dims[2] = {M, cnt * R};
        const int64_t strides[1] = {M * 8};
        const uint32_t box[2] = {(uint32_t)W, (uint32_t)R};
        const int trc = encode_tmap(&O.tm, static_cast<const float2 *>(d_in) + s0 * n, 2, dims, strides, box, 8, 0);
        if (trc != FFTSEG_OK) return trc;
        O.out = p->work;
        O.twL = p->twA;
        O.tw4a = p->tw4a;
        O.tw4b = p->tw4b;
        O.err = p->d_err;
        O.ntiles = cnt * (M / W);
        cudaError_t e = launch_outer(log_r, p->direction, O, st);
        if (e != cudaSuccess) return cuda_error(e, "interleaved four-step: outer pass launch");
        count_launches(1);
        // units of 32 transforms: unit u = s G + b, transforms 32 b .. 32 b + 31 of segment s
        const int64_t units = cnt * (R / 32);
        const int cs = (int)(units < q->ring_cs ? units : q->ring_cs);
        const int64_t slabs = (int64_t)q->ring_nr * cs, ns = 32 * M;
        FourStepWlArgs a{};
        // the workspace as [u N2 + j2][j1][transform c]
        int rc = encode_tmap_3d_swz(&a.tmA, p->work, 32, n1, units * n2, 32 * 8, n1 * 32 * 8, 16, 256, 8, 128);
        if (rc == FFTSEG_OK) {
            // ring blocks [slab][k1][j2][transform]
            const int64_t dims[4] = {32, n2, n1, slabs};
            const int64_t strides[3] = {32 * 8, n2 * 32 * 8, ns * 8};
            const uint32_t box[4] = {16, 256, 1, 1};
            rc = encode_tmap(&a.tmB, q->ring, 4, dims, strides, box, 8, 128);
        }
        const bool power = p->out_kind == FFTSEG_OUT_POWER;
        if (rc == FFTSEG_OK) {  // X[t + R (k1 + N1 k2)] as [segment][k2][R k1 + t]
            if (power)
                rc = encode_tmap_3d_swz(&a.tmO, static_cast<float *>(d_out) + s0 * n, n1 * R, n2, cnt, n1 * R * 4,
                                        n * 4, 32, 256, 4, 128);
            else
                rc = encode_tmap_3d_swz(&a.tmO, static_cast<float2 *>(d_out) + s0 * n, n1 * R, n2, cnt, n1 * R * 8,
                                        n * 8, 16, 256, 8, 128);
        }
        if (rc != FFTSEG_OK) return rc;
        a.out_power = power;
        const int64_t nc = (units + cs - 1) / cs;
        a.ring = q->ring;
        a.twA = q->twA;
        a.twB = q->twA;
        a.w4t = q->w4t;
        a.ctr = q->ctr;
        a.err = q->d_err;
        a.nseg = units;
        a.nchunks = (int)nc;
        a.cs = cs;
        a.nr = q->ring_nr;
        a.la = q->wl_la;
        a.ilv_r = (int)R;
        a.ilv_log_g = log_r - 5;
        e = cudaMemsetAsync(q->ctr, 0, (size_t)(1 + 2 * nc * cs) * sizeof(int), st);
        if (e != cudaSuccess) return cuda_error(e, "four-step counter reset");
        e = launch_fourstep_wl_ilv(p->direction, a, st);
        if (e != cudaSuccess) return cuda_error(e, "interleaved four-step: lane-line launch");
        count_launches(1);
    }
    return FFTSEG_OK;
}

int exec_plan(fftseg_plan p, const void *d_in, void *d_out, int64_t nseg, cudaStream_t st)
{
    if (p->path == PATH_MIXED) {
        MixedArgs a{};
        const int spt = mixed_segments_per_tile(p->n);
        a.in = static_cast<const float2 *>(d_in);
        a.out = d_out;
        a.tw = p->twA;
        a.err = p->d_err;
        a.nseg = nseg;
        a.ntiles = (nseg + spt - 1) / spt;
        a.n = (int)p->n;
        a.segs_per_tile = spt;
        a.nstages = p->mix_nstages;
        a.out_power = p->out_kind == FFTSEG_OUT_POWER;
        a.scale = p->scale;
        int64_t ns = 1;
        for (int t = 0; t < p->mix_nstages; ++t) {
            a.radix[t] = p->mix_radix[t];
            a.ns[t] = (int)ns;
            a.twoff[t] = p->mix_twoff[t];
            a.rm[t] = (float)(1.0 / (double)(p->n / p->mix_radix[t]));
            a.rns[t] = (float)(1.0 / (double)ns);
            ns *= p->mix_radix[t];
        }
        cudaError_t e = launch_mixed(p->direction, a, st);
        if (e != cudaSuccess) return cuda_error(e, "mixed-radix kernel launch");
        count_launches(1);
        return FFTSEG_OK;
    }
    if (p->path == PATH_BLUESTEIN && blue_fused(p)) {
        // M <= 4096: every row on chip from chirp-in to chirp-out, one launch
        BlueBlockArgs a{};
        const int64_t W = block_segments_per_cta(p->log_n);
        a.x = static_cast<const float2 *>(d_in);
        a.out = d_out;
        a.w = p->bw;
        a.bhat = p->bhat;
        a.twL = p->inner->twA;
        a.err = p->d_err;
        a.n = p->n;
        a.nseg = nseg;
        a.ntiles = (nseg + W - 1) / W;
        a.out_power = p->out_kind == FFTSEG_OUT_POWER;
        a.scale = p->scale;
        cudaError_t e = launch_blue_block(p->log_n, a, st);
        if (e != cudaSuccess) return cuda_error(e, "Bluestein block kernel launch");
        count_launches(1);
        return FFTSEG_OK;
    }
    if (p->path == PATH_BLUESTEIN) {
        // chunks of rchunk segments: chirp in, M-point forward transform,
        // product with B, M-point inverse transform, chirp out
        const bool power = p->out_kind == FFTSEG_OUT_POWER;
        for (int64_t s0 = 0; s0 < nseg; s0 += p->rchunk) {
            const int64_t cnt = nseg - s0 < p->rchunk ? nseg - s0 : p->rchunk;
            BlueArgs a{};
            a.x = static_cast<const float2 *>(d_in) + s0 * p->n;
            a.work = p->rwork;
            a.out = static_cast<char *>(d_out) + s0 * p->n * (power ? 4 : 8);
            a.w = p->bw;
            a.bhat = p->bhat;
            a.n = p->n;
            a.m = p->bm;
            a.scale = p->scale;
            cudaError_t e;
            int rc;
            if (blue_inv_fused(p) && p->inner->path == PATH_CLUSTER) {
                // the chirp-in folded into the forward transform's loads
                const fftseg_plan_s *q = p->inner;
                ClusterArgs c{};
                c.in = a.x;
                c.out = p->rwork;
                c.nseg = cnt;
                c.err = p->d_err;
                c.twA = q->twA;
                c.twB = q->twB;
                c.tw4 = q->tw4a;
                c.scale = q->scale;
                c.bl_w = p->bw;
                c.bl_n = p->n;
                e = launch_cluster_blue_fwd(q->log_n, q->log_c, c, st);
                if (e != cudaSuccess) return cuda_error(e, "Bluestein forward cluster launch");
                count_launches(1);
            } else {
                e = launch_blue(0, power, a, cnt, st);
                if (e != cudaSuccess) return cuda_error(e, "chirp-in launch");
                count_launches(1);
                rc = exec_plan(p->inner, p->rwork, p->rwork, cnt, st);
                if (rc != FFTSEG_OK) return rc;
            }
            if (blue_inv_fused(p)) {
                // the product with B, the inverse transform and the chirp-out in one launch
                const fftseg_plan_s *q = p->inner2;
                const int64_t N1 = int64_t(1) << q->log_n1, N2 = int64_t(1) << q->log_n2, M = p->bm;
                ClusterArgs c{};
                rc = encode_tmap_3d(&c.tmap, p->rwork, N2, N1, cnt, N2 * 8, M * 8, (uint32_t)(N2 >> q->log_c),
                                    (uint32_t)N1);
                if (rc != FFTSEG_OK) return rc;
                c.in = p->rwork;
                c.out = a.out;
                c.nseg = cnt;
                c.err = p->d_err;
                c.twA = q->twA;
                c.twB = q->twB;
                c.tw4 = q->tw4a;
                c.out_power = power;
                c.scale = p->scale;
                c.bl_bhat = p->bhat;
                c.bl_w = p->bw;
                c.bl_n = p->n;
                e = launch_cluster_blue_inv(q->log_n, q->log_c, c, st);
                if (e != cudaSuccess) return cuda_error(e, "Bluestein inverse cluster launch");
                count_launches(1);
                continue;
            }
            e = launch_blue(1, power, a, cnt, st);
            if (e != cudaSuccess) return cuda_error(e, "chirp product launch");
            rc = exec_plan(p->inner2, p->rwork, p->rwork, cnt, st);
            if (rc != FFTSEG_OK) return rc;
            e = launch_blue(2, power, a, cnt, st);
            if (e != cudaSuccess) return cuda_error(e, "chirp-out launch");
            count_launches(2);
        }
        return FFTSEG_OK;
    }
    if (p->path == PATH_FRAMES && frames_fused(p)) {
        // n <= 4096: windowed frames straight to their bins, one launch
        FramesBlockArgs a{};
        const int64_t W = block_segments_per_cta(p->log_n);
        a.signal = static_cast<const float2 *>(d_in);
        a.out = d_out;
        a.window = p->fwin;
        a.twL = p->inner->twA;
        a.err = p->d_err;
        a.hop = p->hop;
        a.nframes = nseg;
        a.ntiles = (nseg + W - 1) / W;
        a.out_power = p->out_kind == FFTSEG_OUT_POWER;
        a.scale = p->inner->scale;
        cudaError_t e = launch_block_frames(p->log_n, a, st);
        if (e != cudaSuccess) return cuda_error(e, "frames block kernel launch");
        count_launches(1);
        return FFTSEG_OK;
    }
    if (p->path == PATH_FRAMES && p->frames_wl) {
        // one launch: the frames' column tiles straight from the signal
        const WlFrames fr{p->hop, p->win_row, p->win_col};
        return exec_fourstep_wl(p->inner, d_in, d_out, nseg, st, &fr);
    }
    if (p->path == PATH_FRAMES) {
        // chunks of rchunk frames: windowed frames into an L2-sized
        // intermediate, then the batched complex plan of n points
        const bool power = p->out_kind == FFTSEG_OUT_POWER;
        for (int64_t f0 = 0; f0 < nseg; f0 += p->rchunk) {
            const int64_t cnt = nseg - f0 < p->rchunk ? nseg - f0 : p->rchunk;
            FramesArgs a{};
            a.signal = static_cast<const float2 *>(d_in) + f0 * p->hop;
            a.frames = p->rwork;
            a.window = p->fwin;
            a.hop = p->hop;
            a.n = (int)p->n;
            cudaError_t e = launch_frames(a, cnt, st);
            if (e != cudaSuccess) return cuda_error(e, "frames launch");
            count_launches(1);
            const int rc = exec_plan(p->inner, p->rwork, static_cast<char *>(d_out) + f0 * p->n * (power ? 4 : 8),
                                     cnt, st);
            if (rc != FFTSEG_OK) return rc;
        }
        return FFTSEG_OK;
    }
    if (p->path == PATH_REAL) {
        const int64_t M = p->n / 2;
        const bool power = p->out_kind == FFTSEG_OUT_POWER;
        if (p->direction == FFTSEG_FORWARD && p->inner->path == PATH_BLOCK) {
            // n/2 <= 4096: one pass, the split fused into the block kernel's tiles
            RealBlockArgs a{};
            const int64_t W = block_segments_per_cta(p->inner->log_n);
            a.in = static_cast<const float2 *>(d_in);
            a.out = d_out;
            a.twL = p->inner->twA;
            a.tw = p->rtw;
            a.err = p->d_err;
            a.nseg = nseg;
            a.ntiles = (nseg + W - 1) / W;
            a.out_power = power;
            a.scale = p->scale;
            cudaError_t e = launch_block_r2c(p->inner->log_n, a, st);
            if (e != cudaSuccess) return cuda_error(e, "real-signal block kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        if (real_fused(p) && p->direction == FFTSEG_INVERSE) {
            // n/2 = 2^13..2^17 on the cluster kernel: the join in its column pass's loads
            const fftseg_plan_s *q = p->inner;
            ClusterArgs a{};
            a.in = static_cast<const float2 *>(d_in);
            a.out = d_out;
            a.nseg = nseg;
            a.err = p->d_err;
            a.twA = q->twA;
            a.twB = q->twB;
            a.tw4 = q->tw4a;
            a.rtw = p->rtw;
            a.scale = p->scale;
            cudaError_t e = launch_cluster_c2r(q->log_n, q->log_c, a, st);
            if (e != cudaSuccess) return cuda_error(e, "real-signal cluster kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        if (real_fused(p)) {
            // n/2 = 2^13..2^17 on the cluster kernel: the split in its epilogue
            const fftseg_plan_s *q = p->inner;
            ClusterArgs a{};
            const int64_t N1 = int64_t(1) << q->log_n1, N2 = int64_t(1) << q->log_n2;
            const uint32_t WA = (uint32_t)(N2 >> q->log_c);
            int rc = encode_tmap_3d(&a.tmap, d_in, N2, N1, nseg, N2 * 8, M * 8, WA, (uint32_t)N1);
            if (rc != FFTSEG_OK) return rc;
            a.in = static_cast<const float2 *>(d_in);
            a.out = d_out;
            a.nseg = nseg;
            a.err = p->d_err;
            a.twA = q->twA;
            a.twB = q->twB;
            a.tw4 = q->tw4a;
            a.rtw = p->rtw;
            a.out_power = power;
            a.scale = p->scale;
            cudaError_t e = launch_cluster_r2c(q->log_n, q->log_c, a, st);
            if (e != cudaSuccess) return cuda_error(e, "real-signal cluster kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        // otherwise chunks of rchunk segments: the complex FFT of n/2 points and
        // the split (forward) or join (inverse) pass, through an L2-sized intermediate
        for (int64_t s0 = 0; s0 < nseg; s0 += p->rchunk) {
            const int64_t cnt = nseg - s0 < p->rchunk ? nseg - s0 : p->rchunk;
            RealArgs a{};
            a.m = (int)M;
            a.tw = p->rtw;
            a.scale = p->scale;
            int rc;
            if (p->direction == FFTSEG_FORWARD) {
                rc = exec_plan(p->inner, static_cast<const float2 *>(d_in) + s0 * M, p->rwork, cnt, st);
                if (rc != FFTSEG_OK) return rc;
                a.zin = p->rwork;
                a.out = static_cast<char *>(d_out) + s0 * (M + 1) * (power ? 4 : 8);
                cudaError_t e = launch_real(true, power, a, cnt, st);
                if (e != cudaSuccess) return cuda_error(e, "real-signal split launch");
                count_launches(1);
            } else {
                a.xin = static_cast<const float2 *>(d_in) + s0 * (M + 1);
                a.out = p->rwork;
                cudaError_t e = launch_real(false, false, a, cnt, st);
                if (e != cudaSuccess) return cuda_error(e, "real-signal join launch");
                count_launches(1);
                rc = exec_plan(p->inner, p->rwork, static_cast<float2 *>(d_out) + s0 * M, cnt, st);
                if (rc != FFTSEG_OK) return rc;
            }
        }
        return FFTSEG_OK;
    }
    if (nseg == 0) return FFTSEG_OK;
    const float2 *in = static_cast<const float2 *>(d_in);
    const int sign = p->direction;
    const int power = p->out_kind == FFTSEG_OUT_POWER;
    const int64_t n = p->n;
    cudaError_t e = cudaSuccess;
    switch (p->path) {
        case PATH_BLOCK: {
            BlockArgs a{};
            const int64_t W = block_segments_per_cta(p->log_n);
            a.in = in;
            a.out = d_out;
            a.nseg = nseg;
            a.ntiles = (nseg + W - 1) / W;
            a.twL = p->twA;
            a.err = p->d_err;
            a.out_power = power;
            a.scale = p->scale;
            e = launch_block(p->log_n, sign, kernel_prec(p), a, st);
            if (e != cudaSuccess) return cuda_error(e, "block kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        case PATH_CLUSTER: {
            ClusterArgs a{};
            const int64_t N1 = int64_t(1) << p->log_n1, N2 = int64_t(1) << p->log_n2;
            const uint32_t WA = (uint32_t)(N2 >> p->log_c);
            int rc = encode_tmap_3d(&a.tmap, in, N2, N1, nseg, N2 * 8, n * 8, WA, (uint32_t)N1);
            if (rc != FFTSEG_OK) return rc;
            a.in = in;
            a.out = d_out;
            a.nseg = nseg;
            a.err = p->d_err;
            a.twA = p->twA;
            a.twB = p->twB;
            a.tw4 = p->tw4a;
            a.out_power = power;
            a.scale = p->scale;
            e = launch_cluster(p->log_n, p->log_c, sign, a, st);
            if (e != cudaSuccess) return cuda_error(e, "cluster kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        case PATH_TWOPASS: {
            const int l1 = p->log_n1, l2 = p->log_n2;
            const int64_t n1 = int64_t(1) << l1, n2 = int64_t(1) << l2;
            const int64_t WA = int64_t(1) << pass_log_w(l1), WB = int64_t(1) << pass_log_w(l2);
            for (int64_t s0 = 0; s0 < nseg; s0 += p->work_segs) {
                const int64_t cnt = nseg - s0 < p->work_segs ? nseg - s0 : p->work_segs;
                LinesArgs A{};  // columns: x[j1*n2 + j2] -> Y[k1*n2 + j2] * w_n^{k1 j2}
                A.in = in + s0 * n;
                A.out = p->work;
                A.tiles_per_seg = n2 / WA;
                A.nseg = cnt;
                A.in_seg = A.out_seg = n;
                A.in_tile = A.out_tile = WA;
                A.in_cs = A.out_cs = 1;
                A.in_is = A.out_is = n2;
                A.twL = p->twA;
                A.tw4a = p->tw4a;
                A.tw4b = p->tw4b;
                A.tw_ncols = n2;
                A.tw_log_k = p->tw_log_k;
                A.scale = 1.f;
                e = launch_pass(l1, sign, A, cnt * (n2 / WA), st);
                if (e != cudaSuccess) return cuda_error(e, "column pass launch");
                LinesArgs B{};  // rows: Y[k1*n2 + j2] -> X[k1 + n1*k2]
                B.in = p->work;
                B.out = power ? (void *)(static_cast<float *>(d_out) + s0 * n)
                              : (void *)(static_cast<float2 *>(d_out) + s0 * n);
                B.tiles_per_seg = n1 / WB;
                B.nseg = cnt;
                B.in_seg = B.out_seg = n;
                B.in_tile = WB * n2;
                B.out_tile = WB;
                B.in_cs = n2;
                B.in_is = 1;
                B.out_cs = 1;
                B.out_is = n1;
                B.twL = p->twB;
                B.in_staged = 1;
                B.out_power = power;
                B.scale = p->scale;
                e = launch_pass(l2, sign, B, cnt * (n1 / WB), st);
                if (e != cudaSuccess) return cuda_error(e, "row pass launch");
                count_launches(2);
            }
            return FFTSEG_OK;
        }
        case PATH_FOURSTEP: {
            if (p->ilv_log_r) return exec_fourstep_ilv(p, in, d_out, nseg, st);
            // a batch smaller than a chunk runs as one chunk of its own size, so
            // that the persistent kernels do no work for absent segments
            const int cs = (int)(nseg < p->ring_cs ? nseg : p->ring_cs);
            // the producer/consumer kernel stores row tiles with TMA: a box row must
            // hold at least 16 bytes (not so for 2-point-wide power tiles at 2^24)
            const bool ws = p->precision == FFTSEG_PREC_FP32 && (p->flags & FFTSEG_FLAG_FOURSTEP_PRODUCER) &&
                            (int64_t(1) << p->log_wb) * (power ? 4 : 8) >= 16;
            if (ws) {
                FourStepWsArgs a{};
                const int64_t n1 = int64_t(1) << p->log_n1, n2 = int64_t(1) << p->log_n2;
                const uint32_t boxa = (uint32_t)(n1 < 256 ? n1 : 256), boxb = (uint32_t)(n2 < 256 ? n2 : 256);
                const int64_t slabs = (int64_t)p->ring_nr * cs;
                const int esz = power ? 4 : 8;
                int rc = encode_tmap_3d(&a.tmA, in, n2, n1, nseg, n2 * 8, n * 8, 1u << p->log_wa, boxa);
                if (rc == FFTSEG_OK)
                    rc = encode_tmap_3d(&a.tmB, p->ring, n1, n2, slabs, n1 * 8, n * 8, 1u << p->log_wb, boxb);
                if (rc == FFTSEG_OK)
                    rc = encode_tmap_3d(&a.tmY, p->ring, n1, n2, slabs, n1 * 8, n * 8, boxa, 1u << p->log_wa);
                if (rc == FFTSEG_OK)
                    rc = encode_tmap_3d(&a.tmO, d_out, n1, n2, nseg, n1 * esz, n * esz, 1u << p->log_wb, boxb, esz);
                if (rc != FFTSEG_OK) return rc;
                const int64_t nc = (nseg + cs - 1) / cs;
                a.ring = p->ring;
                a.twA = p->twA;
                a.twB = p->twB;
                a.w4 = p->w4;
                a.w4hi = p->w4hi;
                a.ctr = p->ctr;
                a.err = p->d_err;
                a.nseg = nseg;
                a.nchunks = (int)nc;
                a.cs = cs;
                a.nr = p->ring_nr;
                a.out_power = power;
                a.scale = p->scale;
                e = cudaMemsetAsync(p->ctr, 0, (size_t)(1 + 2 * nc) * sizeof(int), st);
                if (e != cudaSuccess) return cuda_error(e, "four-step counter reset");
                e = launch_fourstep_ws(p->log_n, sign, a, st);
                if (e != cudaSuccess) return cuda_error(e, "four-step kernel launch");
                count_launches(1);
                return FFTSEG_OK;
            }
            if (uses_fourstep_wl(p)) return exec_fourstep_wl(p, in, d_out, nseg, st, nullptr);
            if (uses_fourstep_hw(p)) {
                // n = 256 x 256: warp-local lines, loader and retirer warps, TMA output stores
                FourStepHwArgs a{};
                const int64_t slabs = (int64_t)p->ring_nr * cs;
                int rc = encode_tmap_3d(&a.tmA, in, 256, 256, nseg, 256 * 8, n * 8, 16, 256, 8, true);
                if (rc == FFTSEG_OK) rc = encode_tmap_3d(&a.tmB, p->ring, 256, 256, slabs, 256 * 8, n * 8, 16, 256, 8, true);
                if (rc == FFTSEG_OK) rc = encode_tmap_3d(&a.tmO, d_out, 256, 256, nseg, 256 * 8, n * 8, 16, 256, 8, true);
                if (rc != FFTSEG_OK) return rc;
                const int64_t nc = (nseg + cs - 1) / cs;
                a.ring = p->ring;
                a.twL = p->twA;
                a.w4t = p->w4t;
                a.ctr = p->ctr;
                a.err = p->d_err;
                a.nseg = nseg;
                a.nchunks = (int)nc;
                a.cs = cs;
                a.nr = p->ring_nr;
                e = cudaMemsetAsync(p->ctr, 0, (size_t)(1 + 2 * nc * cs) * sizeof(int), st);
                if (e != cudaSuccess) return cuda_error(e, "four-step counter reset");
                e = launch_fourstep_hw(sign, a, st);
                if (e != cudaSuccess) return cuda_error(e, "four-step kernel launch");
                count_launches(1);
                return FFTSEG_OK;
            }
            FourStepArgs a{};
            const int64_t n1 = int64_t(1) << p->log_n1, n2 = int64_t(1) << p->log_n2;
            const uint32_t boxa = (uint32_t)(n1 < 256 ? n1 : 256), boxb = (uint32_t)(n2 < 256 ? n2 : 256);
            int rc = encode_tmap_3d(&a.tmA, in, n2, n1, nseg, n2 * 8, n * 8, 1u << p->log_wa, boxa);
            if (rc != FFTSEG_OK) return rc;
            rc = encode_tmap_3d(&a.tmB, p->ring, n1, n2, (int64_t)p->ring_nr * cs, n1 * 8, n * 8,
                                1u << p->log_wb, boxb);
            if (rc != FFTSEG_OK) return rc;
            const int64_t nc = (nseg + cs - 1) / cs;
            a.out = d_out;
            a.ring = p->ring;
            a.twA = p->twA;
            a.twB = p->twB;
            a.w4 = p->w4;
            a.w4hi = p->w4hi;
            a.ctr = p->ctr;
            a.err = p->d_err;
            a.nseg = nseg;
            a.nchunks = (int)nc;
            a.cs = cs;
            a.nr = p->ring_nr;
            a.log_k = p->w4_log_k;
            a.out_power = power;
            a.scale = p->scale;
            e = cudaMemsetAsync(p->ctr, 0, (size_t)(1 + 2 * nc) * sizeof(int), st);
            if (e != cudaSuccess) return cuda_error(e, "four-step counter reset");
            e = launch_fourstep(p->log_n, sign, kernel_prec(p), a, st);
            if (e != cudaSuccess) return cuda_error(e, "four-step kernel launch");
            count_launches(1);
            return FFTSEG_OK;
        }
        default: return set_error(FFTSEG_E_INVALID, "corrupt plan");
    }
}

// Real-signal plan: a complex plan of n/2 points (its schedule flags, and an
// autotune request, go to it), the split/join twiddles w_n^k (k <= n/4) and,
// unless the split is fused, an intermediate of kRealSplitChunkBytes between
// the two passes.  (Measured on GB300, 4 GiB of samples at n = 2^16..2^20:
// 512 MiB chunks, 16 launches, 0.33-0.35 of the copy peak; 32 MiB chunks,
// which stay in L2, 256 launches, 0.21-0.25.)  FFTSEG_REAL_CHUNK_MB, read at
// plan creation, sets another size.

int create_real(fftseg_plan *out, int64_t n, int64_t batch, int direction, int norm, int precision, int out_kind,
                unsigned flags)
{
    if (n < 4) return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: real-signal plans need n >= 4");
    if (precision != FFTSEG_PREC_FP32)
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: real-signal plans are FP32 only");
    if (direction == FFTSEG_INVERSE && out_kind == FFTSEG_OUT_POWER)
        return set_error(FFTSEG_E_INVALID, "plan_create: the power output belongs to forward real-signal plans");
    fftseg_plan p = new (std::nothrow) fftseg_plan_s();
    if (!p) return set_error(FFTSEG_E_NOMEM, "plan_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    p->n = n;
    p->batch = batch;
    p->log_n = ilog2(n);
    p->direction = direction;
    p->norm = norm;
    p->precision = precision;
    p->out_kind = out_kind;
    p->flags = flags;
    p->path = PATH_REAL;
    if (norm == FFTSEG_NORM_BACKWARD) p->scale = direction == FFTSEG_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    else if (norm == FFTSEG_NORM_ORTHO) p->scale = (float)(1.0 / sqrt((double)n));
    const int64_t M = n / 2;
    p->log_n1 = ilog2(M);
    int64_t cs = ((int64_t)env_int("FFTSEG_REAL_CHUNK_MB", 512, 1, 4096) << 20) / (M * 8);
    if (cs < 1) cs = 1;
    if (cs > batch) cs = batch;
    p->rchunk = cs;
    unsigned iflags = flags & ~FFTSEG_FLAG_REAL;
    // forward plans of 2^17 samples: the cluster kernel with the split in its
    // epilogue (one pass) measured 0.39 of the copy peak against 0.36 for the
    // chunked lane-line transform plus a split pass (at 2^18: 0.28 against 0.35)
    if (direction == FFTSEG_FORWARD && M == (1 << 16) && !(flags & (kPathFlags | FFTSEG_FLAG_AUTOTUNE)))
        iflags |= FFTSEG_FLAG_CLUSTER_LOG2(4);
    int rc = fftseg_plan_create(&p->inner, M, cs, direction, FFTSEG_NORM_NONE, FFTSEG_PREC_FP32,
                                FFTSEG_OUT_COMPLEX, iflags);
    if (rc == FFTSEG_OK) {
        std::vector<float2> h((size_t)(M / 2 + 1));
        host_roots(h.data(), M / 2 + 1, n, 1);
        rc = upload(&p->rtw, h);
    }
    if (rc == FFTSEG_OK) {
        e = real_fused(p) ? cudaSuccess : cudaMalloc((void **)&p->rwork, (size_t)(cs * M) * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(real-signal intermediate)");
    }
    if (rc != FFTSEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FFTSEG_OK;
}

// Overlapping-segment plan: a forward complex plan of n points over a chunk
// of windowed frames (its schedule flags, and an autotune request, go to it).
int create_frames(fftseg_plan *out, int64_t n, int64_t hop, int window, int64_t batch, int norm, int out_kind,
                  unsigned flags)
{
    fftseg_plan p = new (std::nothrow) fftseg_plan_s();
    if (!p) return set_error(FFTSEG_E_NOMEM, "plan_create_frames: host allocation failed");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    p->n = n;
    p->batch = batch;
    p->log_n = ilog2(n);
    p->log_n1 = p->log_n;
    p->direction = FFTSEG_FORWARD;
    p->norm = norm;
    p->precision = FFTSEG_PREC_FP32;
    p->out_kind = out_kind;
    p->flags = flags;
    p->path = PATH_FRAMES;
    p->hop = hop;
    p->window = window;
    // chunks of windowed frames, 512 MiB (FFTSEG_FRAMES_CHUNK_MB): measured on
    // GB300 at n = 2^14..2^18 with hops that leave the lane-line kernel, 0.27-0.31
    // of the copy peak against 0.17-0.23 in 32 MiB chunks (kept in L2, but 16x
    // the launches of the inner plan)
    int64_t cs = ((int64_t)env_int("FFTSEG_FRAMES_CHUNK_MB", 512, 1, 4096) << 20) / (n * 8);
    if (cs < 1) cs = 1;
    if (cs > batch) cs = batch;
    p->rchunk = cs;
    // the inner plan takes the whole batch: the fused lane-line form runs it
    // in one launch; the chunked form calls it a chunk at a time
    int rc = fftseg_plan_create(&p->inner, n, batch, FFTSEG_FORWARD, norm, FFTSEG_PREC_FP32, out_kind, flags);
    if (rc == FFTSEG_OK && uses_fourstep_wl(p->inner) && hop % (int64_t(1) << p->inner->log_n2) == 0) {
        p->frames_wl = true;
        if (window == FFTSEG_WINDOW_HANN) {
            const int64_t n1 = int64_t(1) << p->inner->log_n1, n2 = int64_t(1) << p->inner->log_n2;
            std::vector<float2> r((size_t)n1), c((size_t)n2);
            host_roots(r.data(), n1, n1, 1);  // (cos, -sin)(2 pi j1 / N1)
            host_roots(c.data(), n2, n, 1);   // (cos, -sin)(2 pi j2 / n)
            for (auto &v : r) v.y = -v.y;
            for (auto &v : c) v.y = -v.y;
            rc = upload(&p->win_row, r);
            if (rc == FFTSEG_OK) rc = upload(&p->win_col, c);
        }
    }
    if (rc == FFTSEG_OK && window == FFTSEG_WINDOW_HANN && !p->frames_wl) {
        // periodic Hann window, w[j] = (1 - cos(2 pi j / n)) / 2, evaluated in double
        std::vector<float> h((size_t)n);
        const double two_pi = 6.283185307179586476925286766559;
        for (int64_t j = 0; j < n; ++j) h[(size_t)j] = (float)(0.5 - 0.5 * cos(two_pi * (double)j / (double)n));
        e = cudaMalloc((void **)&p->fwin, (size_t)n * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(p->fwin, h.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_error(e, "window table");
    }
    if (rc == FFTSEG_OK) {
        // fused frames (n <= 4096, or on the lane-line kernel) need no intermediate
        e = (frames_fused(p) || p->frames_wl) ? cudaSuccess
                                               : cudaMalloc((void **)&p->rwork, (size_t)(cs * n) * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(frames intermediate)");
    }
    if (rc != FFTSEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FFTSEG_OK;
}

// Length n that is not a power of two: Bluestein over M = 2^ceil(log2(2n - 1))
// (see bluestein.cu).  The chirp w[m] = exp(sigma pi i m^2 / n), its phase
// reduced exactly as (m^2 mod 2n) / n, and b = conj(w) placed cyclically and
// divided by M (exact) are evaluated in double on the host; B = FFT_M(b) is
// computed once on the device with the plan's own forward M-point plan.
// Rows with M = 2^13..2^16 take two passes per chunk on the cluster kernel
// (the chirp-in read by the forward transform, the product with B and the
// chirp-out folded into the inverse one), longer rows five.  Chunks of
// 1 GiB of rows: at n = 10007 (M = 32768, 4 GiB of signal) 17.9 ms against
// 18.6 for 256 MiB and 23.0 for L2-sized 32 MiB chunks.
constexpr int kBlueChunkMB = 1024;

int create_bluestein(fftseg_plan *out, int64_t n, int64_t batch, int direction, int norm, int out_kind,
                     unsigned flags)
{
    fftseg_plan p = new (std::nothrow) fftseg_plan_s();
    if (!p) return set_error(FFTSEG_E_NOMEM, "plan_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    int64_t M = 2;
    while (M < 2 * n - 1) M *= 2;
    p->n = n;
    p->batch = batch;
    p->log_n = ilog2(M);
    p->log_n1 = p->log_n;
    p->direction = direction;
    p->norm = norm;
    p->precision = FFTSEG_PREC_FP32;
    p->out_kind = out_kind;
    p->flags = flags;
    p->path = PATH_BLUESTEIN;
    p->bm = M;
    if (norm == FFTSEG_NORM_BACKWARD) p->scale = direction == FFTSEG_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    else if (norm == FFTSEG_NORM_ORTHO) p->scale = (float)(1.0 / sqrt((double)n));
    int64_t cs = ((int64_t)env_int("FFTSEG_BLUE_CHUNK_MB", kBlueChunkMB, 1, 4096) << 20) / (M * 8);
    if (cs < 1) cs = 1;
    if (cs > 65535) cs = 65535;
    if (cs > batch) cs = batch;
    p->rchunk = cs;
    // M = 2^16: the cluster kernel's Bluestein forms (two passes over the
    // M-point rows) rather than five passes around the lane-line kernel
    // (n = 20011, 4 GiB: 22.4 against 26.4 ms; at M = 2^17, n = 40009, the
    // five passes win, 26.5 against 33.0 ms)
    unsigned iflags = flags;
    if (M == (1 << 16) && !(flags & (kPathFlags | FFTSEG_FLAG_AUTOTUNE)))
        iflags |= FFTSEG_FLAG_CLUSTER_LOG2(4);
    int rc = fftseg_plan_create(&p->inner, M, cs, FFTSEG_FORWARD, FFTSEG_NORM_NONE, FFTSEG_PREC_FP32,
                                FFTSEG_OUT_COMPLEX, iflags);
    // M <= 4096 rows run fused (k_blue_block) on the inner plan's stage
    // tables: no inverse plan and no intermediate rows
    const bool fused = rc == FFTSEG_OK && blue_fused(p);
    if (rc == FFTSEG_OK && !fused)
        rc = fftseg_plan_create(&p->inner2, M, cs, FFTSEG_INVERSE, FFTSEG_NORM_NONE, FFTSEG_PREC_FP32,
                                FFTSEG_OUT_COMPLEX, iflags);
    if (rc == FFTSEG_OK) {
        const double pi = 3.141592653589793238462643383279;
        std::vector<float2> w((size_t)n), b((size_t)M, make_float2(0.f, 0.f));
        const double inv_m = 1.0 / (double)M;
        for (int64_t m = 0; m < n; ++m) {
            const int64_t e2 = (int64_t)(((unsigned __int128)m * (unsigned __int128)m) % (unsigned __int128)(2 * n));
            const double a = pi * ((double)e2 / (double)n);
            const double c = cos(a), sn = (double)direction * sin(a);
            w[(size_t)m] = make_float2((float)c, (float)sn);
            const float2 cb = make_float2((float)(c * inv_m), (float)(-sn * inv_m));  // conj(w) / M
            b[(size_t)m] = cb;
            if (m > 0) b[(size_t)(M - m)] = cb;
        }
        rc = upload(&p->bw, w);
        float2 *bdev = nullptr;
        if (rc == FFTSEG_OK) rc = upload(&bdev, b);
        if (rc == FFTSEG_OK) {
            e = cudaMalloc((void **)&p->bhat, (size_t)M * sizeof(float2));
            if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(chirp spectrum)");
        }
        if (rc == FFTSEG_OK) rc = exec_plan(p->inner, bdev, p->bhat, 1, nullptr);
        if (rc == FFTSEG_OK) rc = fftseg_plan_check(p->inner);  // synchronises
        cudaFree(bdev);
    }
    if (rc == FFTSEG_OK) {
        e = fused ? cudaSuccess : cudaMalloc((void **)&p->rwork, (size_t)(cs * M) * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&p->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(Bluestein rows)");
    }
    if (rc != FFTSEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FFTSEG_OK;
}

}  // namespace fftseg

using namespace fftseg;

extern "C" {

// Lengths 2^a 3^b 5^c 7^d <= 4096 that are not powers of two: one pass of
// mixed-radix Stockham stages (k_mixed.cu).  The stage twiddles
// w_{Ns R}^{k r} are evaluated in double on the host and rounded once.
int create_mixed(fftseg_plan *out, int64_t n, int64_t batch, int direction, int norm, int out_kind,
                 unsigned flags, const int *radix, int nstages)
{
    fftseg_plan p = new (std::nothrow) fftseg_plan_s();
    if (!p) return set_error(FFTSEG_E_NOMEM, "plan_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    p->n = n;
    p->batch = batch;
    p->log_n = 0;
    p->direction = direction;
    p->norm = norm;
    p->precision = FFTSEG_PREC_FP32;
    p->out_kind = out_kind;
    p->flags = flags;
    p->path = PATH_MIXED;
    if (norm == FFTSEG_NORM_BACKWARD) p->scale = direction == FFTSEG_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    else if (norm == FFTSEG_NORM_ORTHO) p->scale = (float)(1.0 / sqrt((double)n));
    p->mix_nstages = nstages;
    std::vector<float2> h;
    int64_t ns = 1;
    for (int t = 0; t < nstages; ++t) {
        const int64_t R = radix[t];
        p->mix_radix[t] = (int)R;
        p->mix_twoff[t] = (int)h.size();
        if (ns > 1) {
            const size_t base = h.size();
            h.resize(base + (size_t)((R - 1) * ns));
            for (int64_t r = 1; r < R; ++r) host_roots(h.data() + base + (r - 1) * ns, ns, ns * R, r);
        }
        ns *= R;
    }
    if (h.empty()) h.push_back(make_float2(1.f, 0.f));
    int rc = upload(&p->twA, h);
    if (rc == FFTSEG_OK) {
        e = cudaMalloc((void **)&p->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMalloc(status flag)");
    }
    if (rc != FFTSEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FFTSEG_OK;
}

int fftseg_plan_create(fftseg_plan *out, int64_t n, int64_t batch, int direction, int norm,
                       int precision, int out_kind, unsigned flags)
{
    if (!out) return set_error(FFTSEG_E_INVALID, "plan_create: out is NULL");
    *out = nullptr;
    if (n < 2 || n > (int64_t(1) << FFTSEG_MAX_LOG2N) ||
        (!is_pow2(n) && n > (int64_t(1) << (FFTSEG_MAX_LOG2N - 1))))
        return set_error(FFTSEG_E_UNSUPPORTED,
                         "plan_create: n=%lld outside [2, 2^24] (powers of two) or [3, 2^23] (other lengths)",
                         (long long)n);
    if (batch < 1) return set_error(FFTSEG_E_INVALID, "plan_create: batch must be >= 1");
    if (direction != FFTSEG_FORWARD && direction != FFTSEG_INVERSE)
        return set_error(FFTSEG_E_INVALID, "plan_create: direction must be -1 or +1");
    if (norm < FFTSEG_NORM_NONE || norm > FFTSEG_NORM_ORTHO)
        return set_error(FFTSEG_E_INVALID, "plan_create: bad norm %d", norm);
    if (out_kind != FFTSEG_OUT_COMPLEX && out_kind != FFTSEG_OUT_POWER)
        return set_error(FFTSEG_E_INVALID, "plan_create: bad out_kind %d", out_kind);
    if (precision < FFTSEG_PREC_FP32 || precision > FFTSEG_PREC_TC_BF16)
        return set_error(FFTSEG_E_INVALID, "plan_create: bad precision %d", precision);
    if (batch > (int64_t(1) << 40) / n)
        return set_error(FFTSEG_E_INVALID, "plan_create: batch*n too large");
    if (flags & FFTSEG_FLAG_REAL) {
        if (!is_pow2(n)) return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: real-signal plans need a power of two");
        return create_real(out, n, batch, direction, norm, precision, out_kind, flags);
    }
    if (!is_pow2(n)) {
        if (precision != FFTSEG_PREC_FP32)
            return set_error(FFTSEG_E_UNSUPPORTED, "plan_create: lengths that are not powers of two are FP32 only");
        int radix[kMixMaxStages], nst = 0;
        if (!(flags & FFTSEG_FLAG_BLUESTEIN) && mixed_schedule(n, &nst, radix))
            return create_mixed(out, n, batch, direction, norm, out_kind, flags, radix, nst);
        return create_bluestein(out, n, batch, direction, norm, out_kind, flags);
    }
    if (flags & FFTSEG_FLAG_AUTOTUNE) {  // replace the schedule flags by the fastest measured schedule
        unsigned chosen = 0;
        const int trc = tune_schedule(n, batch, precision, out_kind, &chosen, nullptr);
        if (trc != FFTSEG_OK) return trc;
        flags = (flags & ~(kPathFlags | FFTSEG_FLAG_AUTOTUNE)) | chosen;
    }

    fftseg_plan p = new (std::nothrow) fftseg_plan_s();
    if (!p) return set_error(FFTSEG_E_NOMEM, "plan_create: host allocation failed");
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_error(e, "cudaGetDevice");
    }
    p->n = n;
    p->batch = batch;
    p->log_n = ilog2(n);
    p->direction = direction;
    p->norm = norm;
    p->precision = precision;
    p->out_kind = out_kind;
    p->flags = flags;
    if (norm == FFTSEG_NORM_BACKWARD) p->scale = direction == FFTSEG_INVERSE ? (float)(1.0 / (double)n) : 1.f;
    else if (norm == FFTSEG_NORM_ORTHO) p->scale = (float)(1.0 / sqrt((double)n));
    e = cudaMalloc((void **)&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_error(e, "cudaMalloc(status flag)");
    }
    int rc = precision == FFTSEG_PREC_FP32 ? build_fp32(p) : build_tc(p);
    if (rc != FFTSEG_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return FFTSEG_OK;
}

int fftseg_plan_create_frames(fftseg_plan *out, int64_t n, int64_t hop, int window, int64_t batch, int norm,
                              int out_kind, unsigned flags)
{
    if (!out) return set_error(FFTSEG_E_INVALID, "plan_create_frames: out is NULL");
    *out = nullptr;
    if (!is_pow2(n) || n < 2 || n > (int64_t(1) << FFTSEG_MAX_LOG2N))
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create_frames: n=%lld is not a power of two in [2, 2^24]",
                         (long long)n);
    if (hop < 1) return set_error(FFTSEG_E_INVALID, "plan_create_frames: hop must be >= 1");
    if (window != FFTSEG_WINDOW_RECT && window != FFTSEG_WINDOW_HANN)
        return set_error(FFTSEG_E_INVALID, "plan_create_frames: bad window %d", window);
    if (batch < 1) return set_error(FFTSEG_E_INVALID, "plan_create_frames: batch must be >= 1");
    if (norm < FFTSEG_NORM_NONE || norm > FFTSEG_NORM_ORTHO)
        return set_error(FFTSEG_E_INVALID, "plan_create_frames: bad norm %d", norm);
    if (out_kind != FFTSEG_OUT_COMPLEX && out_kind != FFTSEG_OUT_POWER)
        return set_error(FFTSEG_E_INVALID, "plan_create_frames: bad out_kind %d", out_kind);
    if (flags & FFTSEG_FLAG_REAL)
        return set_error(FFTSEG_E_UNSUPPORTED, "plan_create_frames: frames of a real signal are not built");
    if (batch > (int64_t(1) << 40) / n || hop > (int64_t(1) << 40) / batch)
        return set_error(FFTSEG_E_INVALID, "plan_create_frames: batch*n or batch*hop too large");
    return create_frames(out, n, hop, window, batch, norm, out_kind, flags);
}

int fftseg_plan_destroy(fftseg_plan p)
{
    if (!p) return set_error(FFTSEG_E_INVALID, "plan_destroy: NULL plan");
    free_plan(p);
    return FFTSEG_OK;
}

int fftseg_exec_n(fftseg_plan p, const void *d_in, void *d_out, int64_t nseg, fftseg_stream_t stream)
{
    if (!p) return set_error(FFTSEG_E_INVALID, "exec: NULL plan");
    if (nseg < 0 || nseg > p->batch)
        return set_error(FFTSEG_E_INVALID, "exec: nseg=%lld outside [0, batch=%lld]", (long long)nseg,
                         (long long)p->batch);
    if (nseg == 0) return FFTSEG_OK;
    if (!d_in || !d_out) return set_error(FFTSEG_E_INVALID, "exec: NULL buffer");
    if (((uintptr_t)d_in & 15) || ((uintptr_t)d_out & 15))
        return set_error(FFTSEG_E_INVALID, "exec: buffers must be 16-byte aligned");
    if (d_in == d_out && p->out_kind == FFTSEG_OUT_POWER)
        return set_error(FFTSEG_E_INVALID, "exec: the power output cannot be written in place");
    if (d_in == d_out && (p->path == PATH_REAL || p->path == PATH_FRAMES || p->path == PATH_BLUESTEIN))
        return set_error(FFTSEG_E_INVALID, "exec: real-signal and frame plans work out of place only");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != p->device)
        return set_error(FFTSEG_E_INVALID, "exec: plan belongs to device %d, current device is %d",
                         p->device, dev);
    return exec_plan(p, d_in, d_out, nseg, reinterpret_cast<cudaStream_t>(stream));
}

int fftseg_exec(fftseg_plan p, const void *d_in, void *d_out, fftseg_stream_t stream)
{
    if (!p) return set_error(FFTSEG_E_INVALID, "exec: NULL plan");
    return fftseg_exec_n(p, d_in, d_out, p->batch, stream);
}

int fftseg_plan_info(fftseg_plan p, int64_t info[6])
{
    if (!p || !info) return set_error(FFTSEG_E_INVALID, "plan_info: NULL argument");
    info[0] = p->path;
    info[1] = p->path == PATH_MIXED ? p->n : int64_t(1) << p->log_n1;
    info[2] = (p->path == PATH_BLOCK || p->path == PATH_REAL || p->path == PATH_FRAMES ||
               p->path == PATH_BLUESTEIN || p->path == PATH_MIXED)
                  ? 1
                  : int64_t(1) << p->log_n2;
    info[3] = p->path == PATH_BLUESTEIN ? (p->rwork ? p->rchunk * p->bm * 8 : 0)
              : p->path == PATH_FRAMES ? (p->rwork ? p->rchunk * p->n * 8 : 0)
              : p->path == PATH_REAL ? (p->rwork ? p->rchunk * (p->n / 2) * 8 : 0)
                                    : p->work ? p->work_segs * p->n * 8
                                              : (p->ring ? (int64_t)p->ring_nr * p->ring_cs * p->n * 8 : 0);
    info[4] = (p->path == PATH_REAL || p->path == PATH_FRAMES || p->path == PATH_BLUESTEIN) ? p->rchunk
              : p->path == PATH_MIXED ? mixed_segments_per_tile(p->n)
              : p->work ? p->work_segs : p->ring_cs;
    info[5] = launches_per_exec(p, p->batch);
    return FFTSEG_OK;
}

int fftseg_plan_check(fftseg_plan p)
{
    if (!p) return set_error(FFTSEG_E_INVALID, "plan_check: NULL plan");
    if (p->inner) {
        const int rc = fftseg_plan_check(p->inner);
        if (rc != FFTSEG_OK) return rc;
    }
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "plan_check");
    if (flag) {
        cudaMemset(p->d_err, 0, sizeof(int));
        if (flag & 8)  // only the self-checking build sets it
            return set_error(FFTSEG_E_INVALID, "a kernel found an index out of its buffer (flag %d) and skipped it", flag);
        return set_error(FFTSEG_E_TIMEOUT, "a kernel gave up (flag %d): a bounded wait ran out or a shared buffer was misaligned", flag);
    }
    return FFTSEG_OK;
}

const char *fftseg_last_error(void) { return g_msg; }

int64_t fftseg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
