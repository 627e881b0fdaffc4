// Lengths n = 2^a 3^b 5^c 7^d <= 4096 that are not powers of two, in one
// pass: mixed-radix Stockham stages of radix 2, 3, 4, 5, 7 or 8.
//
// The Cooley-Tukey factorisation (Sec. I of the paper) holds for any
// factorisation n = R_1 R_2 ... R_s; the FFT libraries the paper names handle
// such lengths natively.  Stage t (radix R, Ns = R_1 ... R_{t-1} points
// already combined) runs the n/R butterflies j of every segment:
//   a_r = line[j + r n/R], times w_{Ns R}^{(j mod Ns) r} (r >= 1),
//   A = DFT_R(a),  line'[(j / Ns) Ns R + (j mod Ns) + r Ns] = A_r,
// the self-sorting Stockham form, so the bins come out in natural order.
// The odd radices come first: their Ns = 1 stage stores with an odd stride,
// which no two lanes of a half-warp share a bank pair with.
//
// Each CTA (persistent, two per SM) takes tiles of floor(4096 / n) whole
// segments: the next tile is copied in with 8-byte cp.async copies by every
// thread while the current one runs its stages, ping-ponging between two
// shared buffers with one barrier per stage.  Stage twiddles are read
// through the read-only cache.
#include "engine.cuh"
#include "launch.h"
#include "programmatic.h"

namespace fftseg {

namespace {

constexpr int kMixE = 4096;  // points per tile buffer
constexpr int kMixT = 256;   // threads per CTA

// x / d for 0 <= x < 2^20 and a runtime divisor d with rd ~ 1/d: the float
// quotient is within one of the true one, then one correction step.
FDEV int divq(int x, int d, float rd)
{
    int q = __float2int_rz((float)x * rd);
    const int r = x - q * d;
    if (r < 0) --q;
    else if (r >= d) ++q;
    return q;
}

template <int R, int S>
FDEV void mix_stage(const float2 *src, float2 *dst, int cnt, int n, int ns, float rm, float rns,
                    const float2 *__restrict__ tw, [[maybe_unused]] int *err)
{
    const int m = n / R;
    const int nb = cnt * m;
    // butterfly g = seg m + j, stepped by kMixT without a division per step
    int seg = divq(threadIdx.x, m, rm);
    int j = threadIdx.x - seg * m;
    const int dseg = divq(kMixT, m, rm), dj = kMixT - dseg * m;
    for (int g = threadIdx.x; g < nb; g += kMixT) {
        const int base = seg * n;
        float2 x[R];
        // (self-checking build: the butterfly's points lie in the tile)
        const bool ok = FFTSEG_CHECK(seg < cnt && j < m && base + n <= cnt * n, err);
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = ok ? src[base + j + r * m] : make_float2(0.f, 0.f);
        int jq = j, k = 0;
        if (ns > 1) {
            jq = divq(j, ns, rns);
            k = j - jq * ns;
#pragma unroll
            for (int r = 1; r < R; ++r) x[r] = twmul<S>(x[r], __ldg(tw + (r - 1) * ns + k));
        }
        dft<R, S>(x);
        const int o = base + jq * ns * R + k;
        if (FFTSEG_CHECK(o + (R - 1) * ns < base + n && k < ns, err)) {
#pragma unroll
            for (int r = 0; r < R; ++r) dst[o + r * ns] = x[r];
        }
        seg += dseg;
        j += dj;
        if (j >= m) {
            j -= m;
            ++seg;
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kMixT, 2) k_mixed(const __grid_constant__ MixedArgs a)
{
    extern __shared__ __align__(16) float2 smx[];
    float2 *const buf0 = smx, *const buf1 = smx + kMixE, *const buf2 = smx + 2 * kMixE;
    const int n = a.n, spt = a.segs_per_tile;
    auto count_of = [&](int64_t t) -> int {
        const int64_t left = a.nseg - t * spt;
        return (int)(left < spt ? left : spt);
    };
    // A tile whose bytes start on a 16-byte boundary and are a multiple of 16
    // (an even number of points) arrives by one bulk copy issued by thread 0
    // and completed on an mbarrier; otherwise every thread issues 8-byte
    // cp.async copies.
    __shared__ __align__(8) uint64_t bar[2];
    auto bulk_ok = [&](int64_t t) -> bool {
        return ((t * spt * (int64_t)n) & 1) == 0 && ((count_of(t) * n) & 1) == 0;
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // (launched with programmatic stream serialization, as k_block: the L2
    // fetch of the first two bulk-copied tiles starts before the wait for the
    // previous kernel)
    grid_launch_dependents();
    if (threadIdx.x == 0)
        for (int64_t t = blockIdx.x, q = 0; q < 2 && t < a.ntiles; ++q, t += gridDim.x)
            if (bulk_ok(t))
                prefetch_l2_bulk(a.in + t * spt * (int64_t)n, (uint32_t)(count_of(t) * n * sizeof(float2)));
    grid_dependency_wait();
    uint32_t phase = 0;  // bit b: parity of the next completion of bar[b]
    auto load = [&](int64_t t, float2 *dst, int b) {
        const float2 *src = a.in + t * spt * (int64_t)n;
        const int count = count_of(t) * n;
        if (bulk_ok(t)) {
            if (threadIdx.x == 0) {
                fence_proxy_async();  // this buffer's earlier generic accesses before the copy
                mbar_expect_tx(&bar[b], (uint32_t)(count * sizeof(float2)));
                tma_load_1d(dst, src, (uint32_t)(count * sizeof(float2)), &bar[b]);
            }
        } else {
            for (int e = threadIdx.x; e < count; e += kMixT) cp_async8(dst + e, src + e, 8);
        }
    };
    int64_t t = blockIdx.x;
    if (t < a.ntiles) load(t, buf0, 0);
    cp_async_commit();
    int cur = 0;
    for (; t < a.ntiles; t += gridDim.x) {
        const int64_t tn = t + gridDim.x;
        if (tn < a.ntiles) load(tn, cur ? buf0 : buf1, cur ^ 1);
        cp_async_commit();
        cp_async_wait<1>();  // this tile's copies (the group before the one just issued)
        if (bulk_ok(t)) {
            mbar_wait(&bar[cur], (phase >> cur) & 1, a.err);
            phase ^= 1u << cur;
        }
        __syncthreads();
        const int cnt = count_of(t);
        float2 *src = cur ? buf1 : buf0, *dst = buf2;
        for (int st = 0; st < a.nstages; ++st) {
            const float2 *tw = a.tw + a.twoff[st];
            const int ns = a.ns[st];
            const float rm = a.rm[st], rns = a.rns[st];
            switch (a.radix[st]) {
                case 2: mix_stage<2, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
                case 3: mix_stage<3, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
                case 4: mix_stage<4, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
                case 5: mix_stage<5, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
                case 7: mix_stage<7, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
                default: mix_stage<8, S>(src, dst, cnt, n, ns, rm, rns, tw, a.err); break;
            }
            __syncthreads();
            float2 *tmp = src;
            src = dst;
            dst = tmp;
        }
        const int count = cnt * n;
        const int64_t o0 = t * spt * (int64_t)n;
        const float sc = a.scale;
        if (a.out_power) {
            float *o = static_cast<float *>(a.out) + o0;
            for (int e = threadIdx.x; e < count; e += kMixT) {
                const float2 v = src[e];
                o[e] = (v.x * sc) * (v.x * sc) + (v.y * sc) * (v.y * sc);
            }
        } else {
            float2 *o = static_cast<float2 *>(a.out) + o0;
            for (int e = threadIdx.x; e < count; e += kMixT) {
                const float2 v = src[e];
                o[e] = make_float2(v.x * sc, v.y * sc);
            }
        }
        __syncthreads();  // every read of this tile's buffers is done before they are refilled
        cur ^= 1;
    }
    cp_async_wait<0>();
}

template <int S>
cudaError_t mixed_t(const MixedArgs &a, cudaStream_t st)
{
    auto k = k_mixed<S>;
    constexpr size_t SMEM = 3 * kMixE * sizeof(float2);
    static int per_sm_dev[kMaxDevices] = {};  // per instantiation and device
    int &per_sm = per_sm_dev[current_device_slot()];
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kMixT, SMEM);
        if (e != cudaSuccess) return e;
        if (occ < 1) return cudaErrorLaunchOutOfResources;
        per_sm = occ;
    }
    if (a.ntiles == 0) return cudaSuccess;
    int64_t grid = (int64_t)per_sm * device_sm_count();
    if (grid > a.ntiles) grid = a.ntiles;
    return launch_programmatic(k, (unsigned)grid, kMixT, SMEM, st, a);
}

}  // namespace

int mixed_segments_per_tile(int64_t n) { return n <= kMixE ? (int)(kMixE / n) : 0; }

bool mixed_schedule(int64_t n, int *nstages, int *radix)
{
    if (n < 2 || n > kMixE) return false;
    int64_t m = n;
    int s = 0;
    for (int p : {7, 5, 3}) {
        while (m % p == 0) {
            if (s >= kMixMaxStages) return false;
            radix[s++] = p;
            m /= p;
        }
    }
    while (m % 8 == 0) {
        if (s >= kMixMaxStages) return false;
        radix[s++] = 8;
        m /= 8;
    }
    if (m == 4 || m == 2) {
        if (s >= kMixMaxStages) return false;
        radix[s++] = (int)m;
        m = 1;
    }
    if (m != 1) return false;
    *nstages = s;
    return true;
}

cudaError_t launch_mixed(int sign, const MixedArgs &a, cudaStream_t st)
{
    return sign < 0 ? mixed_t<-1>(a, st) : mixed_t<1>(a, st);
}

}  // namespace fftseg
