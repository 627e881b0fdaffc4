// Host-side launchers of the FP32 kernels (one translation unit per family).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace fftseg {

// Launch-shape caches (occupancy, SM count) are kept per device: index of
// the current device into such a cache (devices past the last slot share it).
constexpr int kMaxDevices = 64;
inline int current_device_slot()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    return dev < kMaxDevices ? dev : kMaxDevices - 1;
}

// Single-pass segment-major tiles for n = 2^log_n <= 4096 (persistent CTAs,
// a.ntiles tiles of block_segments_per_cta segments).  Returns the launch error.
// prec: PREC_FP32, or PREC_FP16 / PREC_BF16 (tensor-core radix-16 stages, n = 16, 256, 4096).
cudaError_t launch_block(int log_n, int sign, int prec, const BlockArgs &a, cudaStream_t st);
int device_sm_count();
// Segments per CTA of the block kernel.
int block_segments_per_cta(int log_n);

// One pass of the two-pass path over lines of length 2^log_l (16..4096),
// interleaved tiles of 2^lines_log_w(log_l) lines; `units` CTAs.
cudaError_t launch_pass(int log_l, int sign, const LinesArgs &a, int64_t units, cudaStream_t st);
// The interleaved four-step's outer pass, persistent and fed by TMA
// (k_outer.cu): n = 2^log_r * 2^16, log_r = 5..8.
struct OuterArgs {
    CUtensorMap tm;      // the input chunk as [segments * R][2^16] complex64, box [4096 / R][R]
    float2 *out;         // the workspace, unit by unit
    const float2 *twL;   // stage tables of an R-point line
    const float2 *tw4a;  // w_n^{(t mod 16) j}, [16][2^16]
    const float2 *tw4b;  // w_n^{16 (t div 16) j}, [R / 16][2^16]
    int *err;            // set when a tile's copy never completed
    int64_t ntiles;      // segments * 2^16 / (4096 / R)
};
cudaError_t launch_outer(int log_r, int sign, const OuterArgs &a, cudaStream_t st);
int pass_log_w(int log_l);

// Single-pass cluster kernel for n = 2^log_n, 2^13..2^17; log_c selects the
// cluster size where two are built (0 = default).
cudaError_t launch_cluster(int log_n, int log_c, int sign, const ClusterArgs &a, cudaStream_t st);
// Forward real-signal segments of 2^(log_n + 1) samples on the cluster kernel
// (the split into the real DFT's bins in its epilogue; a.rtw, a.out_power, a.scale).
cudaError_t launch_cluster_r2c(int log_n, int log_c, const ClusterArgs &a, cudaStream_t st);
// Inverse real-signal segments (n = 2^13, 2^14): the n + 1 bins in (a.in,
// stride n + 1), the 2n samples out (a.out), the join fused into the column
// pass's loads.
cudaError_t launch_cluster_c2r(int log_n, int log_c, const ClusterArgs &a, cudaStream_t st);
// Bluestein rows of M = 2^log_m points: the inverse transform with the
// product with B before it and the chirp-out after it (a.bl_*).
cudaError_t launch_cluster_blue_inv(int log_m, int log_c, const ClusterArgs &a, cudaStream_t st);
// Bluestein rows of M = 2^log_m points: the forward transform of the chirped
// input rows of a.bl_n samples (read directly, zero past them) into a.out.
cudaError_t launch_cluster_blue_fwd(int log_m, int log_c, const ClusterArgs &a, cudaStream_t st);
// Factorisation used for n: *log_n1, *log_n2, default cluster size *log_c.
bool cluster_shape(int log_n, int log_c_req, int *log_n1, int *log_n2, int *log_c);

// Persistent two-pass four-step kernel (L2-resident intermediate), n = 2^14..2^24.
struct FourStepArgs;
// prec as for launch_block (tensor-core stages for n = 2^16, 2^20, 2^24).
cudaError_t launch_fourstep(int log_n, int sign, int prec, const FourStepArgs &a, cudaStream_t st);
// Warp-specialised variant (FP32): producer warp + eight compute warps, TMA
// loads and stores.
struct FourStepWsArgs;
cudaError_t launch_fourstep_ws(int log_n, int sign, const FourStepWsArgs &a, cudaStream_t st);
// Half-warp-line persistent four-step kernel for n = 65536 (FP32, complex
// output): producer warp, three swizzled TMA tile buffers, TMA output stores.
struct FourStepHwArgs;
cudaError_t launch_fourstep_hw(int sign, const FourStepHwArgs &a, cudaStream_t st);
// Lane-line persistent four-step kernel for n = 2^16..2^20 (FP32, complex
// output): lines of 256..1024 points with 32 points per lane, a queue of
// column and row tiles, loader and retirer warps, swizzled TMA tiles.
struct FourStepWlArgs;
cudaError_t launch_fourstep_wl(int log_n, int sign, const FourStepWlArgs &a, cudaStream_t st);
// The same kernel at n = 2^16 over interleaved units of 32 transforms
// (a.ilv_r transforms per segment, a.nseg units).
cudaError_t launch_fourstep_wl_ilv(int sign, const FourStepWlArgs &a, cudaStream_t st);
// Factorisation n = N1 x N2 and log2 of the tile size of the lane-line kernel.
bool fourstep_wl_shape(int log_n, int *log_n1, int *log_n2, int *log_e);
// Real-signal segments (k_real.cu): the pass between a length-n real DFT and
// the length-m = n/2 complex DFT.  post: complex FFT output [nseg][m] -> the
// n/2 + 1 bins [nseg][m + 1] (complex64, or float32 |X|^2 with power); pre:
// bins [nseg][m + 1] -> complex FFT input [nseg][m].  Both apply `scale`.
struct RealArgs {
    const float2 *zin;  // post: [nseg][m]
    const float2 *xin;  // pre: [nseg][m + 1]
    void *out;
    const float2 *tw;   // w_n^k, k = 0 .. m/2 (forward values)
    int64_t blocks_per_seg;  // set by launch_real
    int m;
    float scale;
};
cudaError_t launch_real(bool post, bool power, RealArgs a, int64_t nseg, cudaStream_t st);
// Forward real segments of n = 2^(log_l + 1) <= 8192 points in one pass (the
// block kernel's tiles with the split fused): in [nseg][2^log_l] complex64 view
// of the samples -> out [nseg][2^log_l + 1] bins (or float32 |X|^2).
struct RealBlockArgs {
    const float2 *in;
    void *out;
    const float2 *twL;  // stage tables of the 2^log_l-point line
    const float2 *tw;   // w_n^k, k <= 2^(log_l - 1)
    int *err;
    int64_t nseg, ntiles;
    int out_power;
    float scale;
};
cudaError_t launch_block_r2c(int log_l, const RealBlockArgs &a, cudaStream_t st);
// Overlapping segments (frames.cu): windowed frames f = samples
// [f*hop, f*hop + n) of the signal into [nframes][n] complex64.
struct FramesArgs {
    const float2 *signal;
    float2 *frames;
    const float *window;  // n values, or null for the rectangular window
    int64_t hop;
    int64_t blocks_per_frame;  // set by launch_frames
    int n;
};
cudaError_t launch_frames(FramesArgs a, int64_t nframes, cudaStream_t st);
// Frames of n = 2^log_l <= 4096 points in one fused pass (frames.cu): the
// windowed frames of the signal straight to their forward bins.
struct FramesBlockArgs {
    const float2 *signal;  // frame f starts at signal + f * hop
    void *out;             // [nframes][n] complex64, or float32 |X|^2
    const float *window;   // n values, or null for the rectangular window
    const float2 *twL;     // stage tables of the n-point line
    int *err;              // set to 1 if a copy never completed
    int64_t hop, nframes, ntiles;
    int out_power;
    float scale;
};
cudaError_t launch_block_frames(int log_l, const FramesBlockArgs &a, cudaStream_t st);
// Lengths that are not powers of two (bluestein.cu): step 0 chirps x into the
// M-point work rows (zero-padded), step 1 multiplies them by B, step 2 chirps
// the first n points out into d_out ([nseg][n], complex64 or float32 |X|^2,
// times scale).  nseg <= 65535 per launch.
struct BlueArgs {
    const float2 *x;     // step 0: [nseg][n]
    float2 *work;        // [nseg][m]
    void *out;           // step 2
    const float2 *w;     // chirp, n values
    const float2 *bhat;  // FFT_M of the conjugate chirp, divided by M
    int64_t n, m;
    float scale;
};
cudaError_t launch_blue(int step, bool power, const BlueArgs &a, int64_t nseg, cudaStream_t st);
// Bluestein rows with M = 2^log_m <= 4096 in one fused pass (bluestein.cu).
struct BlueBlockArgs {
    const float2 *x;     // [nseg][n]
    void *out;           // [nseg][n] complex64, or float32 |X|^2
    const float2 *w;     // chirp, n values
    const float2 *bhat;  // FFT_M of the conjugate chirp, divided by M
    const float2 *twL;   // stage tables of the M-point line
    int *err;            // set to 1 if a copy never completed
    int64_t n, nseg, ntiles;
    int out_power;
    float scale;
};
cudaError_t launch_blue_block(int log_m, const BlueBlockArgs &a, cudaStream_t st);
// Lengths n = 2^a 3^b 5^c 7^d <= 4096 (not powers of two) in one pass
// (k_mixed.cu): mixed-radix Stockham stages over tiles of whole segments.
constexpr int kMixMaxStages = 16;
struct MixedArgs {
    const float2 *in;   // [nseg][n] complex64
    void *out;          // [nseg][n] complex64, or float32 |X|^2
    const float2 *tw;   // stage twiddles: stage t at twoff[t], [r-1][k] = w_{ns R}^{k r}, k < ns
    int *err;
    int64_t nseg, ntiles;
    int n, segs_per_tile, nstages, out_power;
    int radix[kMixMaxStages], ns[kMixMaxStages], twoff[kMixMaxStages];
    float rm[kMixMaxStages], rns[kMixMaxStages];  // 1 / (n / radix), 1 / ns
    float scale;
};
cudaError_t launch_mixed(int sign, const MixedArgs &a, cudaStream_t st);
// The radix schedule for n (odd radices 7, 5, 3 first, then 8s and one 4 or
// 2); false if n has another prime factor or is too long for one tile.
bool mixed_schedule(int64_t n, int *nstages, int *radix);
int mixed_segments_per_tile(int64_t n);
// Factorisation and tile widths used for n.
bool fourstep_shape(int log_n, int *log_n1, int *log_n2, int *log_wa, int *log_wb);
// The four-step twiddle w_n^{j2 k1} is the product of two table entries,
// w_n^{j2 (k1 mod K)} and w_n^{j2 K (k1 div K)}, with K = 2^fourstep_log_k(log2 N1).
__host__ __device__ constexpr int fourstep_log_k(int log_n1) { return log_n1 / 2; }

}  // namespace fftseg
