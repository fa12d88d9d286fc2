// hb_common.cuh -- parameter blocks and launch wrappers shared by the CUDA
// translation units of libhb.  Internal: not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>
#ifndef HB_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace hb {

// NVTX range around host-side enqueue work (a profiler's timeline shows the library's calls,
// stages and serving batches); a no-op unless a tool is attached.
struct NvtxRange {
#ifndef HB_NO_NVTX
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char*) {}
#endif
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kThreads = 256;       // threads per CTA of every kernel here
constexpr int kMaxLevels = 6;
constexpr int kStripCols = 512;     // pixel columns per CTA of the two-column-per-lane transforms

// Pixel columns per CTA of the register transforms for 0..4 levels: two per lane for 1..3
// levels (the strip kernels), one per lane otherwise and for the intensity low pass.
__host__ __device__ constexpr int tile_cols(int levels, int ll_intensity) {
    return (levels >= 1 && levels <= 3 && !ll_intensity) ? kStripCols : kThreads;
}

// Frame geometry and the per-coefficient Tikhonov operator (Eq. 5).
struct TransformParams {
    int H, W;                 // frame size in pixels
    int levels;               // Haar levels n (0..6)
    int fmt;                  // 0 = f32 HWC, 1 = u8 HWC
    float eps;                // intensity floor before the logarithm (f32 input)
    int tile_w;               // tile width in pixels (multiple of 2^n)
    int hl, wl;               // low-pass band size: ceil(H / 2^n) x ceil(W / 2^n)
    int tikhonov_lowpass;     // 1: low pass through M as well
    int ll_intensity;         // 1: ybar = -log(block mean of intensity), Eq. 8 (analysis, levels <= 4)
    float M[6];               // M[j*3 + c], j = HbO2/Hb, c = R/G/B
    float ls_L[6];            // least-squares low pass (HB_LOWPASS_LS): c = ls_L ybar, same layout
};

// Constants of the grid posterior, prepared in FP64 on the host.
// Grid node (i, j) sits at (lo0 + i h0, lo1 + j h1).  Relative to a reference
// node (i0, j0) the base-2 log-likelihood ratio of node (i0 + di, j0 + dj) is
//   U di + V dj + Aq di^2 + 2 Bq di dj + Cq dj^2,
// with U, V per pixel and Aq, Bq, Cq per grid.
struct BayesParams {
    int n0, n1;
    double lo0, h0, lo1, h1, hi0, hi1;
    double A[6];              // A[c*2 + j]
    float Af[6];              // same, FP32
    float G00, G01, G11;      // A^T A (FP32, for choosing the reference node)
    float Gi00, Gi01, Gi11;   // (A^T A)^-1
    double u_scale[3];        // 2 kappa h0 a0[c]: U = sum_c r0[c] u_scale[c]
    double v_scale[3];        // 2 kappa h1 a1[c]
    float Aq, Bq, Cq;
    // FP32 copies for the per-pixel set-up (FP64 is slow on this GPU)
    float lo0f, hi0f, lo1f, hi1f, h0f, h1f;
    float inv_h0f, inv_h1f, inv_G00, inv_G11;  // reciprocals (0 where undefined)
    float u_scalef[3], v_scalef[3];
    // A c at the grid origin and per grid step, as float (hi, lo) pairs:
    //   A c_ij = base + i * step0 + j * step1
    float base_hi[3], base_lo[3], step0_hi[3], step0_lo[3], step1_hi[3], step1_lo[3];
    // Rows whose every weight is exactly zero in FP32 are not enumerated.  Over real dj the
    // largest exponent of row di is  -sup_alpha di^2 + (U - sup_r V) di + sup_c V^2;  rows
    // where that stays below -(kSupportCut + 1e-6 * (sup_mg + |U| n0 + |V| n1)) have all
    // 2^t below 2^-150 (the FP32 evaluation error of t is far inside the margin), which
    // ex2.approx.ftz returns as 0.  sup_rows = 0 enumerates every row.
    int sup_rows;
    float sup_alpha, sup_r, sup_c, sup_mg;
    float sup_inv_alpha;      // 0.5 / (-sup_alpha)
    float sup_inv_aq;         // 0.5 / Aq
    float sup_inv_k1;         // 1 / (-sup_r) where the edge-column pieces apply, else 0
    // Within row di the exponent is a concave quadratic in dj (Cq < 0), so the columns that
    // can hold a non-zero weight form one interval: centre j0 + V span_cv - sup_r di,
    // half-width sqrt(((span_a2 di + b2) di + c2)) with b2 = (U - sup_r V) span_inv_acq and
    // c2 = (sup_c V^2 + cut) span_inv_acq (same cut).  sup_cols = 1 enumerates only those
    // intervals (needs sup_rows and Cq < 0).
    int sup_cols;
    // Cut of the column intervals: nodes below 2^-span_cut of the reference node's weight
    // (exactly 1, and at most the total) are left out; with span_cut = 30 + log2(n0 n1) they
    // carry together less than 2^-30 of the posterior mass, far below the FP32 rounding of
    // the sums (at most kSupportCut: beyond it FP32 weights are zero anyway).
    float span_cut;
    float span_a2;            // -sup_alpha / |Cq|
    float span_inv_acq;       // 1 / |Cq|
    float span_cv;            // -0.5 / Cq
    float span_an2;           // sup_alpha n0^2 (size of the quadratic term, for the rounding guard)
    // Row kernel: along a grid row the weights of every second column form a sequence whose
    // consecutive ratios grow by the constant factor row_q = 2^(8 Cq) (the weights are a
    // Gaussian in the column index).  rows_ok = 1 when the column intervals apply and
    // -2 <= Cq < 0 (row_q >= 2^-16).
    float row_q;
    int rows_ok;
    int illum;                // 1: A holds (I - 11^T/3) A and the set-up removes ybar's channel mean
    // Closed-form row sums of the row kernel (row_tab set; needs rows_ok).  Along row di the
    // base-2 log weight is t* + Cq (j - mu)^2 (t* the row's maximum over real columns, mu its
    // column), so over all integer columns the row's weights add up to 2^t* K with
    // K = sqrt(pi / (-Cq ln 2)), and their mean column is mu, up to the Poisson terms below
    // (Poisson summation).
    // A row whose interval the grid cuts off on one side is the one-sided sum
    // F(x) = sum_{k >= 0} 2^(Cq (k - x)^2), x = the peak's distance from the edge column, whose
    // mean is m(x) columns from the edge: row_tab holds, per interval [x_k, x_k + 1/tab_inv_step)
    // of x in [tab_x0, tab_x0 + tab_n / tab_inv_step), the cubic in u = (x - x_k) tab_inv_step of
    // log2 F (float4 2k) and of m (float4 2k + 1), Hermite interpolants of direct FP64 sums,
    // checked on the host against those sums.  Beyond the table's right end F = K and m = x.
    const float4* row_tab;
    float tab_x0, tab_inv_step;
    int tab_n;
    float log2_kfull;         // log2 K
    // The first Poisson term, kept where it exceeds 1e-14 (rows narrower than about 1.5
    // columns): over all integer columns the sum is 2^t* K (1 + 2 q cos(2 pi mu)) and the mean
    // column mu - (2 pi / a) q sin(2 pi mu) / (1 + 2 q cos(2 pi mu)), q = exp(-pi^2 / a),
    // a = -Cq ln 2, up to a relative 2 q^4; the host requires q^4 below 7e-13 (pi^2 / a >= 7).
    // pois_q = q and pois_m = 2 pi q / a, or both 0.
    float pois_q, pois_m;
};

// Where the analysis writes the least-squares low-pass estimates (c = nullptr: it writes the
// posterior records instead): c per low-pass pixel, and optionally 2^n c.
struct LsOut {
    float2* c = nullptr;
    float2* c_scaled = nullptr;
    float scale = 1.f;
};
constexpr float kSupportCut = 150.f;

// Per low-pass pixel record written by the analysis kernel for the posterior kernel.
struct __align__(16) BayesRec {
    int i0, j0;               // reference node (nearest node to the box-constrained maximiser)
    float U, V;               // linear coefficients of the log2-likelihood ratio
};

// Scratch of the posterior kernel: per-part partial sums of each pixel and a per-pixel
// arrival counter (zero between launches; the kernel resets what it uses).
struct PosteriorScratch {
    float* partial;           // npix * max_parts * 3
    unsigned* count;          // npix
    int max_parts;
    unsigned long long* nodes = nullptr;  // optional: grid nodes enumerated, added per warp
};
constexpr int kMaxParts = 8;

// One frame of a serving batch: its geometry, buffers, and where its tiles and low-pass
// pixels sit in the batch-wide grid and arrays.
struct FrameJob {
    TransformParams tp;
    const unsigned char* frame;
    size_t stride;
    float* thb;
    float* so2;
    long ll_offset;           // first low-pass pixel of this frame in the batch arrays
    int tile_begin;           // first CTA of this frame in the batched grids
    int tiles_x;              // tile columns (tiles = tiles_x * hl)
};
constexpr int kMaxBatchJobs = 64;

// Launch wrappers (defined in the .cu files).  All return the launch status; pdl: PDL launch.
cudaError_t launch_analysis(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                            const float2* lut, double* ybar, BayesRec* rec, cudaStream_t s, float* ybar_f = nullptr,
                            const LsOut& ls = LsOut{}, bool pdl = false);
cudaError_t launch_setup(const BayesParams& bp, const double* ybar, long npix, BayesRec* rec, cudaStream_t s);
// Optional gate of the posterior launch: when run is set the kernel takes every pixel if
// *run is non-zero (the decision the learned stand-in's sampled check leaves behind), and
// otherwise only the *count pixels of list (none without a list: the pixels the learned
// stand-in's route sends to the exact posterior), adding how many to *listed_total.
struct PosteriorGate {
    const unsigned* run;
    const int* list = nullptr;
    const unsigned* count = nullptr;
    unsigned long long* listed_total = nullptr;
};
cudaError_t launch_posterior(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                             float2* chat, float2* chat_scaled, float scale, bool pdl, cudaStream_t s,
                             const PosteriorGate& gate = PosteriorGate{nullptr});
// The fused low pass (block means, posterior records and posterior means in one launch, for
// the plain grid posterior at 1..3 levels): whether it applies, and its launch.
bool lowpass_fused_ok(const TransformParams& tp, const BayesParams& bp);
// The closed-form row sums' table for bp (host, FP64; BayesParams::row_tab): fills tab and bp's
// table fields other than row_tab, or returns false when the closed form does not apply.
bool row_table(BayesParams& bp, std::vector<float4>& tab);
cudaError_t launch_lowpass_fused(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                                 const float2* lut, float2* chat, float2* chat_scaled, float scale,
                                 unsigned long long* nodes, bool pdl, cudaStream_t s);
// The single-pass frame kernel (every step of the path in one launch, for the plain grid
// posterior at 1..3 levels with the closed-form rows): whether it applies, and its launch.
// chat (and chat_scaled, if set) receive the low-pass posterior means as a by-product.
bool frame_kernel_ok(const TransformParams& tp, const BayesParams& bp);
cudaError_t launch_frame(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                         const float2* lut, float2* chat, float2* chat_scaled, float scale, float* out0, float* out1,
                         int debug_conc, unsigned long long* nodes, bool pdl, cudaStream_t s);
// Whether launch_posterior takes npix pixels with the kernel it uses for large launches (two
// pixels per warp: the span kernel, or the pair kernel without column intervals); each
// pixel's result then does not depend on the other pixels of the launch.
bool posterior_uses_pairs(const BayesParams& bp, long npix);
cudaError_t launch_synthesis(const TransformParams& tp, const void* frame, size_t stride, const float2* lut,
                             const float2* chat, float* out0, float* out1, int debug_conc, bool pdl, cudaStream_t s);
size_t transform_smem_bytes(const TransformParams& tp);
// Serving batches: one launch per stage for all jobs (levels 0..4 per job).  jobs is a
// device array of njobs entries; total_tiles = sum of tiles_x * hl.
cudaError_t launch_batch_analysis(const BayesParams& bp, const FrameJob* jobs, int njobs, int total_tiles,
                                  const float2* lut, BayesRec* rec_all, cudaStream_t s);
cudaError_t launch_batch_synthesis(const FrameJob* jobs, int njobs, int total_tiles, const float2* lut,
                                   const float2* chat_all, cudaStream_t s);

}  // namespace hb
