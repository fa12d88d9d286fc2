// hb_api.cu -- the C ABI declared in include/hb.h: argument checks, the host-side
// FP64 preparation of the operator and grid constants, context-owned scratch,
// and the launch sequence of one frame.
#include "hb.h"
#include "hb_common.cuh"
#include "hb_mlp.cuh"

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using hb::BayesParams;
using hb::BayesRec;
using hb::TransformParams;

// What a captured hb_estimate_host sequence depends on besides the context itself.
struct HostKey {
    const void* frame;
    size_t stride;
    float* thb;
    float* so2;
    cudaStream_t stream;
    int first, nb;
    bool operator==(const HostKey& o) const {
        return frame == o.frame && stride == o.stride && thb == o.thb && so2 == o.so2 && stream == o.stream &&
               first == o.first && nb == o.nb;
    }
};

struct hb_ctx {
    int device = 0;
    int W = 0, H = 0, levels = 0, fmt = 0;
    unsigned flags = 0;
    int hl = 0, wl = 0;
    long npix_ll = 0;
    double gamma = 0.0;
    TransformParams tp{};
    BayesParams bp{};
    float2* d_lut = nullptr;      // 256 (hi, lo) log-attenuation values of the 8-bit codes
    BayesRec* d_rec = nullptr;    // per low-pass pixel posterior constants
    float2* d_chat = nullptr;     // per low-pass pixel posterior mean
    float* d_partial = nullptr;   // posterior kernel: per-part partial sums
    unsigned* d_count = nullptr;  // posterior kernel: per-pixel arrival counters (kept at zero)
    long rec_cap = 0;             // capacity of the four arrays above in pixels
    // device staging of hb_estimate_host
    void* d_frame = nullptr;
    float* d_thb = nullptr;
    float* d_so2 = nullptr;
    std::atomic<long> launches{0};
    // learned stand-in
    float* d_mlp = nullptr;       // FP32 masters | Adam m | Adam v | BF16 copies | grad, 5 x kNParams
    void* d_mlp_img = nullptr;    // the inference kernel's packed image of the BF16 parameters
    bool mlp_img_dirty = true;    // parameters changed since the image was packed
    float* d_mlp_gpart = nullptr; // per-CTA partial gradients
    float* d_mlp_lpart = nullptr; // per-CTA partial losses
    float* d_mlp_loss = nullptr;  // loss per training step
    long mlp_loss_cap = 0;
    hb::MlpNorm mlp_norm{};
    float mlp_ext0 = 1.f, mlp_ext1 = 1.f;  // box extents: the fallback check's error scale
    double sigma_l = 0.0;
    bool mlp_ready = false;
    int adam_t = 0;
    int lowpass_mode = HB_MODE_BAYES;
    float mlp_tol = 1e-3f;
    int mlp_nsample = 256;
    float* d_ybar_f = nullptr;    // block means for the network (npix_ll x 3)
    // [0] check arrivals, [1] fallback count, [2] run the exact posterior on every pixel,
    // [4 + (frame & 1)] pixels the route listed, [6, 7] listed pixels taken (64-bit total)
    unsigned* d_flags = nullptr;
    int* d_route = nullptr;       // the route's list (npix_ll)
    unsigned char* d_trust = nullptr;  // certification map (trust_k0 x trust_k1)
    hb::MlpRoute route{};         // trust set while a certification holds for the parameters
    float* d_err = nullptr;       // per sampled pixel error of the stand-in (mlp_err_cap)
    int mlp_err_cap = 0;
    unsigned long long* d_nodes = nullptr;  // timed posterior launches: [0] nodes summed one by one,
                                            // [1] rows summed in closed form, [2] of those cut
                                            // off by the box edge
    float4* d_rowtab = nullptr;   // the closed-form row sums' table (BayesParams::row_tab)
    long mlp_frames = 0;
    unsigned frame_seq = 0;
    // hb_estimate_host: copy streams and per-band events (created on first use)
    cudaStream_t s_in = nullptr, s_out = nullptr, s_alt = nullptr;
    std::vector<cudaEvent_t> host_ev;
    // hb_estimate_host_async: a second staging set (the first is d_frame, d_thb, d_so2), the
    // compute stream of the even bands, and per set the event after its last output copy
    void* d_frame2 = nullptr;
    float* d_thb2 = nullptr;
    float* d_so22 = nullptr;
    cudaStream_t s_c0 = nullptr;
    cudaEvent_t set_free[2] = {nullptr, nullptr};
    int set_next = 0;
    bool async_pending = false;
    HostKey hg_key{};                 // the buffers etc. of the last call, and its captured graph
    bool hg_seen = false;
    cudaGraphExec_t hg_exec = nullptr;
    long hg_kernels = 0;
    // per-stage timing
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_stage;
    int ev_used = 0;
    bool timing = false;
};

namespace {

// Row bands of the synchronous host entry point (at most).  The copies of a 1920x1080 u8
// frame need ~98 us with both directions of the host link (~190 GB/s each) busy; a call
// measures ~157 us with 3 bands (201 us unbanded, more with 4 or more), and the synthesis
// storing THb/SO2 straight into pinned host memory instead of the output copies measured
// the same.
#ifndef HB_HOST_BANDS
#define HB_HOST_BANDS 3
#endif
constexpr int kHostBands = HB_HOST_BANDS;
// Row bands of the asynchronous host entry point (at most).  Successive frames overlap there,
// which keeps the host link busy without splitting a frame: a 1920x1080 u8 frame measured
// 101 us per frame in steady state with one band, 107 us with two and 112 us with three
// (the two copies alone need ~98 us).
#ifndef HB_ASYNC_BANDS
#define HB_ASYNC_BANDS 1
#endif
constexpr int kAsyncBands = HB_ASYNC_BANDS < HB_HOST_BANDS ? HB_ASYNC_BANDS : HB_HOST_BANDS;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t elem_size(int fmt) { return fmt == HB_IN_U8_HWC ? 1 : 4; }

// Operator of Eq. 5 and the grid constants, in FP64.
void prepare(hb_ctx* c, const hb_mixing* mix, const hb_grid* g, double lambda) {
    const double(*Ain)[2] = mix->A;
    double G[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) G[j][k] = Ain[0][j] * Ain[0][k] + Ain[1][j] * Ain[1][k] + Ain[2][j] * Ain[2][k];
    c->gamma = (c->flags & HB_LAMBDA_ABSOLUTE) ? lambda : lambda * (G[0][0] + G[1][1]) / 2.0;
    // The 2x3 operator (A^T A + gamma I)^-1 A^T (Eq. 5), or with the illumination term the
    // HbO2 and Hb rows of (xi^T xi + gamma I)^-1 xi^T for xi = [A | 1] (Eq. 8's constant term).
    // gamma = 0 gives the least-squares fit of the maximisation step (Eq. 9).
    auto operator_2x3 = [&](double gamma, float (&out)[6]) {
        if (!(c->flags & HB_ILLUMINATION)) {
            const double R00 = G[0][0] + gamma, R11 = G[1][1] + gamma, R01 = G[0][1];
            const double det = R00 * R11 - R01 * R01;
            for (int ch = 0; ch < 3; ++ch) {
                out[0 * 3 + ch] = (float)((R11 * Ain[ch][0] - R01 * Ain[ch][1]) / det);
                out[1 * 3 + ch] = (float)((-R01 * Ain[ch][0] + R00 * Ain[ch][1]) / det);
            }
            return;
        }
        double xi[3][3], R[3][3], Ri[3][3];
        for (int ch = 0; ch < 3; ++ch) {
            xi[ch][0] = Ain[ch][0];
            xi[ch][1] = Ain[ch][1];
            xi[ch][2] = 1.0;
        }
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                R[j][k] = xi[0][j] * xi[0][k] + xi[1][j] * xi[1][k] + xi[2][j] * xi[2][k] + (j == k ? gamma : 0.0);
        const double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1]) -
                           R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0]) +
                           R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                const int a0 = (k + 1) % 3, a1 = (k + 2) % 3, b0 = (j + 1) % 3, b1 = (j + 2) % 3;
                Ri[j][k] = (R[a0][b0] * R[a1][b1] - R[a0][b1] * R[a1][b0]) / det;
            }
        for (int j = 0; j < 2; ++j)
            for (int ch = 0; ch < 3; ++ch)
                out[j * 3 + ch] = (float)(Ri[j][0] * xi[ch][0] + Ri[j][1] * xi[ch][1] + Ri[j][2] * xi[ch][2]);
    };
    operator_2x3(c->gamma, c->tp.M);
    operator_2x3(0.0, c->tp.ls_L);
    // The posterior's mixing matrix.  With the illumination term the likelihood after
    // integrating kappa out is that of P (ybar - A c), P = I - (1,1,1)(1,1,1)^T / 3; using
    // P A in place of A gives it exactly, since the part of ybar along (1,1,1) is the same
    // for every node and cancels from the weights relative to the reference node.
    double A[3][2];
    for (int j = 0; j < 2; ++j) {
        const double m = (c->flags & HB_ILLUMINATION) ? (Ain[0][j] + Ain[1][j] + Ain[2][j]) / 3.0 : 0.0;
        for (int ch = 0; ch < 3; ++ch) A[ch][j] = Ain[ch][j] - m;
    }
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) G[j][k] = A[0][j] * A[0][k] + A[1][j] * A[1][k] + A[2][j] * A[2][k];
    BayesParams& bp = c->bp;
    bp.illum = (c->flags & HB_ILLUMINATION) ? 1 : 0;
    bp.n0 = g->n0;
    bp.n1 = g->n1;
    bp.lo0 = g->lo0;
    bp.lo1 = g->lo1;
    bp.h0 = g->n0 > 1 ? (g->hi0 - g->lo0) / (g->n0 - 1) : 0.0;
    bp.h1 = g->n1 > 1 ? (g->hi1 - g->lo1) / (g->n1 - 1) : 0.0;
    // hull of the grid nodes (a single node when n = 1): the reference-node search box
    bp.hi0 = g->n0 > 1 ? g->hi0 : g->lo0;
    bp.hi1 = g->n1 > 1 ? g->hi1 : g->lo1;
    for (int ch = 0; ch < 3; ++ch)
        for (int j = 0; j < 2; ++j) {
            bp.A[ch * 2 + j] = A[ch][j];
            bp.Af[ch * 2 + j] = (float)A[ch][j];
        }
    bp.G00 = (float)G[0][0];
    bp.G01 = (float)G[0][1];
    bp.G11 = (float)G[1][1];
    double gd = G[0][0] * G[1][1] - G[0][1] * G[0][1];
    double r = 0.0;
    if (!(gd > 1e-12 * G[0][0] * G[1][1])) r = 1e-6 * (G[0][0] + G[1][1] + 1e-300);  // near-collinear columns
    gd = (G[0][0] + r) * (G[1][1] + r) - G[0][1] * G[0][1];
    bp.Gi00 = (float)((G[1][1] + r) / gd);
    bp.Gi01 = (float)(-G[0][1] / gd);
    bp.Gi11 = (float)((G[0][0] + r) / gd);
    // base-2 log-likelihood: log2(e) / (2 sigma^2) * (-|residual|^2)
    const double kappa = 1.0 / (2.0 * g->sigma_l * g->sigma_l * std::log(2.0));
    const double a0a0 = G[0][0], a0a1 = G[0][1], a1a1 = G[1][1];
    bp.Aq = (float)(-kappa * bp.h0 * bp.h0 * a0a0);
    bp.Bq = (float)(-kappa * bp.h0 * bp.h1 * a0a1);
    bp.Cq = (float)(-kappa * bp.h1 * bp.h1 * a1a1);
    for (int ch = 0; ch < 3; ++ch) {
        bp.u_scale[ch] = 2.0 * kappa * bp.h0 * A[ch][0];
        bp.v_scale[ch] = 2.0 * kappa * bp.h1 * A[ch][1];
        bp.u_scalef[ch] = (float)bp.u_scale[ch];
        bp.v_scalef[ch] = (float)bp.v_scale[ch];
    }
    bp.lo0f = (float)bp.lo0;
    bp.hi0f = (float)bp.hi0;
    bp.lo1f = (float)bp.lo1;
    bp.hi1f = (float)bp.hi1;
    bp.h0f = (float)bp.h0;
    bp.h1f = (float)bp.h1;
    bp.inv_h0f = bp.h0 > 0 ? (float)(1.0 / bp.h0) : 0.f;
    bp.inv_h1f = bp.h1 > 0 ? (float)(1.0 / bp.h1) : 0.f;
    bp.inv_G00 = G[0][0] > 0 ? (float)(1.0 / G[0][0]) : 0.f;
    bp.inv_G11 = G[1][1] > 0 ? (float)(1.0 / G[1][1]) : 0.f;
    // rows of the grid that can hold a non-zero FP32 weight (see BayesParams::sup_rows)
    {
        const double aq = -kappa * bp.h0 * bp.h0 * a0a0, bq = -kappa * bp.h0 * bp.h1 * a0a1,
                     cq = -kappa * bp.h1 * bp.h1 * a1a1;
        double alpha = 0.0, rr = 0.0, cc = 0.0;
        if (cq < 0.0) {
            alpha = -(aq - bq * bq / cq);
            rr = bq / cq;
            cc = -1.0 / (4.0 * cq);
        } else if (bq == 0.0) {  // a single grid column: t = Aq di^2 + U di
            alpha = -aq;
        }
        const double mg = std::fabs(aq) * g->n0 * g->n0 + 2.0 * std::fabs(bq) * g->n0 * g->n1 +
                          std::fabs(cq) * g->n1 * g->n1;
        bp.sup_rows = (!(c->flags & HB_FULL_GRID) && g->n0 > 1 && alpha > 0.0 && std::isfinite(alpha) &&
                       std::isfinite(rr) && std::isfinite(cc) && std::isfinite(mg) && mg < 1e30)
                          ? 1
                          : 0;
        bp.sup_alpha = (float)alpha;
        bp.sup_r = (float)rr;
        bp.sup_c = (float)cc;
        bp.sup_mg = (float)mg;
        bp.sup_inv_alpha = alpha > 0.0 ? (float)(-0.5 / alpha) : 0.f;
        bp.sup_inv_aq = aq < 0.0 ? (float)(0.5 / aq) : 0.f;
        bp.sup_inv_k1 = (cq < 0.0 && aq < 0.0 && rr != 0.0 && std::isfinite(1.0 / rr)) ? (float)(-1.0 / rr) : 0.f;
        bp.sup_cols = (bp.sup_rows && cq < 0.0 && std::isfinite(1.0 / cq) && (float)cq < 0.f &&
                       std::isfinite((float)(alpha / cq)) && std::isfinite((float)(alpha * g->n0 * g->n0)))
                          ? 1
                          : 0;
        bp.span_cut = (float)std::min((double)hb::kSupportCut, 30.0 + std::log2((double)g->n0 * (double)g->n1));
        bp.span_a2 = bp.sup_cols ? (float)(alpha / cq) : 0.f;
        bp.span_inv_acq = bp.sup_cols ? (float)(-1.0 / cq) : 0.f;
        bp.span_cv = bp.sup_cols ? (float)(-0.5 / cq) : 0.f;
        bp.span_an2 = bp.sup_cols ? (float)(alpha * g->n0 * g->n0) : 0.f;
        const double q8 = std::exp2(8.0 * (double)bp.Cq);
        bp.row_q = (float)q8;
        // (steeper rows, |Cq| > 2, have a few nodes each and go to the span kernel: there the
        // widened ends of a row can lie so far below the cut that the chains' range would not do)
        bp.rows_ok = (bp.sup_cols && bp.Cq < 0.f && bp.Cq >= -2.f && q8 <= 1.0) ? 1 : 0;
    }
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (int ch = 0; ch < 3; ++ch) {
        split(A[ch][0] * bp.lo0 + A[ch][1] * bp.lo1, bp.base_hi[ch], bp.base_lo[ch]);
        split(A[ch][0] * bp.h0, bp.step0_hi[ch], bp.step0_lo[ch]);
        split(A[ch][1] * bp.h1, bp.step1_hi[ch], bp.step1_lo[ch]);
    }
}

hb_status ensure_rec(hb_ctx* c, long npix) {
    if (npix <= c->rec_cap) return HB_OK;
    cudaFree(c->d_rec);
    cudaFree(c->d_chat);
    cudaFree(c->d_partial);
    cudaFree(c->d_count);
    c->d_rec = nullptr;
    c->d_chat = nullptr;
    c->d_partial = nullptr;
    c->d_count = nullptr;
    c->rec_cap = 0;
    if (cudaMalloc(&c->d_rec, sizeof(BayesRec) * npix) != cudaSuccess ||
        cudaMalloc(&c->d_chat, sizeof(float2) * npix) != cudaSuccess ||
        cudaMalloc(&c->d_partial, sizeof(float) * 3 * hb::kMaxParts * npix) != cudaSuccess ||
        cudaMalloc(&c->d_count, sizeof(unsigned) * npix) != cudaSuccess) {
        cudaGetLastError();
        return HB_ERR_OOM;
    }
    if (cudaMemset(c->d_count, 0, sizeof(unsigned) * npix) != cudaSuccess) return HB_ERR_CUDA;
    c->rec_cap = npix;
    return HB_OK;
}

}  // namespace

namespace hb {
// The FP64 preparation of the operator and grid constants for code outside a context.
void prepare_constants(const hb_mixing* mix, const hb_grid* grid, double lambda, unsigned flags, float M[6],
                       BayesParams& bp) {
    hb_ctx holder;
    holder.flags = flags;
    prepare(&holder, mix, grid, lambda);
    for (int k = 0; k < 6; ++k) M[k] = holder.tp.M[k];
    bp = holder.bp;
}

namespace {
// The one-sided row sum F(x) = sum_{k >= 0} 2^(cq (k - x)^2) by direct FP64 summation: log2 F,
// its derivative, the mean column m(x) = sum k 2^(...) / F and its derivative
// (d log2 F / dx = -2 cq (m - x), dm / dx = -2 cq ln 2 Var(k)).
void one_sided_sum(double cq, double x, double& lf, double& dlf, double& m, double& dm) {
    const double tmax = x < 0.0 ? cq * x * x : 0.0;  // the largest exponent, at k = 0 or near x
    const long kmax = (long)(std::max(x, 0.0) + std::sqrt(120.0 / -cq)) + 2;  // later terms < 2^-120
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;  // moments about x
    for (long k = 0; k <= kmax; ++k) {
        const double e = (double)k - x;
        const double w = std::exp2(cq * e * e - tmax);
        s0 += w;
        s1 += w * e;
        s2 += w * e * e;
    }
    const double mean = s1 / s0;
    lf = std::log2(s0) + tmax;
    m = x + mean;
    dlf = -2.0 * cq * mean;
    dm = -2.0 * cq * std::log(2.0) * std::max(s2 / s0 - mean * mean, 0.0);
}
}  // namespace

// The closed-form row sums' table (BayesParams::row_tab): over x in [-(hc + 4), hc + 4) (ends
// rounded outwards to a whole step), hc = sqrt((span_cut + 2) / -Cq) the widest half-interval
// of a row whose peak is at most the reference node's weight, cubic Hermite pieces of log2 F
// and m.  The step starts at the power of two nearest below sigma / 16 (sigma = the row's
// Gaussian width in columns, 1 / sqrt(-2 Cq ln 2); at most 1/8 of a column below sigma = 4)
// and is halved, three times at most, until every piece agrees with the direct sums at
// u = 1/4, 1/2, 3/4 (log2 F within 4e-6 + 1e-7 |log2 F|, m within 1e-5 columns + 1e-6 sigma,
// with the FP32-rounded coefficients).
// Sets bp's table fields except row_tab, and the first Poisson term (pois_q, pois_m) where it
// matters; false (no closed form) when the grid has no row kernel, when the second Poisson
// term exp(-4 pi^2 / a) exceeds 7e-13 (pi^2 / a < 7), when the table's right end differs from
// the full sum, or when no step passes.
bool row_table(BayesParams& bp, std::vector<float4>& tab) {
    tab.clear();
    if (!bp.rows_ok || !(bp.Cq < 0.f)) return false;
    const double cq = (double)bp.Cq, a = -cq * std::log(2.0);
    if (M_PI * M_PI / a < 7.0) return false;
    const double q = std::exp(-M_PI * M_PI / a);
    const double hc = std::sqrt(((double)bp.span_cut + 2.0) / -cq);
    const double x1 = hc + 4.0, x0 = -x1;
    const double log2k = 0.5 * std::log2(M_PI / a);
    {
        // at the right end the one-sided sum must be the full one (the two-sided sum, with its
        // Poisson term)
        double lf, dlf, m, dm;
        one_sided_sum(cq, x1, lf, dlf, m, dm);
        const double c = std::cos(2.0 * M_PI * x1), sn = std::sin(2.0 * M_PI * x1), den = 1.0 + 2.0 * q * c;
        const double lf_full = log2k + std::log2(den), m_full = x1 - 2.0 * M_PI / a * q * sn / den;
        if (!(std::fabs(lf - lf_full) <= 1e-9 && std::fabs(m - m_full) <= 1e-7)) return false;
    }
    const double sigma = 1.0 / std::sqrt(2.0 * a);
    const double s_start = std::exp2(std::floor(std::log2(sigma / 16.0)));
    for (double s = s_start; s >= s_start / 8.0; s *= 0.5) {
        const double xa = -std::ceil(-x0 / s) * s;  // a whole number of steps: exact in FP32
        const int n = (int)std::ceil((x1 - xa) / s);
        if (n > 8192) return false;
        std::vector<double> lf(n + 1), dlf(n + 1), m(n + 1), dm(n + 1);
        for (int k = 0; k <= n; ++k) one_sided_sum(cq, xa + k * s, lf[k], dlf[k], m[k], dm[k]);
        tab.assign(2 * (size_t)n, float4{});
        bool ok = true;
        for (int k = 0; k < n && ok; ++k) {
            auto cubic = [&](const std::vector<double>& f, const std::vector<double>& df) {
                const double f0 = f[k], f1 = f[k + 1], d0 = s * df[k], d1 = s * df[k + 1];
                return float4{(float)f0, (float)d0, (float)(3.0 * (f1 - f0) - 2.0 * d0 - d1),
                              (float)(2.0 * (f0 - f1) + d0 + d1)};
            };
            const float4 p = cubic(lf, dlf), q = cubic(m, dm);
            tab[2 * k] = p;
            tab[2 * k + 1] = q;
            for (double u : {0.25, 0.5, 0.75}) {
                double elf, edlf, em, edm;
                one_sided_sum(cq, xa + (k + u) * s, elf, edlf, em, edm);
                const double ilf = p.x + u * (p.y + u * (p.z + u * (double)p.w));
                const double im = q.x + u * (q.y + u * (q.z + u * (double)q.w));
                if (!(std::fabs(ilf - elf) <= 4e-6 + 1e-7 * std::fabs(elf) && std::fabs(im - em) <= 1e-5 + 1e-6 * sigma))
                    ok = false;
            }
        }
        if (!ok) continue;
        bp.tab_x0 = (float)xa;
        bp.tab_inv_step = (float)(1.0 / s);
        bp.tab_n = n;
        bp.log2_kfull = (float)log2k;
        bp.pois_q = q > 1e-14 ? (float)q : 0.f;
        bp.pois_m = q > 1e-14 ? (float)(2.0 * M_PI * q / a) : 0.f;
        return true;
    }
    tab.clear();
    return false;
}
}  // namespace hb

namespace {

// Asynchronous host calls still in flight run on the context's own streams and share its
// low-pass arrays (and, in learned mode, its network and flags) with every other call: wait
// for them first.
hb_status settle_async(hb_ctx* c) {
    if (!c->async_pending) return HB_OK;
    for (cudaStream_t st : {c->s_in, c->s_c0, c->s_alt, c->s_out})
        if (st && cudaStreamSynchronize(st) != cudaSuccess) return HB_ERR_CUDA;
    c->async_pending = false;
    return HB_OK;
}

// Posterior scratch for the low-pass pixels from ll_off on (launches that may run at the same
// time take disjoint pixel ranges, so their counters are disjoint as well).
hb::PosteriorScratch post_scratch(const hb_ctx* c, long ll_off = 0) {
    return hb::PosteriorScratch{c->d_partial + (size_t)3 * hb::kMaxParts * ll_off, c->d_count + ll_off, hb::kMaxParts,
                                c->timing ? c->d_nodes : nullptr};
}

// Event bracket around one launch when timing is armed.
const char* const kStageNames[HB_NUM_STAGES] = {"hb.analysis", "hb.lowpass", "hb.synthesis", "hb.frame"};

struct StageTimer {
    hb_ctx* c;
    cudaStream_t s;
    int slot = -1;
    hb::NvtxRange range;
    StageTimer(hb_ctx* c_, cudaStream_t s_, int stage) : c(c_), s(s_), range(kStageNames[stage]) {
        if (c->timing && 2 * (c->ev_used + 1) <= (int)c->ev.size()) {
            slot = c->ev_used++;
            c->ev_stage[slot] = stage;
            cudaEventRecord(c->ev[2 * slot], s);
        }
    }
    ~StageTimer() {
        if (slot >= 0) cudaEventRecord(c->ev[2 * slot + 1], s);
    }
};

hb_status check_frame_args(const hb_ctx* c, const void* frame, size_t stride) {
    if (!frame) return HB_ERR_ARG;
    const size_t es = elem_size(c->fmt);
    if (stride < (size_t)c->W * 3 * es) return HB_ERR_ARG;
    if (es == 4 && ((reinterpret_cast<uintptr_t>(frame) & 3) || (stride & 3))) return HB_ERR_ARG;
    return HB_OK;
}

// One frame.  Bayesian low pass: analysis kernel (block means and the per-pixel
// posterior records), posterior over the records, synthesis.  The posterior and the
// synthesis are launched with programmatic dependent launch (each waits for its
// predecessor inside the kernel) unless per-stage timing is armed, since timing events
// between the kernels serialise them anyway.  All-Tikhonov mode: the synthesis alone.
// The packed image for inference, rebuilt on `s` if the parameters changed.
const void* mlp_image(hb_ctx* c, cudaStream_t s, cudaError_t& e) {
    if (c->mlp_img_dirty) {
        e = hb::launch_mlp_pack(c->d_mlp + 3 * hb::kNParams, c->d_mlp_img, s);
        c->launches++;
        if (e != cudaSuccess) return nullptr;
        c->mlp_img_dirty = false;
    }
    return c->d_mlp_img;
}

// A band of whole superblock rows of the frame: superblocks never straddle two bands, so a
// band is processed as a frame of its own (its rows, the frame's width) whose low-pass
// pixels sit at ll_off in the context's arrays.  Only the band holding the frame's last
// row meets the bottom edge, so the edge replication is the whole frame's.
struct Band {
    TransformParams tp;
    long ll_off;
    long npix;
};

Band whole_frame(const hb_ctx* c) { return Band{c->tp, 0, c->npix_ll}; }

// chain: the frame is already on the device and the analysis may be launched as a
// programmatic dependent of whatever kernel precedes it on the stream (it waits for that
// kernel before reading); host bands, whose analysis follows a copy, pass false.
hb_status run_band(hb_ctx* c, const Band& b, const void* frame, size_t stride, double* ybar, float* out0, float* out1,
                   float2* conc_scaled, int debug, cudaStream_t s, bool chain = false) {
    cudaError_t e = cudaSuccess;
    // the low pass: the grid posterior (possibly through the learned stand-in), least squares
    // (written by the analysis itself), or nothing separate (Tikhonov on every band)
    const bool lowpass = !(c->flags & HB_LOWPASS_TIKHONOV);
    const bool ls = lowpass && (c->flags & HB_LOWPASS_LS);
    const bool bayes = lowpass && !ls;
    const bool pdl = !c->timing;
    const bool mlp = bayes && c->lowpass_mode != HB_MODE_BAYES;
    BayesRec* rec = c->d_rec + b.ll_off;
    float2* chat = c->d_chat + b.ll_off;
    const float scale = (float)(1 << c->levels);
    if (bayes && !mlp && !ybar && out0 && out1 && hb::frame_kernel_ok(b.tp, c->bp)) {
        // every step in one launch
        StageTimer t(c, s, HB_STAGE_FRAME);
        e = hb::launch_frame(b.tp, c->bp, frame, stride, c->d_lut, chat, conc_scaled, scale, out0, out1, debug,
                             c->timing ? c->d_nodes : nullptr, pdl && chain, s);
        c->launches++;
        return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
    }
    if (bayes && !mlp && !ybar && hb::lowpass_fused_ok(b.tp, c->bp)) {
        // block means, records and posterior means in one launch
        StageTimer t(c, s, HB_STAGE_LOWPASS);
        e = hb::launch_lowpass_fused(b.tp, c->bp, frame, stride, c->d_lut, chat, conc_scaled, scale,
                                     c->timing ? c->d_nodes : nullptr, pdl && chain, s);
        c->launches++;
        if (e != cudaSuccess) return HB_ERR_CUDA;
    } else if (lowpass) {
        {
            StageTimer t(c, s, HB_STAGE_ANALYSIS);
            hb::LsOut lso;
            if (ls) {
                lso.c = chat;
                lso.c_scaled = conc_scaled;
                lso.scale = scale;
            }
            e = hb::launch_analysis(b.tp, c->bp, frame, stride, c->d_lut, ybar, rec, s,
                                    mlp ? c->d_ybar_f + 3 * b.ll_off : nullptr, lso, pdl && chain);
            c->launches++;
        }
        if (e != cudaSuccess) return HB_ERR_CUDA;
    }
    if (bayes && (mlp || ybar || !hb::lowpass_fused_ok(b.tp, c->bp))) {
        StageTimer t(c, s, HB_STAGE_LOWPASS);
        if (mlp) {
            // network estimate together with the sampled exact check (one launch), then the
            // exact recomputation only if the check failed; each kernel waits for its
            // predecessor in-kernel (PDL)
            const void* img = mlp_image(c, s, e);
            const unsigned seq = c->frame_seq++;
            hb::MlpCheck ck{c->mlp_nsample, 0, seq, 1.f / c->mlp_ext0, 1.f / c->mlp_ext1, c->mlp_tol,
                            c->lowpass_mode == HB_MODE_MLP ? 1 : 0, c->d_err, c->d_flags};
            // with a certification, the pixels of untrusted cells go to the exact posterior
            hb::MlpRoute rt = c->route;
            hb::PosteriorGate gate{c->d_flags + 2};
            // every learned frame clears the next frame's counter, routed or not, so that
            // each frame starts its list from zero
            rt.next_count = c->d_flags + 4 + ((seq + 1u) & 1u);
            if (rt.trust) {
                rt.list = c->d_route + b.ll_off;
                rt.count = c->d_flags + 4 + (seq & 1u);
                gate.list = rt.list;
                gate.count = rt.count;
                gate.listed_total = reinterpret_cast<unsigned long long*>(c->d_flags + 6);
            }
            if (img)
                e = hb::launch_mlp_forward_check(img, c->mlp_norm, c->d_ybar_f + 3 * b.ll_off, b.npix, chat,
                                                 conc_scaled, scale, c->bp, rec, ck, rt, pdl, s);
            if (e == cudaSuccess)
                e = hb::launch_posterior(c->bp, rec, b.npix, post_scratch(c, b.ll_off), chat, conc_scaled, scale, pdl,
                                         s, gate);
            c->launches += 2;
            c->mlp_frames++;
        } else {
            e = hb::launch_posterior(c->bp, rec, b.npix, post_scratch(c, b.ll_off), chat, conc_scaled, scale, pdl,
                                     s);
            c->launches++;
        }
    }
    if (e != cudaSuccess) return HB_ERR_CUDA;
    if (out0 || out1) {
        StageTimer t(c, s, HB_STAGE_SYNTHESIS);
        e = hb::launch_synthesis(b.tp, frame, stride, c->d_lut, chat, out0, out1, debug, lowpass && pdl, s);
        c->launches++;
    }
    return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status run_frame(hb_ctx* c, const void* frame, size_t stride, double* ybar, float* out0, float* out1,
                    float2* conc_scaled, int debug, cudaStream_t s) {
    return run_band(c, whole_frame(c), frame, stride, ybar, out0, out1, conc_scaled, debug, s, true);
}

}  // namespace

extern "C" {

hb_status hb_create(const hb_mixing* mix, const hb_grid* grid, int levels, double lambda, int width, int height,
                    int in_format, unsigned flags, hb_ctx** out) {
    if (!out) return HB_ERR_ARG;
    *out = nullptr;
    if (!mix || !grid) return HB_ERR_ARG;
    if (in_format != HB_IN_F32_HWC && in_format != HB_IN_U8_HWC) return HB_ERR_ARG;
    if (flags & ~(unsigned)(HB_LAMBDA_ABSOLUTE | HB_LOWPASS_TIKHONOV | HB_FULL_GRID | HB_ILLUMINATION |
                            HB_LOWPASS_INTENSITY | HB_LOWPASS_LS | HB_NODE_SUMS))
        return HB_ERR_ARG;
    if ((flags & HB_LOWPASS_INTENSITY) && ((flags & HB_LOWPASS_TIKHONOV) || levels > 4)) return HB_ERR_ARG;
    if ((flags & HB_LOWPASS_LS) && (flags & HB_LOWPASS_TIKHONOV)) return HB_ERR_ARG;
    if (width <= 0 || height <= 0 || levels < 0 || levels > hb::kMaxLevels) return HB_ERR_SHAPE;
    if (grid->n0 < 1 || grid->n1 < 1 || !(grid->hi0 >= grid->lo0) || !(grid->hi1 >= grid->lo1) ||
        !(grid->sigma_l > 0.0))
        return HB_ERR_SHAPE;
    if (levels == 0 && (flags & HB_LOWPASS_TIKHONOV)) return HB_ERR_ARG;
    if (!std::isfinite(lambda) || lambda < 0.0) return HB_ERR_ARG;
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 2; ++j)
            if (!std::isfinite(mix->A[c][j])) return HB_ERR_ARG;

    hb_ctx* c = new (std::nothrow) hb_ctx();
    if (!c) return HB_ERR_OOM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return HB_ERR_CUDA;
    }
    c->W = width;
    c->H = height;
    c->levels = levels;
    c->fmt = in_format;
    c->flags = flags;
    const int B = 1 << levels;
    c->hl = (height + B - 1) / B;
    c->wl = (width + B - 1) / B;
    c->npix_ll = (long)c->hl * c->wl;
    c->sigma_l = grid->sigma_l;
    prepare(c, mix, grid, lambda);

    TransformParams& tp = c->tp;
    tp.H = height;
    tp.W = width;
    tp.levels = levels;
    tp.fmt = in_format;
    tp.eps = 1e-6f;
    const int Wp = c->wl * B;
    int tw = 2048 / B;
    if (tw < B) tw = B;
    if (tw > Wp) tw = Wp;
    tp.tile_w = tw;
    tp.hl = c->hl;
    tp.wl = c->wl;
    tp.tikhonov_lowpass = (flags & HB_LOWPASS_TIKHONOV) ? 1 : 0;
    tp.ll_intensity = (flags & HB_LOWPASS_INTENSITY) ? 1 : 0;

    float2 lut[256];
    for (int k = 0; k < 256; ++k) {
        const double y = -std::log((double)(k > 0 ? k : 1) / 255.0);
        const float hi = (float)y;
        lut[k] = make_float2(hi, (float)(y - (double)hi));
    }
    hb_status st = HB_OK;
    if (cudaMalloc(&c->d_lut, sizeof(lut)) != cudaSuccess) st = HB_ERR_OOM;
    if (st == HB_OK && cudaMemcpy(c->d_lut, lut, sizeof(lut), cudaMemcpyHostToDevice) != cudaSuccess) st = HB_ERR_CUDA;
    if (st == HB_OK) st = ensure_rec(c, c->npix_ll);
    std::vector<float4> rowtab;
    if (st == HB_OK && !(flags & HB_NODE_SUMS) && hb::row_table(c->bp, rowtab)) {
        if (cudaMalloc(&c->d_rowtab, sizeof(float4) * rowtab.size()) != cudaSuccess) st = HB_ERR_OOM;
        if (st == HB_OK && cudaMemcpy(c->d_rowtab, rowtab.data(), sizeof(float4) * rowtab.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess)
            st = HB_ERR_CUDA;
        if (st == HB_OK) c->bp.row_tab = c->d_rowtab;
    }
    if (st != HB_OK) {
        cudaGetLastError();
        hb_destroy(c);
        return st;
    }
    *out = c;
    return HB_OK;
}

void hb_destroy(hb_ctx* c) {
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    cudaFree(c->d_lut);
    cudaFree(c->d_rec);
    cudaFree(c->d_chat);
    cudaFree(c->d_partial);
    cudaFree(c->d_count);
    cudaFree(c->d_mlp);
    cudaFree(c->d_mlp_img);
    cudaFree(c->d_mlp_gpart);
    cudaFree(c->d_mlp_lpart);
    cudaFree(c->d_mlp_loss);
    cudaFree(c->d_ybar_f);
    cudaFree(c->d_flags);
    cudaFree(c->d_err);
    cudaFree(c->d_route);
    cudaFree(c->d_trust);
    cudaFree(c->d_nodes);
    cudaFree(c->d_rowtab);
    cudaFree(c->d_frame);
    cudaFree(c->d_thb);
    cudaFree(c->d_so2);
    cudaFree(c->d_frame2);
    cudaFree(c->d_thb2);
    cudaFree(c->d_so22);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->host_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->set_free)
        if (e) cudaEventDestroy(e);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    if (c->s_alt) cudaStreamDestroy(c->s_alt);
    if (c->s_c0) cudaStreamDestroy(c->s_c0);
    if (c->hg_exec) cudaGraphExecDestroy(c->hg_exec);
    cudaGetLastError();
    delete c;
}

hb_status hb_estimate(hb_ctx* c, const void* frame_dev, size_t row_stride_bytes, float* thb_dev, float* so2_dev,
                      void* stream) {
    if (!c || !thb_dev || !so2_dev) return HB_ERR_ARG;
    hb_status st = check_frame_args(c, frame_dev, row_stride_bytes);
    if (st != HB_OK) return st;
    DeviceGuard g(c->device);
    hb::NvtxRange r("hb_estimate");
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    return run_frame(c, frame_dev, row_stride_bytes, nullptr, thb_dev, so2_dev, nullptr, 0,
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Staging buffers of one host call: the frame, THb and SO2 on the device.
struct HostSet {
    unsigned char* frame;
    float* thb;
    float* so2;
};

// Everything of one host call in stream order.  Synchronous calls (async = false): the side
// streams start after the work queued earlier on s, the even bands compute on s, and every
// side stream is joined back into s (so that the sequence can also be captured as a graph).
// Asynchronous calls: nothing waits for s; the input copies wait until the staging set's
// previous frame has finished its output copies (free_set), the even bands compute on s_c0,
// and free_set is recorded after the last output copy, which s then waits for.  Band k always
// computes on the same stream, so the low-pass records and estimates of a band, shared by
// successive frames, are reused in stream order.
hb_status enqueue_host_bands(hb_ctx* c, const void* frame_host, size_t row_stride_bytes, float* thb_host,
                             float* so2_host, cudaStream_t s, const int* bounds, int nb, const HostSet& set,
                             bool async, cudaEvent_t free_set) {
    const int TH = 1 << c->levels;
    const size_t row = (size_t)c->W * 3 * elem_size(c->fmt);
    cudaEvent_t ev_start = c->host_ev[2 * nb], ev_alt = c->host_ev[2 * nb + 1], ev_out = c->host_ev[2 * nb + 2];
    if (async) {
        if (cudaStreamWaitEvent(c->s_in, free_set, 0) != cudaSuccess) return HB_ERR_CUDA;
    } else if (cudaEventRecord(ev_start, s) != cudaSuccess || cudaStreamWaitEvent(c->s_in, ev_start, 0) ||
               cudaStreamWaitEvent(c->s_out, ev_start, 0) || cudaStreamWaitEvent(c->s_alt, ev_start, 0)) {
        // the staging buffers may still be in use by work queued earlier on s
        return HB_ERR_CUDA;
    }
    const unsigned char* fh = static_cast<const unsigned char*>(frame_host);
    for (int k = 0; k < nb; ++k) {
        const int r0 = bounds[k] * TH, r1 = std::min(c->H, bounds[k + 1] * TH);
        if (cudaMemcpy2DAsync(set.frame + (size_t)r0 * row, row, fh + (size_t)r0 * row_stride_bytes,
                              row_stride_bytes, row, r1 - r0, cudaMemcpyHostToDevice, c->s_in) != cudaSuccess ||
            cudaEventRecord(c->host_ev[2 * k], c->s_in) != cudaSuccess)
            return HB_ERR_CUDA;
    }
    for (int k = 0; k < nb; ++k) {
        const int b0 = bounds[k], b1 = bounds[k + 1];
        const int r0 = b0 * TH, r1 = std::min(c->H, b1 * TH);
        Band b = whole_frame(c);
        b.tp.H = r1 - r0;
        b.tp.hl = b1 - b0;
        b.ll_off = (long)b0 * c->wl;
        b.npix = (long)(b1 - b0) * c->wl;
        const size_t o = (size_t)r0 * c->W, n = (size_t)(r1 - r0) * c->W;
        // alternate bands between two compute streams: neighbouring bands share no data, and
        // one band's kernels fill the ramp and tail of the other's
        cudaStream_t cs = (k & 1) ? c->s_alt : (async ? c->s_c0 : s);
        if (cudaStreamWaitEvent(cs, c->host_ev[2 * k], 0) != cudaSuccess) return HB_ERR_CUDA;
        hb_status st = run_band(c, b, set.frame + (size_t)r0 * row, row, nullptr, set.thb + o, set.so2 + o, nullptr, 0,
                                cs);
        if (st != HB_OK) return st;
        if (cudaEventRecord(c->host_ev[2 * k + 1], cs) != cudaSuccess ||
            cudaStreamWaitEvent(c->s_out, c->host_ev[2 * k + 1], 0) != cudaSuccess ||
            cudaMemcpyAsync(thb_host + o, set.thb + o, n * 4, cudaMemcpyDeviceToHost, c->s_out) != cudaSuccess ||
            cudaMemcpyAsync(so2_host + o, set.so2 + o, n * 4, cudaMemcpyDeviceToHost, c->s_out) != cudaSuccess)
            return HB_ERR_CUDA;
    }
    if (async) {  // every band's output copy follows its kernels, so s_out's end covers all
        if (cudaEventRecord(free_set, c->s_out) != cudaSuccess || cudaStreamWaitEvent(s, free_set, 0) != cudaSuccess)
            return HB_ERR_CUDA;
        return HB_OK;
    }
    // later work on s is ordered after every band and every copy
    if (cudaEventRecord(ev_alt, c->s_alt) != cudaSuccess || cudaStreamWaitEvent(s, ev_alt, 0) != cudaSuccess ||
        cudaEventRecord(ev_out, c->s_out) != cudaSuccess || cudaStreamWaitEvent(s, ev_out, 0) != cudaSuccess)
        return HB_ERR_CUDA;
    return HB_OK;
}

// What both host entry points need: arguments checked, staging sets (two for asynchronous
// calls), side streams and events created, and the band bounds.
// Bands of whole superblock rows, pipelined: band k's frame rows go up on s_in while band
// k-1 computes (on an even-band stream or s_alt) and band k-2's THb/SO2 rows come back on
// s_out.  The learned low pass takes the whole frame at once (its fallback decision is per
// frame).  Bands are used only where every band's posterior takes the two-pixel kernel, as
// the whole frame's does: each pixel's result is then the same as in hb_estimate.  The first
// band is kept small, so that the first output copy starts early: the fewest superblock
// rows that still take the two-pixel posterior (or a 2*kHostBands-th of the frame without a
// posterior); the other rows are shared evenly among the other bands, none smaller than the
// first.
hb_status host_prepare(hb_ctx* c, const void* frame_host, size_t row_stride_bytes, const float* thb_host,
                       const float* so2_host, bool two_sets, int max_bands, int* bounds, int& nb, bool& mlp) {
    if (!c || !frame_host || !thb_host || !so2_host) return HB_ERR_ARG;
    const size_t row = (size_t)c->W * 3 * elem_size(c->fmt);
    if (row_stride_bytes < row) return HB_ERR_ARG;
    const size_t npx = (size_t)c->W * c->H;
    auto alloc = [&](void*& f, float*& t, float*& o) {
        if (f) return true;
        if (cudaMalloc(&f, row * c->H) == cudaSuccess && cudaMalloc(&t, npx * 4) == cudaSuccess &&
            cudaMalloc(&o, npx * 4) == cudaSuccess)
            return true;
        cudaGetLastError();
        cudaFree(f);
        cudaFree(t);
        cudaFree(o);
        f = nullptr;
        t = nullptr;
        o = nullptr;
        return false;
    };
    if (!alloc(c->d_frame, c->d_thb, c->d_so2) || (two_sets && !alloc(c->d_frame2, c->d_thb2, c->d_so22)))
        return HB_ERR_OOM;
    const bool bayes = !(c->flags & (HB_LOWPASS_TIKHONOV | HB_LOWPASS_LS));
    mlp = bayes && c->lowpass_mode != HB_MODE_BAYES;
    bounds[0] = 0;
    bounds[1] = c->hl;
    nb = 1;
    if (!mlp && max_bands > 1) {
        int first = std::max(1, c->hl / (2 * max_bands));
        if (bayes)
            while (first < c->hl && !hb::posterior_uses_pairs(c->bp, (long)first * c->wl)) ++first;
        const int rest = c->hl - first;
        int m = std::min(max_bands - 1, first > 0 ? rest / first : 0);
        if (m >= 1) {
            nb = m + 1;
            bounds[1] = first;
            for (int k = 1; k <= m; ++k) bounds[k + 1] = first + (int)((long)rest * k / m);
        }
    }
    if (!c->s_in) {
        if (cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->s_alt, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return HB_ERR_CUDA;
        }
    }
    if (two_sets && !c->s_c0) {
        if (cudaStreamCreateWithFlags(&c->s_c0, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->set_free[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->set_free[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return HB_ERR_CUDA;
        }
    }
    while ((int)c->host_ev.size() < 2 * kHostBands + 3) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HB_ERR_CUDA;
        c->host_ev.push_back(e);
    }
    return HB_OK;
}

}  // namespace

extern "C" {

hb_status hb_estimate_host(hb_ctx* c, const void* frame_host, size_t row_stride_bytes, float* thb_host,
                           float* so2_host, void* stream) {
    if (!c) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    hb::NvtxRange r("hb_estimate_host");
    int bounds[kHostBands + 1];
    int nb = 1;
    bool mlp = false;
    hb_status pst =
        host_prepare(c, frame_host, row_stride_bytes, thb_host, so2_host, false, kHostBands, bounds, nb, mlp);
    if (pst != HB_OK) return pst;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    const HostSet set{static_cast<unsigned char*>(c->d_frame), c->d_thb, c->d_so2};
    // The same buffers, stream and banding twice in a row: capture the sequence as a CUDA
    // graph, then replay it (one launch instead of some twenty calls).  Not for the learned
    // low pass (whose sampled pixels change per frame), nor with stage timing armed, nor on
    // the legacy default stream (which cannot be captured).
    const HostKey key{frame_host, row_stride_bytes, thb_host, so2_host, s, bounds[1], nb};
    const bool graphable = !mlp && !c->timing && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
    if (graphable && c->hg_exec && c->hg_key == key) {
        if (cudaGraphLaunch(c->hg_exec, s) != cudaSuccess) return HB_ERR_CUDA;
        c->launches += c->hg_kernels;
        return cudaStreamSynchronize(s) == cudaSuccess ? HB_OK : HB_ERR_CUDA;
    }
    if (graphable && c->hg_seen && c->hg_key == key) {
        const long before = c->launches.load();
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return HB_ERR_CUDA;
        hb_status st =
            enqueue_host_bands(c, frame_host, row_stride_bytes, thb_host, so2_host, s, bounds, nb, set, false, nullptr);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(s, &graph);
        const long kernels = c->launches.load() - before;
        c->launches -= kernels;  // captured, not run
        cudaGraphExec_t exec = nullptr;
        if (st == HB_OK && ee == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            if (c->hg_exec) cudaGraphExecDestroy(c->hg_exec);
            c->hg_exec = exec;
            c->hg_kernels = kernels;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (c->hg_exec && c->hg_key == key && exec) {
            if (cudaGraphLaunch(c->hg_exec, s) != cudaSuccess) return HB_ERR_CUDA;
            c->launches += c->hg_kernels;
            return cudaStreamSynchronize(s) == cudaSuccess ? HB_OK : HB_ERR_CUDA;
        }
        c->hg_seen = false;  // capture failed: stay eager
        if (st != HB_OK) return st;
    } else {
        if (c->hg_exec && !(c->hg_key == key)) {  // a graph of other buffers: drop it
            cudaGraphExecDestroy(c->hg_exec);
            c->hg_exec = nullptr;
        }
        c->hg_key = key;
        c->hg_seen = graphable;
    }
    hb_status st =
        enqueue_host_bands(c, frame_host, row_stride_bytes, thb_host, so2_host, s, bounds, nb, set, false, nullptr);
    if (st != HB_OK) return st;
    return cudaStreamSynchronize(s) == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status hb_estimate_host_async(hb_ctx* c, const void* frame_host, size_t row_stride_bytes, float* thb_host,
                                 float* so2_host, void* stream) {
    if (!c) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    hb::NvtxRange r("hb_estimate_host_async");
    if (c->timing) return HB_ERR_STATE;
    int bounds[kHostBands + 1];
    int nb = 1;
    bool mlp = false;
    hb_status pst =
        host_prepare(c, frame_host, row_stride_bytes, thb_host, so2_host, true, kAsyncBands, bounds, nb, mlp);
    if (pst != HB_OK) return pst;
    const int j = c->set_next;
    const HostSet set = j == 0 ? HostSet{static_cast<unsigned char*>(c->d_frame), c->d_thb, c->d_so2}
                               : HostSet{static_cast<unsigned char*>(c->d_frame2), c->d_thb2, c->d_so22};
    hb_status st = enqueue_host_bands(c, frame_host, row_stride_bytes, thb_host, so2_host,
                                      static_cast<cudaStream_t>(stream), bounds, nb, set, true, c->set_free[j]);
    c->async_pending = true;
    if (st != HB_OK) return st;
    c->set_next = j ^ 1;
    return HB_OK;
}

hb_status hb_estimate_debug(hb_ctx* c, const void* frame_dev, size_t row_stride_bytes, double* ybar_dev,
                            float* conc_dev, float* hbo2_dev, float* hb_dev, void* stream) {
    if (!c) return HB_ERR_ARG;
    if ((hbo2_dev == nullptr) != (hb_dev == nullptr)) return HB_ERR_ARG;
    if (conc_dev && (reinterpret_cast<uintptr_t>(conc_dev) & 7)) return HB_ERR_ARG;
    hb_status st = check_frame_args(c, frame_dev, row_stride_bytes);
    if (st != HB_OK) return st;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    return run_frame(c, frame_dev, row_stride_bytes, ybar_dev, hbo2_dev, hb_dev, reinterpret_cast<float2*>(conc_dev),
                     1, static_cast<cudaStream_t>(stream));
}

hb_status hb_posterior_mean(hb_ctx* c, const double* ybar_dev, long npix, float* conc_dev, void* stream) {
    if (!c || npix < 0) return HB_ERR_ARG;
    if (npix == 0) return HB_OK;
    if (!ybar_dev || !conc_dev || (reinterpret_cast<uintptr_t>(conc_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(ybar_dev) & 7))
        return HB_ERR_ARG;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (npix > c->rec_cap) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return HB_ERR_CUDA;
        hb_status st = ensure_rec(c, npix);
        if (st != HB_OK) return st;
    }
    cudaError_t e = hb::launch_setup(c->bp, ybar_dev, npix, c->d_rec, s);
    c->launches++;
    if (e != cudaSuccess) return HB_ERR_CUDA;
    StageTimer t(c, s, HB_STAGE_LOWPASS);
    e = hb::launch_posterior(c->bp, c->d_rec, npix, post_scratch(c), reinterpret_cast<float2*>(conc_dev), nullptr, 1.f,
                             false, s);
    c->launches++;
    return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status hb_lowpass_shape(const hb_ctx* c, int* hl, int* wl) {
    if (!c || !hl || !wl) return HB_ERR_ARG;
    *hl = c->hl;
    *wl = c->wl;
    return HB_OK;
}

long hb_launch_count(const hb_ctx* c) { return c ? c->launches.load() : 0; }

hb_status hb_timing_start(hb_ctx* c, int max_launches) {
    if (!c || max_launches <= 0) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    while ((int)c->ev.size() < 2 * max_launches) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return HB_ERR_CUDA;
        c->ev.push_back(e);
    }
    c->ev_stage.assign(c->ev.size() / 2, -1);
    if (!c->d_nodes && cudaMalloc(&c->d_nodes, 3 * sizeof(unsigned long long)) != cudaSuccess) {
        c->d_nodes = nullptr;
        cudaGetLastError();
        return HB_ERR_OOM;
    }
    if (cudaMemset(c->d_nodes, 0, 3 * sizeof(unsigned long long)) != cudaSuccess) return HB_ERR_CUDA;
    c->ev_used = 0;
    c->timing = true;
    return HB_OK;
}

hb_status hb_timing_nodes(hb_ctx* c, unsigned long long* nodes) {
    if (!c || !nodes) return HB_ERR_ARG;
    if (!c->timing || !c->d_nodes) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(nodes, c->d_nodes, sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HB_ERR_CUDA;
    return HB_OK;
}

hb_status hb_timing_rows(hb_ctx* c, unsigned long long rows[2]) {
    if (!c || !rows) return HB_ERR_ARG;
    if (!c->timing || !c->d_nodes) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(rows, c->d_nodes + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HB_ERR_CUDA;
    return HB_OK;
}

hb_status hb_timing_read(hb_ctx* c, double ms[HB_NUM_STAGES], long launches[HB_NUM_STAGES]) {
    if (!c || !ms || !launches) return HB_ERR_ARG;
    if (!c->timing) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    for (int k = 0; k < HB_NUM_STAGES; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    hb_status st = HB_OK;
    for (int i = 0; i < c->ev_used; ++i) {
        float t = 0.f;
        if (cudaEventSynchronize(c->ev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&t, c->ev[2 * i], c->ev[2 * i + 1]) != cudaSuccess) {
            st = HB_ERR_CUDA;
            break;
        }
        ms[c->ev_stage[i]] += t;
        launches[c->ev_stage[i]] += 1;
    }
    c->timing = false;
    c->ev_used = 0;
    return st;
}

// ------------------------------------------------------------------------------------
// Learned stand-in: parameters, training, inference and the low-pass mode.
// ------------------------------------------------------------------------------------
namespace {

constexpr int kMlpMaxBlocks = 1024;  // batch <= 65536 samples (64 per training CTA)
#ifndef HB_MLP_INPUT_SCALE
#define HB_MLP_INPUT_SCALE 4.0
#endif

float bf16_round(float v) {  // round to nearest even on the upper 16 bits
    uint32_t u;
    std::memcpy(&u, &v, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return v;
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    std::memcpy(&v, &u, 4);
    return v;
}

uint64_t splitmix64(uint64_t& x) {  // Steele, Lea and Flood's SplitMix64 output function
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr int kMlpFlags = 8;

hb_status ensure_mlp(hb_ctx* c) {
    if (c->d_mlp) return HB_OK;
    // the baseline needs a box with an extent on both axes
    if (c->bp.n0 < 2 || c->bp.n1 < 2 || !(c->bp.hi0 > c->bp.lo0) || !(c->bp.hi1 > c->bp.lo1)) return HB_ERR_STATE;
    const size_t np = hb::kNParams;
    if (cudaMalloc(&c->d_mlp, sizeof(float) * 5 * np) != cudaSuccess ||
        cudaMalloc(&c->d_mlp_img, hb::mlp_image_bytes()) != cudaSuccess ||
        cudaMalloc(&c->d_mlp_gpart, sizeof(float) * kMlpMaxBlocks * np) != cudaSuccess ||
        cudaMalloc(&c->d_mlp_lpart, sizeof(float) * kMlpMaxBlocks) != cudaSuccess ||
        cudaMalloc(&c->d_ybar_f, sizeof(float) * 3 * c->npix_ll) != cudaSuccess ||
        cudaMalloc(&c->d_flags, sizeof(unsigned) * kMlpFlags) != cudaSuccess ||
        cudaMalloc(&c->d_route, sizeof(int) * c->npix_ll) != cudaSuccess) {
        cudaGetLastError();
        return HB_ERR_OOM;
    }
    if (cudaMemset(c->d_mlp, 0, sizeof(float) * 5 * np) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, sizeof(unsigned) * kMlpFlags) != cudaSuccess)
        return HB_ERR_CUDA;
    // least-squares baseline, input transform and output scale (FP64 here)
    const double* A = c->bp.A;
    const double lo[2] = {c->bp.lo0, c->bp.lo1}, hi[2] = {c->bp.hi0, c->bp.hi1};
    double G[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) G[j][k] = A[0 + j] * A[0 + k] + A[2 + j] * A[2 + k] + A[4 + j] * A[4 + k];
    const double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
    if (!(det > 0)) return HB_ERR_STATE;  // collinear columns: no least-squares baseline
    const double Gi[2][2] = {{G[1][1] / det, -G[0][1] / det}, {-G[1][0] / det, G[0][0] / det}};
    double P[2][3];
    for (int ch = 0; ch < 3; ++ch) {
        P[0][ch] = Gi[0][0] * A[ch * 2] + Gi[0][1] * A[ch * 2 + 1];
        P[1][ch] = Gi[1][0] * A[ch * 2] + Gi[1][1] * A[ch * 2 + 1];
    }
    hb::MlpNorm& nm = c->mlp_norm;
    const double K = HB_MLP_INPUT_SCALE;  // the box maps to [-K, K]
    for (int j = 0; j < 2; ++j) {
        const double half = hi[j] > lo[j] ? 0.5 * (hi[j] - lo[j]) : 1.0, centre = 0.5 * (lo[j] + hi[j]);
        for (int ch = 0; ch < 3; ++ch) {
            nm.Ap[j * 3 + ch] = (float)P[j][ch];
            nm.T[j * 3 + ch] = (float)(K * P[j][ch] / half);
        }
        nm.t0[j] = (float)(-K * centre / half);
    }
    // unit normal of the range of A (cross product of its columns), in sigma_l units
    const double nx = A[2] * A[5] - A[4] * A[3], ny = A[4] * A[1] - A[0] * A[5], nz = A[0] * A[3] - A[2] * A[1];
    const double nn = std::sqrt(nx * nx + ny * ny + nz * nz), sl = c->sigma_l;
    nm.T[6] = (float)(nx / nn / sl);
    nm.T[7] = (float)(ny / nn / sl);
    nm.T[8] = (float)(nz / nn / sl);
    nm.t0[2] = 0.f;
    nm.lo0 = (float)lo[0];
    nm.hi0 = (float)hi[0];
    nm.lo1 = (float)lo[1];
    nm.hi1 = (float)hi[1];
    nm.osc0 = (float)(sl * std::sqrt(Gi[0][0]));
    nm.osc1 = (float)(sl * std::sqrt(Gi[1][1]));
    // the baseline's four edges (see MlpNorm): S = sl^2 Gi, v_e = sgn_e S[:, axis] / s_axis
    for (int e = 0; e < 4; ++e) {
        const int ax = e / 2;
        const double sgn = (e & 1) ? -1.0 : 1.0, pos = (e & 1) ? -hi[ax] : lo[ax];
        const double sa = sl * std::sqrt(Gi[ax][ax]);
        nm.edge_sgn[e] = (float)sgn;
        nm.edge_pos[e] = (float)pos;
        nm.edge_inv_s[e] = (float)(1.0 / sa);
        nm.edge_v0[e] = (float)(sgn * sl * sl * Gi[0][ax] / sa);
        nm.edge_v1[e] = (float)(sgn * sl * sl * Gi[1][ax] / sa);
    }
    c->mlp_ext0 = hi[0] > lo[0] ? (float)(hi[0] - lo[0]) : 1.f;
    c->mlp_ext1 = hi[1] > lo[1] ? (float)(hi[1] - lo[1]) : 1.f;
    return HB_OK;
}

constexpr int kMlpMaxSample = 1 << 24;  // drawn pixels per frame of the learned mode's check
constexpr int kTrustCells = 128;        // certification map: cells per axis
constexpr double kTrustPad = 3.0;       // ... over the box widened by 3 standard deviations

// Network files (hb_mlp_save / hb_mlp_load): header, model, parameters, hash.
constexpr unsigned char kMlpMagic[8] = {'H', 'B', 'M', 'L', 'P', 'v', '1', '\n'};
constexpr int kMlpModelValues = 11;  // A (6), lo0, hi0, lo1, hi1, sigma_l
constexpr size_t kMlpFileBytes = 16 + 8 * kMlpModelValues + 4 * (size_t)hb::kNParams + 4;

// The model a network is trained for, in file order.
void mlp_model(const hb_ctx* c, double (&m)[kMlpModelValues]) {
    for (int k = 0; k < 6; ++k) m[k] = c->bp.A[k];
    m[6] = c->bp.lo0;
    m[7] = c->bp.hi0;
    m[8] = c->bp.lo1;
    m[9] = c->bp.hi1;
    m[10] = c->sigma_l;
}

void put_le(std::vector<unsigned char>& b, uint64_t v, int bytes) {
    for (int k = 0; k < bytes; ++k) b.push_back((unsigned char)(v >> (8 * k)));
}

uint64_t get_le(const unsigned char* q, int bytes) {
    uint64_t v = 0;
    for (int k = 0; k < bytes; ++k) v |= (uint64_t)q[k] << (8 * k);
    return v;
}

uint32_t fnv1a(const unsigned char* q, size_t n) {  // 32-bit FNV-1a (Fowler, Noll, Vo)
    uint32_t h = 2166136261u;
    for (size_t k = 0; k < n; ++k) h = (h ^ q[k]) * 16777619u;
    return h;
}

// Upload masters, refresh the BF16 copies, zero the Adam state.
hb_status put_params(hb_ctx* c, const float* host) {
    const size_t np = hb::kNParams;
    std::vector<float> buf(5 * np, 0.f);
    for (size_t i = 0; i < np; ++i) {
        buf[i] = host[i];
        buf[3 * np + i] = bf16_round(host[i]);
    }
    if (cudaMemcpy(c->d_mlp, buf.data(), sizeof(float) * 5 * np, cudaMemcpyHostToDevice) != cudaSuccess)
        return HB_ERR_CUDA;
    c->adam_t = 0;
    c->mlp_ready = true;
    c->mlp_img_dirty = true;
    c->route.trust = nullptr;  // a certification holds only for the parameters it checked
    return HB_OK;
}

}  // namespace



hb_status hb_mlp_init(hb_ctx* c, unsigned seed) {
    if (!c) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    hb_status st = ensure_mlp(c);
    if (st != HB_OK) return st;
    std::vector<float> p(hb::kNParams, 0.f);
    uint64_t state = 0x6a09e667f3bcc909ull ^ (uint64_t)seed;
    auto fill = [&](int off, int fan_out, int fan_in) {
        const double b = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_out * fan_in; ++i) {
            const double u = (double)(splitmix64(state) >> 11) * (1.0 / 9007199254740992.0);
            p[off + i] = (float)((2.0 * u - 1.0) * b);
        }
    };
    fill(hb::kOffW1, hb::kHid, hb::kIn);
    fill(hb::kOffW2, hb::kHid, hb::kHid);
    fill(hb::kOffW3, hb::kOut, hb::kHid);
    return put_params(c, p.data());
}

hb_status hb_mlp_set_params(hb_ctx* c, const float* params_host) {
    if (!c || !params_host) return HB_ERR_ARG;
    for (int i = 0; i < hb::kNParams; ++i)
        if (!std::isfinite(params_host[i])) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    hb_status st = ensure_mlp(c);
    if (st != HB_OK) return st;
    return put_params(c, params_host);
}

hb_status hb_mlp_get_params(hb_ctx* c, float* params_host) {
    if (!c || !params_host) return HB_ERR_ARG;
    if (!c->mlp_ready) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    return cudaMemcpy(params_host, c->d_mlp, sizeof(float) * hb::kNParams, cudaMemcpyDeviceToHost) == cudaSuccess
               ? HB_OK
               : HB_ERR_CUDA;
}

hb_status hb_mlp_save(hb_ctx* c, const char* path) {
    if (!c || !path) return HB_ERR_ARG;
    if (!c->mlp_ready) return HB_ERR_STATE;
    std::vector<float> p(hb::kNParams);
    hb_status st = hb_mlp_get_params(c, p.data());
    if (st != HB_OK) return st;
    std::vector<unsigned char> buf;
    buf.reserve(kMlpFileBytes);
    buf.insert(buf.end(), kMlpMagic, kMlpMagic + 8);
    put_le(buf, (uint64_t)hb::kNParams, 4);
    put_le(buf, 0, 4);
    double model[kMlpModelValues];
    mlp_model(c, model);
    for (double v : model) {
        uint64_t u;
        std::memcpy(&u, &v, 8);
        put_le(buf, u, 8);
    }
    for (float v : p) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        put_le(buf, u, 4);
    }
    put_le(buf, fnv1a(buf.data(), buf.size()), 4);
    std::FILE* f = std::fopen(path, "wb");
    if (!f) return HB_ERR_IO;
    const bool ok = std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    return (std::fclose(f) == 0 && ok) ? HB_OK : HB_ERR_IO;
}

hb_status hb_mlp_load(hb_ctx* c, const char* path) {
    if (!c || !path) return HB_ERR_ARG;
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return HB_ERR_IO;
    std::vector<unsigned char> buf(kMlpFileBytes + 1);
    const size_t got = std::fread(buf.data(), 1, buf.size(), f);
    std::fclose(f);
    if (got != kMlpFileBytes) return HB_ERR_IO;  // shorter, or longer than a network file
    const unsigned char* q = buf.data();
    if (std::memcmp(q, kMlpMagic, 8) != 0 || get_le(q + 8, 4) != (uint64_t)hb::kNParams || get_le(q + 12, 4) != 0 ||
        get_le(q + kMlpFileBytes - 4, 4) != fnv1a(q, kMlpFileBytes - 4))
        return HB_ERR_IO;
    double model[kMlpModelValues];
    mlp_model(c, model);
    for (int k = 0; k < kMlpModelValues; ++k) {
        const uint64_t u = get_le(q + 16 + 8 * k, 8);
        double v;
        std::memcpy(&v, &u, 8);
        if (!(v == model[k])) return HB_ERR_STATE;
    }
    std::vector<float> p(hb::kNParams);
    for (int i = 0; i < hb::kNParams; ++i) {
        const uint32_t u = (uint32_t)get_le(q + 16 + 8 * kMlpModelValues + 4 * i, 4);
        std::memcpy(&p[i], &u, 4);
        if (!std::isfinite(p[i])) return HB_ERR_IO;
    }
    return hb_mlp_set_params(c, p.data());
}

hb_status hb_lowpass_pairs(hb_ctx* c, const void* frame_dev, size_t row_stride_bytes, float* ybar_dev,
                           float* conc_dev, void* stream) {
    if (!c || !ybar_dev || !conc_dev || (reinterpret_cast<uintptr_t>(conc_dev) & 7)) return HB_ERR_ARG;
    hb_status st = check_frame_args(c, frame_dev, row_stride_bytes);
    if (st != HB_OK) return st;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = hb::launch_analysis(c->tp, c->bp, frame_dev, row_stride_bytes, c->d_lut, nullptr, c->d_rec, s,
                                        ybar_dev);
    c->launches++;
    if (e == cudaSuccess)
        e = hb::launch_posterior(c->bp, c->d_rec, c->npix_ll, post_scratch(c), reinterpret_cast<float2*>(conc_dev),
                                 nullptr, 1.f, false, s);
    c->launches++;
    return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status hb_mlp_train(hb_ctx* c, const float* ybar_dev, const float* target_dev, long n, int steps, int batch,
                       double lr, unsigned seed, float* loss_host, void* stream) {
    if (!c || !ybar_dev || !target_dev || n <= 0 || steps < 0 || batch <= 0 || !(lr > 0.0)) return HB_ERR_ARG;
    if (batch > kMlpMaxBlocks * hb::kMlpTrainSamples) return HB_ERR_SHAPE;
    if (!c->mlp_ready) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (steps > c->mlp_loss_cap) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return HB_ERR_CUDA;
        cudaFree(c->d_mlp_loss);
        c->d_mlp_loss = nullptr;
        c->mlp_loss_cap = 0;
        if (cudaMalloc(&c->d_mlp_loss, sizeof(float) * steps) != cudaSuccess) {
            cudaGetLastError();
            return HB_ERR_OOM;
        }
        c->mlp_loss_cap = steps;
    }
    const size_t np = hb::kNParams;
    float *master = c->d_mlp, *m = c->d_mlp + np, *v = c->d_mlp + 2 * np, *wbf = c->d_mlp + 3 * np,
          *grad = c->d_mlp + 4 * np;
    const int nblocks = (batch + hb::kMlpTrainSamples - 1) / hb::kMlpTrainSamples;
    for (int k = 0; k < steps; ++k) {
        cudaError_t e = hb::launch_mlp_train(wbf, c->mlp_norm, ybar_dev, target_dev, n, batch, seed, k, 0,
                                             c->d_mlp_gpart, c->d_mlp_lpart, s);
        if (e == cudaSuccess)
            e = hb::launch_mlp_adam(c->d_mlp_gpart, c->d_mlp_lpart, nblocks, batch, grad, c->d_mlp_loss + k, master,
                                    m, v, wbf, (float)lr, 0.9f, 0.999f, 1e-8f, ++c->adam_t, s);
        c->launches += 2;
        c->mlp_img_dirty = true;
        c->route.trust = nullptr;
        if (e != cudaSuccess) return HB_ERR_CUDA;
    }
    if (loss_host && steps > 0) {
        if (cudaMemcpyAsync(loss_host, c->d_mlp_loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HB_ERR_CUDA;
    }
    return HB_OK;
}

hb_status hb_mlp_gradient(hb_ctx* c, const float* ybar_dev, const float* target_dev, long n, float* grad_dev,
                          float* loss_dev, void* stream) {
    if (!c || !ybar_dev || !target_dev || !grad_dev || !loss_dev || n <= 0) return HB_ERR_ARG;
    if (n > (long)kMlpMaxBlocks * hb::kMlpTrainSamples) return HB_ERR_SHAPE;
    if (!c->mlp_ready) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t np = hb::kNParams;
    const int nblocks = (int)((n + hb::kMlpTrainSamples - 1) / hb::kMlpTrainSamples);
    cudaError_t e = hb::launch_mlp_train(c->d_mlp + 3 * np, c->mlp_norm, ybar_dev, target_dev, n, (int)n, 0, 0, 1,
                                         c->d_mlp_gpart, c->d_mlp_lpart, s);
    if (e == cudaSuccess)
        e = hb::launch_mlp_adam(c->d_mlp_gpart, c->d_mlp_lpart, nblocks, (int)n, grad_dev, loss_dev, nullptr,
                                nullptr, nullptr, nullptr, 0.f, 0.9f, 0.999f, 1e-8f, 1, s);
    c->launches += 2;
    return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status hb_mlp_forward(hb_ctx* c, const float* ybar_dev, long n, float* conc_dev, void* stream) {
    if (!c || !ybar_dev || !conc_dev || n < 0 || (reinterpret_cast<uintptr_t>(conc_dev) & 7)) return HB_ERR_ARG;
    if (!c->mlp_ready) return HB_ERR_STATE;
    if (n == 0) return HB_OK;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    const void* img = mlp_image(c, static_cast<cudaStream_t>(stream), e);
    if (img)
        e = hb::launch_mlp_forward(img, c->mlp_norm, ybar_dev, n, reinterpret_cast<float2*>(conc_dev), false,
                                   static_cast<cudaStream_t>(stream));
    c->launches++;
    return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

hb_status hb_set_lowpass_mode(hb_ctx* c, int mode, double tol, int nsample) {
    if (!c) return HB_ERR_ARG;
    if (mode != HB_MODE_BAYES && mode != HB_MODE_MLP && mode != HB_MODE_MLP_MEAN_GATE) return HB_ERR_ARG;
    {
        DeviceGuard g(c->device);
        if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    }
    if (mode != HB_MODE_BAYES) {
        if (!(tol >= 0.0) || nsample < 1 || nsample > kMlpMaxSample) return HB_ERR_ARG;
        if (!c->mlp_ready) return HB_ERR_STATE;
        if (c->flags & (HB_LOWPASS_TIKHONOV | HB_LOWPASS_LS | HB_ILLUMINATION | HB_LOWPASS_INTENSITY))
            return HB_ERR_STATE;
        if (nsample > c->mlp_err_cap) {
            DeviceGuard g(c->device);
            cudaFree(c->d_err);
            c->d_err = nullptr;
            c->mlp_err_cap = 0;
            if (cudaMalloc(&c->d_err, sizeof(float) * nsample) != cudaSuccess) {
                cudaGetLastError();
                return HB_ERR_OOM;
            }
            c->mlp_err_cap = nsample;
        }
        c->mlp_tol = (float)tol;
        c->mlp_nsample = nsample;
    }
    c->lowpass_mode = mode;
    return HB_OK;
}

hb_status hb_lowpass_stats(hb_ctx* c, long* mlp_frames, long* fallbacks, long* routed_pixels) {
    if (!c || !mlp_frames || !fallbacks) return HB_ERR_ARG;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    unsigned f[kMlpFlags] = {0};
    if (c->d_flags && cudaMemcpy(f, c->d_flags, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess) return HB_ERR_CUDA;
    unsigned long long routed = 0;
    std::memcpy(&routed, f + 6, sizeof(routed));
    *mlp_frames = c->mlp_frames;
    *fallbacks = f[1];
    if (routed_pixels) *routed_pixels = (long)routed;
    return HB_OK;
}

hb_status hb_mlp_certify(hb_ctx* c, double tol, double* trusted_fraction, void* stream) {
    if (!c || !(tol >= 0.0)) return HB_ERR_ARG;
    if (!c->mlp_ready) return HB_ERR_STATE;
    DeviceGuard g(c->device);
    if (settle_async(c) != HB_OK) return HB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The lattice: kTrustCells^2 cells over the box widened by kTrustPad standard deviations on
    // every side; points at every cell corner and centre, each with three values of the
    // component of ybar outside the range of A (-1.5, 0, 1.5 sigma_l), to which the exact
    // posterior is blind and the network should be.
    constexpr int K = kTrustCells;
    const hb::MlpNorm& nm = c->mlp_norm;
    const double sl = c->sigma_l;
    const double osc[2] = {nm.osc0, nm.osc1};
    const double lo[2] = {c->bp.lo0 - kTrustPad * osc[0], c->bp.lo1 - kTrustPad * osc[1]};
    const double hi[2] = {c->bp.hi0 + kTrustPad * osc[0], c->bp.hi1 + kTrustPad * osc[1]};
    const double cell[2] = {(hi[0] - lo[0]) / K, (hi[1] - lo[1]) / K};
    const double* A = c->bp.A;
    const double nx = A[2] * A[5] - A[4] * A[3], ny = A[4] * A[1] - A[0] * A[5], nz = A[0] * A[3] - A[2] * A[1];
    const double nn = std::sqrt(nx * nx + ny * ny + nz * nz);
    const double nrm[3] = {nx / nn, ny / nn, nz / nn};
    const double offs[3] = {-1.5, 0.0, 1.5};
    const long ncorner = (long)(K + 1) * (K + 1), ncentre = (long)K * K, npt = 3 * (ncorner + ncentre);
    std::vector<double> yd(3 * npt);
    std::vector<float> yf(3 * npt);
    for (int o = 0; o < 3; ++o)
        for (long q = 0; q < ncorner + ncentre; ++q) {
            double c0, c1;
            if (q < ncorner) {
                c0 = lo[0] + cell[0] * (double)(q / (K + 1));
                c1 = lo[1] + cell[1] * (double)(q % (K + 1));
            } else {
                const long r = q - ncorner;
                c0 = lo[0] + cell[0] * ((double)(r / K) + 0.5);
                c1 = lo[1] + cell[1] * ((double)(r % K) + 0.5);
            }
            const long i = (long)o * (ncorner + ncentre) + q;
            for (int ch = 0; ch < 3; ++ch) {
                yd[3 * i + ch] = A[ch * 2] * c0 + A[ch * 2 + 1] * c1 + offs[o] * sl * nrm[ch];
                yf[3 * i + ch] = (float)yd[3 * i + ch];
            }
        }
    double* d_yd = nullptr;
    float* d_yf = nullptr;
    float2 *d_exact = nullptr, *d_net = nullptr;
    BayesRec* d_rec = nullptr;
    float* d_part = nullptr;
    unsigned* d_cnt = nullptr;
    hb_status st = HB_OK;
    if (cudaMalloc(&d_yd, sizeof(double) * 3 * npt) != cudaSuccess ||
        cudaMalloc(&d_yf, sizeof(float) * 3 * npt) != cudaSuccess ||
        cudaMalloc(&d_exact, sizeof(float2) * npt) != cudaSuccess ||
        cudaMalloc(&d_net, sizeof(float2) * npt) != cudaSuccess ||
        cudaMalloc(&d_rec, sizeof(BayesRec) * npt) != cudaSuccess ||
        cudaMalloc(&d_part, sizeof(float) * 3 * hb::kMaxParts * npt) != cudaSuccess ||
        cudaMalloc(&d_cnt, sizeof(unsigned) * npt) != cudaSuccess || (!c->d_trust &&
        cudaMalloc(&c->d_trust, (size_t)K * K) != cudaSuccess))
        st = HB_ERR_OOM;
    std::vector<float2> ex(npt), net(npt);
    cudaError_t e = cudaSuccess;
    if (st == HB_OK) {
        e = cudaMemcpyAsync(d_yd, yd.data(), sizeof(double) * 3 * npt, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_yf, yf.data(), sizeof(float) * 3 * npt, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(unsigned) * npt, s);
        if (e == cudaSuccess) e = hb::launch_setup(c->bp, d_yd, npt, d_rec, s);
        if (e == cudaSuccess)
            e = hb::launch_posterior(c->bp, d_rec, npt, hb::PosteriorScratch{d_part, d_cnt, hb::kMaxParts}, d_exact,
                                     nullptr, 1.f, false, s);
        const void* img = e == cudaSuccess ? mlp_image(c, s, e) : nullptr;
        if (img) e = hb::launch_mlp_forward(img, c->mlp_norm, d_yf, npt, d_net, false, s);
        c->launches += 3;
        if (e == cudaSuccess) e = cudaMemcpyAsync(ex.data(), d_exact, sizeof(float2) * npt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(net.data(), d_net, sizeof(float2) * npt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = HB_ERR_CUDA;
    }
    std::vector<unsigned char> map((size_t)K * K, 0);
    long trusted = 0;
    if (st == HB_OK) {
        // error of one point relative to the box extents (NaN counts as out of tolerance)
        auto ok = [&](long q) {
            for (int o = 0; o < 3; ++o) {
                const long i = (long)o * (ncorner + ncentre) + q;
                const double d0 = std::fabs((double)net[i].x - ex[i].x) / c->mlp_ext0;
                const double d1 = std::fabs((double)net[i].y - ex[i].y) / c->mlp_ext1;
                if (!(d0 <= tol && d1 <= tol)) return false;
            }
            return true;
        };
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j) {
                const bool t = ok((long)i * (K + 1) + j) && ok((long)(i + 1) * (K + 1) + j) &&
                               ok((long)i * (K + 1) + j + 1) && ok((long)(i + 1) * (K + 1) + j + 1) &&
                               ok(ncorner + (long)i * K + j);
                map[(size_t)i * K + j] = t ? 1 : 0;
                trusted += t;
            }
        if (cudaMemcpyAsync(c->d_trust, map.data(), map.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = HB_ERR_CUDA;
    }
    cudaFree(d_yd);
    cudaFree(d_yf);
    cudaFree(d_exact);
    cudaFree(d_net);
    cudaFree(d_rec);
    cudaFree(d_part);
    cudaFree(d_cnt);
    if (st != HB_OK) {
        cudaGetLastError();
        c->route.trust = nullptr;
        return st;
    }
    c->route.trust = c->d_trust;
    c->route.k0 = K;
    c->route.k1 = K;
    c->route.org0 = (float)lo[0];
    c->route.org1 = (float)lo[1];
    c->route.inv0 = (float)(1.0 / cell[0]);
    c->route.inv1 = (float)(1.0 / cell[1]);
    if (trusted_fraction) *trusted_fraction = (double)trusted / ((double)K * K);
    return HB_OK;
}

// ------------------------------------------------------------------------------------
// Allocation-free posterior step.  Its working memory is this one file-scope device
// array; host code passes its device address (looked up once per device) to the
// same set-up and posterior kernels the context path uses.
// ------------------------------------------------------------------------------------
namespace {

constexpr long kStaticPixels = HB_STATIC_MAX_PIXELS;
constexpr int kStaticParts = 4;
constexpr size_t kStaticRecBytes = sizeof(BayesRec) * kStaticPixels;
constexpr size_t kStaticPartialBytes = sizeof(float) * 3 * kStaticParts * kStaticPixels;
constexpr size_t kStaticCountBytes = sizeof(unsigned) * kStaticPixels;
constexpr size_t kStaticBytes = kStaticRecBytes + kStaticPartialBytes + kStaticCountBytes;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices];  // device address of g_static_scratch, per device

// Device address of the array on the current device (looked up on first use).
hb_status static_scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HB_ERR_CUDA;
    }
    if (dev < 0 || dev >= kStaticMaxDevices) return HB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HB_ERR_CUDA;
        }
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return HB_OK;
}

}  // namespace

hb_status hb_posterior_mean_static(const hb_mixing* mix, const hb_grid* grid, const double* ybar_dev, long npix,
                                   float* conc_dev, void* stream) {
    if (!mix || !grid || npix < 0) return HB_ERR_ARG;
    if (grid->n0 < 1 || grid->n1 < 1 || !(grid->hi0 >= grid->lo0) || !(grid->hi1 >= grid->lo1) ||
        !(grid->sigma_l > 0.0))
        return HB_ERR_SHAPE;
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < 2; ++j)
            if (!std::isfinite(mix->A[c][j])) return HB_ERR_ARG;
    if (npix > kStaticPixels) return HB_ERR_SHAPE;
    if (npix == 0) return HB_OK;
    if (!ybar_dev || !conc_dev || (reinterpret_cast<uintptr_t>(ybar_dev) & 7) ||
        (reinterpret_cast<uintptr_t>(conc_dev) & 7))
        return HB_ERR_ARG;
    void* base = nullptr;
    hb_status st = static_scratch_address(&base);
    if (st != HB_OK) return st;
    // host-side constants only: the context object here is a parameter holder on the stack
    hb_ctx holder;
    prepare(&holder, mix, grid, 0.0);
    unsigned char* b = static_cast<unsigned char*>(base);
    BayesRec* rec = reinterpret_cast<BayesRec*>(b);
    float* partial = reinterpret_cast<float*>(b + kStaticRecBytes);
    unsigned* count = reinterpret_cast<unsigned*>(b + kStaticRecBytes + kStaticPartialBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counters must start at zero; whatever an earlier call left is cleared
    if (cudaMemsetAsync(count, 0, sizeof(unsigned) * npix, s) != cudaSuccess) return HB_ERR_CUDA;
    if (hb::launch_setup(holder.bp, ybar_dev, npix, rec, s) != cudaSuccess) return HB_ERR_CUDA;
    const hb::PosteriorScratch sc{partial, count, kStaticParts};
    if (hb::launch_posterior(holder.bp, rec, npix, sc, reinterpret_cast<float2*>(conc_dev), nullptr, 1.f, false, s) !=
        cudaSuccess)
        return HB_ERR_CUDA;
    return HB_OK;
}

const char* hb_strerror(hb_status s) {
    switch (s) {
        case HB_OK: return "ok";
        case HB_ERR_ARG: return "invalid argument";
        case HB_ERR_SHAPE: return "invalid size or level count";
        case HB_ERR_CUDA: return "CUDA error";
        case HB_ERR_OOM: return "out of memory";
        case HB_ERR_BUDGET: return "memory budget exceeded";
        case HB_ERR_TIMEOUT: return "timed out";
        case HB_ERR_STATE: return "invalid state";
        case HB_ERR_IO: return "file error";
    }
    return "unknown status";
}

}  // extern "C"
