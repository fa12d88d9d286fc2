// hb_transform.cu -- the HBM-bound passes of the estimator.
//
//   analysis kernel  : frame tile -> log-attenuation -> n levels of the 2x2-window
//                      Haar transform (Eq. 1-2) -> low-pass block means ybar, plus the
//                      per-pixel constants of the grid posterior (reference node, U, V).
//   synthesis kernel : frame tile -> log-attenuation -> n analysis levels -> Tikhonov
//                      operator M on every directional coefficient (Eq. 5) -> low pass
//                      from the posterior step -> n inverse levels (Eq. 4, H = H*) ->
//                      THb and SO2 (Section 3).
//
// Both kernels work on tiles of one 2^n-row band of superblocks (2^n x 2^n pixel
// blocks; Haar windows never cross a superblock, so tiles need no halo), in one of three
// layouts by level count:
//   strip (1..3 levels): a warp takes 64 columns, two per lane, so the first level stays
//       inside the lane (hb_strip.cuh); CTAs of 512 columns;
//   warp (0 and 4 levels, and the intensity low pass): a lane per column, levels across
//       lanes by shuffles; CTAs of 256 columns;
//   shared-memory tile (5..6 levels): the tile is copied from HBM with coalesced 16-byte
//       loads into shared memory and the whole multi-level transform runs in place there
//       (Mallat layout: after level l the low pass of each 2^l block sits at its top-left
//       position and the three directional coefficients at the other window positions).
// With 1..3 levels and the row kernel's grids the exact path runs no analysis kernel: the
// fused low-pass kernel (hb_bayes.cu) forms the block means itself.
//
// Numerics.  Before the transform every pixel's log-attenuation has the value of
// its superblock's top-left pixel subtracted (per channel).  The transform is
// linear, so the directional coefficients are unchanged and the low pass shifts by
// 2^n times that offset, which is added back in FP64 (analysis) or as the posterior
// estimate after synthesis.  This keeps every FP32 sum at the scale of the
// within-block variation instead of the level-n low pass (up to 2^n * 5.5).  For 8-bit
// input the logarithm comes from a 256-entry table of FP64 values split as
// float hi + float lo.
#include "hb_common.cuh"
#include "hb_device.cuh"
#include "hb_strip.cuh"

#include <math.h>

#ifndef HB_AN_EARLY_DEPENDENTS
#define HB_AN_EARLY_DEPENDENTS 0
#endif

namespace hb {

namespace {

struct TileSmem {
    unsigned char* raw;  // TH * TW * 3 elements of the input format
    float2* lut;         // 256 entries (8-bit input)
    float* D;            // 3 planes of TH * TW floats
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t raw_bytes(int TH, int TW, int fmt) {
    return align16((size_t)TH * TW * 3 * (fmt == 1 ? 1 : 4));
}

__device__ inline TileSmem carve(unsigned char* base, int TH, int TW, int fmt) {
    TileSmem t;
    t.raw = base;
    t.lut = reinterpret_cast<float2*>(base + raw_bytes(TH, TW, fmt));
    t.D = reinterpret_cast<float*>(base + raw_bytes(TH, TW, fmt) + 256 * sizeof(float2));
    return t;
}

// Copy the TH x TW pixel tile at (ty0, tx0) into shared memory, replicating the
// last row / column for positions outside the frame (edge padding).
__device__ void load_tile(const TransformParams& tp, const unsigned char* frame, size_t stride, int ty0, int tx0,
                          int TH, int TW, const float2* lut_g, TileSmem sm) {
    const int es = tp.fmt == 1 ? 1 : 4;
    const int rowbytes = TW * 3 * es;
    if (tp.fmt == 1)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) sm.lut[i] = lut_g[i];
    for (int r = 0; r < TH; ++r) {
        const int gy = min(ty0 + r, tp.H - 1);
        const unsigned char* src = frame + (size_t)gy * stride + (size_t)tx0 * 3 * es;
        unsigned char* dst = sm.raw + (size_t)r * rowbytes;
        const bool vec = (tx0 + TW <= tp.W) && ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (rowbytes % 16 == 0);
        if (vec) {
            const uint4* s4 = reinterpret_cast<const uint4*>(src);
            uint4* d4 = reinterpret_cast<uint4*>(dst);
            for (int i = threadIdx.x; i < rowbytes / 16; i += blockDim.x) d4[i] = __ldg(s4 + i);
        } else {
            const unsigned char* rowp = frame + (size_t)gy * stride;
            for (int e = threadIdx.x; e < TW * 3; e += blockDim.x) {
                const int x = min(tx0 + e / 3, tp.W - 1);
                const int ch = e % 3;
                if (es == 1)
                    dst[e] = rowp[(size_t)x * 3 + ch];
                else
                    reinterpret_cast<float*>(dst)[e] = reinterpret_cast<const float*>(rowp)[(size_t)x * 3 + ch];
            }
        }
    }
}

// Log-attenuation of one raw sample as (hi, lo) with hi + lo = -ln(max(I, eps)).
__device__ __forceinline__ float2 log_atten(const TransformParams& tp, const TileSmem& sm, int idx) {
    if (tp.fmt == 1) return sm.lut[sm.raw[idx]];
    const float I = reinterpret_cast<const float*>(sm.raw)[idx];
    return make_float2(-logf(fmaxf(I, tp.eps)), 0.f);
}

// y(p) - y(top-left of p's superblock), per channel, into the three D planes.
__device__ void offset_log(const TransformParams& tp, const TileSmem& sm, int TH, int TW) {
    const int n = TH * TW;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int r = p / TW, c = p - r * TW;
        const int cref = c & ~(TH - 1);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float2 y = log_atten(tp, sm, p * 3 + ch);
            const float2 yr = log_atten(tp, sm, cref * 3 + ch);
            sm.D[ch * n + r * TW + c] = (y.x - yr.x) + (y.y - yr.y);
        }
    }
}

// n in-place analysis levels on `nch` planes.  LL_ONLY skips the directional outputs.
template <bool LL_ONLY>
__device__ void analysis_levels(float* D, int nch, int TH, int TW, int levels) {
    const int n = TH * TW;
    for (int l = 1; l <= levels; ++l) {
        const int s = 1 << (l - 1), step = 2 * s;
        const int wr = TH / step, wc = TW / step, nwin = wr * wc;
        for (int t = threadIdx.x; t < nwin * nch; t += blockDim.x) {
            const int ch = t / nwin, w = t - ch * nwin;
            const int r = (w / wc) * step, c = (w % wc) * step;
            float* P = D + ch * n;
            const float a = P[r * TW + c], b = P[r * TW + c + s];
            const float cc = P[(r + s) * TW + c], d = P[(r + s) * TW + c + s];
            const float s1 = a + b, s2 = cc + d;
            P[r * TW + c] = 0.5f * (s1 + s2);                 // low pass
            if (!LL_ONLY) {
                const float d1 = a - b, d2 = cc - d;
                P[r * TW + c + s] = 0.5f * (s1 - s2);         // rows differ    [1, 1,-1,-1]
                P[(r + s) * TW + c] = 0.5f * (d1 - d2);       // diagonal       [1,-1,-1, 1]
                P[(r + s) * TW + c + s] = 0.5f * (d1 + d2);   // columns differ [1,-1, 1,-1]
            }
        }
        __syncthreads();
    }
}

// n in-place inverse levels (H is its own inverse) on `nch` planes.
__device__ void synthesis_levels(float* D, int nch, int TH, int TW, int levels) {
    const int n = TH * TW;
    for (int l = levels; l >= 1; --l) {
        const int s = 1 << (l - 1), step = 2 * s;
        const int wr = TH / step, wc = TW / step, nwin = wr * wc;
        for (int t = threadIdx.x; t < nwin * nch; t += blockDim.x) {
            const int ch = t / nwin, w = t - ch * nwin;
            const int r = (w / wc) * step, c = (w % wc) * step;
            float* P = D + ch * n;
            const float ll = P[r * TW + c], d1 = P[r * TW + c + s];
            const float d2 = P[(r + s) * TW + c], d3 = P[(r + s) * TW + c + s];
            const float p = ll + d1, q = ll - d1, u = d2 + d3, v = d2 - d3;
            P[r * TW + c] = 0.5f * (p + u);
            P[r * TW + c + s] = 0.5f * (p - u);
            P[(r + s) * TW + c] = 0.5f * (q - v);
            P[(r + s) * TW + c + s] = 0.5f * (q + v);
        }
        __syncthreads();
    }
}

}  // namespace


namespace {

__global__ void __launch_bounds__(kThreads) analysis_kernel(TransformParams tp, BayesParams bp,
                                                            const unsigned char* __restrict__ frame, size_t stride,
                                                            const float2* __restrict__ lut, double* __restrict__ ybar,
                                                            BayesRec* __restrict__ rec, float* __restrict__ ybar_f,
                                                            LsOut ls) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int TH = 1 << tp.levels, TW = tp.tile_w;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    TileSmem sm = carve(smem, TH, TW, tp.fmt);
    asm volatile("griddepcontrol.wait;" ::: "memory");  // as in analysis_warp_kernel
    load_tile(tp, frame, stride, ty0, tx0, TH, TW, lut, sm);
    __syncthreads();
    offset_log(tp, sm, TH, TW);
    __syncthreads();
    analysis_levels<true>(sm.D, 3, TH, TW, tp.levels);
    const int nsb = TW / TH, n = TH * TW;
    const float inv = 1.f / (float)TH;
    for (int t = threadIdx.x; t < nsb; t += blockDim.x) {
        const int gx = tx0 / TH + t;
        if (gx >= tp.wl) continue;
        float yhi[3], ylo[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float2 yr = log_atten(tp, sm, t * TH * 3 + ch);
            yhi[ch] = yr.x;
            ylo[ch] = yr.y + sm.D[ch * n + t * TH] * inv;
        }
        const size_t o = (size_t)blockIdx.y * tp.wl + gx;
        if (ybar) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar[o * 3 + ch] = (double)yhi[ch] + (double)ylo[ch];
        }
        if (ybar_f) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar_f[o * 3 + ch] = yhi[ch] + ylo[ch];
        }
        low_pass_out(yhi, ylo, tp, bp, o, rec, ls);
    }
}

__global__ void __launch_bounds__(kThreads) setup_kernel(BayesParams bp, const double* __restrict__ ybar, long npix,
                                                         BayesRec* __restrict__ rec) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float yhi[3], ylo[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const double y = ybar[p * 3 + ch];
        yhi[ch] = (float)y;
        ylo[ch] = (float)(y - (double)yhi[ch]);
    }
    rec[p] = bayes_setup(yhi, ylo, bp);
}

__global__ void __launch_bounds__(kThreads) synthesis_kernel(TransformParams tp, const unsigned char* __restrict__ frame,
                                                             size_t stride, const float2* __restrict__ lut,
                                                             const float2* __restrict__ chat, float* __restrict__ out0,
                                                             float* __restrict__ out1, int debug_conc) {
    asm volatile("griddepcontrol.launch_dependents;");  // as in synthesis_warp_kernel
    extern __shared__ __align__(16) unsigned char smem[];
    const int TH = 1 << tp.levels, TW = tp.tile_w;
    const int ty0 = blockIdx.y * TH, tx0 = blockIdx.x * TW;
    TileSmem sm = carve(smem, TH, TW, tp.fmt);
    load_tile(tp, frame, stride, ty0, tx0, TH, TW, lut, sm);
    __syncthreads();
    offset_log(tp, sm, TH, TW);
    __syncthreads();
    analysis_levels<false>(sm.D, 3, TH, TW, tp.levels);
    // Tikhonov operator on every directional coefficient (3 colours -> 2 concentrations);
    // the low-pass position takes 0 (posterior estimate added after synthesis) or, in the
    // all-Tikhonov mode, M applied to the offset-free low pass.
    const int n = TH * TW;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int r = p / TW, c = p - r * TW;
        const float v0 = sm.D[p], v1 = sm.D[n + p], v2 = sm.D[2 * n + p];
        const bool is_ll = (r == 0) && ((c & (TH - 1)) == 0);
        float o0 = tp.M[0] * v0 + tp.M[1] * v1 + tp.M[2] * v2;
        float o1 = tp.M[3] * v0 + tp.M[4] * v1 + tp.M[5] * v2;
        if (is_ll && !tp.tikhonov_lowpass) o0 = o1 = 0.f;
        sm.D[p] = o0;
        sm.D[n + p] = o1;
    }
    __syncthreads();
    synthesis_levels(sm.D, 2, TH, TW, tp.levels);
    if (!tp.tikhonov_lowpass) asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        const int r = p / TW, c = p - r * TW;
        const int gy = ty0 + r, gx = tx0 + c;
        if (gy >= tp.H || gx >= tp.W) continue;
        float off0, off1;
        if (tp.tikhonov_lowpass) {
            const int cref = c & ~(TH - 1);
            const float2 ya = log_atten(tp, sm, cref * 3 + 0);
            const float2 yb = log_atten(tp, sm, cref * 3 + 1);
            const float2 yc = log_atten(tp, sm, cref * 3 + 2);
            off0 = (tp.M[0] * ya.x + tp.M[1] * yb.x + tp.M[2] * yc.x) + (tp.M[0] * ya.y + tp.M[1] * yb.y + tp.M[2] * yc.y);
            off1 = (tp.M[3] * ya.x + tp.M[4] * yb.x + tp.M[5] * yc.x) + (tp.M[3] * ya.y + tp.M[4] * yb.y + tp.M[5] * yc.y);
        } else {
            const float2 ch = chat[(size_t)blockIdx.y * tp.wl + (gx >> tp.levels)];
            off0 = ch.x;
            off1 = ch.y;
        }
        const float hbo2 = sm.D[p] + off0, hb = sm.D[n + p] + off1;
        const size_t o = (size_t)gy * tp.W + gx;
        if (debug_conc) {
            out0[o] = hbo2;
            out1[o] = hb;
        } else {
            const float thb = hbo2 + hb;
            out0[o] = thb;
            out1[o] = thb > 0.f ? hbo2 / thb : 0.f;
        }
    }
}

// ------------------------------------------------------------------------------------
// Register (warp-column) variants for n <= 4.  Lane l of a warp owns pixel column
// x = 32 w + l for the 2^n rows of one superblock band, so a superblock spans 2^n
// neighbouring lanes.  Level l pairs rows r, r+s inside the lane and columns x, x+s
// across lanes (s = 2^(l-1), shuffle with lane ^ s); the in-place layout is the same
// as in the shared-memory kernels (low pass at the window's top-left, directional
// coefficients at the other three positions), and so is every FP32 operation.
// ------------------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

template <int L, bool LL_ONLY>
__device__ __forceinline__ void warp_analysis(float (&v)[3][1 << L], int lane) {
    constexpr int TH = 1 << L;
#pragma unroll
    for (int l = 1; l <= L; ++l) {
        const int s = 1 << (l - 1);
        const bool active = (lane & (s - 1)) == 0;
        const bool right = (lane & s) != 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += 2 * s) {
                const float x = v[ch][r], z = v[ch][r + s];
                const float xp = __shfl_xor_sync(kFull, x, s), zp = __shfl_xor_sync(kFull, z, s);
                const float a = right ? xp : x, b = right ? x : xp, c = right ? zp : z, d = right ? z : zp;
                const float s1 = a + b, s2 = c + d, d1 = a - b, d2 = c - d;
                if (active) {
                    if (!right) {
                        v[ch][r] = 0.5f * (s1 + s2);                    // low pass
                        if (!LL_ONLY) v[ch][r + s] = 0.5f * (d1 - d2);  // diagonal
                    } else if (!LL_ONLY) {
                        v[ch][r] = 0.5f * (s1 - s2);                    // rows differ
                        v[ch][r + s] = 0.5f * (d1 + d2);                // columns differ
                    }
                }
            }
    }
}

template <int L>
__device__ __forceinline__ void warp_synthesis(float (&c)[2][1 << L], int lane) {
    constexpr int TH = 1 << L;
#pragma unroll
    for (int l = L; l >= 1; --l) {
        const int s = 1 << (l - 1);
        const bool active = (lane & (s - 1)) == 0;
        const bool right = (lane & s) != 0;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += 2 * s) {
                const float x = c[ch][r], z = c[ch][r + s];
                const float xp = __shfl_xor_sync(kFull, x, s), zp = __shfl_xor_sync(kFull, z, s);
                const float ll = right ? xp : x, d1 = right ? x : xp, d2 = right ? zp : z, d3 = right ? z : zp;
                const float p = ll + d1, q = ll - d1, u = d2 + d3, w = d2 - d3;
                if (active) {
                    if (!right) {
                        c[ch][r] = 0.5f * (p + u);
                        c[ch][r + s] = 0.5f * (q - w);
                    } else {
                        c[ch][r] = 0.5f * (p - u);
                        c[ch][r + s] = 0.5f * (q + w);
                    }
                }
            }
    }
}

// Raw samples of the lane's column (codes or intensities), the superblock's top-left
// log-attenuation (hi, lo) and the offset-free values d = y - y_ref.  SUMS: also the
// column's sum of floored intensities per channel (ish + isl; for 8-bit input the exact
// integer sum of the codes, each at least 1, i.e. in units of 1/255).
template <int L, bool SUMS = false>
__device__ __forceinline__ void warp_load(const TransformParams& tp, const unsigned char* __restrict__ frame,
                                          size_t stride, const float2* lut, int by, int x, int lane,
                                          float (&v)[3][1 << L], float2 (&yref)[3], float* ish = nullptr,
                                          float* isl = nullptr) {
    constexpr int TH = 1 << L;
    const int xs = min(x, tp.W - 1);
    const int src_lane = lane & ~(TH - 1);
    if (tp.fmt == 1) {
        int k[3][TH];
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            const unsigned char* row = frame + (size_t)min(by * TH + r, tp.H - 1) * stride + (size_t)xs * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) k[ch][r] = __ldg(row + ch);
        }
        if (SUMS) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                int t = 0;
#pragma unroll
                for (int r = 0; r < TH; ++r) t += max(k[ch][r], 1);
                ish[ch] = (float)t;
                isl[ch] = 0.f;
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const int kr = __shfl_sync(kFull, k[ch][0], src_lane);
            yref[ch] = __ldg(lut + kr);
#pragma unroll
            for (int r = 0; r < TH; ++r) {
                const float2 y = __ldg(lut + k[ch][r]);
                v[ch][r] = (y.x - yref[ch].x) + (y.y - yref[ch].y);
            }
        }
    } else {
        if (SUMS) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ish[ch] = isl[ch] = 0.f;
        }
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            const float* row =
                reinterpret_cast<const float*>(frame + (size_t)min(by * TH + r, tp.H - 1) * stride) + (size_t)xs * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float I = fmaxf(__ldg(row + ch), tp.eps);
                if (SUMS) detail::dd_sub(ish[ch], isl[ch], -I, 0.f);
                v[ch][r] = -logf(I);
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float yr = __shfl_sync(kFull, v[ch][0], src_lane);
            yref[ch] = make_float2(yr, 0.f);
#pragma unroll
            for (int r = 0; r < TH; ++r) v[ch][r] = v[ch][r] - yr;
        }
    }
}

// Analysis of one tile (tile column tx of superblock band by): block means of the
// tile's superblocks and their posterior records.  sb_hi / sb_lo: kThreads x 3 floats of
// shared memory.  Called by whole CTAs.
template <int L>
__device__ __forceinline__ void analysis_tile(const TransformParams& tp, const BayesParams& bp,
                                              const unsigned char* __restrict__ frame, size_t stride,
                                              const float2* lut, int tx, int by, double* __restrict__ ybar,
                                              BayesRec* __restrict__ rec, float* __restrict__ ybar_f,
                                              float (*sb_hi)[3], float (*sb_lo)[3], const LsOut& ls = LsOut{}) {
    constexpr int TH = 1 << L;
    constexpr int NSB = kThreads / TH;  // superblocks per tile (kThreads columns)
    const int lane = threadIdx.x & 31;
    const int x0 = (tx * (kThreads / 32) + (threadIdx.x >> 5)) * 32;
    const int x = x0 + lane;
    if (x0 < tp.wl * TH) {  // whole warps right of the padded frame skip the transform
        float v[3][TH];
        float2 yref[3];
        if (!tp.ll_intensity) {
            warp_load<L>(tp, frame, stride, lut, by, x, lane, v, yref);
            warp_analysis<L, true>(v, lane);
            if ((lane & (TH - 1)) == 0) {
                const int t = threadIdx.x / TH;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    sb_hi[t][ch] = yref[ch].x;
                    sb_lo[t][ch] = yref[ch].y + v[ch][0] * (1.f / TH);
                }
            }
        } else {
            // Eq. 8 literally: the low pass of the intensities, then -log of its block mean
            float ish[3], isl[3];
            warp_load<L, true>(tp, frame, stride, lut, by, x, lane, v, yref, ish, isl);
#pragma unroll
            for (int s = 1; s < TH; s <<= 1)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float oh = __shfl_xor_sync(kFull, ish[ch], s), ol = __shfl_xor_sync(kFull, isl[ch], s);
                    detail::dd_sub(ish[ch], isl[ch], -oh, -ol);
                }
            if ((lane & (TH - 1)) == 0) {
                const int t = threadIdx.x / TH;
                const float d = (tp.fmt == 1 ? 255.f : 1.f) * (float)(TH * TH);  // exact
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float mh = __fdiv_rn(ish[ch], d);
                    const float ml = __fdiv_rn(fmaf(-mh, d, ish[ch]) + isl[ch], d);
                    sb_hi[t][ch] = -logf(mh);
                    sb_lo[t][ch] = -__fdiv_rn(ml, mh);
                }
            }
        }
    }
    __syncthreads();
    // one superblock per thread for the posterior set-up, so whole warps do it together
    for (int t = threadIdx.x; t < NSB; t += blockDim.x) {
        const int gx = (tx * kThreads) / TH + t;
        if (gx >= tp.wl) continue;
        float yhi[3], ylo[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            yhi[ch] = sb_hi[t][ch];
            ylo[ch] = sb_lo[t][ch];
        }
        const size_t o = (size_t)by * tp.wl + gx;
        if (ybar) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar[o * 3 + ch] = (double)yhi[ch] + (double)ylo[ch];
        }
        if (ybar_f) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar_f[o * 3 + ch] = yhi[ch] + ylo[ch];
        }
        low_pass_out(yhi, ylo, tp, bp, o, rec, ls);
    }
}

template <int L>
__global__ void __launch_bounds__(kThreads) analysis_warp_kernel(TransformParams tp, BayesParams bp,
                                                                 const unsigned char* __restrict__ frame,
                                                                 size_t stride, const float2* __restrict__ lut_g,
                                                                 double* __restrict__ ybar,
                                                                 BayesRec* __restrict__ rec,
                                                                 float* __restrict__ ybar_f, LsOut ls) {
    __shared__ float sb_hi[kThreads][3], sb_lo[kThreads][3];
    // launched as a programmatic dependent of the preceding kernel (the previous frame's
    // synthesis, or whatever wrote the frame): wait for it before reading anything
    asm volatile("griddepcontrol.wait;" ::: "memory");
    analysis_tile<L>(tp, bp, frame, stride, lut_g, blockIdx.x, blockIdx.y, ybar, rec, ybar_f, sb_hi, sb_lo, ls);
    // the posterior kernel may be scheduled now; it waits for this grid before reading rec
    asm volatile("griddepcontrol.launch_dependents;");
}

// Synthesis of one tile: analysis, Tikhonov operator on the directional coefficients,
// inverse transform, THb and SO2 (or HbO2 and Hb when debug_conc).  Whole warps return
// early, so it must be called last in a kernel.
template <int L>
__device__ __forceinline__ void synthesis_tile(const TransformParams& tp, const unsigned char* __restrict__ frame,
                                               size_t stride, const float2* lut, const float2* __restrict__ chat,
                                               float* __restrict__ out0, float* __restrict__ out1, int debug_conc,
                                               int tx, int by) {
    constexpr int TH = 1 << L;
    const int lane = threadIdx.x & 31;
    const int x0 = (tx * (kThreads / 32) + (threadIdx.x >> 5)) * 32;
    if (x0 >= tp.wl * TH) return;
    const int x = x0 + lane;
    float v[3][TH];
    float2 yref[3];
    warp_load<L>(tp, frame, stride, lut, by, x, lane, v, yref);
    warp_analysis<L, false>(v, lane);
    // Tikhonov operator on every directional coefficient; the low-pass position takes 0
    // (posterior estimate added after synthesis) or M applied to it (all-Tikhonov mode).
    float c[2][TH];
#pragma unroll
    for (int r = 0; r < TH; ++r) {
        const float v0 = v[0][r], v1 = v[1][r], v2 = v[2][r];
        float o0 = tp.M[0] * v0 + tp.M[1] * v1 + tp.M[2] * v2;
        float o1 = tp.M[3] * v0 + tp.M[4] * v1 + tp.M[5] * v2;
        if (r == 0 && (lane & (TH - 1)) == 0 && !tp.tikhonov_lowpass) o0 = o1 = 0.f;
        c[0][r] = o0;
        c[1][r] = o1;
    }
    warp_synthesis<L>(c, lane);
    float off0, off1;
    if (tp.tikhonov_lowpass) {
        off0 = (tp.M[0] * yref[0].x + tp.M[1] * yref[1].x + tp.M[2] * yref[2].x) +
               (tp.M[0] * yref[0].y + tp.M[1] * yref[1].y + tp.M[2] * yref[2].y);
        off1 = (tp.M[3] * yref[0].x + tp.M[4] * yref[1].x + tp.M[5] * yref[2].x) +
               (tp.M[3] * yref[0].y + tp.M[4] * yref[1].y + tp.M[5] * yref[2].y);
    } else {
        // everything above is independent of the posterior step; wait for it here
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const float2 ch = chat[(size_t)by * tp.wl + min(x >> L, tp.wl - 1)];
        off0 = ch.x;
        off1 = ch.y;
    }
    if (x >= tp.W) return;
#pragma unroll
    for (int r = 0; r < TH; ++r) {
        const int gy = by * TH + r;
        if (gy >= tp.H) break;
        const float hbo2 = c[0][r] + off0, hb = c[1][r] + off1;
        const size_t o = (size_t)gy * tp.W + x;
        if (debug_conc) {
            out0[o] = hbo2;
            out1[o] = hb;
        } else {
            const float thb = hbo2 + hb;
            out0[o] = thb;
            // SO2 needs 1e-3 absolute: the fast reciprocal-based division (2 ulp) is plenty
            out1[o] = thb >= 1.17549435e-38f ? __fdividef(hbo2, thb) : (thb > 0.f ? hbo2 / thb : 0.f);
        }
    }
}


template <int L>
__global__ void __launch_bounds__(kThreads) synthesis_warp_kernel(TransformParams tp,
                                                                  const unsigned char* __restrict__ frame,
                                                                  size_t stride, const float2* __restrict__ lut_g,
                                                                  const float2* __restrict__ chat,
                                                                  float* __restrict__ out0, float* __restrict__ out1,
                                                                  int debug_conc) {
    // the next frame's analysis may be scheduled as CTAs of this grid retire; it waits for
    // this grid before reading anything
    asm volatile("griddepcontrol.launch_dependents;");
    synthesis_tile<L>(tp, frame, stride, lut_g, chat, out0, out1, debug_conc, blockIdx.x, blockIdx.y);
}

static_assert(kStripCols == 64 * (kThreads / 32), "two columns per lane");

// Analysis of one strip tile (tile column tx of superblock band by): block means of the
// tile's superblocks and their posterior records.  sb_hi / sb_lo: kThreads x 3 floats of
// shared memory (kStripCols / 2^L <= kThreads superblocks).  Called by whole CTAs.
template <int L>
__device__ __forceinline__ void analysis_strip_tile(const TransformParams& tp, const BayesParams& bp,
                                                    const unsigned char* __restrict__ frame, size_t stride,
                                                    const float2* lut, int tx, int by, double* __restrict__ ybar,
                                                    BayesRec* __restrict__ rec, float* __restrict__ ybar_f,
                                                    float (*sb_hi)[3], float (*sb_lo)[3], const LsOut& ls = LsOut{}) {
    constexpr int TH = 1 << L;
    constexpr int NSB = kStripCols / TH;  // superblocks per tile
    const int lane = threadIdx.x & 31;
    const int x0w = tx * kStripCols + (threadIdx.x >> 5) * 64;  // the warp's first column
    if (x0w < tp.wl * TH) {  // whole warps right of the padded frame skip the transform
        float v[3][TH][2];
        float2 yref[3];
        strip_load<L>(tp, frame, stride, lut, by, x0w + 2 * lane, lane, v, yref);
        strip_analysis<L, 3, true>(v, lane);
        if ((lane & ((TH >> 1) - 1)) == 0) {
            const int t = (threadIdx.x * 2) / TH;  // superblock within the tile
            constexpr float inv = 1.f / (float)(TH * TH);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                sb_hi[t][ch] = yref[ch].x;
                sb_lo[t][ch] = fmaf(v[ch][0][0], inv, yref[ch].y);
            }
        }
    }
    __syncthreads();
    // one superblock per thread for the posterior set-up, so whole warps do it together
    for (int t = threadIdx.x; t < NSB; t += blockDim.x) {
        const int gx = (tx * kStripCols) / TH + t;
        if (gx >= tp.wl) continue;
        float yhi[3], ylo[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            yhi[ch] = sb_hi[t][ch];
            ylo[ch] = sb_lo[t][ch];
        }
        const size_t o = (size_t)by * tp.wl + gx;
        if (ybar) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar[o * 3 + ch] = (double)yhi[ch] + (double)ylo[ch];
        }
        if (ybar_f) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) ybar_f[o * 3 + ch] = yhi[ch] + ylo[ch];
        }
        low_pass_out(yhi, ylo, tp, bp, o, rec, ls);
    }
}

template <int L>
__global__ void __launch_bounds__(kThreads, 4) analysis_strip_kernel(TransformParams tp, BayesParams bp,
                                                                  const unsigned char* __restrict__ frame,
                                                                  size_t stride, const float2* __restrict__ lut_g,
                                                                  double* __restrict__ ybar,
                                                                  BayesRec* __restrict__ rec,
                                                                  float* __restrict__ ybar_f, LsOut ls) {
    __shared__ float sb_hi[kThreads][3], sb_lo[kThreads][3];
    // launched as a programmatic dependent of the preceding kernel (the previous frame's
    // synthesis, or whatever wrote the frame): wait for it before reading anything
    asm volatile("griddepcontrol.wait;" ::: "memory");
#if HB_AN_EARLY_DEPENDENTS
    // the posterior kernel may be scheduled as SMs free up; it waits for this whole grid
    // before reading rec
    asm volatile("griddepcontrol.launch_dependents;");
#endif
    analysis_strip_tile<L>(tp, bp, frame, stride, lut_g, blockIdx.x, blockIdx.y, ybar, rec, ybar_f, sb_hi, sb_lo,
                           ls);
#if !HB_AN_EARLY_DEPENDENTS
    // the posterior kernel may be scheduled now; it waits for this grid before reading rec
    asm volatile("griddepcontrol.launch_dependents;");
#endif
}

// Synthesis of one strip tile: analysis, Tikhonov operator on the directional
// coefficients (M 4^-l at level l), inverse transform, THb and SO2 (or HbO2 and Hb when
// debug_conc).  Whole warps return early, so it must be called last in a kernel.
template <int L>
__device__ __forceinline__ void synthesis_strip_tile(const TransformParams& tp,
                                                     const unsigned char* __restrict__ frame, size_t stride,
                                                     const float2* lut, const float2* __restrict__ chat,
                                                     float* __restrict__ out0, float* __restrict__ out1,
                                                     int debug_conc, int tx, int by) {
    constexpr int TH = 1 << L;
    const int lane = threadIdx.x & 31;
    const int x0w = tx * kStripCols + (threadIdx.x >> 5) * 64;
    if (x0w >= tp.wl * TH) return;
    const int x = x0w + 2 * lane;
    float v[3][TH][2];
    float2 yref[3];
    strip_load<L>(tp, frame, stride, lut, by, x, lane, v, yref);
    strip_analysis<L, 3, false>(v, lane);
    float c[2][TH][2];
    strip_tikhonov<L>(tp, v, lane, c);
    strip_synthesis<L>(c, lane);
    float off0, off1;
    if (tp.tikhonov_lowpass) {
        strip_tikhonov_offset(tp, yref, off0, off1);
    } else {
        // everything above is independent of the posterior step; wait for it here
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const float2 ch = chat[(size_t)by * tp.wl + min(x >> L, tp.wl - 1)];
        off0 = ch.x;
        off1 = ch.y;
    }
    strip_store<L>(tp, c, off0, off1, x, by, out0, out1, debug_conc);
}

template <int L>
__global__ void __launch_bounds__(kThreads, 4) synthesis_strip_kernel(TransformParams tp,
                                                                   const unsigned char* __restrict__ frame,
                                                                   size_t stride, const float2* __restrict__ lut_g,
                                                                   const float2* __restrict__ chat,
                                                                   float* __restrict__ out0, float* __restrict__ out1,
                                                                   int debug_conc) {
    // the next frame's analysis may be scheduled as CTAs of this grid retire; it waits for
    // this grid before reading anything
    asm volatile("griddepcontrol.launch_dependents;");
    synthesis_strip_tile<L>(tp, frame, stride, lut_g, chat, out0, out1, debug_conc, blockIdx.x, blockIdx.y);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t transform_smem_bytes(const TransformParams& tp) {
    const int TH = 1 << tp.levels, TW = tp.tile_w;
    return raw_bytes(TH, TW, tp.fmt) + 256 * sizeof(float2) + (size_t)3 * TH * TW * sizeof(float);
}

static dim3 tile_grid(const TransformParams& tp) {
    const int TH = 1 << tp.levels;
    const int Wp = tp.wl * TH;
    return dim3((Wp + tp.tile_w - 1) / tp.tile_w, tp.hl);
}

// Launch with or without programmatic dependent launch (PDL): with it, CTAs of this
// kernel may start once every CTA of the preceding kernel on the stream has started (or
// asked for it, griddepcontrol.launch_dependents); they wait (griddepcontrol.wait) for that
// kernel to finish before touching what it wrote.
template <typename... Args>
static cudaError_t launch_maybe_pdl(void (*kernel)(Args...), dim3 grid, size_t smem, cudaStream_t s, bool pdl,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_analysis(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                            const float2* lut, double* ybar, BayesRec* rec, cudaStream_t s, float* ybar_f,
                            const LsOut& ls, bool pdl) {
    const unsigned char* f = static_cast<const unsigned char*>(frame);
    if (tp.levels <= 4) {
        const int TH = 1 << tp.levels, cols = tile_cols(tp.levels, tp.ll_intensity);
        const dim3 grid((tp.wl * TH + cols - 1) / cols, tp.hl);
#define HB_AN_ARGS grid, 0, s, pdl, tp, bp, f, stride, lut, ybar, rec, ybar_f, ls
        if (cols == kStripCols) switch (tp.levels) {
                case 1: return launch_maybe_pdl(analysis_strip_kernel<1>, HB_AN_ARGS);
                case 2: return launch_maybe_pdl(analysis_strip_kernel<2>, HB_AN_ARGS);
                default: return launch_maybe_pdl(analysis_strip_kernel<3>, HB_AN_ARGS);
            }
        switch (tp.levels) {
            case 0: return launch_maybe_pdl(analysis_warp_kernel<0>, HB_AN_ARGS);
            case 1: return launch_maybe_pdl(analysis_warp_kernel<1>, HB_AN_ARGS);
            case 2: return launch_maybe_pdl(analysis_warp_kernel<2>, HB_AN_ARGS);
            case 3: return launch_maybe_pdl(analysis_warp_kernel<3>, HB_AN_ARGS);
            default: return launch_maybe_pdl(analysis_warp_kernel<4>, HB_AN_ARGS);
        }
#undef HB_AN_ARGS
    }
    const size_t sm = transform_smem_bytes(tp);
    cudaError_t e = set_smem(analysis_kernel, sm);
    if (e != cudaSuccess) return e;
    return launch_maybe_pdl(analysis_kernel, tile_grid(tp), sm, s, pdl, tp, bp, f, stride, lut, ybar, rec, ybar_f, ls);
}

cudaError_t launch_setup(const BayesParams& bp, const double* ybar, long npix, BayesRec* rec, cudaStream_t s) {
    if (npix <= 0) return cudaSuccess;
    setup_kernel<<<(unsigned)((npix + kThreads - 1) / kThreads), kThreads, 0, s>>>(bp, ybar, npix, rec);
    return cudaGetLastError();
}

cudaError_t launch_synthesis(const TransformParams& tp, const void* frame, size_t stride, const float2* lut,
                             const float2* chat, float* out0, float* out1, int debug_conc, bool pdl, cudaStream_t s) {
    const unsigned char* f = static_cast<const unsigned char*>(frame);
    if (tp.levels <= 4) {
        const int TH = 1 << tp.levels, cols = tile_cols(tp.levels, tp.ll_intensity);
        const dim3 grid((tp.wl * TH + cols - 1) / cols, tp.hl);
        if (cols == kStripCols) switch (tp.levels) {
                case 1: return launch_maybe_pdl(synthesis_strip_kernel<1>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
                case 2: return launch_maybe_pdl(synthesis_strip_kernel<2>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
                default: return launch_maybe_pdl(synthesis_strip_kernel<3>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
            }
        switch (tp.levels) {
            case 0: return launch_maybe_pdl(synthesis_warp_kernel<0>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
            case 1: return launch_maybe_pdl(synthesis_warp_kernel<1>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
            case 2: return launch_maybe_pdl(synthesis_warp_kernel<2>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
            case 3: return launch_maybe_pdl(synthesis_warp_kernel<3>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
            default: return launch_maybe_pdl(synthesis_warp_kernel<4>, grid, 0, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
        }
    }
    const size_t sm = transform_smem_bytes(tp);
    cudaError_t e = set_smem(synthesis_kernel, sm);
    if (e != cudaSuccess) return e;
    return launch_maybe_pdl(synthesis_kernel, tile_grid(tp), sm, s, pdl, tp, f, stride, lut, chat, out0, out1, debug_conc);
}

// ------------------------------------------------------------------------------------
// Serving batches: every CTA finds its frame in the job table (jobs sorted by
// tile_begin) and runs the single-frame tile body for that frame's level count, so
// frames of different sizes and levels share one launch per stage.
// ------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ int find_job(const FrameJob* jobs, int njobs, int block) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {  // last job with tile_begin <= block
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_begin <= block) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kThreads) batch_analysis_kernel(BayesParams bp, const FrameJob* __restrict__ jobs,
                                                                  int njobs, const float2* __restrict__ lut_g,
                                                                  BayesRec* __restrict__ rec_all) {
    __shared__ float sb_hi[kThreads][3], sb_lo[kThreads][3];
    const FrameJob& job = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int local = blockIdx.x - job.tile_begin;
    const int by = local / job.tiles_x, tx = local - by * job.tiles_x;
    BayesRec* rec = rec_all + job.ll_offset;
    if (tile_cols(job.tp.levels, job.tp.ll_intensity) == kStripCols) {
        switch (job.tp.levels) {
            case 1: analysis_strip_tile<1>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
            case 2: analysis_strip_tile<2>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
            default: analysis_strip_tile<3>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
        }
        return;
    }
    switch (job.tp.levels) {
        case 0: analysis_tile<0>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
        case 1: analysis_tile<1>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
        case 2: analysis_tile<2>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
        case 3: analysis_tile<3>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
        default: analysis_tile<4>(job.tp, bp, job.frame, job.stride, lut_g, tx, by, nullptr, rec, nullptr, sb_hi, sb_lo); break;
    }
}

__global__ void __launch_bounds__(kThreads) batch_synthesis_kernel(const FrameJob* __restrict__ jobs, int njobs,
                                                                   const float2* __restrict__ lut_g,
                                                                   const float2* __restrict__ chat_all) {
    const FrameJob& job = jobs[find_job(jobs, njobs, blockIdx.x)];
    const int local = blockIdx.x - job.tile_begin;
    const int by = local / job.tiles_x, tx = local - by * job.tiles_x;
    const float2* chat = chat_all + job.ll_offset;
    if (tile_cols(job.tp.levels, job.tp.ll_intensity) == kStripCols) {
        switch (job.tp.levels) {
            case 1: synthesis_strip_tile<1>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
            case 2: synthesis_strip_tile<2>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
            default: synthesis_strip_tile<3>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
        }
        return;
    }
    switch (job.tp.levels) {
        case 0: synthesis_tile<0>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
        case 1: synthesis_tile<1>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
        case 2: synthesis_tile<2>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
        case 3: synthesis_tile<3>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
        default: synthesis_tile<4>(job.tp, job.frame, job.stride, lut_g, chat, job.thb, job.so2, 0, tx, by); break;
    }
}

}  // namespace

cudaError_t launch_batch_analysis(const BayesParams& bp, const FrameJob* jobs, int njobs, int total_tiles,
                                  const float2* lut, BayesRec* rec_all, cudaStream_t s) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    batch_analysis_kernel<<<total_tiles, kThreads, 0, s>>>(bp, jobs, njobs, lut, rec_all);
    return cudaGetLastError();
}

cudaError_t launch_batch_synthesis(const FrameJob* jobs, int njobs, int total_tiles, const float2* lut,
                                   const float2* chat_all, cudaStream_t s) {
    if (njobs <= 0 || total_tiles <= 0) return cudaSuccess;
    batch_synthesis_kernel<<<total_tiles, kThreads, 0, s>>>(jobs, njobs, lut, chat_all);
    return cudaGetLastError();
}

}  // namespace hb
