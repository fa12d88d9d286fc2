// hb_bayes.cu -- posterior mean of (HbO2, Hb) over the concentration grid for every
// low-pass pixel (the Bayesian estimate on the low-pass band, Section 2).
//
// For a pixel with block-mean log-attenuation ybar the posterior over grid node k is
// proportional to exp(-|ybar - A c_k|^2 / (2 sigma^2)) (flat prior).  Expanded around
// a reference node c_ref = (i0, j0) with residual r0 = ybar - A c_ref, the base-2 log
// weight of node (i0 + di, j0 + dj) relative to the reference is
//
//     t = U di + V dj + Aq di^2 + 2 Bq di dj + Cq dj^2
//       = di * (Aq di + Q_j) + P_j,     Q_j = U + 2 Bq dj,  P_j = V dj + Cq dj^2,
//
// i.e. the -(|r0|^2 - 2 r0.A delta + |A delta|^2) expansion with the per-pixel terms
// (U, V from r0) and the per-grid terms (Aq, Bq, Cq from |A delta|^2) separated.  The
// weight is 2^t (MUFU ex2).  The reference node is the node nearest the likelihood's
// maximiser over the grid's hull, so its weight is exactly 1 and no node's weight can
// overflow; a pixel whose sums still come out non-finite (only possible for inputs far
// outside the model) is recomputed with an explicit maximum pass.
//
// Work split: a unit is (pixel, part); the rs parts of a pixel take contiguous row
// ranges of the grid, lane l of the warp takes columns l, l+32, l+64, ...  Warps are
// persistent (one grid of resident CTAs walks all units) and prefetch the next unit's
// constants.  Per grid node a lane issues 2 packed FP32x2 instructions for t, one ex2
// and 2 packed instructions for the sums (sum w, sum w*di per column): 3 issue slots
// per node for 1 MUFU op.  Warp shuffles combine lanes; the last part of a pixel to
// finish (atomic counter) adds the parts' sums in a fixed order, so results do not
// depend on scheduling.
#include "hb_common.cuh"
#include "hb_device.cuh"

#include <math.h>

#ifndef HB_POST_UNROLL
#define HB_POST_UNROLL 4   // grid rows per unrolled step of the posterior loop
#endif
#ifdef HB_POST_MINB       // minimum resident CTAs per SM requested from the register allocator
#define HB_POST_BOUNDS __launch_bounds__(kThreads, HB_POST_MINB)
#else
#define HB_POST_BOUNDS __launch_bounds__(kThreads)
#endif

namespace hb {
namespace {

typedef unsigned long long u64;
constexpr int kPostUnroll = HB_POST_UNROLL;

__device__ __forceinline__ u64 pk(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Column constants of one lane for the column block starting at j_base.
template <int CPL>
__device__ __forceinline__ void column_terms(const BayesParams& bp, const BayesRec& rec, int lane, int j_base,
                                             float shift, float (&dj)[CPL], float (&P)[CPL], float (&Q)[CPL]) {
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
        const int j = j_base + lane + 32 * s;
        dj[s] = (float)(j - rec.j0);
        P[s] = j < bp.n1 ? fmaf(bp.Cq * dj[s], dj[s], rec.V * dj[s]) - shift : -INFINITY;
        Q[s] = fmaf(2.f * bp.Bq, dj[s], rec.U);
    }
}

// sum w, sum w di, sum w dj over rows [rb, re) and the lane's columns (all column blocks),
// with weights 2^(t - shift).
template <int CPL>
__device__ __forceinline__ void grid_sums(const BayesParams& bp, const BayesRec& rec, int lane, int rb, int re,
                                          float shift, float& sw, float& sdi, float& sdj) {
    for (int jb = 0; jb < bp.n1; jb += 32 * CPL) {
        float dj[CPL], P[CPL], Q[CPL];
        column_terms<CPL>(bp, rec, lane, jb, shift, dj, P, Q);
        float S[CPL], T[CPL];
        if constexpr (CPL == 1) {
            S[0] = 0.f;
            T[0] = 0.f;
            float di = (float)(rb - rec.i0);
#pragma unroll 4
            for (int i = rb; i < re; ++i, di += 1.f) {
                const float w = ex2(fmaf(di, fmaf(bp.Aq, di, Q[0]), P[0]));
                S[0] += w;
                T[0] = fmaf(w, di, T[0]);
            }
        } else {
            u64 Pp[CPL / 2], Qp[CPL / 2], Sp[CPL / 2], Tp[CPL / 2];
#pragma unroll
            for (int q = 0; q < CPL / 2; ++q) {
                Pp[q] = pk(P[2 * q], P[2 * q + 1]);
                Qp[q] = pk(Q[2 * q], Q[2 * q + 1]);
                Sp[q] = pk(0.f, 0.f);
                Tp[q] = pk(0.f, 0.f);
            }
            const u64 AA = pk(bp.Aq, bp.Aq), ONE = pk(1.f, 1.f);
            const float di0 = (float)(rb - rec.i0);
            u64 dd = pk(di0, di0);
#pragma unroll kPostUnroll
            for (int i = rb; i < re; ++i) {
#pragma unroll
                for (int q = 0; q < CPL / 2; ++q) {
                    const u64 X = fma2(dd, AA, Qp[q]);
                    const u64 t = fma2(dd, X, Pp[q]);
                    float t0, t1;
                    upk(t, t0, t1);
                    const u64 w = pk(ex2(t0), ex2(t1));
                    Sp[q] = add2(Sp[q], w);
                    Tp[q] = fma2(w, dd, Tp[q]);
                }
                dd = add2(dd, ONE);
            }
#pragma unroll
            for (int q = 0; q < CPL / 2; ++q) {
                upk(Sp[q], S[2 * q], S[2 * q + 1]);
                upk(Tp[q], T[2 * q], T[2 * q + 1]);
            }
        }
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
            sw += S[s];
            sdi += T[s];
            sdj = fmaf(S[s], dj[s], sdj);
        }
    }
}

// Largest exponent t over rows [rb, re) and the lane's columns.
template <int CPL>
__device__ float grid_max(const BayesParams& bp, const BayesRec& rec, int lane, int rb, int re) {
    float m = -INFINITY;
    for (int jb = 0; jb < bp.n1; jb += 32 * CPL) {
        float dj[CPL], P[CPL], Q[CPL];
        column_terms<CPL>(bp, rec, lane, jb, 0.f, dj, P, Q);
        float di = (float)(rb - rec.i0);
        for (int i = rb; i < re; ++i, di += 1.f)
#pragma unroll
            for (int s = 0; s < CPL; ++s) m = fmaxf(m, fmaf(di, fmaf(bp.Aq, di, Q[s]), P[s]));
    }
    return m;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Recomputation of a pixel whose sums are not usable: explicit maximum, then the sums
// with that shift.  Out of line so that it costs the main path no registers.
template <int CPL>
__device__ __noinline__ void rescue_sums(const BayesParams& bp, const BayesRec& rec, int lane, float& sw, float& sdi,
                                         float& sdj) {
    float m = grid_max<CPL>(bp, rec, lane, 0, bp.n0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    sw = sdi = sdj = 0.f;
    grid_sums<CPL>(bp, rec, lane, 0, bp.n0, m, sw, sdi, sdj);
    sw = warp_sum(sw);
    sdi = warp_sum(sdi);
    sdj = warp_sum(sdj);
}

// Posterior mean from the sums; recomputes the pixel with an explicit maximum when the
// sums are not usable.  Warp-uniform; lane 0 writes.
template <int CPL>
__device__ void finish_pixel(const BayesParams& bp, const BayesRec& rec, long p, int lane, float sw, float sdi,
                             float sdj, float2* chat, float2* chat_scaled, float scale) {
    if (!(sw > 0.f) || !isfinite(sw) || !isfinite(sdi) || !isfinite(sdj)) rescue_sums<CPL>(bp, rec, lane, sw, sdi, sdj);
    if (lane == 0) {
        const double c0 = bp.lo0 + rec.i0 * bp.h0 + bp.h0 * ((double)sdi / (double)sw);
        const double c1 = bp.lo1 + rec.j0 * bp.h1 + bp.h1 * ((double)sdj / (double)sw);
        chat[p] = make_float2((float)c0, (float)c1);
        if (chat_scaled) chat_scaled[p] = make_float2((float)(c0 * scale), (float)(c1 * scale));
    }
}

// Sums of one unit, then either the pixel's result (rs == 1) or the unit's partial sums;
// the last part of a pixel to arrive adds the parts in order and finishes the pixel.
template <int CPL>
__device__ __forceinline__ void run_unit(const BayesParams& bp, const BayesRec& rec, long p, int part, int rs,
                                         int lane, float* partial, unsigned* count, float2* chat,
                                         float2* chat_scaled, float scale) {
    const int rb = (int)((long)bp.n0 * part / rs), re = (int)((long)bp.n0 * (part + 1) / rs);
    float sw = 0.f, sdi = 0.f, sdj = 0.f;
    grid_sums<CPL>(bp, rec, lane, rb, re, 0.f, sw, sdi, sdj);
    sw = warp_sum(sw);
    sdi = warp_sum(sdi);
    sdj = warp_sum(sdj);
    if (rs == 1) {
        finish_pixel<CPL>(bp, rec, p, lane, sw, sdi, sdj, chat, chat_scaled, scale);
        return;
    }
    unsigned prior = 0;
    if (lane == 0) {
        float* slot = partial + ((size_t)p * rs + part) * 3;
        slot[0] = sw;
        slot[1] = sdi;
        slot[2] = sdj;
        __threadfence();
        prior = atomicAdd(&count[p], 1u);
    }
    prior = __shfl_sync(0xffffffffu, prior, 0);
    if (prior == (unsigned)(rs - 1)) {
        __threadfence();
        float a = 0.f, b = 0.f, c = 0.f;
        if (lane == 0) {
            const volatile float* slots = partial + (size_t)p * rs * 3;
            for (int k = 0; k < rs; ++k) {
                a += slots[3 * k];
                b += slots[3 * k + 1];
                c += slots[3 * k + 2];
            }
            count[p] = 0u;
        }
        a = __shfl_sync(0xffffffffu, a, 0);
        b = __shfl_sync(0xffffffffu, b, 0);
        c = __shfl_sync(0xffffffffu, c, 0);
        finish_pixel<CPL>(bp, rec, p, lane, a, b, c, chat, chat_scaled, scale);
    }
}

// Posterior over precomputed per-pixel records (the stand-alone posterior entry point).
template <int CPL>
__global__ void HB_POST_BOUNDS posterior_kernel(BayesParams bp, const BayesRec* __restrict__ recs, long npix, int rs,
                                                float* partial, unsigned* count, float2* __restrict__ chat,
                                                float2* __restrict__ chat_scaled, float scale) {
    const int lane = threadIdx.x & 31;
    const long nw = (long)gridDim.x * (kThreads / 32);
    const long units = npix * rs;
    long u = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    BayesRec next = {0, 0, 0.f, 0.f};
    if (u < units) next = recs[u / rs];
    for (; u < units; u += nw) {
        const long p = u / rs;
        const BayesRec rec = next;
        if (u + nw < units) next = recs[(u + nw) / rs];
        run_unit<CPL>(bp, rec, p, (int)(u - p * rs), rs, lane, partial, count, chat, chat_scaled, scale);
    }
}

// ------------------------------------------------------------------------------------
// Posterior straight from the frame.  A unit's warp first forms the low pass of its
// pixel's 2^n x 2^n superblock: lane l holds the superblock pixels whose Morton index
// (column bit, row bit, column bit, ...) is l, l+32, ...; a butterfly over the index bits
// pairs columns, then rows, level by level, so every sum is the 0.5((a+b)+(c+d)) of one
// Haar window (Eq. 1-2, low-pass row of H) in the same order and rounding as the
// transform kernels.  The next unit's pixels are loaded before the current unit's grid
// loop so that the loads overlap it.
// ------------------------------------------------------------------------------------
template <int L>
struct Superblock {
    static constexpr int kPixels = 1 << (2 * L);
    static constexpr int kPerLane = kPixels >= 32 ? kPixels / 32 : 1;
};

__device__ __forceinline__ int compact_bits(int x) {  // keeps bits 0, 2, 4, ... packed together
    x &= 0x5555;
    x = (x | (x >> 1)) & 0x3333;
    x = (x | (x >> 2)) & 0x0F0F;
    x = (x | (x >> 4)) & 0x00FF;
    return x;
}

template <int L>
__device__ __forceinline__ void sb_load(const TransformParams& tp, const unsigned char* __restrict__ frame,
                                        size_t stride, long p, int lane, float (&raw)[3][Superblock<L>::kPerLane]) {
    constexpr int B = 1 << L;
    const int by = (int)(p / tp.wl), bx = (int)(p - (long)by * tp.wl);
#pragma unroll
    for (int k = 0; k < Superblock<L>::kPerLane; ++k) {
        const int m = (lane + 32 * k) & (Superblock<L>::kPixels - 1);
        const int gy = min(by * B + compact_bits(m >> 1), tp.H - 1);
        const int gx = min(bx * B + compact_bits(m), tp.W - 1);
        const unsigned char* px = frame + (size_t)gy * stride + (size_t)gx * 3 * (tp.fmt == 1 ? 1 : 4);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            raw[ch][k] = tp.fmt == 1 ? (float)__ldg(px + ch) : __ldg(reinterpret_cast<const float*>(px) + ch);
    }
}

template <int L>
__device__ __forceinline__ BayesRec sb_setup(const TransformParams& tp, const BayesParams& bp, const float2* lut,
                                             const float (&raw)[3][Superblock<L>::kPerLane]) {
    constexpr int K = Superblock<L>::kPerLane;
    float yhi[3], ylo[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float2 y[K];
#pragma unroll
        for (int k = 0; k < K; ++k)
            y[k] = tp.fmt == 1 ? lut[(int)raw[ch][k]] : make_float2(-logf(fmaxf(raw[ch][k], tp.eps)), 0.f);
        const float rx = __shfl_sync(0xffffffffu, y[0].x, 0), ry = __shfl_sync(0xffffffffu, y[0].y, 0);
        float d[K];
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = (y[k].x - rx) + (y[k].y - ry);
#pragma unroll
        for (int l = 1; l <= L; ++l) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = 2 * (l - 1) + h;  // Morton bit: column (h = 0) then row (h = 1)
                if (b < 5) {
#pragma unroll
                    for (int k = 0; k < K; ++k) d[k] += __shfl_xor_sync(0xffffffffu, d[k], 1 << b);
                } else {
                    const int kb = 1 << (b - 5);
#pragma unroll
                    for (int k = 0; k < K; ++k)
                        if (!(k & kb)) d[k] = d[k] + d[k | kb];
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) d[k] *= 0.5f;
        }
        yhi[ch] = rx;
        ylo[ch] = ry + d[0] * (1.f / (1 << L));
    }
    return bayes_setup(yhi, ylo, bp);
}

template <int CPL, int L>
__global__ void HB_POST_BOUNDS posterior_frame_kernel(TransformParams tp, BayesParams bp,
                                                      const unsigned char* __restrict__ frame, size_t stride,
                                                      const float2* __restrict__ lut_g, int rs, float* partial,
                                                      unsigned* count, float2* __restrict__ chat,
                                                      float2* __restrict__ chat_scaled, float scale) {
    __shared__ float2 lut[256];
    if (tp.fmt == 1)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = lut_g[i];
    __syncthreads();
    // the synthesis kernel may be scheduled as soon as SMs free up; it waits for this grid
    asm volatile("griddepcontrol.launch_dependents;");
    const int lane = threadIdx.x & 31;
    const long npix = (long)tp.hl * tp.wl;
    const long nw = (long)gridDim.x * (kThreads / 32);
    const long units = npix * rs;
    long u = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    float raw[3][Superblock<L>::kPerLane];
    if (u < units) sb_load<L>(tp, frame, stride, u / rs, lane, raw);
    for (; u < units; u += nw) {
        const long p = u / rs;
        const BayesRec rec = sb_setup<L>(tp, bp, lut, raw);
        if (u + nw < units) sb_load<L>(tp, frame, stride, (u + nw) / rs, lane, raw);
        run_unit<CPL>(bp, rec, p, (int)(u - p * rs), rs, lane, partial, count, chat, chat_scaled, scale);
    }
}

// Resident CTAs per SM for a kernel (cached per device and kernel) and the SM count.
template <typename K>
cudaError_t residency(K kernel, int& resident, int& sms) {
    static int cache_res[64], cache_sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cache_res[dev] == 0) {
        e = cudaDeviceGetAttribute(&cache_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cache_res[dev], kernel, kThreads, 0);
        if (e != cudaSuccess) return e;
        if (cache_res[dev] < 1) cache_res[dev] = 1;
    }
    resident = cache_res[dev];
    sms = cache_sms[dev];
    return cudaSuccess;
}

// Parts per pixel: enough units per warp that the last round is a small part of the work.
inline long parts_for(long npix, long warps, int max_parts, int n0) {
    long rs = (8 * warps + npix - 1) / npix;
    if (rs < 1) rs = 1;
    if (rs > max_parts) rs = max_parts;
    if (rs > n0) rs = n0;
    return rs;
}

template <int CPL>
cudaError_t launch_cpl(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                       float2* chat, float2* chat_scaled, float scale, cudaStream_t s) {
    int resident = 0, sms = 0;
    cudaError_t e = residency(posterior_kernel<CPL>, resident, sms);
    if (e != cudaSuccess) return e;
    const long rs = parts_for(npix, (long)sms * resident * (kThreads / 32), sc.max_parts, bp.n0);
    long blocks = (npix * rs + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    posterior_kernel<CPL><<<(unsigned)blocks, kThreads, 0, s>>>(bp, rec, npix, (int)rs, sc.partial, sc.count, chat,
                                                                chat_scaled, scale);
    return cudaGetLastError();
}

template <int CPL, int L>
cudaError_t launch_frame_cpl(const TransformParams& tp, const BayesParams& bp, const unsigned char* frame,
                             size_t stride, const float2* lut, const PosteriorScratch& sc, float2* chat,
                             float2* chat_scaled, float scale, cudaStream_t s) {
    int resident = 0, sms = 0;
    cudaError_t e = residency(posterior_frame_kernel<CPL, L>, resident, sms);
    if (e != cudaSuccess) return e;
    const long npix = (long)tp.hl * tp.wl;
    // each unit repeats its pixel's low-pass prologue, so split pixels only when there
    // are fewer pixels than resident warps
    const long warps = (long)sms * resident * (kThreads / 32);
    const long rs = npix >= warps ? 1 : parts_for(npix, warps, sc.max_parts, bp.n0);
    long blocks = (npix * rs + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    posterior_frame_kernel<CPL, L><<<(unsigned)blocks, kThreads, 0, s>>>(tp, bp, frame, stride, lut, (int)rs,
                                                                         sc.partial, sc.count, chat, chat_scaled,
                                                                         scale);
    return cudaGetLastError();
}

template <int CPL>
cudaError_t launch_frame_levels(const TransformParams& tp, const BayesParams& bp, const unsigned char* frame,
                                size_t stride, const float2* lut, const PosteriorScratch& sc, float2* chat,
                                float2* chat_scaled, float scale, cudaStream_t s) {
    switch (tp.levels) {
        case 0: return launch_frame_cpl<CPL, 0>(tp, bp, frame, stride, lut, sc, chat, chat_scaled, scale, s);
        case 1: return launch_frame_cpl<CPL, 1>(tp, bp, frame, stride, lut, sc, chat, chat_scaled, scale, s);
        case 2: return launch_frame_cpl<CPL, 2>(tp, bp, frame, stride, lut, sc, chat, chat_scaled, scale, s);
        case 3: return launch_frame_cpl<CPL, 3>(tp, bp, frame, stride, lut, sc, chat, chat_scaled, scale, s);
        case 4: return launch_frame_cpl<CPL, 4>(tp, bp, frame, stride, lut, sc, chat, chat_scaled, scale, s);
        default: return cudaErrorInvalidValue;  // 5-6 levels go through the analysis kernel and records
    }
}

}  // namespace

cudaError_t launch_posterior(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                             float2* chat, float2* chat_scaled, float scale, cudaStream_t s) {
    if (npix <= 0) return cudaSuccess;
    if (bp.n1 <= 32) return launch_cpl<1>(bp, rec, npix, sc, chat, chat_scaled, scale, s);
    if (bp.n1 <= 64) return launch_cpl<2>(bp, rec, npix, sc, chat, chat_scaled, scale, s);
    if (bp.n1 <= 128) return launch_cpl<4>(bp, rec, npix, sc, chat, chat_scaled, scale, s);
    return launch_cpl<8>(bp, rec, npix, sc, chat, chat_scaled, scale, s);
}

cudaError_t launch_posterior_frame(const TransformParams& tp, const BayesParams& bp, const void* frame,
                                   size_t stride, const float2* lut, const PosteriorScratch& sc, float2* chat,
                                   float2* chat_scaled, float scale, cudaStream_t s) {
    if ((long)tp.hl * tp.wl <= 0) return cudaSuccess;
    if (tp.levels > 4) return cudaErrorInvalidValue;
    const unsigned char* f = static_cast<const unsigned char*>(frame);
    if (bp.n1 <= 32) return launch_frame_levels<1>(tp, bp, f, stride, lut, sc, chat, chat_scaled, scale, s);
    if (bp.n1 <= 64) return launch_frame_levels<2>(tp, bp, f, stride, lut, sc, chat, chat_scaled, scale, s);
    if (bp.n1 <= 128) return launch_frame_levels<4>(tp, bp, f, stride, lut, sc, chat, chat_scaled, scale, s);
    return launch_frame_levels<8>(tp, bp, f, stride, lut, sc, chat, chat_scaled, scale, s);
}

}  // namespace hb
