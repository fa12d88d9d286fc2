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
// Work split: a unit is (pixel, part); lane l of a warp takes grid columns l, l+32,
// l+64, ... and the rs parts of a pixel take contiguous row ranges (rs = 1 unless there
// are fewer pixels than resident warps: a split costs partial sums and an atomic
// hand-off).  Warps are persistent (one grid of resident CTAs walks all units) and
// prefetch the next unit's record.  Per pair of grid nodes a lane issues two packed
// FP32x2 FMAs for the exponents, two MUFU ex2 and two packed instructions for the sums
// (sum w and sum w*di per column; sum w*dj follows from the column sums).  Warp shuffles
// combine lanes; when a pixel is split, the last part to finish (atomic counter) adds
// the parts' sums in a fixed order, so results do not depend on scheduling.
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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__device__ __forceinline__ bool usable(float sw, float sdi, float sdj) {
    return sw > 0.f && isfinite(sw) && isfinite(sdi) && isfinite(sdj);
}

// Posterior mean from the sums, in FP32 (the output is FP32): c = c_ref + h * (sum w d / sum w).
__device__ __forceinline__ void write_mean(const BayesParams& bp, const BayesRec& rec, long p, float sw, float sdi,
                                           float sdj, float2* chat, float2* chat_scaled, float scale) {
    const float c0 = fmaf(bp.h0f, sdi / sw, fmaf((float)rec.i0, bp.h0f, bp.lo0f));
    const float c1 = fmaf(bp.h1f, sdj / sw, fmaf((float)rec.j0, bp.h1f, bp.lo1f));
    chat[p] = make_float2(c0, c1);
    if (chat_scaled) chat_scaled[p] = make_float2(c0 * scale, c1 * scale);
}

// One unit: the sums over its rows, then either the pixel's result (rs == 1) or its
// partial sums; the last part of a pixel to arrive adds the parts in order and writes
// the result.  A pixel whose total sums are not usable (only possible for inputs far
// outside the model) is summed again over all rows with an explicit maximum shift.
// grid_sums has a single call site so that the rare path costs the loop no registers.
template <int CPL>
__device__ __forceinline__ void run_unit(const BayesParams& bp, const BayesRec& rec, long p, int part, int rs,
                                         int lane, float* partial, unsigned* count, float2* chat,
                                         float2* chat_scaled, float scale) {
    int rb = (int)((long)bp.n0 * part / rs), re = (int)((long)bp.n0 * (part + 1) / rs);
    float shift = 0.f;
    bool whole = rs == 1;  // sums cover the whole pixel
    while (true) {
        float sw = 0.f, sdi = 0.f, sdj = 0.f;
        grid_sums<CPL>(bp, rec, lane, rb, re, shift, sw, sdi, sdj);
        sw = warp_sum(sw);
        sdi = warp_sum(sdi);
        sdj = warp_sum(sdj);
        if (!whole) {
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
            if (prior != (unsigned)(rs - 1)) return;
            __threadfence();
            sw = sdi = sdj = 0.f;
            if (lane == 0) {
                const volatile float* slots = partial + (size_t)p * rs * 3;
                for (int k = 0; k < rs; ++k) {
                    sw += slots[3 * k];
                    sdi += slots[3 * k + 1];
                    sdj += slots[3 * k + 2];
                }
                count[p] = 0u;
            }
            sw = __shfl_sync(0xffffffffu, sw, 0);
            sdi = __shfl_sync(0xffffffffu, sdi, 0);
            sdj = __shfl_sync(0xffffffffu, sdj, 0);
            whole = true;
        }
        if (usable(sw, sdi, sdj) || shift != 0.f) {
            if (lane == 0) write_mean(bp, rec, p, sw, sdi, sdj, chat, chat_scaled, scale);
            return;
        }
        rb = 0;
        re = bp.n0;
        shift = warp_max(grid_max<CPL>(bp, rec, lane, 0, bp.n0));
        if (!(shift != 0.f)) shift = -1.f;  // any non-zero shift marks the second pass
    }
}

// Posterior over precomputed per-pixel records (the stand-alone posterior entry point).
template <int CPL>
__global__ void HB_POST_BOUNDS posterior_kernel(BayesParams bp, const BayesRec* __restrict__ recs, long npix, int rs,
                                                float* partial, unsigned* count, float2* __restrict__ chat,
                                                float2* __restrict__ chat_scaled, float scale, PosteriorGate gate) {
    // gated launch (fallback of the learned stand-in): run only when the summed sampled
    // error of the stand-in exceeded its threshold (a NaN sum also runs)
    if (gate.err_sum) {
        if (*gate.err_sum <= gate.threshold) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(gate.fallbacks, 1u);
    }
    const int lane = threadIdx.x & 31;
    const long nw = (long)gridDim.x * (kThreads / 32);
    const long units = npix * rs;
    long u = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    // launched with PDL after the analysis kernel: wait for its records, then let the
    // synthesis kernel be scheduled
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    BayesRec next = {0, 0, 0.f, 0.f};
    if (u < units) next = recs[u / rs];
    for (; u < units; u += nw) {
        const long p = u / rs;
        const BayesRec rec = next;
        if (u + nw < units) next = recs[(u + nw) / rs];
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
                       float2* chat, float2* chat_scaled, float scale, bool pdl, const PosteriorGate& gate,
                       cudaStream_t s) {
    int resident = 0, sms = 0;
    cudaError_t e = residency(posterior_kernel<CPL>, resident, sms);
    if (e != cudaSuccess) return e;
    // splitting a pixel costs partial sums and an atomic hand-off, so only when there
    // are fewer pixels than resident warps
    const long warps = (long)sms * resident * (kThreads / 32);
    const long rs = npix >= warps ? 1 : parts_for(npix, warps, sc.max_parts, bp.n0);
    long blocks = (npix * rs + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, posterior_kernel<CPL>, bp, rec, npix, (int)rs, sc.partial, sc.count, chat,
                              chat_scaled, scale, gate);
}

}  // namespace

cudaError_t launch_posterior(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                             float2* chat, float2* chat_scaled, float scale, bool pdl, cudaStream_t s,
                             const PosteriorGate& gate) {
    if (npix <= 0) return cudaSuccess;
    if (bp.n1 <= 32) return launch_cpl<1>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    if (bp.n1 <= 64) return launch_cpl<2>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    if (bp.n1 <= 128) return launch_cpl<4>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    return launch_cpl<8>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
}

namespace {

// Exact posterior mean of a sample of pixels, compared with another estimate of them:
// each pixel's error relative to the box extents (the larger of the two axes) is added
// to *err_sum (a NaN error makes the sum NaN).
template <int CPL>
__global__ void __launch_bounds__(kThreads) posterior_check_kernel(BayesParams bp, const BayesRec* __restrict__ recs,
                                                                   long npix, int nsample, unsigned seed,
                                                                   const float2* __restrict__ est, float inv_ext0,
                                                                   float inv_ext1, float* err_sum) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (w >= nsample) return;
    unsigned h = seed * 0x9E3779B9U + (unsigned)w * 0x85EBCA6BU;
    h ^= h >> 16;
    h *= 0x7feb352dU;
    h ^= h >> 15;
    h *= 0x846ca68bU;
    h ^= h >> 16;
    const long p = (long)(h % (unsigned long)npix);
    const BayesRec rec = recs[p];
    float shift = 0.f, sw, sdi, sdj;
    for (int pass = 0; pass < 2; ++pass) {
        sw = sdi = sdj = 0.f;
        grid_sums<CPL>(bp, rec, lane, 0, bp.n0, shift, sw, sdi, sdj);
        sw = warp_sum(sw);
        sdi = warp_sum(sdi);
        sdj = warp_sum(sdj);
        if (usable(sw, sdi, sdj)) break;
        shift = warp_max(grid_max<CPL>(bp, rec, lane, 0, bp.n0));
    }
    if (lane == 0) {
        const float c0 = fmaf(bp.h0f, sdi / sw, fmaf((float)rec.i0, bp.h0f, bp.lo0f));
        const float c1 = fmaf(bp.h1f, sdj / sw, fmaf((float)rec.j0, bp.h1f, bp.lo1f));
        const float2 e = est[p];
        const float dx = fabsf(e.x - c0) * inv_ext0, dy = fabsf(e.y - c1) * inv_ext1;
        const float err = isnan(dx) || isnan(dy) ? NAN : fmaxf(dx, dy);
        atomicAdd(err_sum, err);
    }
}

template <int CPL>
cudaError_t launch_check_cpl(const BayesParams& bp, const BayesRec* rec, long npix, int nsample, unsigned seed,
                             const float2* est, float inv_ext0, float inv_ext1, float* err_sum, cudaStream_t s) {
    const int blocks = (nsample + kThreads / 32 - 1) / (kThreads / 32);
    posterior_check_kernel<CPL><<<blocks, kThreads, 0, s>>>(bp, rec, npix, nsample, seed, est, inv_ext0, inv_ext1,
                                                            err_sum);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_posterior_check(const BayesParams& bp, const BayesRec* rec, long npix, int nsample, unsigned seed,
                                   const float2* est, float inv_ext0, float inv_ext1, float* err_sum,
                                   cudaStream_t s) {
    if (npix <= 0 || nsample <= 0) return cudaSuccess;
    if (bp.n1 <= 32) return launch_check_cpl<1>(bp, rec, npix, nsample, seed, est, inv_ext0, inv_ext1, err_sum, s);
    if (bp.n1 <= 64) return launch_check_cpl<2>(bp, rec, npix, nsample, seed, est, inv_ext0, inv_ext1, err_sum, s);
    if (bp.n1 <= 128) return launch_check_cpl<4>(bp, rec, npix, nsample, seed, est, inv_ext0, inv_ext1, err_sum, s);
    return launch_check_cpl<8>(bp, rec, npix, nsample, seed, est, inv_ext0, inv_ext1, err_sum, s);
}

}  // namespace hb
