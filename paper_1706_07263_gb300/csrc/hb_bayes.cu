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

// Posterior mean from the sums; recomputes the pixel with an explicit maximum when the
// sums are not usable.  Warp-uniform; lane 0 writes.
template <int CPL>
__device__ void finish_pixel(const BayesParams& bp, const BayesRec& rec, long p, int lane, float sw, float sdi,
                             float sdj, float2* chat, float2* chat_scaled, float scale) {
    if (!(sw > 0.f) || !isfinite(sw) || !isfinite(sdi) || !isfinite(sdj)) {
        float m = grid_max<CPL>(bp, rec, lane, 0, bp.n0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        sw = sdi = sdj = 0.f;
        grid_sums<CPL>(bp, rec, lane, 0, bp.n0, m, sw, sdi, sdj);
        sw = warp_sum(sw);
        sdi = warp_sum(sdi);
        sdj = warp_sum(sdj);
    }
    if (lane == 0) {
        const double c0 = bp.lo0 + rec.i0 * bp.h0 + bp.h0 * ((double)sdi / (double)sw);
        const double c1 = bp.lo1 + rec.j0 * bp.h1 + bp.h1 * ((double)sdj / (double)sw);
        chat[p] = make_float2((float)c0, (float)c1);
        if (chat_scaled) chat_scaled[p] = make_float2((float)(c0 * scale), (float)(c1 * scale));
    }
}

template <int CPL>
__global__ void HB_POST_BOUNDS posterior_kernel(BayesParams bp, const BayesRec* __restrict__ recs,
                                                             long npix, int rs, float* partial, unsigned* count,
                                                             float2* __restrict__ chat,
                                                             float2* __restrict__ chat_scaled, float scale) {
    const int lane = threadIdx.x & 31;
    const long nw = (long)gridDim.x * (kThreads / 32);
    const long units = npix * rs;
    long u = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    BayesRec next = {0, 0, 0.f, 0.f};
    if (u < units) next = recs[u / rs];
    for (; u < units; u += nw) {
        const long p = u / rs;
        const int part = (int)(u - p * rs);
        const BayesRec rec = next;
        if (u + nw < units) next = recs[(u + nw) / rs];
        const int rb = (int)((long)bp.n0 * part / rs), re = (int)((long)bp.n0 * (part + 1) / rs);
        float sw = 0.f, sdi = 0.f, sdj = 0.f;
        grid_sums<CPL>(bp, rec, lane, rb, re, 0.f, sw, sdi, sdj);
        sw = warp_sum(sw);
        sdi = warp_sum(sdi);
        sdj = warp_sum(sdj);
        if (rs == 1) {
            finish_pixel<CPL>(bp, rec, p, lane, sw, sdi, sdj, chat, chat_scaled, scale);
            continue;
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
            // last part of this pixel: add the parts in order
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
}

template <int CPL>
cudaError_t launch_cpl(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                       float2* chat, float2* chat_scaled, float scale, cudaStream_t s) {
    // CTAs per SM at this kernel's register use, and SM count, cached per device
    static int cache_resident[64], cache_sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int& resident = cache_resident[dev];
    int& sms = cache_sms[dev];
    if (resident == 0) {
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, posterior_kernel<CPL>, kThreads, 0);
        if (e != cudaSuccess) return e;
        if (resident < 1) resident = 1;
    }
    const long warps = (long)sms * resident * (kThreads / 32);
    // enough units per warp that the last round is a small part of the work
    long rs = (8 * warps + npix - 1) / npix;
    if (rs < 1) rs = 1;
    if (rs > sc.max_parts) rs = sc.max_parts;
    if (rs > bp.n0) rs = bp.n0;
    const long units = npix * rs;
    long blocks = (units + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    posterior_kernel<CPL><<<(unsigned)blocks, kThreads, 0, s>>>(bp, rec, npix, (int)rs, sc.partial, sc.count, chat,
                                                                chat_scaled, scale);
    return cudaGetLastError();
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

}  // namespace hb
