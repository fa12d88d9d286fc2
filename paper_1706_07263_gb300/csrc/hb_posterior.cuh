// hb_posterior.cuh -- the grid posterior's per-pixel sums and support bounds, shared by
// the posterior kernels and the learned stand-in's sampled check.  Internal to libhb.
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
// Whole-row kernels enumerate only the grid rows that can hold a non-zero FP32 weight
// (support_rows): outside them every 2^t is below 2^-150 and ex2.approx.ftz returns
// exactly 0, so the sums are those over the whole grid up to the order of the additions.
// The span kernel enumerates, per row, the column interval of span_pixel / span_row, whose
// cut leaves out only nodes carrying together less than 2^-30 of the posterior mass.
//
// Whole-row kernels: lane l of a group takes grid columns l, l+G, l+2G, ... (CPL columns
// per lane).  Per pair of grid nodes a lane issues two packed FP32x2 FMAs for the
// exponents, two MUFU ex2 and two packed instructions for the sums (sum w and sum w*di per
// column; sum w*dj follows from the column sums).
#pragma once

#include "hb_common.cuh"

#include <math.h>

#ifndef HB_POST_UNROLL
#define HB_POST_UNROLL 4   // grid rows per unrolled step of the posterior loop
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
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Column constants of one lane for the column block starting at j_base.  A pixel is
// handled by a group of G lanes (32: a warp; 16: half a warp); lane l of the group takes
// columns j_base + l + G s.
template <int CPL, int G = 32>
__device__ __forceinline__ void column_terms(const BayesParams& bp, const BayesRec& rec, int lane, int j_base,
                                             float shift, float (&dj)[CPL], float (&P)[CPL], float (&Q)[CPL]) {
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
        const int j = j_base + lane + G * s;
        dj[s] = (float)(j - rec.j0);
        P[s] = j < bp.n1 ? fmaf(bp.Cq * dj[s], dj[s], rec.V * dj[s]) - shift : -INFINITY;
        Q[s] = fmaf(2.f * bp.Bq, dj[s], rec.U);
    }
}

// sum w, sum w di, sum w dj over rows [rb, re) and the lane's columns (all column blocks),
// with weights 2^(t - shift).
template <int CPL, int G = 32>
__device__ __forceinline__ void grid_sums(const BayesParams& bp, const BayesRec& rec, int lane, int rb, int re,
                                          float shift, float& sw, float& sdi, float& sdj) {
    for (int jb = 0; jb < bp.n1; jb += G * CPL) {
        float dj[CPL], P[CPL], Q[CPL];
        column_terms<CPL, G>(bp, rec, lane, jb, shift, dj, P, Q);
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
template <int CPL, int G = 32>
__device__ float grid_max(const BayesParams& bp, const BayesRec& rec, int lane, int rb, int re) {
    float m = -INFINITY;
    for (int jb = 0; jb < bp.n1; jb += G * CPL) {
        float dj[CPL], P[CPL], Q[CPL];
        column_terms<CPL, G>(bp, rec, lane, jb, 0.f, dj, P, Q);
        float di = (float)(rb - rec.i0);
        for (int i = rb; i < re; ++i, di += 1.f)
#pragma unroll
            for (int s = 0; s < CPL; ++s) m = fmaxf(m, fmaf(di, fmaf(bp.Aq, di, Q[s]), P[s]));
    }
    return m;
}

// Sum / maximum over the G lanes of a group (xor shuffles stay inside aligned groups).
template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
template <int G>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
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

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// {x : qa x^2 + qb x + qc >= 0} for qa < 0 as [lo, hi] (lo > hi when empty); inv = 0.5 / qa.
// The approximate square root is far inside the row of widening the caller adds.
__device__ __forceinline__ void superlevel(float qa, float qb, float qc, float inv, float& lo, float& hi) {
    const float disc = fmaf(qb, qb, -4.f * qa * qc);
    if (!(disc >= 0.f)) {
        lo = INFINITY;
        hi = -INFINITY;
        return;
    }
    const float sq = sqrt_approx(disc);
    lo = (sq - qb) * inv;
    hi = (-qb - sq) * inv;
}

// Rows [lo, hi) of the grid that can hold a non-zero FP32 weight for this pixel (every
// row when the bound is off or not finite).  The largest exponent of row di over the
// grid's columns is the row maximum over real dj where that maximiser dj*(di) lies on the
// grid, else the exponent at the nearer edge column: a concave function of di made of
// three quadratic pieces.  The rows kept are the union over the pieces of (rows where the
// piece reaches -cut) within (rows where the piece applies, widened by one), widened by
// one more row; the reference row (weight exactly 1) is always kept.
// The exponent below which a node's FP32 weight is exactly zero, for the support bounds:
// kSupportCut plus a margin for the FP32 evaluation error of t.
__device__ __forceinline__ float support_cut(const BayesParams& bp, const BayesRec& rec) {
    return fmaf(1e-6f, fmaf(fabsf(rec.U), (float)bp.n0, fmaf(fabsf(rec.V), (float)bp.n1, bp.sup_mg)), kSupportCut);
}

// Narrows the rows [rlo, rhi] (relative to the reference row) where the unconstrained row
// maximum reaches -cut to those where the row's maximum over the grid's columns does: the
// maximum over real dj where the maximiser dj*(di) lies on the grid, else the exponent at the
// nearer edge column -- three quadratic pieces in di.  The rows kept are the union over the
// pieces of (rows where the piece reaches -cut) within (rows where the piece applies,
// widened by one).  Every grid node of a row left out is below -cut.
__device__ __forceinline__ void clip_rows_to_grid(const BayesParams& bp, const BayesRec& rec, float cut, float& rlo,
                                                  float& rhi) {
    const float k1 = -bp.sup_r;  // dj*(di) = k0 + k1 di
    if (bp.sup_inv_k1 == 0.f || !(rlo <= rhi)) return;
    const float k0 = 2.f * rec.V * bp.sup_c;
    const float ea = (-(float)rec.j0 - k0) * bp.sup_inv_k1, eb = ((float)(bp.n1 - 1 - rec.j0) - k0) * bp.sup_inv_k1;
    // where dj* falls left of the grid (a), on it (m), right of it (b)
    const float da_lo = k1 > 0.f ? -INFINITY : ea - 1.f, da_hi = k1 > 0.f ? ea + 1.f : INFINITY;
    const float db_lo = k1 > 0.f ? eb - 1.f : -INFINITY, db_hi = k1 > 0.f ? INFINITY : eb + 1.f;
    const float dm_lo = fminf(ea, eb) - 1.f, dm_hi = fmaxf(ea, eb) + 1.f;
    float ulo = INFINITY, uhi = -INFINITY;
    auto join = [&](float a0, float a1, float b0, float b1) {
        const float x0 = fmaxf(a0, b0), x1 = fminf(a1, b1);
        if (x0 <= x1) {
            ulo = fminf(ulo, x0);
            uhi = fmaxf(uhi, x1);
        }
    };
    join(rlo, rhi, dm_lo, dm_hi);
    float slo, shi;
    const float ja = -(float)rec.j0, jb = (float)(bp.n1 - 1 - rec.j0);
    superlevel(bp.Aq, fmaf(2.f * bp.Bq, ja, rec.U), fmaf(fmaf(bp.Cq, ja, rec.V), ja, cut), bp.sup_inv_aq, slo, shi);
    join(slo, shi, da_lo, da_hi);
    superlevel(bp.Aq, fmaf(2.f * bp.Bq, jb, rec.U), fmaf(fmaf(bp.Cq, jb, rec.V), jb, cut), bp.sup_inv_aq, slo, shi);
    join(slo, shi, db_lo, db_hi);
    if (!isnan(ulo) && !isnan(uhi) && ulo <= uhi) {
        rlo = fmaxf(rlo, ulo);
        rhi = fminf(rhi, uhi);
    }
}

__device__ __forceinline__ void support_rows(const BayesParams& bp, const BayesRec& rec, int& lo, int& hi) {
    lo = 0;
    hi = bp.n0;
    if (!bp.sup_rows) return;
    const float cut = support_cut(bp, rec);
    // unconstrained row maximum: -alpha di^2 + (U - r V) di + c V^2
    float rlo, rhi;
    superlevel(-bp.sup_alpha, fmaf(-bp.sup_r, rec.V, rec.U), fmaf(rec.V * rec.V, bp.sup_c, cut), bp.sup_inv_alpha,
               rlo, rhi);
    clip_rows_to_grid(bp, rec, cut, rlo, rhi);
    if (!(rlo <= rhi) || isnan(rlo) || isnan(rhi)) return;
    const float lim = (float)bp.n0 + 2.f;
    const int a = rec.i0 + (int)floorf(fmaxf(rlo, -lim)) - 1;
    const int z = rec.i0 + (int)ceilf(fminf(rhi, lim)) + 2;
    lo = min(max(a, 0), rec.i0);
    hi = max(min(z, bp.n0), rec.i0 + 1);
}

// Per-pixel constants of the column intervals (needs bp.sup_cols).  Over real dj the
// exponent of row di peaks at column j0 + dj*(di), dj*(di) = -(V + 2 Bq di) / (2 Cq), with
// the value t*(di) = -alpha di^2 + (U - r V) di + c V^2 (the row maximum of support_rows),
// and stays at or above -cut within h(di) = sqrt((t*(di) + cut) / -Cq) columns of it.
// cut = bp.span_cut plus a margin for the FP32 evaluation of t (as in support_cut): the
// nodes left out weigh less than 2^-span_cut each against the reference node, together
// less than 2^-30 of the posterior mass.  Centre and squared half-width are evaluated
// directly (the two-root formula would cancel).  Rows: where t*(di) >= -cut, widened by one
// row on each side and clipped to the grid (narrowing them further to the rows whose interval
// meets the grid's columns, as support_rows does, costs more per pixel than the rows it
// saves; the row kernel skips slots of rows that all miss the grid instead).  A pixel whose
// terms are so large that their
// FP32 rounding could move the bounds by whole columns (only for inputs far outside the
// model) takes every row and column.
constexpr int kSpanSeg = 16;  // columns per lattice segment

struct SpanPixel {
    float a2, b2, c2;   // h(di)^2 = (a2 di + b2) di + c2
    float k1, cc;       // centre column k1 di + cc
    int rlo, rhi;       // rows [rlo, rhi)
    bool whole;
};

__device__ __forceinline__ SpanPixel span_pixel(const BayesParams& bp, const BayesRec& rec) {
    SpanPixel sp;
    const float cut =
        fmaf(1e-6f, fmaf(fabsf(rec.U), (float)bp.n0, fmaf(fabsf(rec.V), (float)bp.n1, bp.sup_mg)), bp.span_cut);
    const float beta = fmaf(-bp.sup_r, rec.V, rec.U);
    const float gamma = bp.sup_c * rec.V * rec.V;
    sp.a2 = bp.span_a2;
    sp.b2 = beta * bp.span_inv_acq;
    sp.c2 = (gamma + cut) * bp.span_inv_acq;
    sp.k1 = -bp.sup_r;
    sp.cc = fmaf(rec.V, bp.span_cv, (float)rec.j0);
    float lo, hi;
    superlevel(-bp.sup_alpha, beta, gamma + cut, bp.sup_inv_alpha, lo, hi);
    sp.whole = !(fmaf(fabsf(beta), (float)bp.n0, gamma + bp.span_an2) <= 1e6f) || !(lo <= hi);
    if (sp.whole) {
        sp.rlo = 0;
        sp.rhi = bp.n0;
    } else {
        const float lim = (float)bp.n0 + 2.f;
        sp.rlo = min(max(rec.i0 + (int)floorf(fmaxf(lo, -lim)) - 1, 0), rec.i0);
        sp.rhi = max(min(rec.i0 + (int)ceilf(fminf(hi, lim)) + 2, bp.n0), rec.i0 + 1);
    }
    return sp;
}

// Lattice segments [ma, ma + ns) (kSpanSeg columns each; nseg in a row) of row i0 + di that meet
// the row's interval, widened by one column on the left and two on the right (far more than
// the rounding of the centre, the half-width and the approximate square root).
__device__ __forceinline__ void span_row(const SpanPixel& sp, int di, int nseg, int& ma, int& ns) {
    const float d = (float)di;
    const float h2 = fmaf(d, fmaf(sp.a2, d, sp.b2), sp.c2);
    const float c = fmaf(sp.k1, d, sp.cc);
    const float h = sqrt_approx(fmaxf(h2, 0.f));
    const int a = max(__float2int_rd((c - h - 1.f) * (1.f / kSpanSeg)), 0);
    const int b = min(__float2int_ru((c + h + 2.f) * (1.f / kSpanSeg)), nseg);
    ma = sp.whole ? 0 : a;
    ns = sp.whole ? nseg : (h2 >= 0.f ? max(b - a, 0) : 0);
}

// Columns [ja, jb) of row i0 + di: those of the row's interval widened by one column on the
// left and two on the right (the same cut as span_row, without rounding to segments),
// clipped to the grid; ja >= jb when the row holds none.
__device__ __forceinline__ void row_cols(const SpanPixel& sp, const BayesRec& rec, int di, int n1, int& ja,
                                         int& jb) {
    if (sp.whole) {
        ja = 0;
        jb = n1;
        return;
    }
    const float d = (float)di;
    const float h2 = fmaf(d, fmaf(sp.a2, d, sp.b2), sp.c2);
    const float c = fmaf(sp.k1, d, sp.cc);
    const float h = sqrt_approx(fmaxf(h2, 0.f));
    ja = max(__float2int_ru(c - h - 1.f), 0);
    jb = min(__float2int_rd(c + h + 2.f) + 1, n1);
    if (!(h2 >= 0.f) || jb < ja) jb = ja;
    (void)rec;
}

__device__ __forceinline__ bool usable(float sw, float sdi, float sdj) {
    return sw > 0.f && isfinite(sw) && isfinite(sdi) && isfinite(sdj);
}

// The k-th pixel of a seeded pseudo-random sample of npix pixels (an integer hash of
// (seed, k); draws may repeat).
__device__ __forceinline__ long sample_pixel(unsigned seed, int k, long npix) {
    unsigned h = seed * 0x9E3779B9U + (unsigned)k * 0x85EBCA6BU;
    h ^= h >> 16;
    h *= 0x7feb352dU;
    h ^= h >> 15;
    h *= 0x846ca68bU;
    h ^= h >> 16;
    return (long)(h % (unsigned long)npix);
}

// Posterior mean of one pixel computed by a whole CTA (every thread calls it): the support
// rows are shared out over the CTA's warps, whose sums are added in warp order.  The
// result is valid in warp 0.  part: shared scratch of kThreads / 32 x 3 floats.
template <int CPL>
__device__ float2 cta_posterior_mean(const BayesParams& bp, const BayesRec& rec, float (*part)[3]) {
    constexpr int kWarps = kThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lo, hi;
    support_rows(bp, rec, lo, hi);
    const int rb = lo + (hi - lo) * warp / kWarps, re = lo + (hi - lo) * (warp + 1) / kWarps;
    float sw = 0.f, sdi = 0.f, sdj = 0.f;
    grid_sums<CPL>(bp, rec, lane, rb, re, 0.f, sw, sdi, sdj);
    sw = warp_sum(sw);
    sdi = warp_sum(sdi);
    sdj = warp_sum(sdj);
    if (lane == 0) {
        part[warp][0] = sw;
        part[warp][1] = sdi;
        part[warp][2] = sdj;
    }
    __syncthreads();
    float2 c = make_float2(0.f, 0.f);
    if (warp == 0) {
        sw = sdi = sdj = 0.f;
        for (int w = 0; w < kWarps; ++w) {
            sw += part[w][0];
            sdi += part[w][1];
            sdj += part[w][2];
        }
        if (!usable(sw, sdi, sdj)) {  // far outside the model: all rows, explicit maximum shift
            const float shift = warp_max(grid_max<CPL>(bp, rec, lane, 0, bp.n0));
            sw = sdi = sdj = 0.f;
            grid_sums<CPL>(bp, rec, lane, 0, bp.n0, shift, sw, sdi, sdj);
            sw = warp_sum(sw);
            sdi = warp_sum(sdi);
            sdj = warp_sum(sdj);
        }
        c.x = fmaf(bp.h0f, sdi / sw, fmaf((float)rec.i0, bp.h0f, bp.lo0f));
        c.y = fmaf(bp.h1f, sdj / sw, fmaf((float)rec.j0, bp.h1f, bp.lo1f));
    }
    __syncthreads();
    return c;
}

}  // namespace
}  // namespace hb
