// hb_device.cuh -- device helpers shared by the translation units of libhb
// (header-only so that they inline without relocatable device code).
#pragma once

#include "hb_common.cuh"

#include <math.h>

namespace hb {

// Reference node and linear coefficients of the posterior for one low-pass pixel.
// The reference node is the grid node nearest to the maximiser of the likelihood
// over the hull of the grid -- a 2-D box-constrained least-squares problem solved
// exactly by checking the interior optimum and then the four edges.  It only fixes
// where the log-likelihood is expanded (so that the FP32 sums near the posterior
// peak involve small numbers); any node gives the same posterior mean in exact
// arithmetic.  Everything here is FP32: the block mean arrives as an unevaluated
// float pair yhi + ylo, and the residual ybar - A c_ref, where the cancellation
// happens, is formed in double-float arithmetic (error-free sums and products).
namespace detail {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) -= (bh, bl), renormalised
__device__ __forceinline__ void dd_sub(float& hi, float& lo, float bh, float bl) {
    float s, e;
    two_sum(hi, -bh, s, e);
    e += lo - bl;
    hi = s + e;
    lo = e - (hi - s);
}

// With the illumination term the block mean minus its channel mean, (I - 11^T / 3) ybar,
// in double-float: the part along (1,1,1) cancels from the posterior, and removing it
// here keeps the residual -- and so the rounding of U and V -- as small as without the
// term (the posterior is much broader then, so its mean is that much more sensitive).
__device__ __forceinline__ void dd_remove_mean(float (&hi)[3], float (&lo)[3]) {
    float sh = hi[0], sl = lo[0];
    dd_sub(sh, sl, -hi[1], -lo[1]);
    dd_sub(sh, sl, -hi[2], -lo[2]);
    const float mh = sh * (1.f / 3.f);
    const float ml = (fmaf(-3.f, mh, sh) + sl) * (1.f / 3.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) dd_sub(hi[c], lo[c], mh, ml);
}

}  // namespace detail

__device__ __forceinline__ BayesRec bayes_setup(const float yhi_in[3], const float ylo_in[3], const BayesParams& bp) {
    float yhi[3] = {yhi_in[0], yhi_in[1], yhi_in[2]}, ylo[3] = {ylo_in[0], ylo_in[1], ylo_in[2]};
    if (bp.illum) detail::dd_remove_mean(yhi, ylo);
    const float y0 = yhi[0] + ylo[0], y1 = yhi[1] + ylo[1], y2 = yhi[2] + ylo[2];
    const float z0 = bp.Af[0] * y0 + bp.Af[2] * y1 + bp.Af[4] * y2;
    const float z1 = bp.Af[1] * y0 + bp.Af[3] * y1 + bp.Af[5] * y2;
    const float lo0 = bp.lo0f, hi0 = bp.hi0f, lo1 = bp.lo1f, hi1 = bp.hi1f;
    float c0 = bp.Gi00 * z0 + bp.Gi01 * z1;
    float c1 = bp.Gi01 * z0 + bp.Gi11 * z1;
    if (!(c0 >= lo0 && c0 <= hi0 && c1 >= lo1 && c1 <= hi1)) {
        // objective |y - A c|^2 - |y|^2 = c^T G c - 2 z^T c, minimised on each edge
        float best = INFINITY, b0 = lo0, b1 = lo1;
        for (int e = 0; e < 4; ++e) {
            float a0, a1;
            if (e < 2) {
                a0 = e == 0 ? lo0 : hi0;
                a1 = bp.G11 > 0.f ? (z1 - bp.G01 * a0) * bp.inv_G11 : lo1;
                a1 = fminf(fmaxf(a1, lo1), hi1);
            } else {
                a1 = e == 2 ? lo1 : hi1;
                a0 = bp.G00 > 0.f ? (z0 - bp.G01 * a1) * bp.inv_G00 : lo0;
                a0 = fminf(fmaxf(a0, lo0), hi0);
            }
            const float f = a0 * (bp.G00 * a0 + 2.f * bp.G01 * a1) + bp.G11 * a1 * a1 - 2.f * (z0 * a0 + z1 * a1);
            if (f < best) { best = f; b0 = a0; b1 = a1; }
        }
        c0 = b0;
        c1 = b1;
    }
    BayesRec rec;
    rec.i0 = min(max(__float2int_rn((c0 - lo0) * bp.inv_h0f), 0), bp.n0 - 1);
    rec.j0 = min(max(__float2int_rn((c1 - lo1) * bp.inv_h1f), 0), bp.n1 - 1);
    // r = ybar - (base + i0 step0 + j0 step1) in double-float
    const float fi = (float)rec.i0, fj = (float)rec.j0;
    float U = 0.f, V = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float hi = yhi[c], lo = ylo[c];
        detail::dd_sub(hi, lo, bp.base_hi[c], bp.base_lo[c]);
        const float p0 = fi * bp.step0_hi[c];
        detail::dd_sub(hi, lo, p0, fmaf(fi, bp.step0_hi[c], -p0) + fi * bp.step0_lo[c]);
        const float p1 = fj * bp.step1_hi[c];
        detail::dd_sub(hi, lo, p1, fmaf(fj, bp.step1_hi[c], -p1) + fj * bp.step1_lo[c]);
        const float r = hi + lo;
        U = fmaf(r, bp.u_scalef[c], U);
        V = fmaf(r, bp.v_scalef[c], V);
    }
    rec.U = U;
    rec.V = V;
    return rec;
}

// The low-pass output of one superblock o from its block mean yhi + ylo: the posterior
// record, or with a least-squares low pass the estimate itself (the 2x3 operator applied to
// the float pair).  With the illumination term the operator annihilates (1,1,1) only in
// exact arithmetic: ybar's channel mean is removed first, in double-float, so that the
// rounding of the FP32 operator does not meet it (it can be large against the concentrations
// when the system [A | 1] is ill-conditioned).
__device__ __forceinline__ void low_pass_out(const float yhi[3], const float ylo[3], const TransformParams& tp,
                                             const BayesParams& bp, size_t o, BayesRec* rec, const LsOut& ls) {
    if (ls.c) {
        float h[3] = {yhi[0], yhi[1], yhi[2]}, l[3] = {ylo[0], ylo[1], ylo[2]};
        if (bp.illum) detail::dd_remove_mean(h, l);
        float c[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float* L = tp.ls_L + 3 * j;
            c[j] = fmaf(L[0], h[0], fmaf(L[1], h[1], L[2] * h[2])) + fmaf(L[0], l[0], fmaf(L[1], l[1], L[2] * l[2]));
        }
        ls.c[o] = make_float2(c[0], c[1]);
        if (ls.c_scaled) ls.c_scaled[o] = make_float2(c[0] * ls.scale, c[1] * ls.scale);
    } else {
        rec[o] = bayes_setup(yhi, ylo, bp);
    }
}

}  // namespace hb
