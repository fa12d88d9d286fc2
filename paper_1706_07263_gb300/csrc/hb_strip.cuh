// hb_strip.cuh -- the register Haar transforms of the strip kernels (two pixel columns
// per lane, 1..3 levels), shared by the transform kernels and the fused low-pass kernel.
// Internal to libhb (header-only, so that they inline without relocatable device code).
#pragma once

#include "hb_common.cuh"

#include <math.h>

namespace hb {
namespace {

constexpr unsigned kStripFull = 0xffffffffu;

// ------------------------------------------------------------------------------------
// Strip variants for 1..3 levels: lane l of a warp owns the two pixel columns
// x = 2 (32 w + l) + {0, 1} of one superblock band (2^n rows), so the first level's 2x2
// windows lie inside the lane and a superblock spans 2^(n-1) neighbouring lanes.  Every
// level is computed as unscaled butterflies (sums and differences, i.e. 2 H per level):
// the first level inside the lane; level l >= 2 as a butterfly across lanes (lane ^
// 2^(l-2)) on the slots holding level-(l-1) low passes, then one across those slots' rows
// inside the lane.  The lanes taking part in level l are those with lane % 2^(l-2) == 0;
// a slot that a level leaves as a directional coefficient is not touched again.  With the
// unscaled forward the level-l coefficients are 2^l times Eq. 2's; the inverse (Eq. 4,
// H = H*) run as the same unscaled butterflies reproduces the pixels when it is fed the
// level-l coefficients times 4^-l -- the Tikhonov operator is applied as M 4^-l -- and the
// low pass as the block mean.  All these factors are powers of two.
// ------------------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void strip_load(const TransformParams& tp, const unsigned char* __restrict__ frame,
                                           size_t stride, const float2* lut, int by, int x0, int lane,
                                           float (&v)[3][1 << L][2], float2 (&yref)[3]) {
    constexpr int TH = 1 << L;
    const int xa = min(x0, tp.W - 1), xb = min(x0 + 1, tp.W - 1);
    const int src_lane = lane & ~((TH >> 1) - 1);  // the superblock's first lane
    if (tp.fmt == 1) {
        // The lane's six bytes per row (two pixels, x0 even) start at byte 3 x0, 2-byte aligned.
        // With 4-byte aligned rows they lie in the two 32-bit words from (3 x0) & ~3 on, which are
        // loaded whole when they end inside the row (every lane but, at most, the last one of a
        // row); otherwise the bytes are loaded one by one.  Either way a row's bytes are kept
        // packed (lo: pixel x0's three channels and pixel x0 + 1's first, hi: the other two), and
        // the log table is read per row, so the raw data takes 2 registers per row.
        const int b0 = 3 * x0, a0 = b0 & ~3;
        const bool words = ((reinterpret_cast<uintptr_t>(frame) | stride) & 3) == 0 && x0 + 1 < tp.W &&
                           a0 + 8 <= 3 * tp.W;
        const unsigned sel_lo = (b0 & 2) ? 0x5432u : 0x3210u, sel_hi = (b0 & 2) ? 0x0076u : 0x0054u;
        unsigned lo[TH], hi[TH];
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            const unsigned char* row = frame + (size_t)min(by * TH + r, tp.H - 1) * stride;
            if (words) {
                const unsigned w0 = __ldg(reinterpret_cast<const unsigned*>(row + a0));
                const unsigned w1 = __ldg(reinterpret_cast<const unsigned*>(row + a0 + 4));
                lo[r] = __byte_perm(w0, w1, sel_lo);
                hi[r] = __byte_perm(w0, w1, sel_hi);
            } else {
                const unsigned char* pa = row + (size_t)xa * 3;
                const unsigned char* pb = row + (size_t)xb * 3;
                lo[r] = (unsigned)__ldg(pa) | ((unsigned)__ldg(pa + 1) << 8) | ((unsigned)__ldg(pa + 2) << 16) |
                        ((unsigned)__ldg(pb) << 24);
                hi[r] = (unsigned)__ldg(pb + 1) | ((unsigned)__ldg(pb + 2) << 8);
            }
        }
        const unsigned lo_ref = __shfl_sync(kStripFull, lo[0], src_lane);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) yref[ch] = __ldg(lut + ((lo_ref >> (8 * ch)) & 0xff));
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            const unsigned code[3][2] = {{lo[r] & 0xff, lo[r] >> 24},
                                         {(lo[r] >> 8) & 0xff, hi[r] & 0xff},
                                         {(lo[r] >> 16) & 0xff, (hi[r] >> 8) & 0xff}};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float2 y = __ldg(lut + code[ch][c]);
                    v[ch][r][c] = (y.x - yref[ch].x) + (y.y - yref[ch].y);
                }
        }
    } else {
#pragma unroll
        for (int r = 0; r < TH; ++r) {
            const float* row = reinterpret_cast<const float*>(frame + (size_t)min(by * TH + r, tp.H - 1) * stride);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                v[ch][r][0] = -logf(fmaxf(__ldg(row + (size_t)xa * 3 + ch), tp.eps));
                v[ch][r][1] = -logf(fmaxf(__ldg(row + (size_t)xb * 3 + ch), tp.eps));
            }
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float yr = __shfl_sync(kStripFull, v[ch][0][0], src_lane);
            yref[ch] = make_float2(yr, 0.f);
#pragma unroll
            for (int r = 0; r < TH; ++r) {
                v[ch][r][0] -= yr;
                v[ch][r][1] -= yr;
            }
        }
    }
}

// The unscaled forward levels in place.  LL_ONLY: only the low passes are formed (the
// block sum of each superblock), in slot (0, 0) of the superblock's first lane.
template <int L, int NCH, bool LL_ONLY>
__device__ __forceinline__ void strip_analysis(float (&v)[NCH][1 << L][2], int lane) {
    constexpr int TH = 1 << L;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
        for (int r = 0; r < TH; r += 2) {
            const float a = v[ch][r][0], b = v[ch][r][1], c = v[ch][r + 1][0], d = v[ch][r + 1][1];
            const float s1 = a + b, s2 = c + d;
            v[ch][r][0] = s1 + s2;                 // low pass
            if (!LL_ONLY) {
                const float d1 = a - b, d2 = c - d;
                v[ch][r][1] = s1 - s2;             // rows differ
                v[ch][r + 1][0] = d1 - d2;         // diagonal
                v[ch][r + 1][1] = d1 + d2;         // columns differ
            }
        }
#pragma unroll
    for (int l = 2; l <= L; ++l) {
        const int s = 1 << (l - 2), rs = 1 << (l - 1);
        const bool active = (lane & (s - 1)) == 0;
        const float sgn = (lane & s) ? -1.f : 1.f;  // left lane: own + partner; right: partner - own
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += rs) {
                const float x = v[ch][r][0];
                const float q = fmaf(sgn, x, __shfl_xor_sync(kStripFull, x, s));
                if (active) v[ch][r][0] = q;
            }
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += 2 * rs)
                if (active) {
                    const float a = v[ch][r][0], b = v[ch][r + rs][0];
                    v[ch][r][0] = a + b;
                    if (!LL_ONLY) v[ch][r + rs][0] = a - b;
                }
    }
}

// The unscaled inverse levels in place (the forward's steps undone in reverse order).
template <int L>
__device__ __forceinline__ void strip_synthesis(float (&c)[2][1 << L][2], int lane) {
    constexpr int TH = 1 << L;
#pragma unroll
    for (int l = L; l >= 2; --l) {
        const int s = 1 << (l - 2), rs = 1 << (l - 1);
        const bool active = (lane & (s - 1)) == 0;
        const float sgn = (lane & s) ? -1.f : 1.f;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += 2 * rs)
                if (active) {
                    const float a = c[ch][r][0], b = c[ch][r + rs][0];
                    c[ch][r][0] = a + b;
                    c[ch][r + rs][0] = a - b;
                }
#pragma unroll
        for (int ch = 0; ch < 2; ++ch)
#pragma unroll
            for (int r = 0; r < TH; r += rs) {
                const float x = c[ch][r][0];
                const float q = fmaf(sgn, x, __shfl_xor_sync(kStripFull, x, s));
                if (active) c[ch][r][0] = q;
            }
    }
#pragma unroll
    for (int ch = 0; ch < 2; ++ch)
#pragma unroll
        for (int r = 0; r < TH; r += 2) {
            const float ll = c[ch][r][0], dr = c[ch][r][1], dd = c[ch][r + 1][0], dc = c[ch][r + 1][1];
            const float s1 = ll + dr, s2 = ll - dr, d1 = dc + dd, d2 = dc - dd;
            c[ch][r][0] = s1 + d1;
            c[ch][r][1] = s1 - d1;
            c[ch][r + 1][0] = s2 + d2;
            c[ch][r + 1][1] = s2 - d2;
        }
}

// Level of the coefficient left in slot (r, 0), r even, of lane `lane` after the forward
// levels (0: the superblock's low pass).  Level l >= 2 turns a slot into a directional
// coefficient by its butterfly across lanes (lane bit l-2) or across rows (row bit l-1).
__device__ __forceinline__ int strip_slot_level(int r, int lane, int L) {
    for (int l = 2; l <= L; ++l) {
        if ((lane >> (l - 2)) & 1) return l;
        if ((r >> (l - 1)) & 1) return l;
    }
    return 0;
}


// The Tikhonov operator (Eq. 5) on the unscaled forward coefficients v (three channels) into
// c (HbO2, Hb): level-1 coefficients (odd rows, second column) with M / 4; the first
// column's even rows by their level (the low pass: 0, or M 4^-L in the all-Tikhonov mode).
template <int L>
__device__ __forceinline__ void strip_tikhonov(const TransformParams& tp, const float (&v)[3][1 << L][2], int lane,
                                               float (&c)[2][1 << L][2]) {
    constexpr int TH = 1 << L;
    const float* M = tp.M;
#pragma unroll
    for (int r = 0; r < TH; ++r)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float v0 = v[0][r][k], v1 = v[1][r][k], v2 = v[2][r][k];
            float sc = 0.25f;
            if (k == 0 && (r & 1) == 0) {
                const int lv = strip_slot_level(r, lane, L);
                // 4^-lv exactly; the low pass (lv = 0) keeps 4^-L only in the all-Tikhonov mode
                sc = lv ? __int_as_float((127 - 2 * lv) << 23)
                        : (tp.tikhonov_lowpass ? 1.f / (float)(TH * TH) : 0.f);
            }
            c[0][r][k] = sc * fmaf(M[0], v0, fmaf(M[1], v1, M[2] * v2));
            c[1][r][k] = sc * fmaf(M[3], v0, fmaf(M[4], v1, M[5] * v2));
        }
}

// All-Tikhonov mode: the superblock's reference log-attenuation (subtracted before the
// transform) through M, added back after the inverse.
__device__ __forceinline__ void strip_tikhonov_offset(const TransformParams& tp, const float2 (&yref)[3], float& off0,
                                                      float& off1) {
    const float* M = tp.M;
    off0 = (M[0] * yref[0].x + M[1] * yref[1].x + M[2] * yref[2].x) +
           (M[0] * yref[0].y + M[1] * yref[1].y + M[2] * yref[2].y);
    off1 = (M[3] * yref[0].x + M[4] * yref[1].x + M[5] * yref[2].x) +
           (M[3] * yref[0].y + M[4] * yref[1].y + M[5] * yref[2].y);
}

// The lane's two pixel columns x, x + 1 of superblock band by after the inverse transform:
// HbO2 = c[0] + off0, Hb = c[1] + off1 (the low pass enters as the offsets: its inverse is the
// block mean broadcast over the superblock), stored as THb and SO2 (SO2 = 0 where THb <= 0)
// or, with debug_conc, as HbO2 and Hb.  Columns and rows beyond the frame are not stored.
template <int L>
__device__ __forceinline__ void strip_store(const TransformParams& tp, const float (&c)[2][1 << L][2], float off0,
                                            float off1, int x, int by, float* __restrict__ out0,
                                            float* __restrict__ out1, int debug_conc) {
    constexpr int TH = 1 << L;
    if (x >= tp.W) return;
    const bool pair = x + 1 < tp.W;
    const bool vec = pair && ((tp.W & 1) == 0);  // 8-byte aligned pairs of outputs
#pragma unroll
    for (int r = 0; r < TH; ++r) {
        const int gy = by * TH + r;
        if (gy >= tp.H) break;
        float a0, a1, b0, b1;
        const float h0 = c[0][r][0] + off0, h1 = c[0][r][1] + off0;  // HbO2
        const float g0 = c[1][r][0] + off1, g1 = c[1][r][1] + off1;  // Hb
        if (debug_conc) {
            a0 = h0;
            a1 = h1;
            b0 = g0;
            b1 = g1;
        } else {
            a0 = h0 + g0;
            a1 = h1 + g1;
            // SO2 needs 1e-3 absolute: the fast reciprocal-based division (2 ulp) is plenty
            b0 = a0 >= 1.17549435e-38f ? __fdividef(h0, a0) : (a0 > 0.f ? h0 / a0 : 0.f);
            b1 = a1 >= 1.17549435e-38f ? __fdividef(h1, a1) : (a1 > 0.f ? h1 / a1 : 0.f);
        }
        const size_t o = (size_t)gy * tp.W + x;
        if (vec) {
            *reinterpret_cast<float2*>(out0 + o) = make_float2(a0, a1);
            *reinterpret_cast<float2*>(out1 + o) = make_float2(b0, b1);
        } else {
            out0[o] = a0;
            out1[o] = b0;
            if (pair) {
                out0[o + 1] = a1;
                out1[o + 1] = b1;
            }
        }
    }
}

}  // namespace
}  // namespace hb
