// hb_bayes.cu -- posterior mean of (HbO2, Hb) over the concentration grid for every
// low-pass pixel (the Bayesian estimate on the low-pass band, Section 2); the per-pixel
// sums are in hb_posterior.cuh.
//
// Six kernels, all with persistent warps:
//   frame_kernel           every step of the path for a strip of the frame in one warp (1..3
//                          levels with the closed-form rows: the default path);
//   lowpass_fused_kernel   block means, posterior records and posterior means in one launch
//                          (1..3 levels where the row kernel applies, with HB_NODE_SUMS);
//   posterior_rows_kernel  over precomputed records (the default when the records are given):
//                          per pixel the rows of the cut, each summed in closed form (eight
//                          pixels per warp, four lanes each: group_pixel) or, with
//                          HB_NODE_SUMS, node by node over its exact column interval by a
//                          ratio recurrence (two pixels per warp: rows_pixel);
//   posterior_span_kernel  two pixels per warp; per pixel the 16-column segments of each
//                          row that meet the row's column interval (grids the recurrence
//                          does not suit);
//   posterior_pair_kernel  two pixels per warp over whole rows (every node enumerated, or
//                          no column intervals for this grid);
//   posterior_kernel       one warp per unit (pixel, part) for launches with fewer pixels
//                          than twice the resident warps: the rs parts of a pixel take
//                          contiguous ranges of its rows, and the last part to finish
//                          (atomic counter) adds the parts' sums in a fixed order.
// Which warp computes a pixel never changes its result.
#include "hb_common.cuh"
#include "hb_device.cuh"
#include "hb_posterior.cuh"
#include "hb_strip.cuh"

#include <math.h>

// Minimum resident CTAs per SM asked of the register allocator (measured on the 1080p
// workload: 2 for the two-pixel kernel, which then keeps its 8 columns per lane in
// registers; 4 for the one-pixel kernel up to 4 columns per lane).  HB_POST_MINB
// overrides both.
#ifdef HB_POST_MINB
#define HB_POST_BOUNDS(cpl) __launch_bounds__(kThreads, HB_POST_MINB)
#define HB_PAIR_BOUNDS __launch_bounds__(kThreads, HB_POST_MINB)
#else
#define HB_POST_BOUNDS(cpl) __launch_bounds__(kThreads, (cpl) >= 8 ? 3 : 4)
#define HB_PAIR_BOUNDS __launch_bounds__(kThreads, 2)
#endif
// The span kernel: CTAs of 8 warps, two per SM (98 registers).  Measured on the 1080p
// workload against 16 warps with one or two CTAs per SM and 8 warps with three: equal or
// faster, and it takes the fewest pixels to fill the GPU (banded host calls).
#ifndef HB_SPAN_THREADS
#define HB_SPAN_THREADS 256
#endif
#ifndef HB_SPAN_MINB
#define HB_SPAN_MINB 2
#endif
#define HB_SPAN_BOUNDS __launch_bounds__(HB_SPAN_THREADS, HB_SPAN_MINB)

namespace hb {
namespace {

// The pixels a launch takes: all npix, or -- under a gate that did not fire -- the ones the
// gate lists (none without a list); the k-th of them is pixel at(k).  Read after the
// kernel's griddepcontrol.wait.
struct Pixels {
    long n;
    const int* list;
    __device__ __forceinline__ long at(long k) const { return list ? (long)list[k] : k; }
};

__device__ __forceinline__ Pixels gated_pixels(const PosteriorGate& g, long npix) {
    if (!g.run || *g.run != 0u) return Pixels{npix, nullptr};
    if (!g.list) return Pixels{0, nullptr};
    const long c = (long)*g.count;
    const Pixels px{c < npix ? c : npix, g.list};
    if (g.listed_total && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(g.listed_total, (unsigned long long)px.n);
    return px;
}

// Posterior mean from the sums, in FP32 (the output is FP32): c = c_ref + h * (sum w d / sum w).
// The posterior mean (HbO2, Hb) from the sums relative to the reference node.
__device__ __forceinline__ float2 posterior_mean(const BayesParams& bp, const BayesRec& rec, float sw, float sdi,
                                                 float sdj) {
    const float inv = __frcp_rn(sw);
    return make_float2(fmaf(bp.h0f, sdi * inv, fmaf((float)rec.i0, bp.h0f, bp.lo0f)),
                       fmaf(bp.h1f, sdj * inv, fmaf((float)rec.j0, bp.h1f, bp.lo1f)));
}

__device__ __forceinline__ void store_mean(long p, float2 c, float2* chat, float2* chat_scaled, float scale) {
    chat[p] = c;
    if (chat_scaled) chat_scaled[p] = make_float2(c.x * scale, c.y * scale);
}

__device__ __forceinline__ void write_mean(const BayesParams& bp, const BayesRec& rec, long p, float sw, float sdi,
                                           float sdj, float2* chat, float2* chat_scaled, float scale) {
    store_mean(p, posterior_mean(bp, rec, sw, sdi, sdj), chat, chat_scaled, scale);
}

// One unit: the sums over its rows, then either the pixel's result (rs == 1) or its
// partial sums; the last part of a pixel to arrive adds the parts in order and writes
// the result.  A pixel whose total sums are not usable (only possible for inputs far
// outside the model) is summed again over all rows with an explicit maximum shift.
// grid_sums has a single call site so that the rare path costs the loop no registers.
template <int CPL>
__device__ __forceinline__ void run_unit(const BayesParams& bp, const BayesRec& rec, long p, long out, int part,
                                         int rs, int lane, float* partial, unsigned* count, float2* chat,
                                         float2* chat_scaled, float scale, unsigned long long& nodes) {
    int lo, hi;
    support_rows(bp, rec, lo, hi);
    int rb = lo, re = hi;
    if (rs > 1) {
        rb = lo + (hi - lo) * part / rs;
        re = lo + (hi - lo) * (part + 1) / rs;
    }
    nodes += (unsigned long long)(re - rb) * (unsigned)bp.n1;
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
            if (lane == 0) write_mean(bp, rec, out, sw, sdi, sdj, chat, chat_scaled, scale);
            return;
        }
        rb = 0;
        re = bp.n0;
        nodes += 2ull * (unsigned)bp.n0 * (unsigned)bp.n1;
        shift = warp_max(grid_max<CPL>(bp, rec, lane, 0, bp.n0));
        if (!(shift != 0.f)) shift = -1.f;  // any non-zero shift marks the second pass
    }
}

// Posterior over precomputed per-pixel records (the stand-alone posterior entry point).
template <int CPL>
__global__ void HB_POST_BOUNDS(CPL) posterior_kernel(BayesParams bp, const BayesRec* __restrict__ recs, long npix, int rs,
                                                float* partial, unsigned* count, float2* __restrict__ chat,
                                                float2* __restrict__ chat_scaled, float scale, PosteriorGate gate,
                                                unsigned long long* nodes_out) {
    const int lane = threadIdx.x & 31;
    const long nw = (long)gridDim.x * (kThreads / 32);
    long u = (long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    // launched with PDL after the kernel that writes the records (or the gate's errors):
    // wait for it, then let the next kernel be scheduled
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    // gated launch (the learned stand-in's exact posterior): every pixel when its sampled
    // check failed, else the pixels its route listed
    const Pixels px = gated_pixels(gate, npix);
    const long units = px.n * rs;
    // (rs == 1 unless there are few pixels: the unit index is then the pixel's position, and
    // the 64-bit divisions below are skipped; the scratch slots follow the position)
    BayesRec next = {0, 0, 0.f, 0.f};
    if (u < units) next = recs[px.at(rs == 1 ? u : u / rs)];
    unsigned long long nodes = 0;
    for (; u < units; u += nw) {
        const long p = rs == 1 ? u : u / rs;
        const BayesRec rec = next;
        if (u + nw < units) next = recs[px.at(rs == 1 ? u + nw : (u + nw) / rs)];
        run_unit<CPL>(bp, rec, p, px.at(p), rs == 1 ? 0 : (int)(u - p * rs), rs, lane, partial, count, chat,
                      chat_scaled, scale, nodes);
    }
    if (nodes_out && lane == 0 && nodes) atomicAdd(nodes_out, nodes);
}

// One round of the two-pixel kernel below: pixel 2r + half, its sums and its mean.
template <int CPL>
__device__ __forceinline__ void pair_round(const BayesParams& bp, const BayesRec& rec, long r, const Pixels& px,
                                           int gl, int half, float2* chat, float2* chat_scaled, float scale,
                                           unsigned long long& nodes) {
    constexpr int G = 16;
    const long k = 2 * r + half;
    const bool valid = k < px.n;
    int lo, hi;
    support_rows(bp, rec, lo, hi);
    int rb = __reduce_min_sync(0xffffffffu, lo), re = __reduce_max_sync(0xffffffffu, hi);
    if (valid) nodes += (unsigned long long)(re - rb) * (unsigned)bp.n1;
    float shift = 0.f, sw, sdi, sdj;
    for (int pass = 0;; ++pass) {
        sw = sdi = sdj = 0.f;
        grid_sums<CPL, G>(bp, rec, gl, rb, re, shift, sw, sdi, sdj);
        sw = group_sum<G>(sw);
        sdi = group_sum<G>(sdi);
        sdj = group_sum<G>(sdj);
        const bool bad = !usable(sw, sdi, sdj);
        if (pass == 1 || !__any_sync(0xffffffffu, bad)) break;
        const float m = group_max<G>(grid_max<CPL, G>(bp, rec, gl, 0, bp.n0));
        shift = bad ? m : 0.f;
        rb = 0;
        re = bp.n0;
        if (valid && bad) nodes += 2ull * (unsigned)bp.n0 * (unsigned)bp.n1;
    }
    if (valid && gl == 0) write_mean(bp, rec, px.at(k), sw, sdi, sdj, chat, chat_scaled, scale);
}

// Two pixels per warp: half-warp h (lanes 16h .. 16h+15) takes pixel 2r + h of round r, CPL
// columns per lane.  The per-pixel fixed work (row bound, column constants, reductions,
// epilogue) is then shared by two pixels in every warp instruction.  The warp enumerates the
// union of the two pixels' support rows; rows outside a pixel's own support carry weights
// that are exactly zero in FP32, so each pixel's sums equal those over its own rows, and
// over the whole grid.  A pixel whose sums are not usable (inputs far outside the model) is
// summed again over all rows with an explicit maximum shift; its partner repeats its own
// sums unshifted, which leaves them unchanged.
//
// Rounds are dealt to CTAs interleaved (CTA b takes rounds b, b + B, b + 2B, ...: an even
// sample of the frame each) and, inside a CTA, to whichever warp is free next through a
// shared-memory counter, so that warps whose pixels have few support rows take more of
// them.  Each warp holds its next round's record while it computes.  Which warp computes a
// pixel does not change its result.
template <int CPL>
__global__ void HB_PAIR_BOUNDS posterior_pair_kernel(BayesParams bp, const BayesRec* __restrict__ recs, long npix,
                                                     float2* __restrict__ chat, float2* __restrict__ chat_scaled,
                                                     float scale, PosteriorGate gate, unsigned long long* nodes_out) {
    const int lane = threadIdx.x & 31, gl = lane & 15, half = lane >> 4;
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) ticket = 0u;
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const Pixels px = gated_pixels(gate, npix);
    const long rounds = (px.n + 1) / 2;
    unsigned long long nodes = 0;
    auto next_round = [&]() {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(&ticket, 1u);
        return (long)blockIdx.x + (long)__shfl_sync(0xffffffffu, k, 0) * gridDim.x;
    };
    auto load = [&](long r) { return recs[px.at(min(2 * r + half, px.n - 1))]; };
    long r0 = next_round();
    BayesRec rec0 = {0, 0, 0.f, 0.f};
    if (r0 < rounds) rec0 = load(r0);
    while (r0 < rounds) {
        const long r1 = next_round();
        BayesRec rec1 = {0, 0, 0.f, 0.f};
        if (r1 < rounds) rec1 = load(r1);
        pair_round<CPL>(bp, rec0, r0, px, gl, half, chat, chat_scaled, scale, nodes);
        r0 = r1;
        rec0 = rec1;
    }
    if (nodes_out && gl == 0 && nodes) atomicAdd(nodes_out, nodes);
}

// ---- Span kernel: only the nodes inside each row's column interval ---------------------
//
// The nodes of a pixel whose weights matter fill a tilted ellipse over the grid (clipped by
// the grid's edges): taking whole rows would enumerate several times as many.  The span
// kernel enumerates, in every row of the ellipse, the 16-column lattice segments that meet
// the row's column interval (span_pixel, span_row): items of (row, segment), dealt to the 16
// lanes of the pixel's half-warp in order.  For the item table the rows go in chunks of 48,
// three consecutive rows per lane: a lane finds its rows' segments, a scan over the
// half-warp gives each lane its first item, and the lane writes its items into the
// half-warp's table in shared memory.  The nodes outside the intervals carry together less
// than 2^-30 of the posterior mass (BayesParams::span_cut).
constexpr int kSpanThreads = HB_SPAN_THREADS;
constexpr int kSpanRows = 3;                 // rows per lane per chunk
constexpr int kSpanChunk = 16 * kSpanRows;   // rows per chunk
constexpr int kSpanMaxCols = 128;            // n1 limit
constexpr int kSpanMaxSegs = kSpanMaxCols / kSpanSeg;
constexpr int kSpanMaxItems = kSpanChunk * kSpanMaxSegs;

// One item: columns dj0 .. dj0 + 15 of row di (relative to the reference node), in pairs;
// even and odd pairs keep separate sums.  Adds sum w to SW and sum w di to SD (packed:
// the two halves are added at the end), sum w dj to T0/T1.
__device__ __forceinline__ void span_item(const BayesParams& bp, const BayesRec& rec, int di, int dj0, u64& SW,
                                          u64& SD, u64& T0, u64& T1) {
    const float d = (float)di;
    const float R = fmaf(2.f * bp.Bq, d, rec.V);
    const float S = d * fmaf(bp.Aq, d, rec.U);
    const u64 RR = pk(R, R), SS = pk(S, S), CC = pk(bp.Cq, bp.Cq), TWO = pk(2.f, 2.f);
    const float f = (float)dj0;
    u64 dj = pk(f, f + 1.f);
    u64 S0 = pk(0.f, 0.f), S1 = pk(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kSpanSeg / 2; ++q) {
        const u64 X = fma2(CC, dj, RR);
        const u64 t = fma2(dj, X, SS);
        float t0, t1;
        upk(t, t0, t1);
        const u64 w = pk(ex2(t0), ex2(t1));
        if (q & 1) {
            S1 = add2(S1, w);
            T1 = fma2(w, dj, T1);
        } else {
            S0 = add2(S0, w);
            T0 = fma2(w, dj, T0);
        }
        dj = add2(dj, TWO);
    }
    const u64 Sq = add2(S0, S1);
    SW = add2(SW, Sq);
    SD = fma2(pk(d, d), Sq, SD);
}

// The same for a segment cut short by the grid's last column (n1 not a multiple of 16).
__device__ __forceinline__ void span_item_short(const BayesParams& bp, const BayesRec& rec, int di, int dj0, int n,
                                                float& sw, float& sdi, float& sdj) {
    const float d = (float)di;
    const float R = fmaf(2.f * bp.Bq, d, rec.V);
    const float S = d * fmaf(bp.Aq, d, rec.U);
    float s = 0.f;
    for (int c = 0; c < n; ++c) {
        const float dj = (float)(dj0 + c);
        const float w = ex2(fmaf(dj, fmaf(bp.Cq, dj, R), S));
        s += w;
        sdj = fmaf(w, dj, sdj);
    }
    sw += s;
    sdi = fmaf(d, s, sdi);
}

// One round of the span kernel: pixel 2r + half, its sums and its mean.  tab: the
// half-warp's item table.  nodes: this lane's share of the enumerated-node count.
template <bool RAGGED>
__device__ __forceinline__ void span_round(const BayesParams& bp, const BayesRec& rec, long r, const Pixels& px,
                                           int gl, int half, unsigned short* tab, float2* chat, float2* chat_scaled,
                                           float scale, unsigned long long& nodes) {
    constexpr int G = 16;
    const long k = 2 * r + half;
    const bool valid = k < px.n;
    const SpanPixel sp = span_pixel(bp, rec);
    const int nseg = (bp.n1 + kSpanSeg - 1) / kSpanSeg;
    u64 SW = pk(0.f, 0.f), SD = pk(0.f, 0.f), T0 = pk(0.f, 0.f), T1 = pk(0.f, 0.f);
    float xw = 0.f, xdi = 0.f, xdj = 0.f;  // short segments
    for (int c0 = sp.rlo; __any_sync(0xffffffffu, c0 < sp.rhi); c0 += kSpanChunk) {
        int ma[kSpanRows], ns[kSpanRows], tot = 0;
#pragma unroll
        for (int q = 0; q < kSpanRows; ++q) {
            const int i = c0 + kSpanRows * gl + q;
            span_row(sp, i - rec.i0, nseg, ma[q], ns[q]);
            if (i >= sp.rhi) ns[q] = 0;
            tot += ns[q];
        }
        int inc = tot;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, d, G);
            if (gl >= d) inc += v;
        }
        const int K = __shfl_sync(0xffffffffu, inc, G - 1, G);
        int at = inc - tot;
#pragma unroll
        for (int q = 0; q < kSpanRows; ++q) {
            const unsigned v = ((unsigned)(kSpanRows * gl + q) << 8) | (unsigned)ma[q];
#pragma unroll
            for (int m = 0; m < kSpanMaxSegs; ++m)
                if (m < ns[q]) tab[at + m] = (unsigned short)(v + m);
            at += ns[q];
        }
        __syncwarp();
        if (valid && gl == 0) nodes += (unsigned)K * kSpanSeg;
        for (int k = gl; k < K; k += G) {
            const unsigned e = tab[k];
            const int di = c0 + (int)(e >> 8) - rec.i0;
            const int j = (int)(e & 255u) * kSpanSeg;
            if (RAGGED && j + kSpanSeg > bp.n1) {
                span_item_short(bp, rec, di, j - rec.j0, bp.n1 - j, xw, xdi, xdj);
                if (valid) nodes -= (unsigned)(j + kSpanSeg - bp.n1);
            } else {
                span_item(bp, rec, di, j - rec.j0, SW, SD, T0, T1);
            }
        }
        __syncwarp();
    }
    float a, b;
    upk(SW, a, b);
    float sw = (a + b) + xw;
    upk(SD, a, b);
    float sdi = (a + b) + xdi;
    const u64 T = add2(T0, T1);
    upk(T, a, b);
    float sdj = (a + b) + xdj;
    sw = group_sum<G>(sw);
    sdi = group_sum<G>(sdi);
    sdj = group_sum<G>(sdj);
    const bool bad = !usable(sw, sdi, sdj);
    if (__any_sync(0xffffffffu, bad)) {
        // far outside the model: the whole grid with an explicit maximum shift (the
        // partner half-warp takes part in the shuffles and keeps its own sums)
        const float m = group_max<G>(grid_max<1, G>(bp, rec, gl, 0, bp.n0));
        float fw = 0.f, fdi = 0.f, fdj = 0.f;
        grid_sums<1, G>(bp, rec, gl, 0, bp.n0, bad ? m : 0.f, fw, fdi, fdj);
        fw = group_sum<G>(fw);
        fdi = group_sum<G>(fdi);
        fdj = group_sum<G>(fdj);
        if (bad) {
            sw = fw;
            sdi = fdi;
            sdj = fdj;
            if (valid && gl == 0) nodes += 2ull * (unsigned)bp.n0 * (unsigned)bp.n1;
        }
    }
    if (valid && gl == 0) write_mean(bp, rec, px.at(k), sw, sdi, sdj, chat, chat_scaled, scale);
}

// Two pixels per warp (half-warp h takes pixel 2r + h of round r), rounds dealt as in
// posterior_pair_kernel above.
template <bool RAGGED>
__global__ void HB_SPAN_BOUNDS posterior_span_kernel(BayesParams bp, const BayesRec* __restrict__ recs, long npix,
                                                     float2* __restrict__ chat, float2* __restrict__ chat_scaled,
                                                     float scale, PosteriorGate gate, unsigned long long* nodes_out) {
    const int lane = threadIdx.x & 31, gl = lane & 15, half = lane >> 4;
    __shared__ unsigned short tab[kSpanThreads / 32][2][kSpanMaxItems];
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) ticket = 0u;
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const Pixels px = gated_pixels(gate, npix);
    const long rounds = (px.n + 1) / 2;
    unsigned short* my = tab[threadIdx.x >> 5][half];
    unsigned long long nodes = 0;
    auto next_round = [&]() {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(&ticket, 1u);
        return (long)blockIdx.x + (long)__shfl_sync(0xffffffffu, k, 0) * gridDim.x;
    };
    auto load = [&](long r) { return recs[px.at(min(2 * r + half, px.n - 1))]; };
    long r0 = next_round();
    BayesRec rec0 = {0, 0, 0.f, 0.f};
    if (r0 < rounds) rec0 = load(r0);
    while (r0 < rounds) {
        const long r1 = next_round();
        BayesRec rec1 = {0, 0, 0.f, 0.f};
        if (r1 < rounds) rec1 = load(r1);
        span_round<RAGGED>(bp, rec0, r0, px, gl, half, my, chat, chat_scaled, scale, nodes);
        r0 = r1;
        rec0 = rec1;
    }
    if (nodes_out) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nodes += __shfl_xor_sync(0xffffffffu, nodes, off);
        if (lane == 0 && nodes) atomicAdd(nodes_out, nodes);
    }
}

// ---- Row kernel: the span kernel's cut, exact column intervals, weights by recurrence ----
//
// Per pixel (a half-warp of 16 lanes) the rows of span_pixel are dealt to the lanes in
// slots of 16 (lane g takes rows rlo + g, rlo + g + 16, ...), and each lane sums its row
// over the row's column interval (row_span: the span kernel's cut without rounding to
// segments).  Along a row the base-2 log weight is the quadratic t(j) = Cq j^2 + R j + S in
// the column offset j, so the weights of every second column satisfy w(j + 2) = w(j) r(j)
// with r(j + 2) = r(j) row_q, row_q = 2^(8 Cq): the lane evaluates 2^t with ex2 only at the
// first two columns (and their ratios), then advances the two chains (even and odd
// columns from the start) together in FP32x2 -- two multiplies and two adds per pair of
// nodes, no MUFU.  The sums are accumulated as A = sum w and B = sum of the running A, from
// which sum w k = m A - B over the m steps of a chain.
//
// Every lane of the warp runs the same number of steps (the warp's longest row), so the
// loop needs no per-lane test: a chain starts at the row's end that the grid cuts off (or at
// the left end), and the steps beyond its interval continue the same Gaussian into the
// row's tail, where every weight is below 2^-cut of the reference node's -- nodes the cut
// would leave out anyway, on or beyond the grid's edge alike (together far below the FP32
// rounding of the sums).  Only a row cut off by the grid at both ends (a posterior wider
// than the grid) must stop at the grid's edge; a warp holding one takes a loop with a
// per-lane test.  Pixels whose bounds take every row and column (span_pixel's guard for
// inputs far outside the model), and pixels whose sums come out not finite, are summed over
// the whole grid with an explicit maximum shift.
constexpr int kRowThreads = 256;
#ifndef HB_ROWS_CTAS_PER_SM
#define HB_ROWS_CTAS_PER_SM 3
#endif
constexpr int kRowCtasPerSm = HB_ROWS_CTAS_PER_SM;

// The cut's column interval [na, nb) of row i0 + di (grid column indices), not clipped to the
// grid (widened by one column on the left and two on the right, as span_row); na >= nb when
// the row holds none.
__device__ __forceinline__ void row_span(const SpanPixel& sp, int di, int& na, int& nb) {
    const float d = (float)di;
    const float h2 = fmaf(d, fmaf(sp.a2, d, sp.b2), sp.c2);
    const float c = fmaf(sp.k1, d, sp.cc);
    const float h = sqrt_approx(fmaxf(h2, 0.f));
    na = __float2int_ru(c - h - 1.f);
    nb = __float2int_rd(c + h + 2.f) + 1;
    if (!(h2 >= 0.f) || nb < na) nb = na;
}

// The warp's counts, added (when counting) to counts[0] (nodes summed one by one), counts[1]
// (rows summed in closed form) and counts[2] (of those, rows the box edge cuts off: the
// table's one-sided sums); rows carries the last two as (edge rows << 32) + rows.
__device__ __forceinline__ void flush_counts(unsigned long long* counts, unsigned long long nodes,
                                             unsigned long long rows, int lane) {
    if (!counts) return;
    unsigned long long r = rows & 0xffffffffull, e = rows >> 32;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nodes += __shfl_xor_sync(0xffffffffu, nodes, off);
        r += __shfl_xor_sync(0xffffffffu, r, off);
        e += __shfl_xor_sync(0xffffffffu, e, off);
    }
    if (lane == 0 && nodes) atomicAdd(counts, nodes);
    if (lane == 0 && r) atomicAdd(counts + 1, r);
    if (lane == 0 && e) atomicAdd(counts + 2, e);
}

// The posterior mean of the half-warp's pixel (record rec) into chat[out] (and chat_scaled)
// when valid, every row summed node by node (the grids without the closed-form rows, and
// HB_NODE_SUMS); both half-warps of the warp call it together.  nodes counts the grid nodes
// summed.
__device__ __forceinline__ void rows_pixel(const BayesParams& bp, const BayesRec& rec, bool valid, long out, int gl,
                                           float2* chat, float2* chat_scaled, float scale,
                                           unsigned long long& nodes, unsigned long long& rows) {
    constexpr int G = 16;
    const SpanPixel sp = span_pixel(bp, rec);
    const bool direct = sp.whole;  // summed over the whole grid below instead
    const int nslots = __reduce_max_sync(0xffffffffu, direct ? 0 : (sp.rhi - sp.rlo + G - 1) / G);
    const u64 QQ = pk(bp.row_q, bp.row_q), CC = pk(bp.Cq, bp.Cq);
    float sw = 0.f, sdi = 0.f, sdj = 0.f;
    unsigned cnt = 0;
    for (int slot = 0; slot < nslots; ++slot) {
        const int i = sp.rlo + slot * G + gl;
        int na = 0, nb = 0;
        if (!direct && i < sp.rhi) row_span(sp, i - rec.i0, na, nb);
        const int ja = max(na, 0), jb = min(nb, bp.n1);  // clipped to the grid
        const bool live = jb > ja;
#ifndef HB_ROWS_NO_DEAD_SKIP
        // rows whose interval misses the grid's columns add exactly nothing: a slot where
        // every lane's row does is skipped (about a fifth of the slots on the 1080p frame)
        if (!__any_sync(0xffffffffu, live)) continue;
#endif
        const bool lclip = na < 0, rclip = nb > bp.n1;
        const float d = (float)(i - rec.i0);
        const float R = fmaf(2.f * bp.Bq, d, rec.V);
        const float S = d * fmaf(bp.Aq, d, rec.U);
        float rs = 0.f, rm = 0.f;
        const bool walk = live;
        {
            const bool full = walk && lclip && rclip;
            const bool back = walk && rclip && !lclip;  // start at the right end, walk left
            const bool any_full = __any_sync(0xffffffffu, full);
            // steps: the warp's longest row; a lane with a full row takes only its own, and the
            // grid's last column on its own when the row has an odd number of columns
            const int len = walk ? jb - ja : 0;
            const int own = full ? (len >> 1) : ((len + 1) >> 1);
            const int steps = __reduce_max_sync(0xffffffffu, own);
            const bool extra = full && (len & 1);
            const float dir = back ? -1.f : 1.f;
            const float s0 = (float)((back ? jb - 1 : ja) - rec.j0);  // the first chain's first column
            const u64 J = pk(s0, s0 + dir);
            const u64 T = fma2(J, fma2(CC, J, pk(R, R)), pk(S, S));
            // t(j + 2 dir) - t(j) = Cq (4 dir j + 4) + 2 dir R
            const u64 D = fma2(CC, fma2(pk(4.f * dir, 4.f * dir), J, pk(4.f, 4.f)), pk(2.f * dir * R, 2.f * dir * R));
            float t0, t1, d0, d1;
            upk(T, t0, t1);
            upk(D, d0, d1);
            // a chain whose first weight would be below 2^-100 starts 2^sh higher and its sums are
            // scaled back (a weight flushed to zero would stop the recurrence)
            const float sh = walk ? fmaxf(0.f, -100.f - fminf(t0, t1)) : 0.f;
            u64 w = walk ? pk(ex2(t0 + sh), ex2(t1 + sh)) : pk(0.f, 0.f);
            u64 q = walk ? pk(ex2(d0), ex2(d1)) : pk(0.f, 0.f);
            u64 A = pk(0.f, 0.f), B = pk(0.f, 0.f);
            if (!any_full) {
#pragma unroll 4
                for (int st = 0; st < steps; ++st) {
                    A = add2(A, w);
                    B = add2(B, A);
                    w = mul2(w, q);
                    q = mul2(q, QQ);
                }
            } else {
                for (int st = 0; st < steps; ++st) {
                    if (st < own) {
                        A = add2(A, w);
                        B = add2(B, A);
                        w = mul2(w, q);
                        q = mul2(q, QQ);
                    }
                }
            }
            if (sh > 0.f) {
                const float u = ex2(-sh);
                A = mul2(A, pk(u, u));
                B = mul2(B, pk(u, u));
            }
            const int m = any_full ? own : steps;  // the steps this lane summed
            float a0, a1, b0, b1;
            upk(A, a0, a1);
            upk(B, b0, b1);
            const float fm = (float)m;
            float ws = a0 + a1;
            // chain c: sum w (j - j0) = (its first column) A + 2 dir (m A - B)
            float wm = fmaf(s0, a0, fmaf(s0 + dir, a1, 2.f * dir * (fmaf(fm, a0, -b0) + fmaf(fm, a1, -b1))));
            if (extra) {  // the grid's last column of an odd full row
                const float jx = (float)(bp.n1 - 1 - rec.j0);
                const float wx = ex2(fmaf(jx, fmaf(bp.Cq, jx, R), S));
                ws += wx;
                wm = fmaf(wx, jx, wm);
            }
            if (walk) {
                rs = ws;
                rm = wm;
                cnt += 2u * (unsigned)m + (extra ? 1u : 0u);
            }
        }
        sw += rs;
        sdj += rm;
        sdi = fmaf(d, rs, sdi);
    }
    sw = group_sum<G>(sw);
    sdi = group_sum<G>(sdi);
    sdj = group_sum<G>(sdj);
    if (valid) nodes += cnt;
    (void)rows;
    const bool bad = direct || !usable(sw, sdi, sdj);
    if (__any_sync(0xffffffffu, bad)) {
        // the whole grid with an explicit maximum shift (the partner half-warp takes part in
        // the shuffles and keeps its own sums)
        const float mx = group_max<G>(grid_max<1, G>(bp, rec, gl, 0, bp.n0));
        float fw = 0.f, fdi = 0.f, fdj = 0.f;
        grid_sums<1, G>(bp, rec, gl, 0, bp.n0, bad ? mx : 0.f, fw, fdi, fdj);
        fw = group_sum<G>(fw);
        fdi = group_sum<G>(fdi);
        fdj = group_sum<G>(fdj);
        if (bad) {
            sw = fw;
            sdi = fdi;
            sdj = fdj;
            if (valid && gl == 0) nodes += (unsigned long long)bp.n0 * (unsigned)bp.n1 * 2ull;
        }
    }
    if (valid && gl == 0) write_mean(bp, rec, out, sw, sdi, sdj, chat, chat_scaled, scale);
}

// ---- Closed-form rows: G = 4 lanes per pixel ----
//
// With the closed-form row sums (BayesParams::row_tab) a row costs a few dozen instructions,
// so the warp-wide steps of rows_pixel (every lane running the longest row) are no longer
// needed: a group of kGroup lanes takes a pixel, lane g of the group the rows rlo + g,
// rlo + g + kGroup, ... of span_pixel, each lane on its own (rows whose interval misses the
// grid's columns are passed over).  Rows cut off on both sides, or whose peak lies beyond the
// table, are summed node by node with one ex2 per node.  The group's sums are added by
// shuffles in a fixed order, so a pixel's result depends only on its record: the fused
// kernel and posterior_rows_kernel give the same bits.
constexpr int kGroup = 4;
constexpr int kGroupPixels = 32 / kGroup;  // pixels per warp

// The sums of the group's pixel (the same bits in every lane of the group); every lane of
// the warp calls it together.  The rows are those of span_pixel narrowed to the rows whose
// cut interval meets the grid's columns (clip_rows_to_grid).  A row's terms and class are
// computed without branches: its cut interval, widened by one column on the left and two on
// the right as in row_span, has centre cen (the row's peak column) and squared half-width
// h2; it is cut off on the left when cen - h - 1 < 0 and on the right when
// cen + h + 2 > n1 - 1 (compared squared, no square root).  Inside the grid it takes the
// full-line sum, cut off on one side the table's one-sided sum (the table read at an index
// clamped into it, the result used only when in range).  Rows cut off on both sides, or with
// the peak beyond the table's left end, are summed node by node in a second pass (rare).
// Rows whose interval misses the grid add nothing.
// A row's class from its cut interval, widened by one column on the left and two on the right
// as in row_span (centre cen, half-width sqrt(h2)): cut off on the left when it starts left of
// column 0, on the right when it ends right of column n1 - 1.  A row whose interval misses the
// grid, or whose h2 is negative (its maximum below the cut), is classed by its centre alone and
// its sums are the true, negligible ones.
__device__ __forceinline__ void row_class(float h2, float cen, float n1f, bool& lclip, bool& rclip) {
    const float h = sqrt_approx(fmaxf(h2, 0.f));
    lclip = cen - h < 1.f;
    rclip = cen + h > n1f - 3.f;
}

// COUNT: add the rows summed in closed form (and those of them cut off by an edge) and the nodes
// summed one by one to the counters.
template <bool COUNT>
__device__ __forceinline__ void group_sums(const BayesParams& bp, const BayesRec& rec, bool valid, int gl, float& sw,
                                           float& sdi, float& sdj, unsigned long long& nodes,
                                           unsigned long long& rows) {
    constexpr int G = kGroup;
    const SpanPixel sp = span_pixel(bp, rec);
    sw = 0.f;
    sdi = 0.f;
    sdj = 0.f;
    unsigned cnt = 0, rcnt = 0, ecnt = 0;
    int ra = sp.rlo, rb = sp.rhi;
    if (!sp.whole) {
        float lo = (float)(ra - rec.i0), hi = (float)(rb - 1 - rec.i0);
        clip_rows_to_grid(bp, rec, fmaf(1e-6f, fmaf(fabsf(rec.U), (float)bp.n0, fmaf(fabsf(rec.V), (float)bp.n1,
                                                                                     bp.sup_mg)),
                                        bp.span_cut),
                          lo, hi);
        if (lo <= hi) {  // widened by a row on each side; the reference row is always kept
            ra = max(ra, min(rec.i0 + (int)floorf(lo) - 1, rec.i0));
            rb = min(rb, max(rec.i0 + (int)ceilf(hi) + 2, rec.i0 + 1));
        }
    }
    const float n1f = (float)bp.n1, edge_r = (float)(bp.n1 - 1 - rec.j0), edge_l = (float)rec.j0;
    bool walked = false;
    if (valid && !sp.whole) {
        for (int i = ra + gl; i < rb; i += G) {
            const float d = (float)(i - rec.i0);
            const float h2 = fmaf(d, fmaf(sp.a2, d, sp.b2), sp.c2);
            const float cen = fmaf(sp.k1, d, sp.cc);
            bool lclip, rclip;
            row_class(h2, cen, n1f, lclip, rclip);
            const float R = fmaf(2.f * bp.Bq, d, rec.V);
            const float S = d * fmaf(bp.Aq, d, rec.U);
            const float js = R * bp.span_cv;          // the row's peak, in columns from j0
            const float ts = fmaf(0.5f * R, js, S);   // its base-2 log weight t*
            const float x = lclip ? edge_l + js : edge_r - js;  // the peak's distance from the cut-off edge
            const float f = (x - bp.tab_x0) * bp.tab_inv_step;
            const int k = min(max((int)f, 0), bp.tab_n - 1);
            const float u = f - (float)k;
            const float4 p = __ldg(bp.row_tab + 2 * k), q = __ldg(bp.row_tab + 2 * k + 1);
            const bool one = lclip != rclip, in_tab = f < (float)bp.tab_n;
            const float lf_t = fmaf(u, fmaf(u, fmaf(u, p.w, p.z), p.y), p.x);
            const float m_t = fmaf(u, fmaf(u, fmaf(u, q.w, q.z), q.y), q.x);  // mean, columns from the edge
            float lf_full = bp.log2_kfull, mc_full = js;  // over all integer columns
            if (bp.pois_q > 0.f) {  // the first Poisson term (rows narrower than ~1.5 columns)
                float sn, cs;
                sincospif(2.f * (js - floorf(js)), &sn, &cs);
                const float e = 2.f * bp.pois_q * cs;  // |e| < 2e-3: ln(1 + e) to e^4
                lf_full = fmaf(e * fmaf(e, fmaf(e, 1.f / 3.f, -0.5f), 1.f), 1.4426950408889634f, lf_full);
                mc_full = fmaf(-bp.pois_m, __fdividef(sn, 1.f + e), js);
            }
            const float lf = (one && in_tab) ? lf_t : lf_full;
            const float mc = (one && in_tab) ? (lclip ? m_t - edge_l : edge_r - m_t) : mc_full;
            const bool walk = (lclip && rclip) || (one && !(f >= 0.f));
            const float rs = walk ? 0.f : ex2(ts + lf);
            sw += rs;
            sdj = fmaf(mc, rs, sdj);
            sdi = fmaf(d, rs, sdi);
            if (COUNT) {
                rcnt += walk ? 0u : 1u;
                ecnt += (!walk && one) ? 1u : 0u;
            }
            walked |= walk;
        }
    }
    if (__any_sync(0xffffffffu, walked) && walked) {
        // the rows taken node by node, one ex2 per node over the row's widened interval
        for (int i = ra + gl; i < rb; i += G) {
            const float d = (float)(i - rec.i0);
            const float h2 = fmaf(d, fmaf(sp.a2, d, sp.b2), sp.c2);
            const float cen = fmaf(sp.k1, d, sp.cc);
            bool lclip, rclip;
            row_class(h2, cen, n1f, lclip, rclip);
            const float R = fmaf(2.f * bp.Bq, d, rec.V);
            const float js = R * bp.span_cv;
            const float x = lclip ? edge_l + js : edge_r - js;
            const float f = (x - bp.tab_x0) * bp.tab_inv_step;
            if (!((lclip && rclip) || (lclip != rclip && !(f >= 0.f)))) continue;
            int na, nb;
            row_span(sp, i - rec.i0, na, nb);
            const int ja = max(na, 0), jb = min(nb, bp.n1);
            const float S = d * fmaf(bp.Aq, d, rec.U);
            float rs = 0.f, rm = 0.f;
            for (int j = ja; j < jb; ++j) {
                const float dj = (float)(j - rec.j0);
                const float w = ex2(fmaf(dj, fmaf(bp.Cq, dj, R), S));
                rs += w;
                rm = fmaf(w, dj, rm);
            }
            cnt += (unsigned)max(jb - ja, 0);
            sw += rs;
            sdj += rm;
            sdi = fmaf(d, rs, sdi);
        }
    }
    sw = group_sum<G>(sw);
    sdi = group_sum<G>(sdi);
    sdj = group_sum<G>(sdj);
    if (COUNT && valid) {
        nodes += cnt;
        rows += ((unsigned long long)ecnt << 32) + rcnt;
    }
    const bool bad = valid && (sp.whole || !usable(sw, sdi, sdj));
    if (__any_sync(0xffffffffu, bad)) {
        // the whole grid with an explicit maximum shift (the other groups take part in the
        // shuffles and keep their own sums)
        const float mx = group_max<G>(grid_max<1, G>(bp, rec, gl, 0, bp.n0));
        float fw = 0.f, fdi = 0.f, fdj = 0.f;
        grid_sums<1, G>(bp, rec, gl, 0, bp.n0, bad ? mx : 0.f, fw, fdi, fdj);
        fw = group_sum<G>(fw);
        fdi = group_sum<G>(fdi);
        fdj = group_sum<G>(fdj);
        if (bad) {
            sw = fw;
            sdi = fdi;
            sdj = fdj;
            if (COUNT && gl == 0) nodes += (unsigned long long)bp.n0 * (unsigned)bp.n1;
        }
    }
}

__device__ __forceinline__ void group_pixel(const BayesParams& bp, const BayesRec& rec, bool valid, long out, int gl,
                                            float2* chat, float2* chat_scaled, float scale,
                                            unsigned long long& nodes, unsigned long long& rows) {
    float sw, sdi, sdj;
    group_sums<true>(bp, rec, valid, gl, sw, sdi, sdj, nodes, rows);
    if (valid && gl == 0) write_mean(bp, rec, out, sw, sdi, sdj, chat, chat_scaled, scale);
}

// Two pixels per warp (half-warp h takes pixel 2r + h of round r), rounds dealt as in
// posterior_pair_kernel.
template <bool CLOSED>
__global__ void __launch_bounds__(kRowThreads, 3) posterior_rows_kernel(BayesParams bp,
                                                                       const BayesRec* __restrict__ recs, long npix,
                                                                       float2* __restrict__ chat,
                                                                       float2* __restrict__ chat_scaled, float scale,
                                                                       PosteriorGate gate,
                                                                       unsigned long long* nodes_out) {
    // pixels per warp and round: two (a half-warp each) node by node, eight (kGroup lanes
    // each) with the closed-form rows
    constexpr int PPW = CLOSED ? kGroupPixels : 2, G = 32 / PPW;
    const int lane = threadIdx.x & 31, gl = lane % G, half = lane / G;
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) ticket = 0u;
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const Pixels px = gated_pixels(gate, npix);
    const long rounds = (px.n + PPW - 1) / PPW;
    unsigned long long nodes = 0, rows = 0;
    auto next_round = [&]() {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&ticket, 1u);
        return (long)blockIdx.x + (long)__shfl_sync(0xffffffffu, t, 0) * gridDim.x;
    };
    auto load = [&](long rr) { return recs[px.at(min(PPW * rr + half, px.n - 1))]; };
    long r0 = next_round();
    BayesRec rec0 = {0, 0, 0.f, 0.f};
    if (r0 < rounds) rec0 = load(r0);
    while (r0 < rounds) {
        const long r1 = next_round();
        BayesRec rec1 = {0, 0, 0.f, 0.f};
        if (r1 < rounds) rec1 = load(r1);
        const long k = PPW * r0 + half;
        if constexpr (CLOSED)
            group_pixel(bp, rec0, k < px.n, k < px.n ? px.at(k) : 0, gl, chat, chat_scaled, scale, nodes, rows);
        else
            rows_pixel(bp, rec0, k < px.n, k < px.n ? px.at(k) : 0, gl, chat, chat_scaled, scale, nodes, rows);
        r0 = r1;
        rec0 = rec1;
    }
    flush_counts(nodes_out, nodes, rows, lane);
}

// ---- Fused low pass: block means, posterior records and posterior means in one kernel ----
//
// For 1..3 levels with the row kernel's bounds.  A unit is one warp's strip of the frame:
// 64 pixel columns of one superblock band (64 / 2^n superblocks).  Warp w of the W warps of
// the launch takes tickets w, w + W, w + 2W, ... (no counter: a global ticket counter cost
// 2.3 us of the 1080p frame's 22.9, its same-address atomics serialising in L2); for each,
// the warp forms the superblocks' block means by the strip analysis (the same code as the
// analysis kernel), computes their posterior records on lanes 0 .. 64/2^n - 1
// (bayes_setup), and then the posterior means two superblocks at a time (rows_pixel) or,
// with the closed-form rows, eight at a time (group_pixel), so a superblock's record never
// leaves the warp and the frame's loads overlap other warps' posterior sums.
//
// Tail.  With U units over W warps, U mod W units are left once every warp has taken its
// share of whole units; dealt whole, they would keep that many warps busy for a whole unit
// while the others idle.  Those tail units are instead dealt in P pieces each (P a power of
// two up to the unit's rounds, with P x tail <= W / 2): a piece redoes its unit's analysis
// and records and takes 1/P of its rounds.  Each superblock is still computed by exactly
// one warp with the same code, so the results do not depend on the split.
constexpr int kFusedThreads = 256;
#ifndef HB_FUSED_MINB
#define HB_FUSED_MINB 3  // resident CTAs per SM asked of the register allocator (80 registers)
#endif

struct FusedTickets {
    unsigned full, per_unit, total;  // whole units first, then per_unit pieces per tail unit
};

__device__ __forceinline__ FusedTickets fused_tickets(unsigned nunits, unsigned warps, unsigned rounds) {
    const unsigned tail = nunits % warps;
    unsigned p = 1;
#ifndef HB_FUSED_WHOLE_UNITS
    while (2 * p <= rounds && tail > 0 && 4ull * p * tail <= warps) p *= 2;
#endif
    if (p == 1) return FusedTickets{nunits, 1, nunits};
    return FusedTickets{nunits - tail, p, nunits - tail + tail * p};
}

template <int L, bool CLOSED>
__global__ void __launch_bounds__(kFusedThreads, HB_FUSED_MINB)
    lowpass_fused_kernel(TransformParams tp, BayesParams bp, const unsigned char* __restrict__ frame, size_t stride,
                         const float2* __restrict__ lut, float2* __restrict__ chat, float2* __restrict__ chat_scaled,
                         float scale, unsigned long long* nodes_out) {
    // rounds per unit: superblocks two at a time (rows_pixel) or, with the closed-form rows,
    // eight at a time (group_pixel)
    constexpr int TH = 1 << L, NSB = 64 / TH, PPR = CLOSED ? kGroupPixels : 2, NR = (NSB + PPR - 1) / PPR;
    constexpr int G = 32 / PPR;
    const int lane = threadIdx.x & 31, gl = lane % G, half = lane / G;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int ux = (tp.wl * TH + 63) / 64;  // units per superblock band
    const unsigned nunits = (unsigned)ux * (unsigned)tp.hl;
    const FusedTickets tk = fused_tickets(nunits, gridDim.x * (kFusedThreads / 32), NR);
    unsigned long long nodes = 0, rows = 0;
    const unsigned nwarps = gridDim.x * (kFusedThreads / 32);
    for (unsigned tix = blockIdx.x * (kFusedThreads / 32) + (threadIdx.x >> 5); tix < tk.total; tix += nwarps) {
        // ticket -> unit and its rounds [k0, k1)
        unsigned u = tix;
        int k0 = 0, k1 = NR;
        if (tix >= tk.full) {
            const unsigned q = tix - tk.full, per = NR / tk.per_unit;
            u = tk.full + q / tk.per_unit;
            k0 = (int)((q % tk.per_unit) * per);
            k1 = k0 + (int)per;
        }
        const int by = (int)(u / (unsigned)ux), x0w = (int)(u % (unsigned)ux) * 64;
        float v[3][TH][2];
        float2 yref[3];
        strip_load<L>(tp, frame, stride, lut, by, x0w + 2 * lane, lane, v, yref);
        strip_analysis<L, 3, true>(v, lane);
        // superblock t's sum sits in lane t * 2^(n-1): lane t < NSB gathers it
        const int src = (lane * (TH / 2)) & 31;
        float yhi[3], ylo[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float sum = __shfl_sync(0xffffffffu, v[ch][0][0], src);
            yhi[ch] = __shfl_sync(0xffffffffu, yref[ch].x, src);
            ylo[ch] = fmaf(sum, 1.f / (float)(TH * TH), __shfl_sync(0xffffffffu, yref[ch].y, src));
        }
        const int sb0 = x0w / TH, nsb = min(NSB, tp.wl - sb0);  // superblocks of this unit
        BayesRec rec = {0, 0, 0.f, 0.f};
        if (lane < nsb) rec = bayes_setup(yhi, ylo, bp);
        for (int k = k0; k < k1 && PPR * k < nsb; ++k) {
            const int t = PPR * k + half;
            BayesRec rr;
            rr.i0 = __shfl_sync(0xffffffffu, rec.i0, t);
            rr.j0 = __shfl_sync(0xffffffffu, rec.j0, t);
            rr.U = __shfl_sync(0xffffffffu, rec.U, t);
            rr.V = __shfl_sync(0xffffffffu, rec.V, t);
            if constexpr (CLOSED)
                group_pixel(bp, rr, t < nsb, (long)by * tp.wl + sb0 + t, gl, chat, chat_scaled, scale, nodes, rows);
            else
                rows_pixel(bp, rr, t < nsb, (long)by * tp.wl + sb0 + t, gl, chat, chat_scaled, scale, nodes, rows);
        }
    }
    flush_counts(nodes_out, nodes, rows, lane);
}

// ---- One launch per frame: every step of the path for a strip in one warp ----
//
// For the plain posterior at 1..3 levels with the closed-form rows.  A warp takes a strip
// (64 pixel columns of one superblock band: 64 / 2^n superblocks) and, in registers:
// log-attenuation and the forward Haar levels (strip_load, strip_analysis); the Tikhonov
// operator on the directional coefficients (strip_tikhonov); the superblocks' block means
// and posterior records (bayes_setup on lanes 0 .. 64/2^n - 1); their posterior means eight
// at a time, four lanes each (group_sums); the inverse levels (strip_synthesis) with each
// superblock's mean as its low pass; THb and SO2 (strip_store).  A superblock's synthesis
// needs only its own mean, so no step waits for another warp: the frame is read once and
// nothing but the outputs (and the means, 8 bytes per superblock) is written.  For 3 levels
// a superblock's columns are the lanes of the group that computes its mean; for 1 and 2
// levels the means reach their lanes by shuffles.  The arithmetic is that of the separate
// analysis, posterior and synthesis kernels, so the outputs are the same bits.  Warp w of W
// takes strips w, w + W, ...
// Seven warps per CTA and four CTAs per SM (72 registers): 28 resident warps per SM, 4,256
// on the GPU, so the 4,050 strips of a 1920x1080 frame at 3 levels are taken in one round
// (eight warps and three CTAs per SM, 80 registers, left 402 strips for a second round: 22.5
// against 20.5 us per frame).
#ifndef HB_FRAME_THREADS
#define HB_FRAME_THREADS 224
#endif
#ifndef HB_FRAME_MINB
#define HB_FRAME_MINB 4
#endif
constexpr int kFrameThreads = HB_FRAME_THREADS;

template <int L, bool COUNT>
__global__ void __launch_bounds__(kFrameThreads, HB_FRAME_MINB)
    frame_kernel(TransformParams tp, BayesParams bp, const unsigned char* __restrict__ frame, size_t stride,
                 const float2* __restrict__ lut, float2* __restrict__ chat, float2* __restrict__ chat_scaled,
                 float scale, float* __restrict__ out0, float* __restrict__ out1, int debug_conc,
                 int pieces, unsigned long long* nodes_out) {
    constexpr int TH = 1 << L, NSB = 64 / TH, SBL = TH / 2;  // superblocks per strip, lanes per superblock
    constexpr int NR = NSB / kGroupPixels;                   // rounds of eight superblocks
    const int lane = threadIdx.x & 31, gl = lane % kGroup, grp = lane / kGroup, mine_sb = lane / SBL;
    // the frame (and the output buffers) may be written by the kernel before this one
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int ux = (tp.wl * TH + 63) / 64;  // strips per superblock band
    const unsigned nunits = (unsigned)ux * (unsigned)tp.hl;
    const int P = NR > 1 ? pieces : 1;  // pieces per strip (a strip of one round has one)
    const unsigned nwarps = gridDim.x * (kFrameThreads / 32), ntix = nunits * (unsigned)P;
    const int per = NR / P;  // rounds per piece
    unsigned long long nodes = 0, rows = 0;
    for (unsigned tix = blockIdx.x * (kFrameThreads / 32) + (threadIdx.x >> 5); tix < ntix; tix += nwarps) {
        const unsigned u = tix / (unsigned)P;
        const int k0 = (int)(tix % (unsigned)P) * per, k1 = k0 + per;  // this piece's rounds
        const int by = (int)(u / (unsigned)ux), x0w = (int)(u % (unsigned)ux) * 64, x = x0w + 2 * lane;
        float c[2][TH][2];
        float yhi[3], ylo[3];
        {
            float v[3][TH][2];
            float2 yref[3];
            strip_load<L>(tp, frame, stride, lut, by, x, lane, v, yref);
            strip_analysis<L, 3, false>(v, lane);
            // superblock t's sum sits in lane t * 2^(n-1): lane t < NSB gathers it
            const int src = (lane * SBL) & 31;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float sum = __shfl_sync(0xffffffffu, v[ch][0][0], src);
                yhi[ch] = __shfl_sync(0xffffffffu, yref[ch].x, src);
                ylo[ch] = fmaf(sum, 1.f / (float)(TH * TH), __shfl_sync(0xffffffffu, yref[ch].y, src));
            }
            strip_tikhonov<L>(tp, v, lane, c);
        }
        const int sb0 = x0w / TH, nsb = min(NSB, tp.wl - sb0);  // superblocks of this strip
        BayesRec rec = {0, 0, 0.f, 0.f};
        if (lane < nsb) rec = bayes_setup(yhi, ylo, bp);
        float2 mean = make_float2(0.f, 0.f);  // the posterior mean of this lane's superblock
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            if (k < k0) continue;
            if (k >= k1 || kGroupPixels * k >= nsb) break;
            const int t = kGroupPixels * k + grp;
            BayesRec rr;
            rr.i0 = __shfl_sync(0xffffffffu, rec.i0, t);
            rr.j0 = __shfl_sync(0xffffffffu, rec.j0, t);
            rr.U = __shfl_sync(0xffffffffu, rec.U, t);
            rr.V = __shfl_sync(0xffffffffu, rec.V, t);
            float sw, sdi, sdj;
            group_sums<COUNT>(bp, rr, t < nsb, gl, sw, sdi, sdj, nodes, rows);
            float2 m = make_float2(0.f, 0.f);
            if (t < nsb) {
                m = posterior_mean(bp, rr, sw, sdi, sdj);
                if (gl == 0) store_mean((long)by * tp.wl + sb0 + t, m, chat, chat_scaled, scale);
            }
            if constexpr (SBL == kGroup) {  // 3 levels: the group's lanes are the superblock's
                mean = m;
            } else {
                const int from = kGroup * (mine_sb % kGroupPixels);
                const float mx = __shfl_sync(0xffffffffu, m.x, from), my = __shfl_sync(0xffffffffu, m.y, from);
                if (mine_sb / kGroupPixels == k) mean = make_float2(mx, my);
            }
        }
        strip_synthesis<L>(c, lane);
        const int kr = mine_sb / kGroupPixels;  // the round of this lane's superblock
        if (kr >= k0 && kr < k1) strip_store<L>(tp, c, mean.x, mean.y, x, by, out0, out1, debug_conc);
    }
    if (COUNT) flush_counts(nodes_out, nodes, rows, lane);
}

// Resident CTAs per SM for a kernel (cached per device and kernel) and the SM count.
template <typename K>
cudaError_t residency(K kernel, int& resident, int& sms, int threads = kThreads) {
    static K cache_k[64];
    static int cache_res[64], cache_sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cache_res[dev] == 0 || cache_k[dev] != kernel) {
        e = cudaDeviceGetAttribute(&cache_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cache_res[dev], kernel, threads, 0);
        if (e != cudaSuccess) return e;
        if (cache_res[dev] < 1) cache_res[dev] = 1;
        cache_k[dev] = kernel;
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
                              chat_scaled, scale, gate, sc.nodes);
}

// The pair kernel when there are at least two pixels per resident warp (cudaErrorNotReady
// when there are fewer: the caller then uses the one-pixel-per-unit kernel).
template <int CPL>
cudaError_t launch_pair(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                        float2* chat, float2* chat_scaled, float scale, bool pdl, const PosteriorGate& gate,
                        cudaStream_t s) {
    int resident = 0, sms = 0;
    cudaError_t e = residency(posterior_pair_kernel<CPL>, resident, sms);
    if (e != cudaSuccess) return e;
    const long warps = (long)sms * resident * (kThreads / 32);
    if (npix < 2 * warps) return cudaErrorNotReady;
    const long rounds = (npix + 1) / 2;
    long blocks = (rounds + kThreads / 32 - 1) / (kThreads / 32);
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
    return cudaLaunchKernelEx(&cfg, posterior_pair_kernel<CPL>, bp, rec, npix, chat, chat_scaled, scale, gate,
                              sc.nodes);
}

// The span kernel under the same rule as the pair kernel.
template <bool RAGGED>
cudaError_t launch_span(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                        float2* chat, float2* chat_scaled, float scale, bool pdl, const PosteriorGate& gate,
                        cudaStream_t s) {
    int resident = 0, sms = 0;
    cudaError_t e = residency(posterior_span_kernel<RAGGED>, resident, sms, kSpanThreads);
    if (e != cudaSuccess) return e;
    const long warps = (long)sms * resident * (kSpanThreads / 32);
    if (npix < 2 * warps) return cudaErrorNotReady;
    const long rounds = (npix + 1) / 2;
    long blocks = (rounds + kSpanThreads / 32 - 1) / (kSpanThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kSpanThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, posterior_span_kernel<RAGGED>, bp, rec, npix, chat, chat_scaled, scale, gate,
                              sc.nodes);
}

// The row kernel under the same rule as the pair kernel.
cudaError_t launch_rows(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                        float2* chat, float2* chat_scaled, float scale, bool pdl, const PosteriorGate& gate,
                        cudaStream_t s) {
    int resident = 0, sms = 0;
    const bool closed = bp.row_tab != nullptr;
    auto kernel = closed ? posterior_rows_kernel<true> : posterior_rows_kernel<false>;
    cudaError_t e = residency(kernel, resident, sms, kRowThreads);
    if (e != cudaSuccess) return e;
    if (resident > kRowCtasPerSm) resident = kRowCtasPerSm;
    const long warps = (long)sms * resident * (kRowThreads / 32);
    if (npix < 2 * warps) return cudaErrorNotReady;
    const int ppw = closed ? kGroupPixels : 2;
    const long rounds = (npix + ppw - 1) / ppw;
    long blocks = (rounds + kRowThreads / 32 - 1) / (kRowThreads / 32);
    // at most kRowCtasPerSm CTAs per SM (resident above), leaving room beside them for CTAs
    // of the synthesis launched as its programmatic dependent (its transform runs before it
    // waits for the posterior)
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kRowThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, bp, rec, npix, chat, chat_scaled, scale, gate, sc.nodes);
}

bool uses_rows(const BayesParams& bp) {
#ifdef HB_POST_NO_ROWS
    return false;
#else
    return bp.rows_ok != 0;
#endif
}

bool uses_span(const BayesParams& bp) {
#ifdef HB_POST_NO_SPAN
    return false;
#else
    return bp.sup_cols && bp.n1 <= kSpanMaxCols;
#endif
}

}  // namespace

bool posterior_uses_pairs(const BayesParams& bp, long npix) {
    int resident = 0, sms = 0;
    cudaError_t e;
    if (uses_rows(bp)) {
        e = residency(bp.row_tab ? posterior_rows_kernel<true> : posterior_rows_kernel<false>, resident, sms,
                      kRowThreads);
        if (resident > kRowCtasPerSm) resident = kRowCtasPerSm;
        return e == cudaSuccess && npix >= 2L * sms * resident * (kRowThreads / 32);
    }
    if (uses_span(bp)) {
        e = bp.n1 % kSpanSeg ? residency(posterior_span_kernel<true>, resident, sms, kSpanThreads)
                             : residency(posterior_span_kernel<false>, resident, sms, kSpanThreads);
        return e == cudaSuccess && npix >= 2L * sms * resident * (kSpanThreads / 32);
    } else {
#ifdef HB_POST_NO_PAIRS
        return false;
#else
        if (bp.n1 > 128) return false;
        e = bp.n1 <= 16   ? residency(posterior_pair_kernel<1>, resident, sms)
            : bp.n1 <= 32 ? residency(posterior_pair_kernel<2>, resident, sms)
            : bp.n1 <= 64 ? residency(posterior_pair_kernel<4>, resident, sms)
                          : residency(posterior_pair_kernel<8>, resident, sms);
#endif
    }
    return e == cudaSuccess && npix >= 2L * sms * resident * (kThreads / 32);
}

bool lowpass_fused_ok(const TransformParams& tp, const BayesParams& bp) {
#ifdef HB_NO_FUSED_LOWPASS
    return false;
#else
    // where the separate posterior launch would take the row kernel too, so that each pixel's
    // result is the same either way (the learned stand-in's fallback runs the separate launch)
    return tp.levels >= 1 && tp.levels <= 3 && !tp.ll_intensity && uses_rows(bp) &&
           posterior_uses_pairs(bp, (long)tp.hl * tp.wl);
#endif
}

bool frame_kernel_ok(const TransformParams& tp, const BayesParams& bp) {
#ifdef HB_NO_FRAME_KERNEL
    return false;
#else
    return bp.row_tab != nullptr && !tp.tikhonov_lowpass && lowpass_fused_ok(tp, bp);
#endif
}

cudaError_t launch_frame(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                         const float2* lut, float2* chat, float2* chat_scaled, float scale, float* out0, float* out1,
                         int debug_conc, unsigned long long* nodes, bool pdl, cudaStream_t s) {
    int resident = 0, sms = 0;
    // the counting variant only when counters are given (timing armed)
    auto kernel = nodes ? (tp.levels == 1 ? frame_kernel<1, true> : tp.levels == 2 ? frame_kernel<2, true>
                                                                                    : frame_kernel<3, true>)
                        : (tp.levels == 1 ? frame_kernel<1, false> : tp.levels == 2 ? frame_kernel<2, false>
                                                                                     : frame_kernel<3, false>);
    cudaError_t e = residency(kernel, resident, sms, kFrameThreads);
    if (e != cudaSuccess) return e;
    const long units = (long)((tp.wl * (1 << tp.levels) + 63) / 64) * tp.hl;
    // a strip's rounds (1 at 3 levels, 2 at 2, 4 at 1) are split over as many warps as fill the
    // resident ones: each piece redoes the strip's analysis and stores its superblocks' columns
    const long warps = (long)sms * resident * (kFrameThreads / 32);
    const int nr = (64 >> tp.levels) / kGroupPixels;
    int pieces = 1;
    while (pieces < nr && units * 2 * pieces <= warps) pieces *= 2;
    long blocks = (units * pieces + kFrameThreads / 32 - 1) / (kFrameThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kFrameThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const unsigned char* f = static_cast<const unsigned char*>(frame);
    return cudaLaunchKernelEx(&cfg, kernel, tp, bp, f, stride, lut, chat, chat_scaled, scale, out0, out1, debug_conc,
                              pieces, nodes);
}

cudaError_t launch_lowpass_fused(const TransformParams& tp, const BayesParams& bp, const void* frame, size_t stride,
                                 const float2* lut, float2* chat, float2* chat_scaled, float scale,
                                 unsigned long long* nodes, bool pdl, cudaStream_t s) {
    int resident = 0, sms = 0;
    const bool closed = bp.row_tab != nullptr;
    auto kernel = closed ? (tp.levels == 1 ? lowpass_fused_kernel<1, true>
                            : tp.levels == 2 ? lowpass_fused_kernel<2, true>
                                             : lowpass_fused_kernel<3, true>)
                         : (tp.levels == 1 ? lowpass_fused_kernel<1, false>
                            : tp.levels == 2 ? lowpass_fused_kernel<2, false>
                                             : lowpass_fused_kernel<3, false>);
    cudaError_t e = residency(kernel, resident, sms, kFusedThreads);
    if (e != cudaSuccess) return e;
    const long units = (long)((tp.wl * (1 << tp.levels) + 63) / 64) * tp.hl;
    long blocks = (units + kFusedThreads / 32 - 1) / (kFusedThreads / 32);
    if (blocks > (long)sms * resident) blocks = (long)sms * resident;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const unsigned char* f = static_cast<const unsigned char*>(frame);
    return cudaLaunchKernelEx(&cfg, kernel, tp, bp, f, stride, lut, chat, chat_scaled, scale, nodes);
}

cudaError_t launch_posterior(const BayesParams& bp, const BayesRec* rec, long npix, const PosteriorScratch& sc,
                             float2* chat, float2* chat_scaled, float scale, bool pdl, cudaStream_t s,
                             const PosteriorGate& gate) {
    if (npix <= 0) return cudaSuccess;
    if (uses_rows(bp)) {
        cudaError_t e = launch_rows(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
        if (e != cudaErrorNotReady) return e;
    } else if (uses_span(bp)) {
        cudaError_t e = bp.n1 % kSpanSeg ? launch_span<true>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s)
                                         : launch_span<false>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
        if (e != cudaErrorNotReady) return e;
    }
#ifndef HB_POST_NO_PAIRS
    else if (bp.n1 <= 128) {
        cudaError_t e = bp.n1 <= 16   ? launch_pair<1>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s)
                        : bp.n1 <= 32 ? launch_pair<2>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s)
                        : bp.n1 <= 64 ? launch_pair<4>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s)
                                      : launch_pair<8>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
        if (e != cudaErrorNotReady) return e;
    }
#endif
    if (bp.n1 <= 32) return launch_cpl<1>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    if (bp.n1 <= 64) return launch_cpl<2>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    if (bp.n1 <= 128) return launch_cpl<4>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
    return launch_cpl<8>(bp, rec, npix, sc, chat, chat_scaled, scale, pdl, gate, s);
}

}  // namespace hb
