// hb_mlp.cu -- learned stand-in for the low-pass posterior step: a 3 -> 64 -> 64 -> 2
// multilayer perceptron with erf GELU, BF16 weights and activations and FP32
// accumulation, trained on (block-mean log-attenuation -> posterior mean) pairs that the
// posterior kernel produces.  The paper has no learned component; the network only
// stands in for its low-pass Bayesian estimate.
//
// Model.  x = T ybar + t0;  z1 = W1 x + b1;  h1 = bf16(gelu(z1));
//         z2 = W2 h1 + b2;  h2 = bf16(gelu(z2));  o = W3 h2 + b3;
//         c = b(ybar) + osc * o
// where b is the least-squares point moved by each box edge as if that edge alone cut the
// Gaussian likelihood (MlpNorm); the network learns what b leaves of the posterior mean
// (the corners, where two edges act together, and the grid's discreteness), in units of
// the posterior standard deviation osc; its input is ybar in least-squares coordinates.
// Loss: mean over samples and both outputs of (o - t)^2, t = (c_target - b(ybar)) / osc.
//
// Kernels.  mlp_train_kernel: a CTA of 4 warps takes 64 samples of a minibatch (16 per
// warp), runs the forward pass, the loss gradient and the backward pass, and writes its
// partial parameter gradients; the two 64x64 products per direction run on tensor cores
// (mma.sync m16n8k16, BF16 in, FP32 accumulate), the 3- and 2-wide layers on the FP32
// pipes.  mlp_adam_kernel adds the partials in a fixed order (deterministic) and applies
// Adam to the FP32 master weights, refreshing the BF16 copies.  mlp_forward_kernel:
// inference, 8 samples per warp held in tensor-core fragments.  mlp_forward_check_kernel:
// the same inference with the per-frame sampled exact check in extra CTAs of the launch,
// so that the check runs beside the inference instead of after it.  Weights are BF16;
// activations are rounded to BF16 at h1 and h2, and so is the gradient dz2 fed to the
// tensor cores; erf is evaluated to FP32 accuracy (see gelu); the input x
// stays FP32 (the correction varies fast near the box edges, so the input needs more
// resolution than BF16's 8 bits); accumulation is FP32 throughout.
#include "hb_common.cuh"
#include "hb_mlp.cuh"
#include "hb_posterior.cuh"

#include <cuda_bf16.h>
#include <math.h>

namespace hb {
namespace {

constexpr int kWarpsT = 4;                 // warps per training CTA
constexpr int kSamplesT = 16 * kWarpsT;    // samples per training CTA
constexpr float kInvSqrt2 = 0.70710678118654752440f;
constexpr float kInvSqrt2Pi = 0.39894228040143267794f;

// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 with erf by Abramowitz & Stegun 7.1.26
// (Hastings' rational approximation):
//   1 - erf(x) = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),  t = 1 / (1 + p x),
// x >= 0, |error| <= 1.5e-7 -- the accuracy of FP32 erff, in a third of the instructions
// (one reciprocal and one exponential on the MUFU).  1 + erf is formed as 2 - q for z >= 0
// and as q itself for z < 0 (erf is odd), so no digits cancel on the negative side.
__device__ __forceinline__ float gelu(float z) {
    const float x = z * kInvSqrt2, ax = fabsf(x);
    float t, e;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, ax, 1.f)));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * ax * ax));
    float poly = fmaf(1.061405429f, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    const float q = poly * t * e;
    return 0.5f * z * (x >= 0.f ? 2.f - q : q);
}
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * kInvSqrt2)) + z * kInvSqrt2Pi * expf(-0.5f * z * z);
}
#ifndef HB_MLP_ACT_FP32
#define HB_MLP_ACT_FP32 0  // 1: keep activations in FP32 (precision study only)
#endif
__device__ __forceinline__ float bf(float v) {
#if HB_MLP_ACT_FP32
    return v;
#else
    return __bfloat162float(__float2bfloat16_rn(v));
#endif
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);  // .x = lo (low 16 bits)
    return *reinterpret_cast<const unsigned*>(&p);
}

// D = A B + D for one m16n8k16 tile; a[4], b[2] packed bf16 pairs, d[4] FP32.
__device__ __forceinline__ void mma16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment helpers.  A(m, k) and B(k, n) are read through functors so that the same
// code serves transposed operands.  Layout of m16n8k16 (PTX ISA): g = lane / 4,
// q = lane % 4; A regs: (g, 2q..2q+1), (g+8, 2q..), (g, 2q+8..), (g+8, 2q+8..);
// B regs: (k = 2q..2q+1, n = g), (k = 2q+8.., n = g); C: (g, 2q..2q+1), (g+8, 2q..).
template <typename FA>
__device__ __forceinline__ void load_a(unsigned (&a)[4], FA A, int m0, int k0, int lane) {
    const int g = lane >> 2, q = lane & 3;
    a[0] = pack_bf16(A(m0 + g, k0 + 2 * q), A(m0 + g, k0 + 2 * q + 1));
    a[1] = pack_bf16(A(m0 + g + 8, k0 + 2 * q), A(m0 + g + 8, k0 + 2 * q + 1));
    a[2] = pack_bf16(A(m0 + g, k0 + 2 * q + 8), A(m0 + g, k0 + 2 * q + 9));
    a[3] = pack_bf16(A(m0 + g + 8, k0 + 2 * q + 8), A(m0 + g + 8, k0 + 2 * q + 9));
}
template <typename FB>
__device__ __forceinline__ void load_b(unsigned (&b)[2], FB B, int k0, int n0, int lane) {
    const int g = lane >> 2, q = lane & 3;
    b[0] = pack_bf16(B(k0 + 2 * q, n0 + g), B(k0 + 2 * q + 1, n0 + g));
    b[1] = pack_bf16(B(k0 + 2 * q + 8, n0 + g), B(k0 + 2 * q + 9, n0 + g));
}

// Parameters in shared memory (BF16 values held as float; they are exact in FP32).
struct SmemParams {
    float W1[kHid * kIn], b1[kHid], W2[kHid * kHid], b2[kHid], W3[kOut * kHid], b3[kOut];
};

__device__ void load_params(SmemParams& P, const float* __restrict__ wbf) {
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {
        const float v = wbf[i];
        if (i < kOffB1) P.W1[i - kOffW1] = v;
        else if (i < kOffW2) P.b1[i - kOffB1] = v;
        else if (i < kOffB2) P.W2[i - kOffW2] = v;
        else if (i < kOffW3) P.b2[i - kOffB2] = v;
        else if (i < kOffB3) P.W3[i - kOffW3] = v;
        else P.b3[i - kOffB3] = v;
    }
}

__device__ __forceinline__ float2 least_squares(const MlpNorm& nm, const float y[3]) {
    return make_float2(fmaf(nm.Ap[0], y[0], fmaf(nm.Ap[1], y[1], nm.Ap[2] * y[2])),
                       fmaf(nm.Ap[3], y[0], fmaf(nm.Ap[4], y[1], nm.Ap[5] * y[2])));
}

// The baseline b from the least-squares point (see MlpNorm): lambda(d) = phi(d) / Phi(d) as
// sqrt(2/pi) / erfcx(-d / sqrt 2), finite on both sides of the edge (erfcx overflows to
// infinity only far inside, where lambda is 0).
__device__ __forceinline__ float2 baseline(const MlpNorm& nm, float2 c) {
    constexpr float kSqrt2OverPi = 0.79788456080286535588f;
    float b0 = c.x, b1 = c.y;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float d = (nm.edge_sgn[e] * (e < 2 ? c.x : c.y) - nm.edge_pos[e]) * nm.edge_inv_s[e];
        const float lam = kSqrt2OverPi / erfcxf(-d * kInvSqrt2);
        b0 = fmaf(lam, nm.edge_v0[e], b0);
        b1 = fmaf(lam, nm.edge_v1[e], b1);
    }
    return make_float2(b0, b1);
}

// Whether the route sends the pixel with least-squares point c to the network (true) or
// lists it for the exact posterior.
__device__ __forceinline__ bool trusted(const MlpRoute& rt, float2 c) {
    if (!rt.trust) return true;
    const float u = (c.x - rt.org0) * rt.inv0, v = (c.y - rt.org1) * rt.inv1;
    if (!(u >= 0.f && v >= 0.f && u < (float)rt.k0 && v < (float)rt.k1)) return false;  // NaN too
    const int i = min((int)u, rt.k0 - 1), j = min((int)v, rt.k1 - 1);
    return rt.trust[i * rt.k1 + j] != 0;
}

// Per-warp forward for 16 samples whose inputs are ys[s][3].  TRAIN keeps z1 and z2
// for the backward pass; inference writes h2 straight from the tensor-core results.
template <bool TRAIN>
struct WarpBufT {
    float x[16][kIn];
    float h1[16][kHid], h2[16][kHid];
    float z1[TRAIN ? 16 : 1][kHid], z2[TRAIN ? 16 : 1][kHid];
    float o[16][kOut];
};
typedef WarpBufT<true> WarpBuf;

template <bool TRAIN>
__device__ void warp_forward(const SmemParams& P, const MlpNorm& nm, WarpBufT<TRAIN>& B, const float (*ys)[3],
                             int lane) {
    if (lane < 16)
        for (int c = 0; c < kIn; ++c)
            B.x[lane][c] = nm.T[c * 3] * ys[lane][0] + nm.T[c * 3 + 1] * ys[lane][1] + nm.T[c * 3 + 2] * ys[lane][2] +
                           nm.t0[c];
    __syncwarp();
    // layer 1 (FP32 pipes): 16 samples x 64 units, 32 per lane
    for (int e = lane; e < 16 * kHid; e += 32) {
        const int s = e / kHid, u = e % kHid;
        float z = P.b1[u];
        for (int c = 0; c < kIn; ++c) z = fmaf(P.W1[u * kIn + c], B.x[s][c], z);
        if (TRAIN) B.z1[s][u] = z;
        B.h1[s][u] = bf(gelu(z));
    }
    __syncwarp();
    // layer 2 on tensor cores: z2 (16 x 64) = h1 (16 x 64) W2^T
    const int g = lane >> 2, q = lane & 3;
    for (int nt = 0; nt < kHid / 8; ++nt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        for (int kt = 0; kt < kHid / 16; ++kt) {
            unsigned a[4], b[2];
            load_a(a, [&](int m, int k) { return B.h1[m][k]; }, 0, kt * 16, lane);
            load_b(b, [&](int k, int n) { return P.W2[n * kHid + k]; }, kt * 16, nt * 8, lane);
            mma16816(d, a, b);
        }
        const int n = nt * 8 + 2 * q;
        const float z00 = d[0] + P.b2[n], z01 = d[1] + P.b2[n + 1];
        const float z10 = d[2] + P.b2[n], z11 = d[3] + P.b2[n + 1];
        if (TRAIN) {
            B.z2[g][n] = z00;
            B.z2[g][n + 1] = z01;
            B.z2[g + 8][n] = z10;
            B.z2[g + 8][n + 1] = z11;
        }
        B.h2[g][n] = bf(gelu(z00));
        B.h2[g][n + 1] = bf(gelu(z01));
        B.h2[g + 8][n] = bf(gelu(z10));
        B.h2[g + 8][n + 1] = bf(gelu(z11));
    }
    __syncwarp();
    // layer 3 (FP32 pipes): 16 samples x 2 outputs, one per lane
    {
        const int s = lane >> 1, j = lane & 1;
        float o = P.b3[j];
        for (int u = 0; u < kHid; ++u) o = fmaf(P.W3[j * kHid + u], B.h2[s][u], o);
        B.o[s][j] = o;
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned hash_u32(unsigned x) {
    // integer hash (a variant of the well-known "lowbias32" mixing function)
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

struct TrainSmem {
    SmemParams P;
    WarpBuf W[kWarpsT];
    float dz2[kSamplesT][kHid];  // BF16 values
    float h1[kSamplesT][kHid];   // copy of the CTA's h1 for dW2
    float dz1[kSamplesT][kHid];
    float do_[kSamplesT][kOut];
    float ys[kSamplesT][3];
    float red[kWarpsT];
};

// One CTA: 64 samples of the minibatch -> partial gradients (kNParams floats) and the
// partial sum of squared errors.  Samples index into (ybar, target) through a hash of
// (seed, step, position) unless idx_direct is set (sample b of the batch is row b).
__global__ void __launch_bounds__(32 * kWarpsT) mlp_train_kernel(const float* __restrict__ wbf, MlpNorm nm,
                                                                 const float* __restrict__ ybar,
                                                                 const float* __restrict__ target, long n, int batch,
                                                                 unsigned seed, int step, int idx_direct,
                                                                 float* __restrict__ gpart,
                                                                 float* __restrict__ lpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_params(S.P, wbf);
    // gather the CTA's samples
    float* tgt_local = &S.do_[0][0];  // targets staged here, replaced by dL/do below
    for (int s = threadIdx.x; s < kSamplesT; s += blockDim.x) {
        const long b = (long)blockIdx.x * kSamplesT + s;
        long r = 0;
        const bool valid = b < batch;
        if (valid) r = idx_direct ? b : (long)(hash_u32(seed ^ hash_u32((unsigned)step * 0x9E3779B9U + (unsigned)b)) % (unsigned long)n);
        for (int c = 0; c < 3; ++c) S.ys[s][c] = valid ? ybar[r * 3 + c] : 0.f;
        for (int j = 0; j < kOut; ++j) tgt_local[s * kOut + j] = valid ? target[r * 2 + j] : 0.f;
    }
    __syncthreads();
    WarpBuf& B = S.W[warp];
    const int s0 = warp * 16;
    warp_forward<true>(S.P, nm, B, &S.ys[s0], lane);
    // loss and dL/do = (o - t) / (batch * kOut) * 2  (mean over batch * 2 elements)
    float sq = 0.f;
    {
        const int s = lane >> 1, j = lane & 1;
        const long b = (long)blockIdx.x * kSamplesT + s0 + s;
        const float* y = S.ys[s0 + s];
        const float osc = j == 0 ? nm.osc0 : nm.osc1;
        const float2 bl = baseline(nm, least_squares(nm, y));
        const float t = (tgt_local[(s0 + s) * kOut + j] - (j == 0 ? bl.x : bl.y)) / osc;
        const float err = b < batch ? B.o[s][j] - t : 0.f;
        sq = err * err;
        S.do_[s0 + s][j] = err * (2.f / ((float)batch * kOut));
    }
    for (int off = 16; off > 0; off >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, off);
    if (lane == 0) S.red[warp] = sq;
    __syncwarp();
    // dz2 = (W3^T do) * gelu'(z2), rounded to BF16 for the tensor cores
    for (int e = lane; e < 16 * kHid; e += 32) {
        const int s = e / kHid, u = e % kHid;
        const float dh = S.P.W3[u] * S.do_[s0 + s][0] + S.P.W3[kHid + u] * S.do_[s0 + s][1];
        S.dz2[s0 + s][u] = bf(dh * gelu_grad(B.z2[s][u]));
        S.h1[s0 + s][u] = B.h1[s][u];
    }
    __syncwarp();
    // dh1 (16 x 64) = dz2 (16 x 64) W2 on tensor cores, then dz1 = dh1 * gelu'(z1)
    {
        const int g = lane >> 2, q = lane & 3;
        for (int nt = 0; nt < kHid / 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int kt = 0; kt < kHid / 16; ++kt) {
                unsigned a[4], b[2];
                load_a(a, [&](int m, int k) { return S.dz2[s0 + m][k]; }, 0, kt * 16, lane);
                load_b(b, [&](int k, int nn) { return S.P.W2[k * kHid + nn]; }, kt * 16, nt * 8, lane);
                mma16816(d, a, b);
            }
            const int nn = nt * 8 + 2 * q;
            S.dz1[s0 + g][nn] = d[0] * gelu_grad(B.z1[g][nn]);
            S.dz1[s0 + g][nn + 1] = d[1] * gelu_grad(B.z1[g][nn + 1]);
            S.dz1[s0 + g + 8][nn] = d[2] * gelu_grad(B.z1[g + 8][nn]);
            S.dz1[s0 + g + 8][nn + 1] = d[3] * gelu_grad(B.z1[g + 8][nn + 1]);
        }
    }
    __syncthreads();
    float* gp = gpart + (size_t)blockIdx.x * kNParams;
    // dW2 (64 x 64) = dz2^T (64 x 64 samples) h1 (64 samples x 64): warp w takes rows 16w..16w+15
    {
        const int g = lane >> 2, q = lane & 3, m0 = warp * 16;
        for (int nt = 0; nt < kHid / 8; ++nt) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            for (int kt = 0; kt < kSamplesT / 16; ++kt) {
                unsigned a[4], b[2];
                load_a(a, [&](int m, int k) { return S.dz2[k][m]; }, m0, kt * 16, lane);
                load_b(b, [&](int k, int nn) { return S.h1[k][nn]; }, kt * 16, nt * 8, lane);
                mma16816(d, a, b);
            }
            const int nn = nt * 8 + 2 * q;
            gp[kOffW2 + (m0 + g) * kHid + nn] = d[0];
            gp[kOffW2 + (m0 + g) * kHid + nn + 1] = d[1];
            gp[kOffW2 + (m0 + g + 8) * kHid + nn] = d[2];
            gp[kOffW2 + (m0 + g + 8) * kHid + nn + 1] = d[3];
        }
    }
    // the small layers and the biases: one thread per parameter, fixed-order sums over samples
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) {
        if (i >= kOffW2 && i < kOffB2) continue;
        float acc = 0.f;
        if (i < kOffB1) {
            const int u = (i - kOffW1) / kIn, c = (i - kOffW1) % kIn;
            for (int s = 0; s < kSamplesT; ++s) acc = fmaf(S.dz1[s][u], S.W[s / 16].x[s % 16][c], acc);
        } else if (i < kOffW2) {
            const int u = i - kOffB1;
            for (int s = 0; s < kSamplesT; ++s) acc += S.dz1[s][u];
        } else if (i < kOffW3) {
            const int u = i - kOffB2;
            for (int s = 0; s < kSamplesT; ++s) acc += S.dz2[s][u];
        } else if (i < kOffB3) {
            const int j = (i - kOffW3) / kHid, u = (i - kOffW3) % kHid;
            for (int s = 0; s < kSamplesT; ++s) acc = fmaf(S.do_[s][j], S.W[s / 16].h2[s % 16][u], acc);
        } else {
            const int j = i - kOffB3;
            for (int s = 0; s < kSamplesT; ++s) acc += S.do_[s][j];
        }
        gp[i] = acc;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int w = 0; w < kWarpsT; ++w) l += S.red[w];
        lpart[blockIdx.x] = l;
    }
}

__global__ void mlp_adam_kernel(const float* __restrict__ gpart, const float* __restrict__ lpart, int nblocks,
                                int batch, float* __restrict__ grad, float* __restrict__ loss, float* __restrict__ master,
                                float* __restrict__ m, float* __restrict__ v, float* __restrict__ wbf, float lr,
                                float beta1, float beta2, float eps, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        float l = 0.f;
        for (int b = 0; b < nblocks; ++b) l += lpart[b];
        *loss = l / ((float)batch * kOut);
    }
    if (i >= kNParams) return;
    float gsum = 0.f;
    for (int b = 0; b < nblocks; ++b) gsum += gpart[(size_t)b * kNParams + i];
    grad[i] = gsum;
    if (lr > 0.f && master) {
        const float mi = beta1 * m[i] + (1.f - beta1) * gsum;
        const float vi = beta2 * v[i] + (1.f - beta2) * gsum * gsum;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.f - powf(beta1, (float)t)), vh = vi / (1.f - powf(beta2, (float)t));
        const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
        master[i] = w;
        wbf[i] = bf(w);
    }
}

// Inference.  One warp computes 8 samples at a time entirely in registers, with layer 2
// transposed: z2^T (64 units x 8 samples) = W2 h1^T, so W2 is the m16n8k16 A operand
// (staged once per CTA as ready-made fragments) and the 8 samples are N.  Lane (g, q)
// (g = lane / 4, q = lane % 4) evaluates layer 1 for sample g at exactly the hidden units
// its B fragments hold (k = 16 kt + 2q + {0, 1, 8, 9}), so h1 goes from the FP32 pipes
// straight into the tensor-core operands; the accumulators come back holding units
// 16 mt + g + {0, 8} of samples 2q, 2q + 1, where GELU, the BF16 rounding of h2 and the
// lane's share of layer 3 are applied, and shuffles over g finish layer 3.
constexpr int kWarpsF = 8;
constexpr int kMlpCheckPerCta = kWarpsF / 2;  // drawn pixels a check CTA takes at a time
static_assert(kMlpCheckPerCta == 4, "pair_barrier names one barrier per pair of warps");

// Barrier of the two warps 2 pair, 2 pair + 1 (named barriers 1 .. 4; 0 is __syncthreads).
// The identifiers are literals so that the kernel reserves only the barriers it uses.
__device__ __forceinline__ void pair_barrier(int pair) {
    switch (pair) {
        case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
        case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
        case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
        default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
}
struct __align__(16) InferSmem {
    uint4 w2f[kHid / 16][kHid / 16][32];  // W2 A fragments per (m tile, k tile, lane)
    float4 l1[kHid];                      // W1[u][0..2], b1[u]
    float4 l3[kHid];                      // b2[u], W3[0][u], W3[1][u], 0
    float4 b3;                            // b3[0], b3[1], 0, 0
};
static_assert(sizeof(InferSmem) % 16 == 0, "the image is copied in 16-byte words");

// The network as the inference kernel holds it in shared memory, built once per parameter
// change (mlp_pack_kernel) so that every CTA stages it with coalesced 16-byte loads.
__global__ void __launch_bounds__(256) mlp_pack_kernel(const float* __restrict__ wbf, InferSmem* __restrict__ img) {
    for (int i = threadIdx.x; i < (kHid / 16) * (kHid / 16) * 32; i += blockDim.x) {
        const int l = i & 31, kt = (i >> 5) % (kHid / 16), mt = i / (32 * (kHid / 16));
        const float* w0 = wbf + kOffW2 + (mt * 16 + (l >> 2)) * kHid + kt * 16 + 2 * (l & 3);
        const float* w8 = w0 + 8 * kHid;
        img->w2f[mt][kt][l] = make_uint4(pack_bf16(w0[0], w0[1]), pack_bf16(w8[0], w8[1]), pack_bf16(w0[8], w0[9]),
                                         pack_bf16(w8[8], w8[9]));
    }
    for (int u = threadIdx.x; u < kHid; u += blockDim.x) {
        img->l1[u] = make_float4(wbf[kOffW1 + u * kIn], wbf[kOffW1 + u * kIn + 1], wbf[kOffW1 + u * kIn + 2],
                                 wbf[kOffB1 + u]);
        img->l3[u] = make_float4(wbf[kOffB2 + u], wbf[kOffW3 + u], wbf[kOffW3 + kHid + u], 0.f);
    }
    if (threadIdx.x == 0) img->b3 = make_float4(wbf[kOffB3], wbf[kOffB3 + 1], 0.f, 0.f);
}

// One 8-sample tile (samples 8 tile .. 8 tile + 7) through the network in one warp.  The
// lanes with g < 2 end up holding sample 2q + g: they return its index and leave its
// estimate in val; the other lanes, and samples past n, return -1.  With a route, the
// samples of untrusted cells are appended to its list (their estimates are still written;
// the exact posterior replaces them).
__device__ __forceinline__ long infer_tile(const InferSmem& S, const MlpNorm& nm, const float* __restrict__ ybar,
                                           long n, long tile, int lane, float2& val,
                                           const MlpRoute& rt = MlpRoute{}) {
    const int g = lane >> 2, q = lane & 3;
    const long r = tile * 8 + g;
    float y[3], x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = r < n ? ybar[r * 3 + c] : 0.f;
#pragma unroll
    for (int c = 0; c < kIn; ++c)
        x[c] = nm.T[c * 3] * y[0] + nm.T[c * 3 + 1] * y[1] + nm.T[c * 3 + 2] * y[2] + nm.t0[c];
    // layer 1 into the B fragments of layer 2 (k = unit, n = sample g)
    unsigned bfr[kHid / 16][2];
#pragma unroll
    for (int kt = 0; kt < kHid / 16; ++kt) {
        float h[4];  // units 16 kt + 2q + {0, 1, 8, 9}
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float4 w = S.l1[kt * 16 + 2 * q + (v & 1) + 8 * (v >> 1)];
            float z = w.w;
            z = fmaf(w.x, x[0], z);
            z = fmaf(w.y, x[1], z);
            z = fmaf(w.z, x[2], z);
            h[v] = gelu(z);
        }
        bfr[kt][0] = pack_bf16(h[0], h[1]);
        bfr[kt][1] = pack_bf16(h[2], h[3]);
    }
    // layer 2 on the tensor cores, layer 3 from the accumulators
    float o00 = 0.f, o01 = 0.f, o10 = 0.f, o11 = 0.f;  // (sample 2q / 2q + 1, output 0 / 1)
#pragma unroll
    for (int mt = 0; mt < kHid / 16; ++mt) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kHid / 16; ++kt) {
            const uint4 aw = S.w2f[mt][kt][lane];
            const unsigned af[4] = {aw.x, aw.y, aw.z, aw.w};
            mma16816(d, af, bfr[kt]);
        }
        // d: (unit mt*16 + g, samples 2q, 2q+1), (unit mt*16 + g + 8, samples 2q, 2q+1)
        const float4 la = S.l3[mt * 16 + g], lb = S.l3[mt * 16 + g + 8];
        const float h00 = bf(gelu(d[0] + la.x)), h01 = bf(gelu(d[1] + la.x));
        const float h10 = bf(gelu(d[2] + lb.x)), h11 = bf(gelu(d[3] + lb.x));
        o00 = fmaf(la.y, h00, fmaf(lb.y, h10, o00));
        o01 = fmaf(la.z, h00, fmaf(lb.z, h10, o01));
        o10 = fmaf(la.y, h01, fmaf(lb.y, h11, o10));
        o11 = fmaf(la.z, h01, fmaf(lb.z, h11, o11));
    }
#pragma unroll
    for (int off = 4; off <= 16; off <<= 1) {
        o00 += __shfl_xor_sync(0xffffffffu, o00, off);
        o01 += __shfl_xor_sync(0xffffffffu, o01, off);
        o10 += __shfl_xor_sync(0xffffffffu, o10, off);
        o11 += __shfl_xor_sync(0xffffffffu, o11, off);
    }
    // lanes g = 0 and g = 1 hold samples 2q and 2q + 1; they need those samples' ybar
    const int s = 2 * q + (g & 1);
    const long rs = tile * 8 + s;
    const float ya = __shfl_sync(0xffffffffu, y[0], 4 * s), yb = __shfl_sync(0xffffffffu, y[1], 4 * s),
                yc = __shfl_sync(0xffffffffu, y[2], 4 * s);
    const bool mine = g < 2 && rs < n;
    const float ys[3] = {ya, yb, yc};
    const float2 cls = least_squares(nm, ys);
    if (rt.trust) {
        // warp-aggregated append of the untrusted samples
        const bool out = mine && !trusted(rt, cls);
        const unsigned m = __ballot_sync(0xffffffffu, out);
        if (m) {
            unsigned base = 0;
            if (lane == __ffs(m) - 1) base = atomicAdd(rt.count, (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
            const unsigned at = base + __popc(m & ((1u << lane) - 1u));
            if (out && at < (unsigned long)n) rt.list[at] = (int)rs;  // at most n are ever listed
        }
    }
    if (!mine) return -1;
    const float o0 = (g & 1) ? o10 : o00, o1 = (g & 1) ? o11 : o01;
    const float2 bl = baseline(nm, cls);
    val = make_float2(fmaf(nm.osc0, o0 + S.b3.x, bl.x), fmaf(nm.osc1, o1 + S.b3.y, bl.y));
    return rs;
}

// Every CTA stages the network image before waiting on the kernel that writes ybar (the
// weights do not come from it); then the launch's dependents may start.
__device__ __forceinline__ void stage_image(InferSmem& S, const InferSmem* __restrict__ img) {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(&S);
    for (int i = threadIdx.x; i < (int)(sizeof(InferSmem) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
    // programmatic dependent launch: returns at once after a plain launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
}

__global__ void __launch_bounds__(32 * kWarpsF) mlp_forward_kernel(const InferSmem* __restrict__ img, MlpNorm nm,
                                                                   const float* __restrict__ ybar, long n,
                                                                   float2* __restrict__ chat) {
    __shared__ InferSmem S;
    stage_image(S, img);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long ntile = (n + 7) / 8;
    for (long tile = (long)blockIdx.x * kWarpsF + warp; tile < ntile; tile += (long)gridDim.x * kWarpsF) {
        float2 v;
        const long rs = infer_tile(S, nm, ybar, n, tile, lane, v);
        if (rs >= 0) chat[rs] = v;
    }
}

// Posterior mean of one pixel computed by one warp (CPL grid columns per lane), valid in
// every lane.  Rows: those of the span kernel's cut where it applies (every node left out
// weighs under 2^-span_cut of the reference node, together under 2^-30 of the posterior
// mass), else the rows of non-zero FP32 weight; each row is summed whole.
template <int CPL>
__device__ float2 warp_posterior_mean(const BayesParams& bp, const BayesRec& rec, int lane) {
    int lo, hi;
    if (bp.sup_cols) {
        const SpanPixel sp = span_pixel(bp, rec);
        lo = sp.rlo;
        hi = sp.rhi;
    } else {
        support_rows(bp, rec, lo, hi);
    }
    float sw = 0.f, sdi = 0.f, sdj = 0.f;
    grid_sums<CPL>(bp, rec, lane, lo, hi, 0.f, sw, sdi, sdj);
    sw = warp_sum(sw);
    sdi = warp_sum(sdi);
    sdj = warp_sum(sdj);
    if (!usable(sw, sdi, sdj)) {  // far outside the model: all rows, explicit maximum shift
        const float shift = warp_max(grid_max<CPL>(bp, rec, lane, 0, bp.n0));
        sw = sdi = sdj = 0.f;
        grid_sums<CPL>(bp, rec, lane, 0, bp.n0, shift, sw, sdi, sdj);
        sw = warp_sum(sw);
        sdi = warp_sum(sdi);
        sdj = warp_sum(sdj);
    }
    return make_float2(fmaf(bp.h0f, sdi / sw, fmaf((float)rec.i0, bp.h0f, bp.lo0f)),
                       fmaf(bp.h1f, sdj / sw, fmaf((float)rec.j0, bp.h1f, bp.lo1f)));
}

// Inference and the sampled exact check in one launch.  CTAs 0 .. ck.nctas - 1 check
// kMlpCheckPerCta drawn pixels at a time, one per pair of warps: the even warp computes the
// pixel's exact posterior mean (warp_posterior_mean) while the odd warp runs the pixel's
// 8-sample tile through the same code as the inference CTAs; then err[k] = the larger of
// the two axes' errors relative to the box extents (NaN if either is).  The last check
// CTA to arrive adds the errors in a fixed order and leaves the decision in sync[2]
// (sync[1] counts the failed frames, sync[0] is the arrival counter).  The remaining CTAs
// run inference exactly as mlp_forward_kernel and, if chat_scaled is set, also write the
// estimates times scale there.
template <int CPL>
__global__ void __launch_bounds__(32 * kWarpsF, 4)
    mlp_forward_check_kernel(const InferSmem* __restrict__ img, MlpNorm nm, const float* __restrict__ ybar, long n,
                             float2* __restrict__ chat, float2* __restrict__ chat_scaled, float scale,
                             BayesParams bp, const BayesRec* __restrict__ recs, MlpCheck ck, MlpRoute rt) {
    __shared__ InferSmem S;
    __shared__ float2 est[kMlpCheckPerCta];
    __shared__ float red[kWarpsF];
    __shared__ unsigned redbad[kWarpsF];
    __shared__ unsigned last;
    stage_image(S, img);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // every kernel before this one in the stream has completed (the wait in stage_image), so
    // the previous frame's exact posterior has read its counter: clear it for the next frame
    if (rt.next_count && blockIdx.x == 0 && threadIdx.x == 0) *rt.next_count = 0u;
    if ((int)blockIdx.x >= ck.nctas) {
        const long ntile = (n + 7) / 8, nblk = (long)gridDim.x - ck.nctas;
        for (long tile = ((long)blockIdx.x - ck.nctas) * kWarpsF + warp; tile < ntile; tile += nblk * kWarpsF) {
            float2 v;
            const long rs = infer_tile(S, nm, ybar, n, tile, lane, v, rt);
            if (rs >= 0) {
                chat[rs] = v;
                if (chat_scaled) chat_scaled[rs] = make_float2(scale * v.x, scale * v.y);
            }
        }
        return;
    }
    const int pair = warp >> 1;
    for (int k0 = blockIdx.x * kMlpCheckPerCta; k0 < ck.nsample; k0 += ck.nctas * kMlpCheckPerCta) {
        const int k = k0 + pair;
        const bool on = k < ck.nsample;  // the same for both warps of the pair
        const long p = on ? sample_pixel(ck.seed, k, n) : 0;
        float2 c = make_float2(0.f, 0.f);
        if (on && (warp & 1)) {
            float2 v = make_float2(0.f, 0.f);
            const long rs = infer_tile(S, nm, ybar, n, p >> 3, lane, v);
            const int src = __ffs(__ballot_sync(0xffffffffu, rs == p)) - 1;  // the one lane holding p
            const float ex = __shfl_sync(0xffffffffu, v.x, src), ey = __shfl_sync(0xffffffffu, v.y, src);
            if (lane == 0) est[pair] = make_float2(ex, ey);
        } else if (on) {
            c = warp_posterior_mean<CPL>(bp, recs[p], lane);
        }
        pair_barrier(pair);  // the even warp reads what the odd one wrote
        if (on && !(warp & 1) && lane == 0) {
            const float2 e = est[pair];
            const float dx = fabsf(e.x - c.x) * ck.inv_ext0, dy = fabsf(e.y - c.y) * ck.inv_ext1;
            float err = isnan(dx) || isnan(dy) ? NAN : fmaxf(dx, dy);
            if (rt.trust) {  // a listed pixel gets the exact posterior: nothing to check
                const float yp[3] = {ybar[p * 3], ybar[p * 3 + 1], ybar[p * 3 + 2]};
                if (!trusted(rt, least_squares(nm, yp))) err = 0.f;
            }
            ck.err[k] = err;
        }
        pair_barrier(pair);  // est[pair] free again
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // the CTA's errors (ordered before by the barrier) before the arrival
        last = atomicAdd(&ck.sync[0], 1u) == (unsigned)ck.nctas - 1u ? 1u : 0u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the decision: the largest sampled error (or their mean) against tol; a NaN fails
    const volatile float* ev = ck.err;
    float e = 0.f;
    unsigned bad = 0u;
    for (int k = threadIdx.x; k < ck.nsample; k += blockDim.x) {
        const float v = ev[k];
        bad |= isnan(v) ? 1u : 0u;
        e = ck.use_max ? fmaxf(e, v) : e + v;
    }
    e = ck.use_max ? warp_max(e) : warp_sum(e);
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0) {
        red[warp] = e;
        redbad[warp] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kWarpsF; ++w) {
            t = ck.use_max ? fmaxf(t, red[w]) : t + red[w];
            bad |= redbad[w];
        }
        const float stat = ck.use_max ? t : t / (float)ck.nsample;
        const bool run = bad || !(stat <= ck.tol);
        ck.sync[2] = run ? 1u : 0u;
        if (run) ck.sync[1] += 1u;
        ck.sync[0] = 0u;
    }
}

template <typename K>
cudaError_t set_smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_train(const float* wbf, const MlpNorm& nm, const float* ybar, const float* target, long n,
                             int batch, unsigned seed, int step, int idx_direct, float* gpart, float* lpart,
                             cudaStream_t s) {
    const size_t sm = sizeof(TrainSmem);
    cudaError_t e = set_smem_attr(mlp_train_kernel, sm);
    if (e != cudaSuccess) return e;
    const int blocks = (batch + kSamplesT - 1) / kSamplesT;
    mlp_train_kernel<<<blocks, 32 * kWarpsT, sm, s>>>(wbf, nm, ybar, target, n, batch, seed, step, idx_direct, gpart,
                                                       lpart);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const float* gpart, const float* lpart, int nblocks, int batch, float* grad, float* loss,
                            float* master, float* m, float* v, float* wbf, float lr, float beta1, float beta2,
                            float eps, int t, cudaStream_t s) {
    mlp_adam_kernel<<<(kNParams + 255) / 256, 256, 0, s>>>(gpart, lpart, nblocks, batch, grad, loss, master, m, v,
                                                            wbf, lr, beta1, beta2, eps, t);
    return cudaGetLastError();
}

size_t mlp_image_bytes() { return sizeof(InferSmem); }

cudaError_t launch_mlp_pack(const float* wbf, void* img, cudaStream_t s) {
    mlp_pack_kernel<<<1, 256, 0, s>>>(wbf, static_cast<InferSmem*>(img));
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat, bool pdl,
                               cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long tiles = (n + 7) / 8;
    long blocks = (tiles + kWarpsF - 1) / kWarpsF;  // one tile per warp while that fits
    if (blocks > 8L * sms) blocks = 8L * sms;
    if (blocks < 1) blocks = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(32 * kWarpsF);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, mlp_forward_kernel, static_cast<const InferSmem*>(img), nm, ybar, n, chat);
}

namespace {

template <int CPL>
cudaError_t launch_forward_check_cpl(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat,
                                     float2* chat_scaled, float scale, const BayesParams& bp, const BayesRec* rec,
                                     const MlpCheck& ck, const MlpRoute& rt, unsigned blocks, bool pdl,
                                     cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32 * kWarpsF);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, mlp_forward_check_kernel<CPL>, static_cast<const InferSmem*>(img), nm, ybar, n,
                              chat, chat_scaled, scale, bp, rec, ck, rt);
}

}  // namespace

cudaError_t launch_mlp_forward_check(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat,
                                     float2* chat_scaled, float scale, const BayesParams& bp, const BayesRec* rec,
                                     MlpCheck ck, const MlpRoute& rt, bool pdl, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (ck.nsample <= 0) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // check CTAs first (dispatched first), kMlpCheckPerCta drawn pixels each while 4096 CTAs
    // suffice
    const long need = (ck.nsample + kMlpCheckPerCta - 1) / kMlpCheckPerCta;
    ck.nctas = (int)(need < 4096 ? need : 4096);
    const long tiles = (n + 7) / 8;
    long blocks = (tiles + kWarpsF - 1) / kWarpsF;  // one tile per warp while that fits
    if (blocks > 8L * sms) blocks = 8L * sms;
    if (blocks < 1) blocks = 1;
    blocks += ck.nctas;
#define HB_FC_ARGS img, nm, ybar, n, chat, chat_scaled, scale, bp, rec, ck, rt, (unsigned)blocks, pdl, s
    if (bp.n1 <= 32) return launch_forward_check_cpl<1>(HB_FC_ARGS);
    if (bp.n1 <= 64) return launch_forward_check_cpl<2>(HB_FC_ARGS);
    if (bp.n1 <= 128) return launch_forward_check_cpl<4>(HB_FC_ARGS);
    return launch_forward_check_cpl<8>(HB_FC_ARGS);
#undef HB_FC_ARGS
}

}  // namespace hb
