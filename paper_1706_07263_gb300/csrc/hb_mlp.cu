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

// Inference on the fifth-generation tensor cores.  A warpgroup (128 threads) takes 128
// samples at a time, one per thread: layer 1 on the FP32 pipes, h1 rounded to BF16 and
// written to shared memory as the A operand (128 x 64, K-major); layer 2, z2 = h1 W2^T,
// as four tcgen05.mma of K = 16 (kind::f16, BF16 in, FP32 accumulate) issued by one
// thread, with W2 (64 x 64, K-major) as the B operand in the CTA's copy of the network
// image and the accumulator in 64 columns of tensor memory; the commit arrives on the
// warpgroup's mbarrier, and each thread then reads its sample's row of z2 from tensor
// memory (tcgen05.ld, 16 columns at a time) to apply b2, GELU, the BF16 rounding of h2 and
// layer 3 on the FP32 pipes.  Operand layout (no swizzle): 8 x 16-byte core matrices,
// core matrix (K group kg, row group rg) at byte (kg * R + rg) * 128 for R row groups, so
// the descriptor's leading (K-direction) byte offset is 128 R and its stride (row-direction)
// offset 128; the K = 16 step s starts 2 s core matrices further along K.
constexpr int kWarpsF = 8;                    // 256 threads: two warpgroups
constexpr int kTileF = 128;                   // samples per warpgroup tile
constexpr int kTmemColsF = 128;               // tensor-memory columns per CTA (64 per warpgroup)
constexpr int kMlpCheckPerCta = kWarpsF / 2;  // drawn pixels a check CTA takes at a time
static_assert(kMlpCheckPerCta == 4, "pair_barrier names one barrier per pair of warps");
// h1 tiles of the two warpgroups (dynamic shared memory), plus a pad that keeps a CTA's
// shared memory above a fifth of the SM's, so that at most four CTAs share an SM's 512
// tensor-memory columns
constexpr size_t kTcSmemBytes = 2 * kTileF * kHid * 2 + 4096;

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
// Barrier of the four warps of warpgroup wg (named barriers 5, 6).
__device__ __forceinline__ void wg_barrier(int wg) {
    if (wg == 0) asm volatile("bar.sync 5, 128;" ::: "memory");
    else asm volatile("bar.sync 6, 128;" ::: "memory");
}

// Whether v holds in every thread of warpgroup wg (a barrier of its four warps).
__device__ __forceinline__ bool wg_all(int wg, bool v) {
    uint32_t r;
    if (wg == 0)
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 5, 128, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(r)
            : "r"((uint32_t)v)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 6, 128, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(r)
            : "r"((uint32_t)v)
            : "memory");
    return r != 0;
}

struct __align__(16) InferSmem {
    uint4 w2c[kHid * kHid / 8];  // W2 (row = output unit n, K = input unit) in core matrices
    float4 l1[kHid];             // W1[u][0..2], b1[u]
    float4 l3[kHid];             // b2[u], W3[0][u], W3[1][u], 0
    float4 b3;                   // b3[0], b3[1], 0, 0
};
static_assert(sizeof(InferSmem) % 16 == 0, "the image is copied in 16-byte words");

// 16-byte word of element (row, k) of a K-major operand with `rgroups` row groups.
__device__ __forceinline__ int core_word(int row, int k, int rgroups) {
    return ((k >> 3) * rgroups + (row >> 3)) * 8 + (row & 7);
}

// The network as the inference kernel holds it in shared memory, built once per parameter
// change (mlp_pack_kernel) so that every CTA stages it with coalesced 16-byte loads.
__global__ void __launch_bounds__(256) mlp_pack_kernel(const float* __restrict__ wbf, InferSmem* __restrict__ img) {
    for (int i = threadIdx.x; i < kHid * kHid / 8; i += blockDim.x) {
        const int n = i / (kHid / 8), kg = i % (kHid / 8);
        const float* w = wbf + kOffW2 + n * kHid + kg * 8;
        img->w2c[core_word(n, kg * 8, kHid / 8)] =
            make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]), pack_bf16(w[6], w[7]));
    }
    for (int u = threadIdx.x; u < kHid; u += blockDim.x) {
        img->l1[u] = make_float4(wbf[kOffW1 + u * kIn], wbf[kOffW1 + u * kIn + 1], wbf[kOffW1 + u * kIn + 2],
                                 wbf[kOffB1 + u]);
        img->l3[u] = make_float4(wbf[kOffB2 + u], wbf[kOffW3 + u], wbf[kOffW3 + kHid + u], 0.f);
    }
    if (threadIdx.x == 0) img->b3 = make_float4(wbf[kOffB3], wbf[kOffB3 + 1], 0.f, 0.f);
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

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (row-direction) byte offsets, the fixed version field, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)(lead >> 4) << 16) |
           ((unsigned long long)(stride >> 4) << 32) | (1ull << 46);
}

// Tensor memory and barriers of an inference CTA: warp 0 allocates kTmemColsF columns,
// thread 0 sets up one mbarrier per warpgroup; the whole CTA then synchronises.
struct TcCta {
    uint32_t tmem;        // first column of the allocation (lane 0)
    uint32_t bar[2];      // shared addresses of the warpgroups' mbarriers
};
__device__ __forceinline__ TcCta tc_setup(uint32_t* slot, unsigned long long* bars) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                     "r"(kTmemColsF)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int w = 0; w < 2; ++w)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bars + w)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return TcCta{*slot, {smem_addr(bars), smem_addr(bars + 1)}};
}
// Every warp's tensor-memory reads done, then warp 0 frees the columns.
__device__ __forceinline__ void tc_teardown(const TcCta& t) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(kTmemColsF)
                     : "memory");
    }
}

// Waits for the phase with the given parity of an mbarrier; false after about 2^22 tries
// (far beyond the microseconds a 128 x 64 x 64 product takes).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Sixteen FP32 columns [c0, c0 + 16) of this thread's lane of tensor memory.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// The network's input for ybar y.
__device__ __forceinline__ void net_input(const MlpNorm& nm, const float (&y)[3], float (&x)[kIn]) {
#pragma unroll
    for (int c = 0; c < kIn; ++c)
        x[c] = nm.T[c * 3] * y[0] + nm.T[c * 3 + 1] * y[1] + nm.T[c * 3 + 2] * y[2] + nm.t0[c];
}

// The estimate from the network's outputs o (without b3) and ybar y.
__device__ __forceinline__ float2 net_estimate(const InferSmem& S, const MlpNorm& nm, const float (&y)[3], float o0,
                                               float o1) {
    const float2 bl = baseline(nm, least_squares(nm, y));
    return make_float2(fmaf(nm.osc0, o0 + S.b3.x, bl.x), fmaf(nm.osc1, o1 + S.b3.y, bl.y));
}

// Warpgroup wg's tiles tile0, tile0 + step, ... of 128 samples through the network (see
// above).  a: the warpgroup's A operand (128 x 64 BF16, 16 KB); tmem: its first column.
// With a route, the samples of untrusted cells are appended to its list (their estimates
// are still written; the exact posterior replaces them).  A product that does not complete
// leaves NaN estimates for its tile.
__device__ void wg_infer(const InferSmem& S, uint4* a, uint32_t tmem, uint32_t bar, int wg, const MlpNorm& nm,
                         const float* __restrict__ ybar, long n, long tile0, long step, float2* __restrict__ chat,
                         float2* __restrict__ chat_scaled, float scale, const MlpRoute& rt) {
    const int t = threadIdx.x & (kTileF - 1), lane = threadIdx.x & 31;
    // this thread's lane of tensor memory is its sample's row: warp (w % 4) reads lanes 32 (w % 4) ..
    const uint32_t trow = tmem + ((uint32_t)(t & ~31) << 16);
    const uint32_t a0 = smem_addr(a), b0 = smem_addr(S.w2c);
    constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                                ((uint32_t)(kTileF >> 4) << 24);  // F32 accumulator, BF16 A and B, K-major, 128 x 64
    constexpr uint32_t kLeadA = 128 * (kTileF / 8), kLeadB = 128 * (kHid / 8);
    const long ntile = (n + kTileF - 1) / kTileF;
    uint32_t parity = 0;
    for (long tile = tile0; tile < ntile; tile += step) {
        const long r = tile * kTileF + t;
        float y[3], x[kIn];
#pragma unroll
        for (int c = 0; c < 3; ++c) y[c] = r < n ? ybar[r * 3 + c] : 0.f;
        net_input(nm, y, x);
        // layer 1 into the A operand: row t, units 8 kg .. 8 kg + 7 in one 16-byte word
#pragma unroll 2
        for (int kg = 0; kg < kHid / 8; ++kg) {
            float h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 w = S.l1[kg * 8 + j];
                float z = w.w;
                z = fmaf(w.x, x[0], z);
                z = fmaf(w.y, x[1], z);
                z = fmaf(w.z, x[2], z);
                h[j] = gelu(z);
            }
            a[core_word(t, kg * 8, kTileF / 8)] =
                make_uint4(pack_bf16(h[0], h[1]), pack_bf16(h[2], h[3]), pack_bf16(h[4], h[5]), pack_bf16(h[6], h[7]));
        }
        // the operand's generic-proxy writes made visible to the tensor cores; the previous
        // tile's tensor-memory reads finished (all threads) before the next product
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        wg_barrier(wg);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < kHid / 16; ++s) {
                const unsigned long long da = smem_desc(a0 + s * 2 * kLeadA, kLeadA, 128);
                const unsigned long long db = smem_desc(b0 + s * 2 * kLeadB, kLeadB, 128);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(kIdesc), "r"((uint32_t)s)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
        }
        // one decision for the warpgroup (its threads give up on their own)
        const bool done = wg_all(wg, mbar_wait(bar, parity));
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // layer 2's bias, GELU and BF16 rounding, layer 3, from the accumulator row
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float z[16];
            tmem_ld16(trow + (uint32_t)c0, z);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 l = S.l3[c0 + j];
                const float h2 = bf(gelu(z[j] + l.x));
                o0 = fmaf(l.y, h2, o0);
                o1 = fmaf(l.z, h2, o1);
            }
        }
        const bool mine = r < n;
        float2 val = net_estimate(S, nm, y, o0, o1);
        if (!done) val = make_float2(NAN, NAN);
        if (rt.trust) {
            // warp-aggregated append of the untrusted samples
            const bool out = mine && !trusted(rt, least_squares(nm, y));
            const unsigned m = __ballot_sync(0xffffffffu, out);
            if (m) {
                unsigned base = 0;
                if (lane == __ffs(m) - 1) base = atomicAdd(rt.count, (unsigned)__popc(m));
                base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
                const unsigned at = base + __popc(m & ((1u << lane) - 1u));
                if (out && at < (unsigned long)n) rt.list[at] = (int)r;  // at most n are ever listed
            }
        }
        if (mine) {
            chat[r] = val;
            if (chat_scaled) chat_scaled[r] = make_float2(scale * val.x, scale * val.y);
        }
        if (!done) break;  // the product never completed: leave the rest to the check
    }
}

// One sample's estimate in one warp on the FP32 pipes, for the sampled check: lane l holds
// units l and l + 32 of each layer.  The same arithmetic as wg_infer (BF16 h1 and h2, FP32
// sums) in another order of additions.
__device__ float2 warp_infer_one(const InferSmem& S, const MlpNorm& nm, const float* __restrict__ ybar, long p,
                                 int lane) {
    float y[3], x[kIn];
#pragma unroll
    for (int c = 0; c < 3; ++c) y[c] = ybar[p * 3 + c];
    net_input(nm, y, x);
    float h1[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float4 w = S.l1[lane + 32 * i];
        float z = w.w;
        z = fmaf(w.x, x[0], z);
        z = fmaf(w.y, x[1], z);
        z = fmaf(w.z, x[2], z);
        h1[i] = bf(gelu(z));
    }
    const unsigned short* w2 = reinterpret_cast<const unsigned short*>(S.w2c);
    float z2[2] = {0.f, 0.f};
    for (int k = 0; k < kHid; ++k) {
        const float hk = __shfl_sync(0xffffffffu, h1[k >> 5], k & 31);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int u = lane + 32 * i;
            const float w = __uint_as_float((unsigned)w2[core_word(u, k, kHid / 8) * 8 + (k & 7)] << 16);
            z2[i] = fmaf(w, hk, z2[i]);
        }
    }
    float o0 = 0.f, o1 = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float4 l = S.l3[lane + 32 * i];
        const float h2 = bf(gelu(z2[i] + l.x));
        o0 = fmaf(l.y, h2, o0);
        o1 = fmaf(l.z, h2, o1);
    }
    return net_estimate(S, nm, y, warp_sum(o0), warp_sum(o1));
}

__global__ void __launch_bounds__(32 * kWarpsF) mlp_forward_kernel(const InferSmem* __restrict__ img, MlpNorm nm,
                                                                   const float* __restrict__ ybar, long n,
                                                                   float2* __restrict__ chat) {
    __shared__ InferSmem S;
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t slot;
    extern __shared__ __align__(1024) uint4 tc_a[];
    const TcCta tc = tc_setup(&slot, bars);
    stage_image(S, img);
    const int wg = threadIdx.x >> 7;
    wg_infer(S, tc_a + wg * (kTileF * kHid / 8), tc.tmem + 64u * wg, tc.bar[wg], wg, nm, ybar, n,
             (long)blockIdx.x * 2 + wg, (long)gridDim.x * 2, chat, nullptr, 0.f, MlpRoute{});
    tc_teardown(tc);
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
// pixel's exact posterior mean (warp_posterior_mean) while the odd warp runs the pixel
// through the network on the FP32 pipes (warp_infer_one); then err[k] = the larger of
// the two axes' errors relative to the box extents (NaN if either is).  The last check
// CTA to arrive adds the errors in a fixed order and leaves the decision in sync[2]
// (sync[1] counts the failed frames, sync[0] is the arrival counter).  The remaining CTAs
// run inference on the tensor cores as mlp_forward_kernel and, if chat_scaled is set, also
// write the estimates times scale there.
template <int CPL>
__global__ void __launch_bounds__(32 * kWarpsF, 4)
    mlp_forward_check_kernel(const InferSmem* __restrict__ img, MlpNorm nm, const float* __restrict__ ybar, long n,
                             float2* __restrict__ chat, float2* __restrict__ chat_scaled, float scale,
                             BayesParams bp, const BayesRec* __restrict__ recs, MlpCheck ck, MlpRoute rt) {
    __shared__ InferSmem S;
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t slot;
    extern __shared__ __align__(1024) uint4 tc_a[];
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
        const TcCta tc = tc_setup(&slot, bars);
        const int wg = threadIdx.x >> 7;
        const long nblk = (long)gridDim.x - ck.nctas;
        wg_infer(S, tc_a + wg * (kTileF * kHid / 8), tc.tmem + 64u * wg, tc.bar[wg], wg, nm, ybar, n,
                 ((long)blockIdx.x - ck.nctas) * 2 + wg, nblk * 2, chat, chat_scaled, scale, rt);
        tc_teardown(tc);
        return;
    }
    const int pair = warp >> 1;
    for (int k0 = blockIdx.x * kMlpCheckPerCta; k0 < ck.nsample; k0 += ck.nctas * kMlpCheckPerCta) {
        const int k = k0 + pair;
        const bool on = k < ck.nsample;  // the same for both warps of the pair
        const long p = on ? sample_pixel(ck.seed, k, n) : 0;
        float2 c = make_float2(0.f, 0.f);
        if (on && (warp & 1)) {
            const float2 v = warp_infer_one(S, nm, ybar, p, lane);
            if (lane == 0) est[pair] = v;
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

// Dynamic shared memory of the inference kernels (the warpgroups' A operands), and a check
// that no more CTAs fit on an SM than its 512 tensor-memory columns serve at once (a CTA
// beyond them would wait in its allocation for another CTA to finish).
template <typename K>
cudaError_t tc_prepare(K kernel) {
    cudaError_t e = set_smem_attr(kernel, kTcSmemBytes);
    int resident = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kernel, 32 * kWarpsF, kTcSmemBytes);
    if (e == cudaSuccess && resident * kTmemColsF > 512) e = cudaErrorInvalidConfiguration;
    return e;
}

// Inference CTAs for n samples: two 128-sample tiles per CTA while that fits, at most
// four CTAs per SM.
inline long tc_blocks(long n, int sms) {
    const long tiles = (n + kTileF - 1) / kTileF;
    long blocks = (tiles + 1) / 2;
    if (blocks > 4L * sms) blocks = 4L * sms;
    return blocks < 1 ? 1 : blocks;
}

cudaError_t launch_mlp_forward(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat, bool pdl,
                               cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = tc_prepare(mlp_forward_kernel);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tc_blocks(n, sms));
    cfg.blockDim = dim3(32 * kWarpsF);
    cfg.dynamicSmemBytes = kTcSmemBytes;
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
    cudaError_t e = tc_prepare(mlp_forward_check_kernel<CPL>);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32 * kWarpsF);
    cfg.dynamicSmemBytes = kTcSmemBytes;
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
    const long blocks = tc_blocks(n, sms) + ck.nctas;
#define HB_FC_ARGS img, nm, ybar, n, chat, chat_scaled, scale, bp, rec, ck, rt, (unsigned)blocks, pdl, s
    if (bp.n1 <= 32) return launch_forward_check_cpl<1>(HB_FC_ARGS);
    if (bp.n1 <= 64) return launch_forward_check_cpl<2>(HB_FC_ARGS);
    if (bp.n1 <= 128) return launch_forward_check_cpl<4>(HB_FC_ARGS);
    return launch_forward_check_cpl<8>(HB_FC_ARGS);
#undef HB_FC_ARGS
}

}  // namespace hb
