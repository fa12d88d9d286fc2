// hb_mlp.cuh -- shape, parameter layout and launch wrappers of the learned low-pass
// stand-in (internal to libhb).
#pragma once

#include <cuda_runtime.h>

#include "hb_common.cuh"

namespace hb {

constexpr int kIn = 3, kHid = 64, kOut = 2;
// FP32 master parameters, contiguous: W1[64][3], b1[64], W2[64][64] (row = output unit),
// b2[64], W3[2][64], b3[2]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kOut * kHid;
constexpr int kNParams = kOffB3 + kOut;  // 4546

// Input transform and the least-squares baseline the network corrects:
//   x = T ybar + t0   (rows 0, 1: least-squares concentrations mapped to [-4, 4] over the
//                      box; row 2: the part of ybar outside the range of A, in sigma_l units)
//   c = clip(A+ ybar, box) + osc * o   (osc = posterior standard deviation per axis)
struct MlpNorm {
    float T[9], t0[3];
    float Ap[6];             // pseudo-inverse of A, 2 x 3, row-major
    float lo0, hi0, lo1, hi1;
    float osc0, osc1;        // output scale
};

constexpr int kMlpTrainSamples = 64;  // samples per training CTA

size_t mlp_train_smem_bytes();
cudaError_t launch_mlp_train(const float* wbf, const MlpNorm& nm, const float* ybar, const float* target, long n,
                             int batch, unsigned seed, int step, int idx_direct, float* gpart, float* lpart,
                             cudaStream_t s);
// Sum the partial gradients of nblocks CTAs in order into grad (kNParams) and the loss
// into *loss (mean squared error); then, if lr > 0, one Adam step on the masters.
cudaError_t launch_mlp_adam(const float* gpart, const float* lpart, int nblocks, int batch, float* grad, float* loss,
                            float* master, float* m, float* v, float* wbf, float lr, float beta1, float beta2,
                            float eps, int t, cudaStream_t s);
// The inference kernel's shared-memory image of the network (mlp_image_bytes() bytes),
// packed from the BF16 parameters; to be rebuilt after every parameter change.
size_t mlp_image_bytes();
cudaError_t launch_mlp_pack(const float* wbf, void* img, cudaStream_t s);
// Inference for n samples from a packed image; pdl: launched as a programmatic dependent of
// the preceding kernel in the stream (the kernel waits for it before reading ybar).
cudaError_t launch_mlp_forward(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat, bool pdl,
                               cudaStream_t s);

// The learned stand-in's sampled check, run by extra CTAs of the inference launch: the
// exact posterior of nsample pseudo-randomly drawn pixels (seeded) against the network's
// estimate of them.  err[k] = the larger of |d c0| inv_ext0 and |d c1| inv_ext1 for the
// k-th drawn pixel (NaN if either is); the last check CTA to finish adds the errors in
// a fixed order and sets sync[2] = 1 when their mean exceeds tol or is NaN (then also
// sync[1] += 1), else 0; sync[0] is its arrival counter (zero before and after).
struct MlpCheck {
    int nsample;
    int nctas;  // check CTAs (set by the launch)
    unsigned seed;
    float inv_ext0, inv_ext1, tol;
    float* err;
    unsigned* sync;
};
// Inference for the n samples of a band (the rows of rec) and the sampled check of it in
// one launch; chat_scaled (optional) also receives the estimates times scale; pdl as for
// launch_mlp_forward.  nsample must be positive; n = 0 launches nothing.
cudaError_t launch_mlp_forward_check(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat,
                                     float2* chat_scaled, float scale, const BayesParams& bp, const BayesRec* rec,
                                     MlpCheck ck, bool pdl, cudaStream_t s);

}  // namespace hb
