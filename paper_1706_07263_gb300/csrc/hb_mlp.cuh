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

// Input transform and the baseline the network corrects:
//   x = T ybar + t0   (rows 0, 1: least-squares concentrations mapped to [-4, 4] over the
//                      box; row 2: the part of ybar outside the range of A, in sigma_l units)
//   c = b(ybar) + osc * o   (osc = posterior standard deviation per axis)
// b = c_ls + sum over the box's four edges e of lambda(d_e) v_e, c_ls = A+ ybar: the mean of
// the Gaussian N(c_ls, S), S = sigma_l^2 (A^T A)^-1, cut by the edge alone is c_ls +
// lambda(d_e) v_e, with d_e = (sgn_e c_ls[axis_e] - pos_e) / s_e its distance from the edge in
// standard deviations (positive inside), lambda(d) = phi(d) / Phi(d) = sqrt(2/pi) /
// erfcx(-d / sqrt 2), v_e = sgn_e S[:, axis_e] / s_e and s_e = sqrt(S[axis_e][axis_e]).
// Edges 0, 1: HbO2 >= lo0, HbO2 <= hi0; edges 2, 3: Hb >= lo1, Hb <= hi1.
struct MlpNorm {
    float T[9], t0[3];
    float Ap[6];             // pseudo-inverse of A, 2 x 3, row-major
    float lo0, hi0, lo1, hi1;
    float osc0, osc1;        // output scale
    float edge_sgn[4], edge_pos[4], edge_inv_s[4], edge_v0[4], edge_v1[4];
};

// Routing of the learned mode after a certification (hb_mlp_certify): a map of cells over
// the least-squares concentrations, 1 where the network was found within tolerance.  The
// low-pass pixels whose c_ls falls in a cell marked 0, or outside the map, are listed for
// the exact posterior.  trust = nullptr: every pixel takes the network.
struct MlpRoute {
    const unsigned char* trust = nullptr;  // k0 x k1 cells, row = HbO2 cell
    int k0 = 0, k1 = 0;
    float org0 = 0.f, org1 = 0.f;          // c_ls at the map's first corner
    float inv0 = 0.f, inv1 = 0.f;          // cells per uM
    int* list = nullptr;                   // listed pixel indices (capacity: the launch's pixels)
    unsigned* count = nullptr;             // how many are listed (zero before the launch)
    unsigned* next_count = nullptr;        // the next frame's counter, cleared by this launch
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
// k-th drawn pixel (NaN if either is; 0 for a pixel the route lists for the exact
// posterior); the last check CTA to finish sets sync[2] = 1 when the largest error
// (use_max) or the mean error (in a fixed order of additions) exceeds tol, or any is NaN
// (then also sync[1] += 1), else 0; sync[0] is its arrival counter (zero before and after).
struct MlpCheck {
    int nsample;
    int nctas;  // check CTAs (set by the launch)
    unsigned seed;
    float inv_ext0, inv_ext1, tol;
    int use_max;
    float* err;
    unsigned* sync;
};
// Inference for the n samples of a band (the rows of rec) and the sampled check of it in
// one launch; chat_scaled (optional) also receives the estimates times scale; pdl as for
// launch_mlp_forward.  nsample must be positive; n = 0 launches nothing.
// With rt.trust set, the pixels of untrusted cells are also listed in rt.list / rt.count.
cudaError_t launch_mlp_forward_check(const void* img, const MlpNorm& nm, const float* ybar, long n, float2* chat,
                                     float2* chat_scaled, float scale, const BayesParams& bp, const BayesRec* rec,
                                     MlpCheck ck, const MlpRoute& rt, bool pdl, cudaStream_t s);

}  // namespace hb
