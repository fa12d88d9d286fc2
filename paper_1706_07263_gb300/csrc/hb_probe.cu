// hb_probe.cu -- measurement of the device's MUFU ex2 throughput, the denominator of the
// grid posterior's roofline (one ex2 per evaluated grid node).  Not part of the method.
//
// A throughput kernel fills every SM with independent ex2 chains (8 per thread, one FP32
// multiply between successive ex2 of a chain, so the values stay finite: x -> 2^x / 2
// converges to 1).  With 2 issued instructions per ex2 the issue slots (1 per clock per
// scheduler) allow twice the MUFU rate of 8 lanes per clock per scheduler, so the MUFU
// pipe is what limits the loop.  Each CTA reads the SM's cycle counter around the loop;
// the rate in ex2 per clock per SM follows from the CTAs resident on an SM together,
// independent of the clock frequency.
#include "hb.h"

#include <cuda_runtime.h>

#include <vector>

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) ex2_probe_kernel(int iters, float* sink, long long* cycles) {
    float x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = 0.5f + 0.0625f * k + 1e-6f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) {
            float y;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[k]));
            x[k] = 0.5f * y;
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += x[k];
    if (s == -1.f) sink[threadIdx.x] = s;  // never true: keeps the loop live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" hb_status hb_measure_ex2_rate(double* ex2_per_clock_per_sm, int* sm_count) {
    if (!ex2_per_clock_per_sm || !sm_count) return HB_ERR_ARG;
    int dev = 0, sms = 0, resident = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, ex2_probe_kernel, kProbeThreads, 0) != cudaSuccess ||
        sms < 1 || resident < 1) {
        cudaGetLastError();
        return HB_ERR_CUDA;
    }
    const int blocks = sms * resident;  // one wave: every SM holds `resident` CTAs at once
    const int iters = 4096;
    float* sink = nullptr;
    long long* cycles = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * kProbeThreads) != cudaSuccess ||
        cudaMalloc(&cycles, sizeof(long long) * blocks) != cudaSuccess) {
        cudaFree(sink);
        cudaGetLastError();
        return HB_ERR_OOM;
    }
    hb_status st = HB_OK;
    std::vector<long long> c(blocks);
    for (int rep = 0; rep < 2 && st == HB_OK; ++rep) {  // the first run warms up the clocks
        ex2_probe_kernel<<<blocks, kProbeThreads>>>(iters, sink, cycles);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(c.data(), cycles, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = HB_ERR_CUDA;
    }
    cudaFree(sink);
    cudaFree(cycles);
    if (st != HB_OK) {
        cudaGetLastError();
        return st;
    }
    double mean = 0.0;
    for (long long v : c) mean += (double)v;
    mean /= blocks;
    const double per_cta = (double)kProbeThreads * kProbeChains * iters;
    *ex2_per_clock_per_sm = mean > 0.0 ? resident * per_cta / mean : 0.0;
    *sm_count = sms;
    return HB_OK;
}
