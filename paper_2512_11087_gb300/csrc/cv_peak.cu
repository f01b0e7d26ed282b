// Measured FP32 FMA issue peak of the device (cv_fp32_fma_peak): the denominator of the roofline of
// the ALU-bound kernels (complete clipping issues FP32 / INT32 lane instructions, one per lane and
// clock at most on every SM sub-partition).  A grid of 4 blocks per SM, each thread running 16
// independent FFMA chains whose operands are kernel arguments (nothing to fold), timed with events.
#include "cv_internal.cuh"

namespace {

constexpr int PK_CHAINS = 16;

__global__ void __launch_bounds__(256) k_fma_probe(int iters, float a, float b, int write, float* sink) {
    float f[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) f[c] = (float)(threadIdx.x + c) * 1e-3f;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) f[c] = fmaf(f[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += f[c];
    if (write) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never set: keeps the chains alive
}

}  // namespace

extern "C" cv_status cv_fp32_fma_peak(double* lane_fma_per_s, float* ms_out, void* stream) {
    if (!lane_fma_per_s) { cv_set_error("cv_fp32_fma_peak: null output"); return CV_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CV_CUDA(cudaGetDevice(&dev));
    CV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 4 * sms, threads = 256, iters = 4096;
    cudaEvent_t e0, e1;
    CV_CUDA(cudaEventCreate(&e0));
    CV_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    // a = 1 - 2^-24, b = 2^-20: the chains stay finite and never simplify
    for (int rep = 0; rep < 4; ++rep) {
        CV_CUDA(cudaEventRecord(e0, st));
        k_fma_probe<<<blocks, threads, 0, st>>>(iters, 0.99999994f, 9.5367431640625e-07f, 0, nullptr);
        CV_LAUNCH_CHECK("k_fma_probe");
        CV_CUDA(cudaEventRecord(e1, st));
        CV_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        CV_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best) best = ms;  // the first launch loads the module
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double fmas = (double)blocks * threads * iters * 8.0 * PK_CHAINS;
    *lane_fma_per_s = fmas / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return CV_OK;
}
