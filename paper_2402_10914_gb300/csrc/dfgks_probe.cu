// dfgks_probe.cu -- FP64 FMA throughput probe: independent fused multiply-add chains, timed with
// CUDA events.  Used only to cross-check the FP64 roofline denominator of the solver kernels.
#include <cuda_runtime.h>
#include "../../include/dfgks.h"

namespace {

__global__ void k_dfma_chains(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
    double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
    for (int k = 0; k < iters; ++k) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live without a store per thread
}

}  // namespace

extern "C" DFGKS_API dfgks_status dfgks_probe_fp64(int iters, double* gflops, double* ms) {
    if (iters < 1 || !gflops) return DFGKS_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DFGKS_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DFGKS_ECUDA;
    double* out = nullptr;
    if (cudaMalloc((void**)&out, 65536 * sizeof(double)) != cudaSuccess) return DFGKS_ENOMEM;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_dfma_chains<<<blocks, threads>>>(out, 64, 0.999999, 1e-7);   // warm-up
    cudaEventRecord(e0);
    k_dfma_chains<<<blocks, threads>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return DFGKS_ECUDA;
    const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *gflops = flops / (t * 1e-3) / 1e9;
    if (ms) *ms = t;
    return DFGKS_OK;
}
