// FP64 fused multiply-add throughput probe: the roofline denominator of the
// FP64 numeric kernels.  Eight independent register chains per thread, enough
// resident warps to fill every SM; the result is never stored unless it hits
// an impossible value, so the loop cannot be removed.
#include <cstdio>

#include "kernels.cuh"
#include "../../include/hylu.h"

namespace hylu {

namespace {
__global__ void dfma_probe(double* sink, int iters) {
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
    double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
    const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == -1.0) sink[blockIdx.x] = s;
}
}  // namespace

int measure_fp64_peak(double* gflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HYLU_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 4, threads = 256, iters = 4096;
    double* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(double) * blocks) != cudaSuccess) return HYLU_ERR_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dfma_probe<<<blocks, threads, 0, st>>>(sink, 64);
    count_launch();
    cudaEventRecord(e0, st);
    dfma_probe<<<blocks, threads, 0, st>>>(sink, iters);
    count_launch();
    cudaEventRecord(e1, st);
    int rc = HYLU_OK;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = HYLU_ERR_CUDA;
    else *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) * 1e-9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}

}  // namespace hylu
