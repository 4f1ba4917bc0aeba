// FP64 pipe throughput micro-benchmark: the roofline denominator of the
// FP64-bound stencil (the GPU's FP64 rate is far below its HBM rate per
// byte of this path).  Each thread runs 8 independent dependency chains of
// one FP64 instruction kind; the grid covers every SM several times.
#include <cuda_runtime.h>

#include "adjamr.h"

namespace {

template <int KIND>
__global__ void k_fp64(double *out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (double)(threadIdx.x + k) * 1e-7;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if constexpr (KIND == 0) x[k] = fma(x[k], a, b);
            else if constexpr (KIND == 1) x[k] = x[k] + b;
            else x[k] = x[k] * a;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

}  // namespace

extern "C" adjamr_status adjamr_fp64_peak(int kind, int iters, double *flops_per_s, double *ms_out)
{
    if (!flops_per_s || kind < 0 || kind > 2 || iters < 1) return ADJAMR_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADJAMR_ECUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return ADJAMR_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = nsm * 8;
    auto launch = [&]() {
        if (kind == 0) k_fp64<0><<<blocks, threads>>>(d, iters, 0.999999, 1e-9);
        else if (kind == 1) k_fp64<1><<<blocks, threads>>>(d, iters, 0.999999, 1e-9);
        else k_fp64<2><<<blocks, threads>>>(d, iters, 0.999999, 1e-9);
    };
    launch();  // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (err != cudaSuccess || ms <= 0.f) return ADJAMR_ECUDA;
    double ops = (double)blocks * threads * 8.0 * iters * (kind == 0 ? 2.0 : 1.0);
    *flops_per_s = ops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return ADJAMR_OK;
}
