// Weighted sum for callers that cannot allocate device memory.
//
// Same arithmetic as the functional J of adjamr_integrate_functional: terms
// weight*(q[k]*w[k]) summed by the fixed pairwise tree.  The only memory it
// needs beyond the caller's inputs and output is the term array of the
// tree, which lives here in a file-scope device array instead of being
// allocated per call.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

// Scratch for the terms of the pairwise tree: ADJAMR_NOALLOC_MAX_TERMS
// doubles (8 MiB), held by every GPU that loads the library until exit.
__device__ __align__(256) double g_sum_scratch[ADJAMR_NOALLOC_MAX_TERMS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_dev[kMaxDevices] = {};

// Device address of the scratch array on the current device (the name
// g_sum_scratch is only a host-side stand-in).  Looked up afresh on every
// call whose stream is not being captured -- after a device reset or a
// re-created primary context the array has a new address -- and remembered
// per device for calls made during a stream capture, when the lookup is not
// made (the first call on a device must therefore come before any capture).
cudaError_t scratch_address(cudaStream_t s, double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // treat an unanswerable query as a capture
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sum_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<double *>(p);
    } else if (!g_scratch_dev[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

__global__ void k_weighted_terms(const double *__restrict__ q, const double *__restrict__ w, long long n,
                                 double weight, double *terms)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) terms[t] = weight * (q[t] * w[t]);
}

}  // namespace

extern "C" adjamr_status adjamr_weighted_sum_noalloc(const double *q, const double *w, long long n, double weight,
                                                     double *out, void *stream)
{
    if (n > ADJAMR_NOALLOC_MAX_TERMS) return ADJAMR_EBUDGET;
    if (n < 0 || !out || (n > 0 && (!q || !w))) return ADJAMR_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *terms = nullptr;
    const cudaError_t ea = scratch_address(s, &terms);
    if (ea == cudaErrorStreamCaptureUnsupported) return ADJAMR_ESTATE;  // first call on this device under capture
    if (ea != cudaSuccess) return ADJAMR_ECUDA;
    if (n > 0) {
        const int threads = 256;
        k_weighted_terms<<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(q, w, n, weight, terms);
        if (cudaGetLastError() != cudaSuccess) return ADJAMR_ECUDA;
    }
    // every term the tree reads was written above in this call, so nothing in
    // the scratch has to be cleared first
    if (adjamr::launch_pairwise(terms, n, out, s) != cudaSuccess) return ADJAMR_ECUDA;
    return ADJAMR_OK;
}
