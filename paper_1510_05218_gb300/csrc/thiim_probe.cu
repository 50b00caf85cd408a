// Throughput of the FP64 pipe, measured on the device the caller runs on.
//
// GB300 executes FP64 fused multiply-adds at a small fraction of its FP32
// rate, so an FP64 stencil can be bound by that pipe rather than by HBM.  The
// roofline of such a kernel needs the pipe's peak as its denominator; this
// measures it in the same process and at the same clocks as the kernel it is
// compared with.  Not a step of the paper's method.
#include <cuda_runtime.h>

#include "../../include/thiim.h"

namespace {

constexpr int PROBE_CHAINS = 8;     // independent FMA chains per thread
constexpr int PROBE_ITERS = 4096;   // FMAs per chain
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

__global__ void __launch_bounds__(PROBE_THREADS) dfma_probe(double *sink, double seed) {
    double acc[PROBE_CHAINS];
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) acc[i] = seed + 1e-3 * i + 1e-9 * threadIdx.x;
    const double m = 0.999999999, a = 1e-12;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < PROBE_CHAINS; ++i) acc[i] = fma(acc[i], m, a);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; ++i) s += acc[i];
    if (s == 12345.678) sink[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

}  // namespace

extern "C" int thiim_fp64_pipe_rate(void *cuda_stream, double *fma_per_s) {
    if (!fma_per_s) return THIIM_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
        return THIIM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = nsm * PROBE_BLOCKS_PER_SM;
    double *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = THIIM_OK;
    float best = 0.f;
    if (cudaMalloc(&sink, (size_t)blocks * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return THIIM_ERR_NOMEM; }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { st = THIIM_ERR_CUDA; goto done; }
    dfma_probe<<<blocks, PROBE_THREADS, 0, s>>>(sink, 1.0);   // warm-up
    for (int rep = 0; rep < 5; ++rep) {
        float ms = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = THIIM_ERR_CUDA; goto done; }
        dfma_probe<<<blocks, PROBE_THREADS, 0, s>>>(sink, 1.0 + rep);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) { st = THIIM_ERR_CUDA; goto done; }
        if (best == 0.f || ms < best) best = ms;
    }
    if (cudaGetLastError() != cudaSuccess || !(best > 0.f)) { st = THIIM_ERR_CUDA; goto done; }
    *fma_per_s = (double)blocks * PROBE_THREADS * PROBE_CHAINS * PROBE_ITERS / (best * 1e-3);
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}
