// FP32-pair sweep instantiations that read complex128 fields, and the
// coefficient splitter.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_pair_in_c128(const SweepArgs &a, dim3 grid, cudaStream_t s, bool out_pairs) {
    if (out_pairs)
        sweep_kernel<PairArith<0, 1>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    else
        sweep_kernel<PairArith<0, 0>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

struct SplitArgs {
    const double2 *src[28];
    float4 *dst[28];
};

// hi = the double rounded to float, lo = the remainder rounded to float.
__global__ void split_kernel(const SplitArgs a, size_t n) {
    const double2 *in = a.src[blockIdx.y];
    float4 *out = a.dst[blockIdx.y];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = in[i];
        const fpair r = split_double(v.x), m = split_double(v.y);
        out[i] = make_float4(r.h, r.l, m.h, m.l);
    }
}

cudaError_t split_coeffs(const void *const *src, void *const *dst, int count, size_t n, cudaStream_t s) {
    if (count < 1 || count > 28) return cudaErrorInvalidValue;
    SplitArgs a;
    for (int i = 0; i < count; ++i) {
        a.src[i] = (const double2 *)src[i];
        a.dst[i] = (float4 *)dst[i];
    }
    size_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    split_kernel<<<dim3((unsigned)blocks, (unsigned)count), 256, 0, s>>>(a, n);
    return cudaGetLastError();
}

}  // namespace thiim
