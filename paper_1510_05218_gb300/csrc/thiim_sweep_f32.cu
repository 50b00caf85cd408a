// FP32 (complex64) instantiation of the fused sweep.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_f32(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep_kernel<Native<float>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_correct_f32(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep_kernel<Native<float>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB, SWEEP_CORRECT><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim
