// complex64 instantiation of the two-iteration (temporally blocked) sweep.
#include "thiim_internal.h"
#include "thiim_sweep2.cuh"

namespace thiim {

cudaError_t launch_sweep2_f32(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep2_kernel<Native<float>, SWEEP_TX, SWEEP2_TY, SWEEP2_NT><<<grid, SWEEP2_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim
