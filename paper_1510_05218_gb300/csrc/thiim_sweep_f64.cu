// FP64 (complex128) instantiation of the fused sweep.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_f64(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    typedef Tile<Native<double>> T;
    sweep_kernel<Native<double>, T::TX, T::TY, SWEEP_NT, T::MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_defect_f64(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep_kernel<Native<double>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB, SWEEP_DEFECT><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim
