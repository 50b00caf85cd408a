// FP64 sweeps with part of the binary64 arithmetic on the integer pipe
// (Fp64Int, thiim_arith.cuh): results bit-identical to the FP64 sweep.
#include "thiim_internal.h"

namespace thiim {

template <int OFF>
static void launch_int(const SweepArgs &a, dim3 grid, cudaStream_t s, bool tall) {
    typedef Tile<Fp64Int<OFF>> T;
    if (tall)
        sweep_kernel<Fp64Int<OFF>, T::TX, T::TY, SWEEP_NT, T::MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    else
        sweep_kernel<Fp64Int<OFF>, SWEEP_TX, SWEEP_TY, SWEEP_NT, T::MINB><<<grid, SWEEP_NT, 0, s>>>(a);
}

cudaError_t launch_sweep_f64_int(const SweepArgs &a, dim3 grid, cudaStream_t s, int offload, bool tall) {
    if (offload == 1)
        launch_int<1>(a, grid, s, tall);
    else if (offload == 3)
        launch_int<3>(a, grid, s, tall);
    else if (offload == 4)
        launch_int<4>(a, grid, s, tall);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace thiim
