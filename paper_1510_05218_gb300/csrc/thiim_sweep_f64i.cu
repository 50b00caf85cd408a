// FP64 sweeps with part of the binary64 arithmetic on the integer pipe
// (Fp64Int, thiim_arith.cuh): results bit-identical to the FP64 sweep.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_f64_int(const SweepArgs &a, dim3 grid, cudaStream_t s, int offload) {
    if (offload == 1)
        sweep_kernel<Fp64Int<1>, Tile<Fp64Int<1>>::TX, Tile<Fp64Int<1>>::TY, SWEEP_NT, Tile<Fp64Int<1>>::MINB>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else if (offload == 3)
        sweep_kernel<Fp64Int<3>, Tile<Fp64Int<3>>::TX, Tile<Fp64Int<3>>::TY, SWEEP_NT, Tile<Fp64Int<3>>::MINB>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else if (offload == 4)
        sweep_kernel<Fp64Int<4>, Tile<Fp64Int<4>>::TX, Tile<Fp64Int<4>>::TY, SWEEP_NT, Tile<Fp64Int<4>>::MINB>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace thiim
