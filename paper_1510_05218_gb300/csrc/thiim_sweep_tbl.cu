// Instantiations of the fused sweep that read the coefficients from a
// (material, plane) table selected by a per-cell material id.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_f64_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s, bool tall) {
    typedef Tile<Native<double>> T;
    if (tall)
        sweep_kernel<Native<double>, T::TX, T::TY, SWEEP_NT, T::MINB, SWEEP_PLAIN, true><<<grid, SWEEP_NT, 0, s>>>(a);
    else
        sweep_kernel<Native<double>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s) {
    sweep_kernel<Native<float>, SWEEP_TX, SWEEP_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
        <<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_pair_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s, bool in_pairs, bool out_pairs) {
    if (!in_pairs && out_pairs)
        sweep_kernel<PairArith<0, 1>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else if (!in_pairs)
        sweep_kernel<PairArith<0, 0>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else if (out_pairs)
        sweep_kernel<PairArith<1, 1>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    else
        sweep_kernel<PairArith<1, 0>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB, SWEEP_PLAIN, true>
            <<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim
