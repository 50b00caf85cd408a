// FP32-pair sweep instantiations that read float4-pair fields.
#include "thiim_internal.h"

namespace thiim {

cudaError_t launch_sweep_pair_in_c128(const SweepArgs &a, dim3 grid, cudaStream_t s, bool out_pairs);

cudaError_t launch_sweep_pair(const SweepArgs &a, dim3 grid, cudaStream_t s, bool in_pairs, bool out_pairs) {
    if (!in_pairs) return launch_sweep_pair_in_c128(a, grid, s, out_pairs);
    if (out_pairs)
        sweep_kernel<PairArith<1, 1>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    else
        sweep_kernel<PairArith<1, 0>, SWEEP_PAIR_TX, SWEEP_PAIR_TY, SWEEP_NT, SWEEP_MINB><<<grid, SWEEP_NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace thiim
