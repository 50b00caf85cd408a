// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "thiim_sweep.cuh"

namespace thiim {

// Sweep tile: TX x TY cells per CTA, NT threads.
constexpr int SWEEP_TX = 32;
constexpr int SWEEP_TY = 8;
constexpr int SWEEP_NT = 256;

// Enqueue one fused iteration; grid = (tiles_x * tiles_y, chunks).
cudaError_t launch_sweep_f64(const SweepArgs &a, dim3 grid, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepArgs &a, dim3 grid, cudaStream_t s);
// FP32-pair arithmetic on complex128 data: fields read as complex128
// (in_pairs = false) or float4 pairs, written likewise; coefficients are
// float4 pairs (see split_coeffs).
cudaError_t launch_sweep_pair(const SweepArgs &a, dim3 grid, cudaStream_t s, bool in_pairs, bool out_pairs);

// Split n complex128 values of each of `count` arrays into float4 pairs.
cudaError_t split_coeffs(const void *const *src, void *const *dst, int count, size_t n, cudaStream_t s);

}  // namespace thiim
