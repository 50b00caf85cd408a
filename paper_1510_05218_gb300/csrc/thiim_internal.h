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

}  // namespace thiim
