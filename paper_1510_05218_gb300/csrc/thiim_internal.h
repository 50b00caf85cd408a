// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "thiim_sweep.cuh"

namespace thiim {

// Sweep tile: TX x TY cells per CTA (TX fixed at 32 in the shipped build; the
// macros let a build try other shapes), NT threads, MINB resident CTAs per SM
// requested from the register allocator (0 = no request).
#ifndef THIIM_SWEEP_TY
#define THIIM_SWEEP_TY 8
#endif
#ifndef THIIM_SWEEP_NT
#define THIIM_SWEEP_NT 256
#endif
#ifndef THIIM_SWEEP_MINB
#define THIIM_SWEEP_MINB 0
#endif
#ifndef THIIM_SWEEP_TX
#define THIIM_SWEEP_TX 32
#endif
#ifndef THIIM_SWEEP_PAIR_TX
#define THIIM_SWEEP_PAIR_TX 64
#endif
#ifndef THIIM_SWEEP_PAIR_TY
#define THIIM_SWEEP_PAIR_TY 4
#endif
// Integer-pipe binary64 operations of a new THIIM_C128 context.
#ifndef THIIM_FP64_INT_OPS_DEFAULT
#define THIIM_FP64_INT_OPS_DEFAULT 0u
#endif
// Tile height and threads of the two-iteration (temporally blocked) kernel;
// its tile is SWEEP_TX wide like the single-iteration kernel's.
#ifndef THIIM_SWEEP2_TY
#define THIIM_SWEEP2_TY 8
#endif
#ifndef THIIM_SWEEP2_NT
#define THIIM_SWEEP2_NT 512
#endif
constexpr int SWEEP2_TY = THIIM_SWEEP2_TY;
constexpr int SWEEP2_NT = THIIM_SWEEP2_NT;
constexpr int SWEEP_TX = THIIM_SWEEP_TX;
constexpr int SWEEP_TY = THIIM_SWEEP_TY;
constexpr int SWEEP_NT = THIIM_SWEEP_NT;
constexpr int SWEEP_MINB = THIIM_SWEEP_MINB;
constexpr int SWEEP_PAIR_TX = THIIM_SWEEP_PAIR_TX;
constexpr int SWEEP_PAIR_TY = THIIM_SWEEP_PAIR_TY;

// Tile of each arithmetic policy and the resident CTAs per SM its kernels ask
// of the register allocator.  The FP32-pair sweeps use 64 x 4: their 1 KB rows
// per array and CTA measured 3.5 % faster at 512^3 than 32 x 8.  The FP64
// sweeps of thiim_iterate use 32 x 16 at 2 CTAs per SM (128 registers, the
// 113 KB of shared memory allow two): the halo recomputed per cell shrinks
// (FP64 instructions per cell 146 -> ~140, the FP64 pipe being the bound),
// 3616 vs 3530 MLUP/s at 512^3; 32 x 16 with 80 registers spilled and was
// slower (3413).  complex64 is fastest at 32 x 8.  Host code picks the same
// shape by precision (tiles_x / tiles_y).
#ifndef THIIM_SWEEP_F64_TY
#define THIIM_SWEEP_F64_TY 16
#endif
// Smallest grid (cells) whose FP64 sweep runs on the tall tile: below it the
// 32 x 8 tile fills the GPU better (grid sweep: 32 x 8 faster at 64^3 ..
// 192^3, 32 x 16 from 256^3 on).  Every FP64 sweep variant (plain, material
// table, integer pipe) follows the same rule, so that they stay bit-identical
// down to the per-CTA residual partials.
#ifndef THIIM_F64_TALL_MIN_CELLS
#define THIIM_F64_TALL_MIN_CELLS (1ull << 23)
#endif
template <typename A>
struct Tile { static constexpr int TX = SWEEP_TX, TY = SWEEP_TY, MINB = A::min_blocks; };
template <int I, int O>
struct Tile<PairArith<I, O>> { static constexpr int TX = SWEEP_PAIR_TX, TY = SWEEP_PAIR_TY, MINB = 2; };
template <>
struct Tile<Native<double>> { static constexpr int TX = SWEEP_TX, TY = THIIM_SWEEP_F64_TY, MINB = 2; };
template <int OFF>
struct Tile<Fp64Int<OFF>> { static constexpr int TX = SWEEP_TX, TY = THIIM_SWEEP_F64_TY, MINB = 2; };
static_assert(SWEEP_PAIR_TX * SWEEP_PAIR_TY <= 2 * SWEEP_NT, "pair tile too large for the CTA");

// Enqueue one fused iteration; grid = (tiles_x * tiles_y, chunks) in the
// policy's Tile (launch_sweep_f64_t8: FP64 on 32 x 8 tiles, for callers with
// their own 32 x 8 tiling).
cudaError_t launch_sweep_f64(const SweepArgs &a, dim3 grid, cudaStream_t s);
cudaError_t launch_sweep_f64_t8(const SweepArgs &a, dim3 grid, cudaStream_t s);
cudaError_t launch_sweep_f32(const SweepArgs &a, dim3 grid, cudaStream_t s);
// The FP64 sweep with additions (offload = 1) or additions and the leading
// products (offload = 3) on the integer pipe; bit-identical results.
cudaError_t launch_sweep_f64_int(const SweepArgs &a, dim3 grid, cudaStream_t s, int offload, bool tall);
// FP32-pair arithmetic on complex128 data: fields read as complex128
// (in_pairs = false) or float4 pairs, written likewise; coefficients are
// float4 pairs (see split_coeffs).
cudaError_t launch_sweep_pair(const SweepArgs &a, dim3 grid, cudaStream_t s, bool in_pairs, bool out_pairs);

// The same sweeps reading coefficients from the (material, plane) table
// (a.mat, a.table); pair coefficients are float4 pairs of the table.
cudaError_t launch_sweep_f64_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s, bool tall);
cudaError_t launch_sweep_f32_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s);
cudaError_t launch_sweep_pair_tbl(const SweepArgs &a, dim3 grid, cudaStream_t s, bool in_pairs, bool out_pairs);

// Defect-correction sweeps: FP64 defect r = F(x) - x written as complex64,
// and the complex64 correction iteration delta <- M delta + r (a.xsrc = r).
cudaError_t launch_defect_f64(const SweepArgs &a, dim3 grid, cudaStream_t s);
cudaError_t launch_correct_f32(const SweepArgs &a, dim3 grid, cudaStream_t s);

// Two iterations per launch (temporal blocking), complex64 only; grid
// (tiles_x * ceil(ny / SWEEP2_TY), chunks), partials as the single sweep.
cudaError_t launch_sweep2_f32(const SweepArgs &a, dim3 grid, cudaStream_t s);

// Split n complex128 values of each of `count` arrays into float4 pairs.
cudaError_t split_coeffs(const void *const *src, void *const *dst, int count, size_t n, cudaStream_t s);

}  // namespace thiim
