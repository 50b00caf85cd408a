"""Footprint / code-balance models and the autotuner of the sweep.

The paper prunes its auto-tuner's search with a cache-block-size model
(Eq. 11) and predicts memory traffic with code-balance models (Eqs. 8, 9,
12) and a bottleneck model (Eq. 10), Sec. III.  The same reasoning, written
for the GPU kernels here:

* ``cache_block_bytes`` / ``code_balance_diamond`` / ``bottleneck_mlups`` /
  ``code_balance_naive`` / ``code_balance_spatial`` are the paper's models
  as printed (their worked numbers are unit-tested).
* ``gpu_footprint`` gives, for a launch configuration (iterations per launch,
  z planes per CTA), the shared memory one CTA needs and the data a launch
  must find again in L2; ``gpu_code_balance`` the DRAM bytes per cell and
  iteration including the halo the tiles re-read (32 x 8 cells for
  complex64, 32 x 16 for FP64 on large grids, 64 x 4 for the FP32-pair sweeps).  A candidate is
  admitted if its shared memory fits a CTA, its L2 set stays within half of
  L2 (the paper's "half the cache is usable for tile data" rule, Sec. III-C)
  and its grid fills the resident slots; the library default is always a
  candidate.
* ``autotune`` times the admitted candidates on the caller's problem with
  the real kernels (thiim_set_tuning + thiim_iterate) and keeps the fastest;
  the caller's fields are restored afterwards.
"""
from __future__ import annotations

import math

# ---- the paper's models (Sec. III) -------------------------------------------------


def code_balance_naive(word_bytes: int = 8) -> int:
    """Eq. 8: 4 * (18 + 12 + 12) words per LUP (double precision words)."""
    return 4 * (18 + 12 + 12) * word_bytes


def code_balance_spatial(word_bytes: int = 8) -> int:
    """Eq. 9: the four z-shift loops save 4 words each once two layers fit in cache."""
    return 4 * ((18 - 4) + 12 + 12) * word_bytes


def bottleneck_mlups(bandwidth_gbs: float, bytes_per_lup: float) -> float:
    """Eq. 10: P_mem = b_S / B_C."""
    return bandwidth_gbs * 1e9 / bytes_per_lup / 1e6


def cache_block_bytes(n_x: int, d_w: int, b_z: int) -> float:
    """Eq. 11: C_s = 16 N_x [40 (D_w^2/2 + D_w (B_Z - 1)) + 12 (D_w + W_w)], W_w = D_w + B_Z - 1."""
    w_w = d_w + b_z - 1
    return 16.0 * n_x * (40.0 * (d_w * d_w / 2.0 + d_w * (b_z - 1)) + 12.0 * (d_w + w_w))


def code_balance_diamond(d_w: int) -> float:
    """Eq. 12: B_C = 16 [6 (2 D_w - 1) + (40 D_w + 12)] / (D_w^2 / 2) bytes per LUP."""
    return 16.0 * (6 * (2 * d_w - 1) + (40 * d_w + 12)) / (d_w * d_w / 2.0)


# ---- the same reasoning for the GPU kernels -----------------------------------------

TX, TY = 32, 8                        # cells of one CTA's column (complex128, complex64)
PAIR_TX, PAIR_TY = 64, 4              # the FP32-pair sweeps' column
SMEM_PER_SM = 228 * 1024              # bytes of shared memory per SM (GB300)
SMEM_PER_CTA = 227 * 1024


def elem_bytes(precision: int) -> int:
    return 8 if precision == 1 else 16


F64_TALL_MIN_CELLS = 1 << 23          # FP64 grids from here on run on 32 x 16 tiles


def tile(precision: int, cells=None):
    """(TX, TY) of the sweep kernels a precision runs (FP64: 32 x 16 on grids of
    at least F64_TALL_MIN_CELLS cells or when the size is not given, else 32 x 8)."""
    if precision == 0:
        return (TX, 2 * TY) if cells is None or cells >= F64_TALL_MIN_CELLS else (TX, TY)
    return (PAIR_TX, PAIR_TY) if precision == 2 else (TX, TY)


def gpu_footprint(precision: int, temporal: int, zchunk: int, ctas: int, n_sm: int, l2_bytes: int, cells=None):
    """Shared memory per CTA, resident CTAs and the L2 set that must be reused.

    Shared memory: the full-field sums (3 complex) of every plane the kernel
    keeps — two planes of the E region and two of the H region for one
    iteration; the two-iteration kernel keeps the grown regions of both
    iterations plus the intermediate iterate's splits.  The L2 set is the data
    a launch reads twice and counts on finding in L2: for the two-iteration
    kernel, the coefficients the second iteration re-reads one to two plane
    steps after the first (2 planes x 28 arrays of the H region per resident
    CTA).  The single-iteration kernel relies on L2 only for halo rows and
    has no such requirement.  A candidate fits if its shared memory fits a
    CTA, its L2 set is at most half of L2 (the paper's rule for tile data,
    Sec. III-C) and the grid has at least one CTA per resident slot.
    """
    b = elem_bytes(precision)
    tx, ty = tile(precision, cells)
    if temporal == 1:
        smem = b * 3 * 2 * ((tx + 2) * (ty + 2) + (tx + 1) * (ty + 1))
        per_sm = 5 if precision == 1 else (3 if (precision == 0 and ty == TY) else 2)
        l2_set = 0
    else:
        smem = b * (3 * 2 * ((tx + 4) * (ty + 4) + (tx + 3) * (ty + 3) + (tx + 2) * (ty + 2) + (tx + 1) * (ty + 1))
                    + 6 * 2 * ((tx + 1) * (ty + 1) + tx * ty))
        per_sm = 1
    per_sm = max(1, min(per_sm, SMEM_PER_SM // max(1, smem)))
    resident = per_sm * n_sm
    if temporal != 1:
        l2_set = min(resident, ctas) * 2 * 28 * b * (tx + 1) * (ty + 1)
    return {"smem_per_cta": smem, "ctas_per_sm": per_sm, "resident_ctas": resident, "l2_set": l2_set,
            "fits": smem <= SMEM_PER_CTA and l2_set <= l2_bytes // 2 and ctas >= resident}


def gpu_code_balance(precision: int, temporal: int, zchunk: int, cells=None) -> float:
    """DRAM bytes per cell and iteration if every halo cell is re-read from DRAM.

    One iteration reads 40 arrays (E on the (TX+2)(TY+2) region, H and the
    coefficients on (TX+1)(TY+1)) and writes 12 on the tile; a z chunk adds
    one plane of prologue and one of lookahead.  Two iterations per launch
    read x^0 on the grown regions once and write x^2 once, per two iterations.
    """
    b = elem_bytes(precision)
    TX, TY = tile(precision, cells)
    cells = TX * TY
    z = max(1, zchunk)
    if temporal == 1:
        rd = 6 * (TX + 2) * (TY + 2) + (6 + 14) * (TX + 1) * (TY + 1) + 14 * cells
        per_cell = (rd + 12 * cells) / cells
        return b * per_cell * (z + 2) / z
    rd = 6 * (TX + 4) * (TY + 4) + (6 + 14) * (TX + 3) * (TY + 3) + 14 * (TX + 2) * (TY + 2)
    per_cell = (rd + 12 * cells) / cells / 2.0
    return b * per_cell * (z + 3) / z


def candidates(precision: int, nz: int, tiles: int, n_sm: int, l2_bytes: int, cells=None):
    """(temporal, zchunk) pairs admitted by the footprint model, plus the default (1, 0)."""
    out = [(1, 0)]
    for temporal in ((1, 2) if precision == 1 else (1,)):
        for z in (16, 32, 64, 128, 256):
            if z > nz:
                continue
            fp = gpu_footprint(precision, temporal, z, tiles * math.ceil(nz / z), n_sm, l2_bytes, cells)
            if fp["fits"]:
                out.append((temporal, z))
    return out


def autotune(ctx, fields, nx, ny, nz, precision, iters=20, repeats=2, stream=None):
    """Time the admitted launch configurations on this problem; keep the fastest.

    `fields` are the 12 tensors registered with the context; they are restored
    after timing.  Returns (best (temporal, zchunk), {candidate: seconds}).
    """
    import torch

    from . import thiim as T

    props = torch.cuda.get_device_properties(fields[0].device)
    tx, ty = tile(precision, nx * ny * nz)
    tiles = math.ceil(nx / tx) * math.ceil(ny / ty)
    cands = candidates(precision, nz, tiles, props.multi_processor_count, props.L2_cache_size, nx * ny * nz)
    saved = [f.clone() for f in fields]
    times = {}
    try:
        for cand in cands:
            T.thiim_set_tuning(ctx, cand[0], cand[1])
            T.thiim_iterate(ctx, iters)          # warm-up
            torch.cuda.synchronize()
            best = math.inf
            for _ in range(repeats):
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                s = stream or torch.cuda.current_stream()
                t0.record(s)
                T.thiim_iterate(ctx, iters)
                t1.record(s)
                torch.cuda.synchronize()
                best = min(best, t0.elapsed_time(t1) / 1e3)
            times[cand] = best
    finally:
        for f, g in zip(fields, saved):
            f.copy_(g)
        torch.cuda.synchronize()
    choice = min(times, key=times.get) if times else (1, 0)
    T.thiim_set_tuning(ctx, choice[0], choice[1])
    return choice, times
