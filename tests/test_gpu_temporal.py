"""Temporal blocking (two iterations per launch, complex64): results must be
bit-identical to single-iteration sweeps — each cell's arithmetic is the
same, only the CTA that computes it differs — for ragged grids, every
boundary mix including periodic z, small z chunks (chunk-boundary
recomputation) and odd iteration counts (a single sweep finishes).  The
residual of the last iteration must match too, and the result stays within
the complex64 bound of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields

pytestmark = pytest.mark.gpu

CASES = [((9, 13, 70), 3, 0), ((12, 17, 33), 7, 5), ((5, 8, 32), 0, 2), ((3, 1, 1), 7, 0),
         ((16, 9, 40), 4, 3), ((1, 5, 7), 3, 0), ((20, 24, 64), 3, 7)]


def _run(shape, bc, n, temporal, zchunk, seed=81):
    import paper_1510_05218_gb300 as p
    p.load_library()
    nz, ny, nx = shape
    f = random_fields(nx, ny, nz, seed=seed)
    c = random_coeffs(nx, ny, nz, seed=seed)
    fd, cd = to_dev(f, "complex64"), to_dev(c, "complex64")
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C64, bc)
    try:
        p.thiim_set_tuning(ctx, temporal, zchunk)
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, n)
        r = p.thiim_residual(ctx)
        return to_host(fd), r, f, c
    finally:
        p.thiim_destroy(ctx)


@pytest.mark.parametrize("shape,bc,zchunk", CASES)
@pytest.mark.parametrize("n", [2, 3, 4])
def test_two_iteration_blocking_is_bit_identical(shape, bc, zchunk, n):
    a, ra, _, _ = _run(shape, bc, n, 2, zchunk)
    b, rb, _, _ = _run(shape, bc, n, 1, zchunk)
    for s in range(12):
        assert np.array_equal(a[s], b[s]), s
    assert ra == rb or abs(ra - rb) <= 1e-12 * rb


def test_two_iteration_blocking_matches_oracle():
    shape, bc = (9, 13, 70), 3
    g, _, f, c = _run(shape, bc, 4, 2, 0)
    f32 = [x.astype(np.complex64).astype(np.complex128) for x in f]
    c32 = [x.astype(np.complex64).astype(np.complex128) for x in c]
    oracle.iterate(f32, c32, 4, bc=bc)
    for s in range(12):
        assert rel_l2(g[s], f32[s]) <= 4 * 16 * 2.0 ** -24 * 1.2, s


def test_tuning_rejects_blocking_outside_complex64():
    import paper_1510_05218_gb300 as p
    p.load_library()
    ctx = p.thiim_create(8, 8, 8, p.THIIM_C128, 3)
    try:
        with pytest.raises(p.ThiimError):
            p.thiim_set_tuning(ctx, 2, 0)
        with pytest.raises(p.ThiimError):
            p.thiim_set_tuning(ctx, 3, 0)
        p.thiim_set_tuning(ctx, 1, 4)
    finally:
        p.thiim_destroy(ctx)


def test_autotune_restores_fields_and_picks_a_candidate():
    import torch
    import paper_1510_05218_gb300 as p
    from paper_1510_05218_gb300 import tuning
    p.load_library()
    nz, ny, nx = 64, 64, 64
    f = random_fields(nx, ny, nz, seed=90)
    c = random_coeffs(nx, ny, nz, seed=90)
    fd, cd = to_dev(f, "complex64"), to_dev(c, "complex64")
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C64, 3)
    try:
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        choice, times = tuning.autotune(ctx, fd, nx, ny, nz, p.THIIM_C64, iters=4, repeats=1)
        assert choice in times and (1, 0) in times
        back = to_host(fd)
        for s in range(12):
            assert np.array_equal(back[s], f[s].astype(np.complex64).astype(np.complex128))
    finally:
        p.thiim_destroy(ctx)
    del torch
