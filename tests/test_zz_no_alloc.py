"""thiim_step_noalloc: the iteration entry point for callers that cannot allocate.

Callers running under another framework's memory pool or allocator hooks, or
with all device memory reserved in advance, cannot let the library call
cudaMalloc.  thiim_step_noalloc runs one iteration between caller buffers and
keeps its reduction scratch in a fixed device array.  Here it is called twice
in a row through the C ABI and compared with the FP64 oracle and with
thiim_iterate (the allocating path) after one and two iterations, at the
tolerances the other parity tests use (1e-12 for complex128; the FP32 bound
of test_gpu_sweep for complex64).  Every buffer a kernel could touch is real
device memory.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import full_fields, rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields

pytestmark = pytest.mark.gpu


def _oracle(f0, co, n):
    """n oracle iterations and the relative full-field update of the last one."""
    f = [a.copy() for a in f0]
    prev = None
    for it in range(n):
        if it == n - 1:
            prev = full_fields(f)
        oracle.iterate(f, co, 1, bc=3)
    cur = full_fields(f)
    num = sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(cur, prev))
    den = sum(np.sum(np.abs(a) ** 2) for a in cur)
    return f, math.sqrt(num / den)


# (nz, ny, nx): ragged tiles in x and y with one z chunk; 4 tiles with 8 z chunks
SHAPES = [(11, 21, 75), (64, 16, 64)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_oracle_and_allocating_path_on_two_calls(precision, shape):
    import torch
    import paper_1510_05218_gb300 as p
    p.load_library()
    nz, ny, nx = shape
    dt = "complex128" if precision == 0 else "complex64"
    f0 = random_fields(nx, ny, nz, seed=31)
    c0 = random_coeffs(nx, ny, nz, seed=31)
    co = to_dev(c0, dt)
    a = to_dev(f0, dt)
    b = [torch.empty_like(t) for t in a]
    c = [torch.empty_like(t) for t in a]
    r1 = p.thiim_step_noalloc(nx, ny, nz, precision, 3, a, b, co)
    r2 = p.thiim_step_noalloc(nx, ny, nz, precision, 3, b, c, co)
    got1, got2 = to_host(b), to_host(c)

    # the FP64 oracle (on the complex64-rounded inputs for the complex64 path)
    if precision == 1:
        f0 = [x.astype(np.complex64).astype(np.complex128) for x in f0]
        c0 = [x.astype(np.complex64).astype(np.complex128) for x in c0]
    o1, q1o = _oracle(f0, c0, 1)
    o2, q2o = _oracle(f0, c0, 2)
    tol_f = 1e-12 if precision == 0 else 2 * 16 * 2.0 ** -24
    for s in range(12):
        assert rel_l2(got1[s], o1[s]) <= tol_f, (s, rel_l2(got1[s], o1[s]))
        assert rel_l2(got2[s], o2[s]) <= tol_f, (s, rel_l2(got2[s], o2[s]))
    tol_r = 1e-10 if precision == 0 else 1e-4
    assert abs(r1 - q1o) <= tol_r * q1o and abs(r2 - q2o) <= tol_r * q2o

    # the allocating path: same kernel and CTA layout, so agreement is tight
    ref = to_dev(f0, dt)
    ctx = p.thiim_create(nx, ny, nz, precision, 3)
    try:
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, ref)
        p.thiim_iterate(ctx, 1)
        want1 = to_host(ref)
        q1 = p.thiim_residual(ctx)
        p.thiim_iterate(ctx, 1)
        want2 = to_host(ref)
        q2 = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    for s in range(12):
        assert rel_l2(got1[s], want1[s]) <= 1e-12
        assert rel_l2(got2[s], want2[s]) <= 1e-12
    assert abs(r1 - q1) <= 1e-12 * q1 and abs(r2 - q2) <= 1e-12 * q2
    assert np.isfinite(r1) and r1 > 0


def test_noalloc_at_its_largest_grid_matches_the_allocating_path():
    """Exactly 16384 tiles of 32 x 8 (the scratch array's capacity), two planes:
    every CTA partial slot is used and the fixed-order reduction must cover all
    of them; the residual and fields equal thiim_iterate's (same CTA layout)."""
    import torch
    import paper_1510_05218_gb300 as p
    p.load_library()
    nx, ny, nz = 32 * 128, 8 * 128, 2
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    shape = (nz, ny, nx)

    def rnd(scale):
        return torch.complex(torch.randn(shape, generator=g, device="cuda", dtype=torch.float32),
                             torch.randn(shape, generator=g, device="cuda", dtype=torch.float32)) * scale

    co = [rnd(0.3) for _ in range(28)]
    a = [rnd(1.0) for _ in range(12)]
    b = [torch.empty_like(t) for t in a]
    r = p.thiim_step_noalloc(nx, ny, nz, 1, 3, a, b, co)
    ref = [t.clone() for t in a]
    ctx = p.thiim_create(nx, ny, nz, 1, 3)
    try:
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, ref)
        p.thiim_iterate(ctx, 1)
        q = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    torch.cuda.synchronize()
    assert r == q and np.isfinite(r) and r > 0
    for s in range(12):
        assert torch.equal(b[s], ref[s])


def test_noalloc_rejects_grids_beyond_its_scratch():
    """16512 tiles > 16384: rejected before any launch.  The arrays are real
    device buffers sized for the grid, so even a launch would stay in bounds."""
    import torch
    import paper_1510_05218_gb300 as p
    p.load_library()
    nx, ny, nz = 32 * 129, 8 * 128, 1
    shape = (nz, ny, nx)
    src = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    dst = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    coef = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(p.ThiimError) as e:
        p.thiim_step_noalloc(nx, ny, nz, 1, 3, [src] * 12, [dst] * 12, [coef] * 28)
    assert e.value.code == -1
    torch.cuda.synchronize()
    assert not bool(torch.any(dst != 0))


@pytest.mark.parametrize("nz", [128, 127])
def test_fp64_tile_shape_changes_no_field_bit(nz):
    """The FP64 sweep runs 32 x 16 tiles from 2^23 cells on (256 x 256 x 128
    here) and 32 x 8 below it (nz = 127); thiim_step_noalloc always runs 32 x 8.
    Each cell's arithmetic does not depend on the tile (a halo cell's H is
    recomputed by the same operations in the same order), so the fields agree
    bit for bit either way.  The residual sums per-CTA partials, whose grouping
    follows the tile: equal bit for bit on the same tile, within a few
    rounding errors (1e-13 relative) across tiles."""
    import torch
    import paper_1510_05218_gb300 as p
    p.load_library()
    nx = ny = 256
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    shape = (nz, ny, nx)

    def rnd(scale):
        return torch.complex(torch.randn(shape, generator=g, device="cuda", dtype=torch.float64),
                             torch.randn(shape, generator=g, device="cuda", dtype=torch.float64)) * scale

    co = [rnd(0.3) for _ in range(28)]
    a = [rnd(1.0) for _ in range(12)]
    b = [torch.empty_like(t) for t in a]
    r = p.thiim_step_noalloc(nx, ny, nz, 0, 3, a, b, co)
    ref = [t.clone() for t in a]
    del a
    ctx = p.thiim_create(nx, ny, nz, 0, 3)
    try:
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, ref)
        p.thiim_iterate(ctx, 1)
        q = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    torch.cuda.synchronize()
    for s in range(12):
        assert torch.equal(b[s], ref[s]), s
    assert np.isfinite(r) and r > 0
    if nx * ny * nz < 2 ** 23:
        assert r == q
    else:
        assert abs(r - q) <= 1e-13 * q
