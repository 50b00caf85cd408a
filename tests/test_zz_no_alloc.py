"""thiim_step_noalloc: the iteration entry point for callers that cannot allocate.

Callers running under another framework's memory pool or allocator hooks, or
with all device memory reserved in advance, cannot let the library call
cudaMalloc.  thiim_step_noalloc runs one iteration between caller buffers and
keeps its reduction scratch in a fixed device array.  Here it is called twice
in a row through the C ABI and compared with thiim_iterate (the allocating
path) after one and two iterations, at the 1e-12 tolerance the other parity
tests use.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from tests.gpu_util import rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-12)])
def test_noalloc_matches_allocating_path_on_two_calls(precision, tol):
    import torch
    import paper_1510_05218_gb300 as p
    p.load_library()
    nz, ny, nx = 11, 21, 75          # several tiles, ragged in x and y
    dt = "complex128" if precision == 0 else "complex64"
    f0 = random_fields(nx, ny, nz, seed=31)
    co = to_dev(random_coeffs(nx, ny, nz, seed=31), dt)
    a = to_dev(f0, dt)
    b = [torch.empty_like(t) for t in a]
    c = [torch.empty_like(t) for t in a]
    r1 = p.thiim_step_noalloc(nx, ny, nz, precision, 3, a, b, co)
    r2 = p.thiim_step_noalloc(nx, ny, nz, precision, 3, b, c, co)
    got1, got2 = to_host(b), to_host(c)

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
        assert rel_l2(got1[s], want1[s]) <= tol
        assert rel_l2(got2[s], want2[s]) <= tol
    assert abs(r1 - q1) <= tol * q1 and abs(r2 - q2) <= tol * q2
    assert np.isfinite(r1) and r1 > 0


def test_noalloc_rejects_grids_beyond_its_scratch():
    import paper_1510_05218_gb300 as p
    p.load_library()
    nx, ny, nz = 32 * 129, 8 * 128, 4           # 16512 CTAs > 16384: rejected before any launch
    fake = [4096 * (i + 1) for i in range(12)]
    fake2 = [4096 * (i + 20) for i in range(12)]
    fakec = [4096 * (i + 40) for i in range(28)]
    with pytest.raises(p.ThiimError) as e:
        p.thiim_step_noalloc(nx, ny, nz, 0, 3, fake, fake2, fakec)
    assert e.value.code == -1
