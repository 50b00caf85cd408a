"""Batched solves (thiim_batch_iterate): one persistent launch per iteration
over uneven grids, CUDA graph per convergence-check chunk.

* Every solve of a ragged, uneven batch matches the oracle after the same
  number of iterations at 1e-12 per split (complex128 native and FP32 pairs),
  including a final chunk shorter than check_every and an odd total.
* A solve whose residual reaches tol leaves the batch at that check while the
  others continue; results equal the single-problem path bit for bit
  (same arithmetic, only the work distribution differs).
"""
import math

import numpy as np
import pytest

import oracle
from tests.gpu_util import full_fields, rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields

pytestmark = pytest.mark.gpu

SHAPES = [(9, 13, 70), (5, 17, 33), (40, 9, 31), (3, 1, 1), (12, 8, 32)]
BCS = [3, 7, 0, 3, 6]


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _make(p, shape, bc, seed, precision):
    nz, ny, nx = shape
    f = random_fields(nx, ny, nz, seed=seed)
    c = random_coeffs(nx, ny, nz, seed=seed)
    dt = "complex64" if precision == 1 else "complex128"
    fd, cd = to_dev(f, dt), to_dev(c, dt)
    ctx = p.thiim_create(nx, ny, nz, precision, bc)
    p.thiim_set_coeffs(ctx, cd)
    p.thiim_set_fields(ctx, fd)
    return ctx, f, c, fd, cd


def _full_change(before, after):
    a, b = full_fields(after), full_fields(before)
    num = sum(np.sum(np.abs(x - y) ** 2) for x, y in zip(a, b))
    den = sum(np.sum(np.abs(x) ** 2) for x in a)
    return math.sqrt(num / den)


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("max_iters,check", [(7, 2), (6, 4), (1, 2)])
def test_batch_matches_oracle(precision, max_iters, check):
    p = _lib()
    made = [_make(p, sh, bc, 50 + i, precision) for i, (sh, bc) in enumerate(zip(SHAPES, BCS))]
    try:
        iters, res = p.thiim_batch_iterate([m[0] for m in made], max_iters, check, 0.0)
        got = [to_host(m[3]) for m in made]
        r_ctx = [p.thiim_residual(m[0]) for m in made]
    finally:
        for m in made:
            p.thiim_destroy(m[0])
    assert iters == [max_iters] * len(made)
    for (ctx, f, c, fd, cd), g, bc, r, rc in zip(made, got, BCS, res, r_ctx):
        o = [a.copy() for a in f]
        oracle.iterate(o, c, max_iters - 1, bc=bc)
        before = [a.copy() for a in o]
        oracle.iterate(o, c, 1, bc=bc)
        for s in range(12):
            assert rel_l2(g[s], o[s]) <= 1e-12, (s, rel_l2(g[s], o[s]))
        r_o = _full_change(before, o)
        assert abs(r - r_o) <= 1e-10 * r_o and r == rc


@pytest.mark.parametrize("precision", [0, 1])
def test_converged_solve_retires_and_others_match_single_runs(precision):
    import torch
    p = _lib()
    made = [_make(p, sh, bc, 70 + i, precision) for i, (sh, bc) in enumerate(zip(SHAPES[:3], BCS[:3]))]
    # solve 0: zero fields and zero sources -> its residual is 0 after the first check
    for t in made[0][3]:
        t.zero_()
    for t in made[0][4][24:]:
        t.zero_()
    start = [[t.clone() for t in m[3]] for m in made]
    try:
        iters, res = p.thiim_batch_iterate([m[0] for m in made], 12, 4, 1e-300)
        got = [to_host(m[3]) for m in made]
    finally:
        for m in made:
            p.thiim_destroy(m[0])
    assert iters == [4, 12, 12] and res[0] == 0.0
    for i, m in enumerate(made):
        nz, ny, nx = SHAPES[i]
        ctx = p.thiim_create(nx, ny, nz, precision, BCS[i])
        try:
            fd = [t.clone() for t in start[i]]
            p.thiim_set_coeffs(ctx, m[4])
            p.thiim_set_fields(ctx, fd)
            p.thiim_iterate(ctx, iters[i])
            want = to_host(fd)
        finally:
            p.thiim_destroy(ctx)
        for s in range(12):
            assert np.array_equal(got[i][s], want[s])
    del torch


def test_batch_rejects_mixed_precisions_and_odd_chunks():
    p = _lib()
    a = _make(p, (4, 8, 32), 3, 1, 0)
    b = _make(p, (4, 8, 32), 3, 2, 1)
    try:
        with pytest.raises(p.ThiimError):
            p.thiim_batch_iterate([a[0], b[0]], 4, 2, 0.0)
        with pytest.raises(p.ThiimError):
            p.thiim_batch_iterate([a[0]], 4, 3, 0.0)
    finally:
        p.thiim_destroy(a[0])
        p.thiim_destroy(b[0])


def test_poisoned_solve_fails_alone():
    """A solve with a NaN coefficient is retired at its first check and the call
    reports THIIM_ERR_NONFINITE; the other solves still run to max_iters and
    match their single runs."""
    p = _lib()
    made = [_make(p, sh, bc, 95 + i, 0) for i, (sh, bc) in enumerate(zip(SHAPES[:3], BCS[:3]))]
    made[1][4][0][1, 2, 3] = float("nan")
    start = [[t.clone() for t in m[3]] for m in made]
    try:
        with pytest.raises(p.ThiimError) as e:
            p.thiim_batch_iterate([m[0] for m in made], 8, 4, 0.0)
        assert e.value.code == -6
        got = [to_host(m[3]) for m in made]
    finally:
        for m in made:
            p.thiim_destroy(m[0])
    for i in (0, 2):
        nz, ny, nx = SHAPES[i]
        ctx = p.thiim_create(nx, ny, nz, 0, BCS[i])
        try:
            fd = [t.clone() for t in start[i]]
            p.thiim_set_coeffs(ctx, made[i][4])
            p.thiim_set_fields(ctx, fd)
            p.thiim_iterate(ctx, 8)
            want = to_host(fd)
        finally:
            p.thiim_destroy(ctx)
        for s in range(12):
            assert np.array_equal(got[i][s], want[s])
