"""Mixed precision with FP64 defect correction (thiim_mixed_solve) against the oracle.

* The FP64 defect residual equals the oracle's relative full-field update
  of one iteration (both FP64): 1e-10.
* One outer step with K inner complex64 iterations equals K plain FP64
  iterations up to the FP32 error of the correction: the correction is K
  FP32 sweeps of r rounded to complex64, each adding at most ~16 u relative
  (u = 2^-24, see test_gpu_sweep), so the error relative to the change
  ||x_K - x_0|| is below K * 16 u; K = 3 gives 2.9e-6, taken as 5e-6.
* At convergence the mixed solution's full field components match the
  oracle's converged FP64 solution to 1e-6 (the required bound for
  complex64 vs FP64).  The mixed FP64 residual levels off at a floor
  (~5e-8 with 50 inner iterations on the 32^3 stack; measured 2e-8 / 5e-8 /
  1e-7 for 10 / 50 / 250) set by the FP32 error of corrections that carry
  the undamped split parts inside the absorbing layers; the test runs to
  that floor (<= 1e-7) and checks the 1e-6 accuracy there.  The native FP64
  GPU solve, run to residual 1e-8, meets the same bound.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs as oracle_coeffs
from tests.gpu_util import full_fields, rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields, stack_config

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _c64_ctx(p, shape, coeffs64_host, bc=3):
    import torch
    nz, ny, nx = shape
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C64, bc)
    c32 = to_dev([c.astype(np.complex64) for c in coeffs64_host], "complex64")
    work = [torch.zeros(shape, dtype=torch.complex64, device="cuda") for _ in range(12)]
    p.thiim_set_coeffs(ctx, c32)
    p.thiim_set_fields(ctx, work)
    return ctx, c32, work


def _oracle_full_change(f, co, bc):
    prev = full_fields(f)
    oracle.iterate(f, co, 1, bc=bc)
    cur = full_fields(f)
    num = sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(cur, prev))
    den = sum(np.sum(np.abs(a) ** 2) for a in cur)
    return math.sqrt(num / den)


def test_defect_residual_matches_oracle():
    p = _lib()
    shape = (9, 13, 70)
    nz, ny, nx = shape
    x = random_fields(nx, ny, nz, seed=41)
    co = random_coeffs(nx, ny, nz, seed=41)
    ctx, keep32, keepw = _c64_ctx(p, shape, co)   # the library borrows these arrays
    try:
        xd = to_dev(x)
        c64 = to_dev(co)
        done, r = p.thiim_mixed_solve(ctx, c64, xd, inner_iters=5, max_outer=0, tol=0.0)
        assert done == 0
        xg = to_host(xd)
    finally:
        p.thiim_destroy(ctx)
    for a, b in zip(xg, x):
        assert np.array_equal(a, b)            # max_outer = 0 leaves x untouched
    r_o = _oracle_full_change([a.copy() for a in x], co, 3)
    assert abs(r - r_o) <= 1e-10 * r_o


@pytest.mark.parametrize("bc", [3, 0])
def test_one_correction_equals_k_fp64_iterations(bc):
    p = _lib()
    shape = (7, 11, 45)
    nz, ny, nx = shape
    x = random_fields(nx, ny, nz, seed=42)
    co = random_coeffs(nx, ny, nz, seed=42)
    K = 3
    ctx, keep32, keepw = _c64_ctx(p, shape, co, bc)
    try:
        xd = to_dev(x)
        c64 = to_dev(co)
        done, _ = p.thiim_mixed_solve(ctx, c64, xd, inner_iters=K, max_outer=1, tol=0.0)
        assert done == 1
        xg = to_host(xd)
    finally:
        p.thiim_destroy(ctx)
    o = [a.copy() for a in x]
    oracle.iterate(o, co, K, bc=bc)
    num = sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(xg, o))
    den = sum(np.sum(np.abs(b - a0) ** 2) for b, a0 in zip(o, x))
    assert math.sqrt(num / den) <= 5e-6


def _oracle_converged(st, co, tol):
    f = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    threads = os.cpu_count() or 1
    for _ in range(400):
        oracle.iterate(f, co, 999, bc=3, nthreads=threads)
        if _oracle_full_change(f, co, 3) <= tol:
            return f
    raise AssertionError("oracle did not converge")


def test_mixed_and_native_converge_to_the_fp64_fixed_point():
    import torch
    p = _lib()
    st = stack_config("stack32")
    shape = (st.nz, st.ny, st.nx)
    co = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    ref = full_fields(_oracle_converged(st, co, 1e-10))

    # mixed: complex64 corrections, FP64 defect
    ctx, keep32, keepw = _c64_ctx(p, shape, co)
    try:
        x64 = [torch.zeros(shape, dtype=torch.complex128, device="cuda") for _ in range(12)]
        c64 = to_dev(co)
        done, r = p.thiim_mixed_solve(ctx, c64, x64, inner_iters=50, max_outer=2000, tol=1e-8)
        assert r <= 1e-7, (done, r)
        mixed = full_fields(to_host(x64))
    finally:
        p.thiim_destroy(ctx)
    for comp in range(6):
        assert rel_l2(mixed[comp], ref[comp]) <= 1e-6, (comp, rel_l2(mixed[comp], ref[comp]))

    # native FP64 on the GPU, to the same residual
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3)
    try:
        fd = [torch.zeros(shape, dtype=torch.complex128, device="cuda") for _ in range(12)]
        cd = to_dev(co)
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        for _ in range(400):
            p.thiim_iterate(ctx, 500)
            if p.thiim_residual(ctx) <= 1e-8:
                break
        native = full_fields(to_host(fd))
    finally:
        p.thiim_destroy(ctx)
    for comp in range(6):
        assert rel_l2(native[comp], ref[comp]) <= 1e-6, (comp, rel_l2(native[comp], ref[comp]))


def test_mixed_converged_64_cube_within_1e6_of_native_fp64():
    """The 64^3 stack (the largest grid of the layered workload whose iteration
    converges in reach: native FP64 reaches residual 9e-12 in 250k iterations;
    the 128^3 stack's iteration has a slowly growing mode, see the benchmark's
    extended C2 run) converged by native FP64 and by the mixed solver with an
    FP64 defect every 10 complex64 iterations.  Every full component of the
    mixed solution lies within 1e-6 (relative L2) of the FP64 one at the mixed
    solver's residual floor.  Measured: 3.2e-7 at the floor 1.3e-8 (13500 outer
    steps); with a defect every 50 iterations the floor is 6.8e-8 and the error
    1.5e-6, over the bound."""
    import torch
    p = _lib()
    st = stack_config("stack64")
    shape = (st.nz, st.ny, st.nx)
    eps = torch.from_numpy(st.eps()).to("cuda")
    bargs = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3)
    co64 = [torch.empty(shape, dtype=torch.complex128, device="cuda") for _ in range(28)]
    f64 = [torch.zeros(shape, dtype=torch.complex128, device="cuda") for _ in range(12)]
    try:
        p.thiim_build_coeffs(ctx, eps, *bargs, co64)
        p.thiim_set_coeffs(ctx, co64)
        p.thiim_set_fields(ctx, f64)
        it, r64 = 0, 1.0
        while it < 300000 and r64 > 1e-11:
            p.thiim_iterate(ctx, 5000)
            it += 5000
            r64 = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    assert r64 <= 1e-10, r64
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C64, 3)
    co32 = [torch.empty(shape, dtype=torch.complex64, device="cuda") for _ in range(28)]
    work = [torch.zeros(shape, dtype=torch.complex64, device="cuda") for _ in range(12)]
    x64 = [torch.zeros(shape, dtype=torch.complex128, device="cuda") for _ in range(12)]
    try:
        p.thiim_build_coeffs(ctx, eps, *bargs, co32)
        p.thiim_set_coeffs(ctx, co32)
        p.thiim_set_fields(ctx, work)
        # to the mixed solver's floor: chunks of 500 outer steps until five in a
        # row gain less than 10 % (stopping at residual 2e-8 left 1.3e-6: the
        # slow tail of the iteration)
        outer, best, stall, rm = 0, 1.0, 0, 1.0
        while outer < 20000 and stall < 5:
            done, rm = p.thiim_mixed_solve(ctx, co64, x64, 10, 500, 0.0)
            outer += done
            stall = stall + 1 if rm > 0.9 * best else 0
            best = min(best, rm)
    finally:
        p.thiim_destroy(ctx)
    assert rm <= 3e-8, (outer, rm)
    for c in range(6):
        ref = f64[2 * c] + f64[2 * c + 1]
        mix = x64[2 * c] + x64[2 * c + 1]
        err = float(torch.linalg.vector_norm(mix - ref) / torch.linalg.vector_norm(ref))
        assert err <= 1e-6, (c, err)
