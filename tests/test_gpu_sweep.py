"""GPU parity of the fused THIIM sweep against the FP64 oracle (through the C ABI).

Tolerances (written here, derived from the arithmetic):
  * complex128 path: relative L2 <= 1e-12 per split (the required bound);
    both sides are FP64 and differ only in rounding order and FMA use.
  * complex128 data with FP32-pair arithmetic (THIIM_C128_PAIR): the same
    1e-12 bound.  A pair carries ~48 significant bits (unit 2^-48 ~ 3.6e-15)
    and an update rounds each of its ~5 terms once, so one iteration adds at
    most ~10 * 2^-48 ~ 4e-14 relative; 20 iterations stay below 1e-12.
  * complex64 path: FP32 storage of fields and coefficients (unit roundoff
    u = 2^-24 ~ 6e-8) and FP32 arithmetic.  One update rounds ~4 inputs and
    ~10 operations, so its relative error is below ~16 u ~ 1e-6; errors carry
    over with |t| <= 1 and the curl terms, and after n iterations stay below
    n * 16 u.  The test uses 3 iterations: bound 3 * 16 u ~ 3e-6, taken as 5e-6.
"""
import math

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


def _run_gpu(fields, coeffs, n, bc, precision=0):
    p = _lib()
    nz, ny, nx = fields[0].shape
    dt = "complex64" if precision == 1 else "complex128"
    fd = to_dev(fields, dt)
    cd = to_dev(coeffs, dt)
    ctx = p.thiim_create(nx, ny, nz, precision, bc)
    try:
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, n)
        r = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    return to_host(fd), r


def _run_oracle(fields, coeffs, n, bc):
    f = [a.copy() for a in fields]
    prev = None
    for it in range(n):
        if it == n - 1:
            prev = full_fields(f)
        oracle.iterate(f, coeffs, 1, bc=bc)
    cur = full_fields(f)
    num = sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(cur, prev))
    den = sum(np.sum(np.abs(a) ** 2) for a in cur)
    return f, math.sqrt(num / den)


SHAPES = [  # (nz, ny, nx): several tiles plus ragged tails in x and y, odd z
    (9, 13, 70),
    (5, 17, 33),
    (4, 8, 32),
    (3, 1, 1),
    (1, 5, 7),
    (40, 9, 31),
]


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [3, 7, 0, 1, 6])
def test_c128_sweep_matches_oracle(shape, bc, precision):
    nz, ny, nx = shape
    f = random_fields(nx, ny, nz, seed=7)
    c = random_coeffs(nx, ny, nz, seed=7)
    n = 3
    g, r_gpu = _run_gpu(f, c, n, bc, precision)
    o, r_ora = _run_oracle(f, c, n, bc)
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 1e-12, (oracle.SPLITS[s], rel_l2(g[s], o[s]))
    assert abs(r_gpu - r_ora) <= 1e-10 * r_ora


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_c128_iteration_counts_and_copy_back(n, precision):
    """Odd counts end in the library's second field set and are copied back;
    in pair mode n = 1..4 runs every (input, output) format variant."""
    nz, ny, nx = 6, 10, 40
    f = random_fields(nx, ny, nz, seed=3)
    c = random_coeffs(nx, ny, nz, seed=3)
    g, _ = _run_gpu(f, c, n, 3, precision)
    o, _ = _run_oracle(f, c, n, 3)
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 1e-12


def test_c64_sweep_matches_oracle_within_fp32_bound():
    nz, ny, nx = 9, 13, 70
    f = random_fields(nx, ny, nz, seed=5)
    c = random_coeffs(nx, ny, nz, seed=5)
    n = 3
    g, _ = _run_gpu(f, c, n, 3, precision=1)
    # the oracle runs on the FP32-rounded inputs in FP64
    f32 = [a.astype(np.complex64).astype(np.complex128) for a in f]
    c32 = [a.astype(np.complex64).astype(np.complex128) for a in c]
    o, _ = _run_oracle(f32, c32, n, 3)
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 5e-6, (oracle.SPLITS[s], rel_l2(g[s], o[s]))


def _device_stack(st, precision=0):
    """Coefficients of a layered stack built on the GPU from its permittivity map."""
    import torch
    p = _lib()
    eps = torch.from_numpy(st.eps()).to("cuda")
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, 3)
    dt = torch.complex64 if precision == 1 else torch.complex128
    co = [torch.empty((st.nz, st.ny, st.nx), dtype=dt, device="cuda") for _ in range(28)]
    p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co)
    return ctx, co


@pytest.mark.parametrize("precision", [0, 2])
def test_stack32_twenty_iterations_match_oracle(precision):
    """The 32^3 textured stack, 20 iterations from zero, coefficients built on each side."""
    p = _lib()
    st = stack_config("stack32")
    ctx, co = _device_stack(st, precision)
    try:
        oc = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
        gc = to_host(co)
        for i in range(28):
            assert rel_l2(gc[i], oc[i]) <= 1e-14, (oracle.COEFF_NAMES[i], rel_l2(gc[i], oc[i]))
        import torch
        fd = [torch.zeros((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda") for _ in range(12)]
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, 20)
        r_gpu = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    g = to_host(fd)
    f0 = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    o, r_ora = _run_oracle(f0, oc, 20, 3)
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 1e-12, (oracle.SPLITS[s], rel_l2(g[s], o[s]))
    assert abs(r_gpu - r_ora) <= 1e-10 * r_ora


def test_pair_mode_tracks_native_fp64_over_200_iterations():
    """Drift of the FP32-pair arithmetic against native FP64 (both on the GPU,
    both parity-checked against the oracle above) over the benchmark's 200
    iterations on the 128^3 stack."""
    import torch
    p = _lib()
    st = stack_config("stack128")
    out = []
    for prec in (0, 2):
        ctx, co = _device_stack(st, prec)
        try:
            fd = [torch.zeros((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda") for _ in range(12)]
            p.thiim_set_coeffs(ctx, co)
            p.thiim_set_fields(ctx, fd)
            p.thiim_iterate(ctx, 200)
            torch.cuda.synchronize()
            out.append([t.cpu().numpy() for t in fd])
        finally:
            p.thiim_destroy(ctx)
    a, b = full_fields(out[1]), full_fields(out[0])
    for comp in range(6):
        assert rel_l2(a[comp], b[comp]) <= 1e-12, (comp, rel_l2(a[comp], b[comp]))


def test_pair_mode_resplits_after_new_coefficients():
    """thiim_set_coeffs marks the split coefficients stale: new contents are used."""
    p = _lib()
    nz, ny, nx = 6, 9, 35
    f = random_fields(nx, ny, nz, seed=12)
    c1 = random_coeffs(nx, ny, nz, seed=12)
    c2 = random_coeffs(nx, ny, nz, seed=13)
    fd = to_dev(f)
    cd = to_dev(c1)
    ctx = p.thiim_create(nx, ny, nz, 2, 3)
    try:
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, 2)
        for t, v in zip(cd, to_dev(c2)):
            t.copy_(v)
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_iterate(ctx, 2)
        g = to_host(fd)
    finally:
        p.thiim_destroy(ctx)
    o = [a.copy() for a in f]
    oracle.iterate(o, c1, 2, bc=3)
    oracle.iterate(o, c2, 2, bc=3)
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 1e-12


def test_build_coeffs_c64_rounds_the_fp64_values():
    st = stack_config("stack32")
    ctx, co = _device_stack(st, precision=1)
    _lib().thiim_destroy(ctx)
    oc = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    gc = to_host(co)
    for i in range(28):
        assert np.array_equal(gc[i], oc[i].astype(np.complex64).astype(np.complex128)) or \
            rel_l2(gc[i], oc[i]) <= 2 * U32, oracle.COEFF_NAMES[i]


def test_zero_iterations_and_errors():
    import torch
    p = _lib()
    ctx = p.thiim_create(8, 8, 8, 0, 3)
    try:
        with pytest.raises(p.ThiimError) as e:
            p.thiim_iterate(ctx, 1)            # no fields / coefficients yet
        assert e.value.code == -3
        with pytest.raises(p.ThiimError) as e:
            p.thiim_residual(ctx)
        assert e.value.code == -3
        f = [torch.zeros((8, 8, 8), dtype=torch.complex128, device="cuda") for _ in range(12)]
        c = [torch.zeros((8, 8, 8), dtype=torch.complex128, device="cuda") for _ in range(28)]
        p.thiim_set_fields(ctx, f)
        p.thiim_set_coeffs(ctx, c)
        p.thiim_iterate(ctx, 0)
        with pytest.raises(p.ThiimError) as e:
            p.thiim_iterate(ctx, -1)
        assert e.value.code == -1
        p.thiim_iterate(ctx, 2)
        assert p.thiim_residual(ctx) == 0.0          # all-zero fields
        bad = (ctypes_addr(f[0]) + 8)
        with pytest.raises(p.ThiimError) as e:
            p.thiim_set_fields(ctx, [bad] + f[1:])
        assert e.value.code == -2
    finally:
        p.thiim_destroy(ctx)


def ctypes_addr(t):
    return t.data_ptr()


def test_nonfinite_residual_is_reported():
    import torch
    p = _lib()
    nz, ny, nx = 4, 8, 8
    f = random_fields(nx, ny, nz, seed=1)
    c = random_coeffs(nx, ny, nz, seed=1)
    c[0][1, 2, 3] = np.nan
    fd = to_dev(f)
    cd = to_dev(c)
    ctx = p.thiim_create(nx, ny, nz, 0, 3)
    try:
        p.thiim_set_fields(ctx, fd)
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_iterate(ctx, 1)
        with pytest.raises(p.ThiimError) as e:
            p.thiim_residual(ctx)
        assert e.value.code == -6
    finally:
        p.thiim_destroy(ctx)
    del torch
