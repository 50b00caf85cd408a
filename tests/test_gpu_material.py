"""GPU checks of the compressed-coefficient variant (material map + table).

* The table built on the GPU, expanded on the host through the material map,
  equals the oracle's 28 coefficient arrays of the same stack within 1e-14
  relative per array (the bound the array builder is held to).
* Iterating with the table gives fields and residuals bit-identical to
  iterating with the 28 arrays built from the same materials, for every
  precision, on the 32^3 stack and on a stack with ragged x and y tiles
  (7 iterations: covers the pair mode's complex128 / pair boundaries and the
  odd-count copy-back).  The coefficient values are the same bits and the
  update arithmetic is the same, so exact equality is the expected result.
* Table mode against the oracle directly: 20 iterations of the 32^3 stack
  from zero within the complex128 bound, 1e-12 relative per split.
* A table rebuilt in place and set again is the one used (the pair mode
  splits it again), and leaves the context's state clean for later calls.
* Error returns of the two entry points and of the calls that need the 28
  arrays.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs as oracle_coeffs
from tests.gpu_util import full_fields, rel_l2, to_dev, to_host
from workloads import random_fields, stack_config
from workloads.thiim_workloads import LayeredStack

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _stack(name):
    if name == "ragged":   # 40 x 20: 32 x 8 tiles 32 + 8 by 8 + 8 + 4; 64 x 4 tiles (pair) 40 by 5 x 4
        return LayeredStack(nx=40, ny=20, nz=48, seed=3)
    return stack_config(name)


def _dtype(precision):
    import torch
    return torch.complex64 if precision == 1 else torch.complex128


def _table(p, ctx, st, precision):
    import torch
    em = st.material_eps()
    table = torch.empty(len(em) * st.nz * 28, dtype=_dtype(precision), device="cuda")
    p.thiim_build_material_table(ctx, em, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0,
                                 table)
    return table


def _arrays(p, ctx, st, precision):
    import torch
    eps = torch.from_numpy(st.eps()).to("cuda")
    co = [torch.empty((st.nz, st.ny, st.nx), dtype=_dtype(precision), device="cuda") for _ in range(28)]
    p.thiim_build_coeffs(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0, co)
    return co


@pytest.mark.parametrize("name", ["stack32", "ragged"])
def test_table_expands_to_oracle_coefficients(name):
    p = _lib()
    st = _stack(name)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3)
    try:
        table = _table(p, ctx, st, 0)
        t = to_host([table])[0].reshape(4, st.nz, 28)
    finally:
        p.thiim_destroy(ctx)
    ids = st.material_ids()
    k = np.arange(st.nz)[:, None, None]
    oc = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    for i in range(28):
        got = t[ids, k, i]
        assert rel_l2(got, oc[i]) <= 1e-14, (oracle.COEFF_NAMES[i], rel_l2(got, oc[i]))


def _iterate(p, st, precision, use_table, n, x0, temporal=1):
    import torch
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, 3)
    try:
        if precision == 1:
            p.thiim_set_tuning(ctx, temporal, 0)
        keep = []
        if use_table:
            table = _table(p, ctx, st, precision)
            mat = torch.from_numpy(st.material_ids()).to("cuda")
            p.thiim_set_material_coeffs(ctx, mat, 4, table)
            keep += [table, mat]
        else:
            keep += _arrays(p, ctx, st, precision)
            p.thiim_set_coeffs(ctx, keep)
        fd = to_dev(x0, "complex64" if precision == 1 else "complex128")
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, n)
        r = p.thiim_residual(ctx)
        torch.cuda.synchronize()
        return [f.cpu().numpy() for f in fd], r
    finally:
        p.thiim_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("name", ["stack32", "ragged"])
def test_table_mode_bit_identical_to_arrays(name, precision):
    p = _lib()
    st = _stack(name)
    x0 = [0.01 * a for a in random_fields(st.nx, st.ny, st.nz, seed=17)]
    g_arr, r_arr = _iterate(p, st, precision, False, 7, x0)
    g_tbl, r_tbl = _iterate(p, st, precision, True, 7, x0)
    for s in range(12):
        assert np.array_equal(g_tbl[s], g_arr[s]), oracle.SPLITS[s]
    assert r_tbl == r_arr


def test_table_mode_ignores_temporal_blocking():
    p = _lib()
    st = _stack("stack32")
    x0 = [0.01 * a for a in random_fields(st.nx, st.ny, st.nz, seed=18)]
    g1, r1 = _iterate(p, st, 1, True, 6, x0, temporal=1)
    g2, r2 = _iterate(p, st, 1, True, 6, x0, temporal=2)
    for s in range(12):
        assert np.array_equal(g1[s], g2[s]), oracle.SPLITS[s]
    assert r1 == r2


@pytest.mark.parametrize("precision", [0, 2])
def test_table_mode_matches_oracle(precision):
    p = _lib()
    st = _stack("stack32")
    f0 = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    g, r_gpu = _iterate(p, st, precision, True, 20, f0)
    oc = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    o = [a.copy() for a in f0]
    oracle.iterate(o, oc, 19, bc=3)
    prev = full_fields(o)
    oracle.iterate(o, oc, 1, bc=3)
    cur = full_fields(o)
    r_ora = np.sqrt(sum(np.sum(np.abs(a - b) ** 2) for a, b in zip(cur, prev)) /
                    sum(np.sum(np.abs(a) ** 2) for a in cur))
    for s in range(12):
        assert rel_l2(g[s], o[s]) <= 1e-12, (oracle.SPLITS[s], rel_l2(g[s], o[s]))
    assert abs(r_gpu - r_ora) <= 1e-10 * r_ora


@pytest.mark.parametrize("precision", [1, 2])
def test_rebuilt_table_is_used_on_the_same_context(precision):
    """A table rebuilt in place for other materials, then set again, gives the
    same iterate as a fresh context built for those materials (the pair mode
    splits the table again)."""
    import torch
    p = _lib()
    st = _stack("stack32")
    st2 = LayeredStack(nx=st.nx, ny=st.ny, nz=st.nz, eps_scale=1.2)
    x0 = [0.01 * a for a in random_fields(st.nx, st.ny, st.nz, seed=19)]
    want, r_want = _iterate(p, st2, precision, True, 5, x0)
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, 3)
    try:
        table = _table(p, ctx, st, precision)
        mat = torch.from_numpy(st.material_ids()).to("cuda")
        p.thiim_set_material_coeffs(ctx, mat, 4, table)
        fd = to_dev(x0, "complex64" if precision == 1 else "complex128")
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, 3)
        em = st2.material_eps()
        p.thiim_build_material_table(ctx, em, st2.sigma_pml_e(), st2.sigma_pml_h(), st2.omega, st2.tau, st2.k_s,
                                     1.0, table)
        p.thiim_set_material_coeffs(ctx, mat, 4, table)
        for f, a in zip(fd, x0):
            f.copy_(torch.from_numpy(a))
        p.thiim_iterate(ctx, 5)
        r = p.thiim_residual(ctx)
        torch.cuda.synchronize()
        got = [f.cpu().numpy() for f in fd]
    finally:
        p.thiim_destroy(ctx)
    for s in range(12):
        assert np.array_equal(got[s], want[s]), oracle.SPLITS[s]
    assert r == r_want


def test_table_errors_and_mode_switch():
    import torch
    p = _lib()
    lib = p.load_library()
    st = _stack("stack32")
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C64, 3)
    try:
        table = torch.zeros(4 * st.nz * 28 + 1, dtype=torch.complex64, device="cuda")
        mat = torch.zeros((st.nz, st.ny, st.nx), dtype=torch.uint8, device="cuda")
        em = st.material_eps()
        args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
        for bad in (0, 257):
            assert lib.thiim_set_material_coeffs(ctx, ctypes.c_void_p(mat.data_ptr()), bad,
                                                 ctypes.c_void_p(table.data_ptr())) == -1
        with pytest.raises(p.ThiimError) as e:
            p.thiim_build_material_table(ctx, np.array([1.0, 0.0]), *args, table)
        assert e.value.code == -1                      # zero permittivity
        with pytest.raises(p.ThiimError) as e:
            p.thiim_build_material_table(ctx, np.array([1.0, np.nan]), *args, table)
        assert e.value.code == -1
        odd = ctypes.c_void_p(table.data_ptr() + 4)    # complex64 needs 8-byte alignment
        assert lib.thiim_set_material_coeffs(ctx, ctypes.c_void_p(mat.data_ptr()), 4, odd) == -2
        p.thiim_build_material_table(ctx, em, *args, table)
        p.thiim_set_material_coeffs(ctx, mat, 4, table)
        fd = [torch.zeros((st.nz, st.ny, st.nx), dtype=torch.complex64, device="cuda") for _ in range(12)]
        p.thiim_set_fields(ctx, fd)
        # calls that need the 28 arrays refuse the table mode (before reading any pointer)
        fake28, fake12 = [16] * 28, [16] * 12
        with pytest.raises(p.ThiimError) as e:
            p.thiim_mixed_solve(ctx, fake28, fake12, 4, 1)
        assert e.value.code == -3
        with pytest.raises(p.ThiimError) as e:
            p.thiim_batch_iterate([ctx], 4, 2)
        assert e.value.code == -3
        # back to arrays with thiim_set_coeffs
        co = _arrays(p, ctx, st, 1)
        p.thiim_set_coeffs(ctx, co)
        p.thiim_mixed_solve(ctx, to_dev([c.cpu().numpy() for c in co]), to_dev([f.cpu().numpy() for f in fd]), 4, 1)
    finally:
        p.thiim_destroy(ctx)
    ctx = p.thiim_create(8, 8, 8, p.THIIM_C128, 3)
    try:
        table = torch.zeros(8 * 28, dtype=torch.complex128, device="cuda")
        mat = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
        p.thiim_set_material_coeffs(ctx, mat, 1, table)
        with pytest.raises(p.ThiimError) as e:
            p.thiim_adjoint_iterate(ctx, [16] * 12, [16] * 28, [16] * 12, 1)
        assert e.value.code == -3
    finally:
        p.thiim_destroy(ctx)
