"""GPU checks of general polarisation, absorbed power and the spectrum driver.

* thiim_build_coeffs_jones vs the oracle's builder for a random Jones vector:
  1e-14 relative per array (the array builder's bound).
* y-polarised iteration vs the oracle: 20 iterations of a textured stack from
  zero, 1e-12 relative per split (the complex128 / pair bound).
* thiim_absorbed_power vs the oracle's sum on the same fields: 1e-12
  relative (both FP64 sums of the same terms, in different orders), for all
  three precisions.
* The material table with a Jones vector is bit-identical to the arrays.
* absorption_spectrum (3 wavelengths x 2 polarisations in one batch, a fixed
  200 iterations): each solve's absorbed power within 1e-10 of the oracle's
  200-iteration solve; on a texture that is symmetric under x <-> y the x-
  and y-polarised absorptions agree to 1e-12 (mirror symmetry).
"""
import numpy as np
import pytest

import oracle
from oracle.coeffs import absorbed_power, build_coeffs
from tests.gpu_util import rel_l2, to_dev, to_host
from workloads.thiim_workloads import LayeredStack

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _stack(nx=40, ny=20, nz=48, seed=3):
    return LayeredStack(nx=nx, ny=ny, nz=nz, amp=3.0, seed=seed)


def test_jones_builder_matches_oracle():
    import torch
    p = _lib()
    st = _stack()
    ax, ay = 0.3 - 0.8j, -0.6 + 0.25j
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3)
    try:
        co = [torch.empty((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda") for _ in range(28)]
        eps = torch.from_numpy(st.eps()).to("cuda")
        p.thiim_build_coeffs_jones(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s,
                                   ax, ay, co)
        g = to_host(co)
    finally:
        p.thiim_destroy(ctx)
    oc = build_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, ax, ay))
    for i in range(28):
        assert rel_l2(g[i], oc[i]) <= 1e-14, (oracle.COEFF_NAMES[i], rel_l2(g[i], oc[i]))
    assert np.max(np.abs(oc[24])) > 0 and np.max(np.abs(oc[27])) > 0      # y sources present


@pytest.mark.parametrize("precision", [0, 2])
def test_y_polarised_iteration_matches_oracle(precision):
    import torch
    p = _lib()
    st = _stack()
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, 3)
    try:
        co = [torch.empty((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda") for _ in range(28)]
        eps = torch.from_numpy(st.eps()).to("cuda")
        p.thiim_build_coeffs_jones(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s,
                                   0.0, 1.0, co)
        fd = [torch.zeros((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda") for _ in range(12)]
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, 20)
        g = to_host(fd)
    finally:
        p.thiim_destroy(ctx)
    oc = build_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 0.0, 1.0))
    o = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    oracle.iterate(o, oc, 20, bc=3)
    for s in range(12):
        if np.max(np.abs(o[s])) == 0:
            assert np.max(np.abs(g[s])) == 0, oracle.SPLITS[s]
        else:
            assert rel_l2(g[s], o[s]) <= 1e-12, (oracle.SPLITS[s], rel_l2(g[s], o[s]))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_absorbed_power_matches_oracle_sum(precision):
    import torch
    p = _lib()
    st = _stack()
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, 3)
    dt = torch.complex64 if precision == 1 else torch.complex128
    try:
        co = [torch.empty((st.nz, st.ny, st.nx), dtype=dt, device="cuda") for _ in range(28)]
        eps = torch.from_numpy(st.eps()).to("cuda")
        p.thiim_build_coeffs_jones(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s,
                                   1.0, 0.5j, co)
        fd = [torch.zeros((st.nz, st.ny, st.nx), dtype=dt, device="cuda") for _ in range(12)]
        p.thiim_set_coeffs(ctx, co)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, 30)
        sigma = st.omega * st.eps().imag * st.absorber_mask()
        got = p.thiim_absorbed_power(ctx, torch.from_numpy(sigma).to("cuda"))
        g = to_host(fd)
    finally:
        p.thiim_destroy(ctx)
    want = absorbed_power(g, sigma)
    assert want > 0 and abs(got - want) <= 1e-12 * want


def test_material_table_with_jones_is_bit_identical_to_arrays():
    import torch
    p = _lib()
    st = _stack()
    ax, ay = 0.5 + 0.1j, -0.2 + 0.9j
    x0 = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    out = []
    for use_table in (False, True):
        ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128_PAIR, 3)
        try:
            if use_table:
                em = st.material_eps()
                table = torch.empty(len(em) * st.nz * 28, dtype=torch.complex128, device="cuda")
                p.thiim_build_material_table(ctx, em, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau,
                                             st.k_s, ax, table, amp_y=ay)
                mat = torch.from_numpy(st.material_ids()).to("cuda")
                p.thiim_set_material_coeffs(ctx, mat, len(em), table)
                keep = [table, mat]
            else:
                keep = [torch.empty((st.nz, st.ny, st.nx), dtype=torch.complex128, device="cuda")
                        for _ in range(28)]
                eps = torch.from_numpy(st.eps()).to("cuda")
                p.thiim_build_coeffs_jones(ctx, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau,
                                           st.k_s, ax, ay, keep)
                p.thiim_set_coeffs(ctx, keep)
            fd = to_dev(x0)
            p.thiim_set_fields(ctx, fd)
            p.thiim_iterate(ctx, 9)
            out.append(to_host(fd))
        finally:
            p.thiim_destroy(ctx)
    for s in range(12):
        assert np.array_equal(out[0][s], out[1][s]), oracle.SPLITS[s]


def test_spectrum_matches_oracle_and_mirror_symmetry():
    p = _lib()
    from paper_1510_05218_gb300.spectrum import absorption_spectrum, incident_power
    st = LayeredStack(nx=16, ny=16, nz=32, amp=3.0, seed=7)
    eps = st.eps()
    # symmetric texture: eps[:, j, i] = eps[:, min(i, j), max(i, j)]
    jj, ii = np.meshgrid(np.arange(st.ny), np.arange(st.nx), indexing="ij")
    eps = np.ascontiguousarray(eps[:, np.minimum(ii, jj), np.maximum(ii, jj)])
    assert np.array_equal(eps, eps.transpose(0, 2, 1))
    absorber = (eps.real > 10)
    lams = [16.0, 20.0, 28.0]
    n_it = 200
    r = absorption_spectrum(eps, lams, st.sigma_pml_e(), st.sigma_pml_h(), st.k_s, st.tau, absorber,
                            precision=p.THIIM_C128_PAIR, max_iters=n_it, check_every=50, tol=0.0)
    assert r["iterations"] == [n_it] * 6
    for b, lam in enumerate(lams):
        omega = 2 * np.pi / lam
        sigma = omega * eps.imag * absorber
        for q, (pol, amps) in enumerate((("x", (1.0,)), ("y", (0.0, 1.0)))):
            co = build_coeffs(eps, st.sigma_pml_e(), st.sigma_pml_h(), omega, st.tau, tfsf=(st.k_s,) + amps)
            o = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
            oracle.iterate(o, co, n_it, bc=3)
            want = absorbed_power(o, sigma)
            got = r["power"][2 * b + q]
            assert abs(got - want) <= 1e-10 * want, (lam, pol, got, want)
            a_want = np.cos(omega * st.tau / 2) * want / incident_power(omega, st.tau, st.nx, st.ny)
            assert abs(r["A"][pol][b] - a_want) <= 1e-10 * r["A"][pol][b]
        assert abs(r["A"]["x"][b] - r["A"]["y"][b]) <= 1e-12 * r["A"]["x"][b]
        assert r["A_unpolarised"][b] == pytest.approx(0.5 * (r["A"]["x"][b] + r["A"]["y"][b]), rel=1e-15)


def test_power_and_jones_errors():
    import ctypes
    import torch
    p = _lib()
    lib = p.load_library()
    ctx = p.thiim_create(8, 8, 8, p.THIIM_C128, 3)
    try:
        sigma = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
        out = ctypes.c_double()
        assert lib.thiim_absorbed_power(ctx, ctypes.c_void_p(sigma.data_ptr()), ctypes.byref(out)) == -3
        eps = torch.ones((8, 8, 8), dtype=torch.complex128, device="cuda")
        co = [torch.empty((8, 8, 8), dtype=torch.complex128, device="cuda") for _ in range(28)]
        with pytest.raises(p.ThiimError) as e:
            p.thiim_build_coeffs_jones(ctx, eps, None, None, 0.3, 0.5, 4, float("nan"), 0.0, co)
        assert e.value.code == -1
        fd = [torch.zeros((8, 8, 8), dtype=torch.complex128, device="cuda") for _ in range(12)]
        p.thiim_set_fields(ctx, fd)
        odd = ctypes.c_void_p(sigma.data_ptr() + 4)
        assert lib.thiim_absorbed_power(ctx, odd, ctypes.byref(out)) == -2
        assert p.thiim_absorbed_power(ctx, sigma) == 0.0
    finally:
        p.thiim_destroy(ctx)
