"""Pins of the oracle's y-polarised and general (Jones) plane-wave sources.

No GPU.  The x-polarised source is pinned by the plane-wave and 1D tests in
test_oracle_pins.py; the y-polarised one is checked here against statements
that do not use its formulas:
  * in an air column it carries the same discrete plane wave as the 1D solve
    of the x-polarised problem (E_y = E_x there, H_x = -H_y, E_x = 0);
  * mirror symmetry: swapping x and y maps the x-polarised problem on eps to
    the y-polarised problem on the transposed eps.  E is a polar vector
    (E'_x(i, j) = E_y(j, i), ...) and H an axial one (H'_x(i, j) = -H_y(j, i),
    ...), and the split of each component swaps with its mirror partner
    (Exy <-> Eyx, Exz <-> Eyz, Ezx <-> Ezy; the same for H with a minus sign);
  * linearity: the field of the source (A_x, A_y) is A_x times the
    x-polarised field plus A_y times the y-polarised one;
  * a source with a planted sign error fails the mirror check.
"""
import numpy as np

import oracle
from oracle.coeffs import absorbed_power, build_coeffs
from tests.test_oracle_pins import _flat_1d_system, _iterate_to
from workloads.thiim_workloads import LayeredStack

MIRROR = {"Exy": "Eyx", "Exz": "Eyz", "Eyx": "Exy", "Eyz": "Exz", "Ezx": "Ezy", "Ezy": "Ezx",
          "Hxy": "Hyx", "Hxz": "Hyz", "Hyx": "Hxy", "Hyz": "Hxz", "Hzx": "Hzy", "Hzy": "Hzx"}


def _mirror(fields):
    out = []
    for name in oracle.SPLITS:
        a = fields[oracle.FIELD_INDEX[MIRROR[name]]].transpose(0, 2, 1)
        out.append(np.ascontiguousarray(-a if name[0] == "H" else a))
    return out


def _run(co, shape, n):
    f = [np.zeros(shape, np.complex128) for _ in range(12)]
    oracle.iterate(f, co, n, bc=3)
    return f


def test_y_polarised_plane_wave_in_air():
    nz, L, k_s = 32, 6, 8
    st = LayeredStack(1, 1, nz, lam=20.0, amp=0.0, pml_cells=L)
    eps = np.ones((nz, 1, 1), np.complex128)
    co = build_coeffs(eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(k_s, 0.0, 1.0))
    f = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    _iterate_to(f, co, 3, tol=1e-15, max_iter=200000, chunk=2000)
    E1d, _ = _flat_1d_system(nz, eps[:, 0, 0], st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, k_s)
    Ey = (f[8] + f[9])[:, 0, 0]
    assert np.max(np.abs(Ey - E1d)) <= 1e-10
    for s in ("Exy", "Exz", "Hyx", "Hyz", "Ezx", "Ezy", "Hzx", "Hzy"):
        assert np.all(f[oracle.FIELD_INDEX[s]] == 0), s
    # the x-polarised solve of the same column: H_x(y-pol) = -H_y(x-pol)
    cox = build_coeffs(eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(k_s, 1.0))
    g = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    _iterate_to(g, cox, 3, tol=1e-15, max_iter=200000, chunk=2000)
    assert np.max(np.abs((f[0] + f[1]) + (g[2] + g[3]))) <= 1e-10


def _textured(seed=4):
    st = LayeredStack(nx=8, ny=8, nz=32, amp=3.0, seed=seed)
    eps = st.eps()
    assert not np.allclose(eps, eps.transpose(0, 2, 1))     # the texture is not mirror symmetric
    return st, eps


def test_mirror_symmetry_maps_x_to_y_polarisation():
    st, eps = _textured()
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau)
    fx = _run(build_coeffs(eps, *args, tfsf=(st.k_s, 1.0)), eps.shape, 80)
    epsT = np.ascontiguousarray(eps.transpose(0, 2, 1))
    fy = _run(build_coeffs(epsT, *args, tfsf=(st.k_s, 0.0, 1.0)), eps.shape, 80)
    want = _mirror(fx)
    scale = max(np.max(np.abs(a)) for a in fx)
    for s, name in enumerate(oracle.SPLITS):
        assert np.max(np.abs(fy[s] - want[s])) <= 1e-13 * scale, name
    sigma = st.omega * eps.imag * st.absorber_mask()
    px = absorbed_power(fx, sigma)
    py = absorbed_power(fy, np.ascontiguousarray(sigma.transpose(0, 2, 1)))
    assert px > 0 and abs(px - py) <= 1e-12 * px


def test_mirror_pin_detects_planted_source_sign_error():
    st, eps = _textured()
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau)
    fx = _run(build_coeffs(eps, *args, tfsf=(st.k_s, 1.0)), eps.shape, 80)
    epsT = np.ascontiguousarray(eps.transpose(0, 2, 1))
    co = build_coeffs(epsT, *args, tfsf=(st.k_s, 0.0, 1.0))
    co[24] = -co[24]                                  # planted: wrong sign of SrcHxy
    fy = _run(co, eps.shape, 80)
    want = _mirror(fx)
    err = max(np.max(np.abs(fy[s] - want[s])) for s in range(12))
    assert not (err <= 1e-3)


def test_jones_source_is_the_superposition_of_both_polarisations():
    st, eps = _textured(seed=5)
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau)
    ax, ay = 0.3 - 0.2j, 0.7 + 0.5j
    fx = _run(build_coeffs(eps, *args, tfsf=(st.k_s, 1.0)), eps.shape, 40)
    fy = _run(build_coeffs(eps, *args, tfsf=(st.k_s, 0.0, 1.0)), eps.shape, 40)
    fj = _run(build_coeffs(eps, *args, tfsf=(st.k_s, ax, ay)), eps.shape, 40)
    scale = max(np.max(np.abs(a)) for a in fj)
    for s, name in enumerate(oracle.SPLITS):
        assert np.max(np.abs(fj[s] - (ax * fx[s] + ay * fy[s]))) <= 1e-12 * scale, name
