"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests uses the GPU.  Each checks the oracle (oracle/) against an
independent statement of the same quantity:
  * dense FDFD solves assembled straight from Eqs. 3-7 (fixed point),
  * the 1D reduction of a flat stack, the discrete plane wave closed form and
    a lossy periodic plane wave in closed form,
  * the real arithmetic of the paper's Listings 1-2 and its flop counts,
  * periodic shift invariance.
"""
import cmath
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs
from tests import fdfd_ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _iterate_to(fields, coeffs, bc, tol=1e-15, max_iter=200000, chunk=500):
    """Iterate the oracle until the relative update of the last step is <= tol."""
    done = 0
    while done < max_iter:
        r = oracle.iterate(fields, coeffs, chunk, bc=bc, nthreads=1)
        done += chunk
        if r <= tol:
            return done, r
    return done, r


def _rel(a, b):
    num = sum(np.sum(np.abs(x - y) ** 2) for x, y in zip(a, b))
    den = sum(np.sum(np.abs(y) ** 2) for y in b)
    return math.sqrt(num / den)


def _physical_problem(shape, rng, neg_cells=4, pml=False):
    """Random lossy media: eps in [1, 4] (a few cells at -5), sigma, sigma* in [0.05, 0.3]."""
    nz, ny, nx = shape
    eps = rng.uniform(1.0, 4.0, shape)
    flat = rng.choice(eps.size, neg_cells, replace=False)
    eps.reshape(-1)[flat] = -5.0
    omega, tau = 2 * math.pi / 6.0, 0.5
    sig_mat = rng.uniform(0.05, 0.3, shape)
    sig_star = rng.uniform(0.05, 0.3, shape)
    eps_r = eps + 1j * sig_mat / omega           # physics convention: sigma = omega Im(eps_r)
    if pml:
        sig_pml_e = rng.uniform(0.0, 1.0, nz)
        sig_pml_h = rng.uniform(0.0, 1.0, nz)
    else:
        sig_pml_e = np.zeros(nz)
        sig_pml_h = np.zeros(nz)
    S = {n: (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) for n in ("Hxy", "Hyx", "Exy", "Eyx")}
    return eps, eps_r, omega, tau, sig_mat, sig_star, sig_pml_e, sig_pml_h, S


def _split_conductivities(shape, sig_mat, sig_star, sig_pml_e, sig_pml_h):
    terms = fdfd_ref.split_terms()
    sig_e, sig_h = {}, {}
    kk = np.arange(shape[0])[:, None, None]
    for s in fdfd_ref.SPLITS:
        along_z = terms[s][1] == 2
        if s[0] == "E":
            sig_e[s] = sig_mat + (sig_pml_e[kk] if along_z else 0.0)
        else:
            sig_h[s] = sig_star + (sig_pml_h[kk] if along_z else 0.0)
    return sig_e, sig_h


@pytest.mark.parametrize("shape,bc,pml", [((4, 4, 4), 7, False), ((6, 4, 4), 3, True)])
def test_fixed_point_matches_dense_fdfd_solve(shape, bc, pml):
    """P1: the iteration's fixed point solves the FDFD system of Eqs. 3-7.

    Includes eps < 0 cells (Eq. 5 back iteration), magnetic and electric
    losses so that every mode of the iteration decays, all four source splits,
    and (second case) absorbing-layer conductivities on the z splits with
    zero (Dirichlet) z boundaries.
    """
    rng = np.random.default_rng(11)
    eps, eps_r, omega, tau, sig_mat, sig_star, spe, sph, S = _physical_problem(shape, rng, pml=pml)
    sig_e, sig_h = _split_conductivities(shape, sig_mat, sig_star, spe, sph)
    Sfull = {s: S.get(s, np.zeros(shape)) for s in fdfd_ref.SPLITS}
    A, b = fdfd_ref.assemble(shape, eps, sig_e, sig_h, omega, tau, Sfull,
                             bc=(bool(bc & 1), bool(bc & 2), bool(bc & 4)))
    x_ref = fdfd_ref.to_fields(np.linalg.solve(A, b), shape)

    co = build_coeffs(eps_r, spe, sph, omega, tau, S=S, sigma_star=sig_star)
    f = [np.zeros(shape, np.complex128) for _ in range(12)]
    n, r = _iterate_to(f, co, bc, tol=1e-15)
    assert r <= 1e-15, (n, r)
    assert _rel(f, x_ref) <= 1e-12


def test_fixed_point_pin_detects_planted_sign_error():
    """The P1 comparison is sensitive: flipping one split's curl sign breaks it."""
    shape, bc = (4, 4, 4), 7
    rng = np.random.default_rng(11)
    eps, eps_r, omega, tau, sig_mat, sig_star, spe, sph, S = _physical_problem(shape, rng)
    sig_e, sig_h = _split_conductivities(shape, sig_mat, sig_star, spe, sph)
    Sfull = {s: S.get(s, np.zeros(shape)) for s in fdfd_ref.SPLITS}
    A, b = fdfd_ref.assemble(shape, eps, sig_e, sig_h, omega, tau, Sfull)
    x_ref = fdfd_ref.to_fields(np.linalg.solve(A, b), shape)
    co = build_coeffs(eps_r, spe, sph, omega, tau, S=S, sigma_star=sig_star)
    co[12 + oracle.FIELD_INDEX["Ezx"]] = -co[12 + oracle.FIELD_INDEX["Ezx"]]   # planted mistake
    f = [np.zeros(shape, np.complex128) for _ in range(12)]
    with np.errstate(all="ignore"):
        _iterate_to(f, co, bc, tol=1e-15, max_iter=4000)
        err = _rel(f, x_ref)
    assert not (err <= 1e-3)   # NaN (the flipped sign can make it diverge) also counts


def _flat_1d_system(nz, eps_r, sig_pml_e, sig_pml_h, omega, tau, k_s):
    """2 nz unknowns (E_x(k), H_y(k)) of a normally incident x-polarised wave.

    From Eqs. 3-5 at the fixed point with d/dz as the only derivative:
      H_y (index k, at z = k - 1/2):  w_h H = -(E(k) - E(k-1)) - sig*(k) H
      E_x (at z = k):                 w_e E = -(1/eps) e^{i w tau/2} (H(k+1) - H(k)) - loss
    with zero E below k = 0 and zero H above k = nz - 1, and the plane-wave
    coupling across the plane between H index k_s and E index k_s: H_y(k_s)
    sees E - E_inc, E_x(k_s) sees H + H_inc (total field for k >= k_s).
    """
    e = lambda a: cmath.exp(1j * a)  # noqa: E731
    wt = 2 * math.sin(omega * tau / 2) / tau
    kappa = 2 * math.asin(wt / 2)
    E_inc = lambda k: cmath.exp(-1j * kappa * (k - k_s))  # noqa: E731
    H_inc = lambda k: -(E_inc(k) - E_inc(k - 1)) / (1j * wt)  # noqa: E731
    w_e = (e(omega * tau) - 1) / tau
    w_h = (e(omega * tau / 2) - e(-omega * tau / 2)) / tau
    n = 2 * nz
    A = np.zeros((n, n), np.complex128)
    b = np.zeros(n, np.complex128)
    iE = lambda k: k  # noqa: E731
    iH = lambda k: nz + k  # noqa: E731
    for k in range(nz):
        r = iH(k)
        A[r, r] += w_h + sig_pml_h[k]
        A[r, iE(k)] += 1.0
        if k >= 1:
            A[r, iE(k - 1)] -= 1.0
        if k == k_s:
            b[r] += E_inc(k_s)
        r = iE(k)
        ep = eps_r[k].real
        sg = omega * eps_r[k].imag + sig_pml_e[k]
        A[r, r] += w_e + (sg / ep * e(omega * tau) if ep > 0 else sg / ep)
        g = e(omega * tau / 2) / ep
        if k + 1 < nz:
            A[r, iH(k + 1)] += g
        A[r, iH(k)] -= g
        if k == k_s:
            b[r] += g * H_inc(k_s)
    x = np.linalg.solve(A, b)
    return x[:nz], x[nz:]


@pytest.mark.parametrize("name,maxit,tol", [("stack32", 60000, 2e-16), ("stack128", 600000, 5e-13)])
def test_flat_stack_reduces_to_1d_solve(name, maxit, tol):
    """P2: a flat stack at normal incidence is x, y invariant with only E_x, H_y.

    The oracle runs the full 12-split 3D iteration on an (nz, 2, 2) periodic
    column of the stack without texture; its fixed point must equal the 1D
    FDFD solve of the same layers, absorbing profiles and plane-wave source.
    The 128-deep column (the scaled stack of the 128^3 workloads) takes ~3e5
    iterations (~25 s); the 512-deep one converges too slowly, ~1e6
    iterations, for a 1e-12 comparison in a unit test.
    """
    from workloads import LayeredStack, stack_config
    ref = stack_config(name)
    st = LayeredStack(2, 2, ref.nz, lam=ref.lam, n_sin=ref.n_sin, amp=0.0, seed=0)
    eps = st.eps()
    co = build_coeffs(eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    f = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    n, r = _iterate_to(f, co, 3, tol=tol, max_iter=maxit, chunk=5000)
    E1, H1 = _flat_1d_system(st.nz, eps[:, 0, 0], st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s)
    Ex = f[oracle.FIELD_INDEX["Exy"]] + f[oracle.FIELD_INDEX["Exz"]]
    Hy = f[oracle.FIELD_INDEX["Hyx"]] + f[oracle.FIELD_INDEX["Hyz"]]
    err = math.sqrt((np.sum(np.abs(Ex[:, 0, 0] - E1) ** 2) + np.sum(np.abs(Hy[:, 0, 0] - H1) ** 2))
                    / (np.sum(np.abs(E1) ** 2) + np.sum(np.abs(H1) ** 2)))
    assert err <= 1e-12, (n, r, err)
    for s in ("Exz", "Eyx", "Eyz", "Ezx", "Ezy", "Hxy", "Hxz", "Hyz", "Hzx", "Hzy"):
        assert np.all(f[oracle.FIELD_INDEX[s]] == 0), s
    for a in (Ex, Hy):
        assert np.max(np.abs(a - a[:, :1, :1])) == 0.0


def test_plane_wave_in_air_matches_closed_form():
    """P3: homogeneous air with absorbing layers and the plane-wave source.

    The exact fixed point (the 1D FDFD solve that P2 ties to the oracle's
    iteration) carries, in the total-field region, the discrete plane wave
    E_x(k) = exp(-i kappa (k - k_s)) with 2 sin(kappa/2) = 2 sin(omega tau/2)/tau,
    and the scattered-field region is empty, both up to the reflection of the
    bottom absorbing layer (<= 1e-3 with 32-cell layers at lambda = 20).
    The oracle's own iteration reaches the same field on a short air column.
    """
    from workloads import LayeredStack
    nz, L, k_s = 128, 32, 48
    st = LayeredStack(1, 1, nz, lam=20.0, amp=0.0, pml_cells=L)
    eps = np.ones(nz, np.complex128)
    E, _ = _flat_1d_system(nz, eps, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, k_s)
    wt = 2 * math.sin(st.omega * st.tau / 2) / st.tau
    kappa = 2 * math.asin(wt / 2)
    k_tf = np.arange(k_s, nz - L)
    k_sf = np.arange(L, k_s)
    exact = np.exp(-1j * kappa * (k_tf - k_s))
    assert np.max(np.abs(E[k_tf] - exact)) <= 1e-3
    assert np.max(np.abs(E[k_sf])) <= 1e-3
    # discrete vs continuum wave number: relative difference O((omega h)^2)
    assert abs(kappa - st.omega) / st.omega <= st.omega ** 2 / 8
    assert abs(2 * math.sin(kappa / 2) - wt) <= 1e-15
    # the oracle's iteration on a 32-deep air column converges to the 1D solve
    nz2, L2, ks2 = 32, 6, 8
    st2 = LayeredStack(1, 1, nz2, lam=20.0, amp=0.0, pml_cells=L2)
    eps2 = np.ones((nz2, 1, 1), np.complex128)
    co = build_coeffs(eps2, st2.sigma_pml_e(), st2.sigma_pml_h(), st2.omega, st2.tau, tfsf=(ks2, 1.0))
    f = [np.zeros(eps2.shape, np.complex128) for _ in range(12)]
    _iterate_to(f, co, 3, tol=1e-15, max_iter=200000, chunk=2000)
    E2, _ = _flat_1d_system(nz2, eps2[:, 0, 0], st2.sigma_pml_e(), st2.sigma_pml_h(), st2.omega, st2.tau, ks2)
    Ex = (f[6] + f[7])[:, 0, 0]
    assert np.max(np.abs(Ex - E2)) <= 1e-10


def test_lossy_periodic_plane_wave_closed_form():
    """P4: all-periodic lossy medium driven by S_E = exp(-i kappa0 k) on E_xy.

    The fixed point is A exp(-i kappa0 k) for E_x and B exp(-i kappa0 k) for
    H_y (index k at z = k - 1/2), where, with g = exp(i omega tau/2)/eps,
      w_h B = -(1 - exp(i kappa0)) A
      (w_e + sigma exp(i omega tau)/eps) A = -g (exp(-i kappa0) - 1) B + 1.
    """
    nz, m = 16, 2
    kappa0 = 2 * math.pi * m / nz
    omega, tau = 2 * math.pi / 7.0, 0.5
    eps_v, sig = 2.0, 0.2
    eps_r = np.full((nz, 1, 1), eps_v + 1j * sig / omega)
    k = np.arange(nz)
    S = {"Exy": np.exp(-1j * kappa0 * k)[:, None, None]}
    co = build_coeffs(eps_r, np.zeros(nz), np.zeros(nz), omega, tau, S=S)
    f = [np.zeros((nz, 1, 1), np.complex128) for _ in range(12)]
    _iterate_to(f, co, 7, tol=1e-15, max_iter=100000)
    e = lambda a: cmath.exp(1j * a)  # noqa: E731
    w_e = (e(omega * tau) - 1) / tau
    w_h = (e(omega * tau / 2) - e(-omega * tau / 2)) / tau
    g = e(omega * tau / 2) / eps_v
    # B = -(1 - e^{i k0}) A / w_h ; substitute into the E equation.
    a11 = w_e + sig / eps_v * e(omega * tau) + g * (e(-kappa0) - 1) * (-(1 - e(kappa0)) / w_h)
    A = 1.0 / a11
    B = -(1 - e(kappa0)) * A / w_h
    Ex = (f[6] + f[7])[:, 0, 0]
    Hy = (f[2] + f[3])[:, 0, 0]
    assert np.max(np.abs(Ex - A * np.exp(-1j * kappa0 * k))) <= 1e-12 * abs(A)
    assert np.max(np.abs(Hy - B * np.exp(-1j * kappa0 * k))) <= 1e-12 * abs(B)


def test_periodic_shift_invariance_is_exact():
    """P5: rolling the texture by (di, dj) rolls the result bit for bit."""
    from workloads import LayeredStack
    st = LayeredStack(12, 10, 32, lam=20.0, seed=3)
    eps = st.eps()
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau)
    di, dj = 5, 3
    co_a = build_coeffs(eps, *args, tfsf=(st.k_s, 1.0))
    co_b = build_coeffs(np.roll(eps, (dj, di), axis=(1, 2)), *args, tfsf=(st.k_s, 1.0))
    fa = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    fb = [np.zeros(eps.shape, np.complex128) for _ in range(12)]
    oracle.iterate(fa, co_a, 25, bc=3)
    oracle.iterate(fb, co_b, 25, bc=3)
    for a, b in zip(fa, fb):
        assert np.array_equal(np.roll(a, (dj, di), axis=(1, 2)), b)


def _golden():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as fh:
        return json.load(fh)


def test_listing_arithmetic_and_flop_counts():
    """P8: the oracle's H_yx and H_zx updates equal the real arithmetic of Listings 1-2.

    Listing 1 (H_yx): with (R, I) = E_x(k) - E_x(k-1),
      re' = Hr tr - Hi ti + Sr - cr R + ci I,  im' = Hr ti + Hi tr + Si - cr I - ci R.
    Listing 2 (H_zx): with (R, I) = E_x(j-1) - E_x(j) and no source,
      re' = Hr tr - Hi ti - cr R + ci I,        im' = Hr ti + Hi tr - cr I - ci R.
    Flops: 3 + 3 for the two differences of sums, 8 + 8 (Listing 1) or
    7 + 7 (Listing 2) for the update: 22 and 20; 4*22 + 8*20 = 248 per LUP.
    """
    g = _golden()
    assert 3 + 3 + 8 + 8 == g["flops_listing1"]
    assert 3 + 3 + 7 + 7 == g["flops_listing2"]
    assert 4 * g["flops_listing1"] + 8 * g["flops_listing2"] == g["flops_per_lup"]
    assert 12 + 4 * 3 + 8 * 2 == g["arrays_per_cell"]
    assert 16 * g["arrays_per_cell"] == g["bytes_per_cell"]

    rng = np.random.default_rng(5)
    shape = (3, 3, 3)
    f = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(12)]
    co = [rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for _ in range(28)]
    f0 = [a.copy() for a in f]
    oracle.iterate(f, co, 1, bc=7)
    k, j, i = 1, 1, 1
    Ex = f0[6] + f0[7]
    ix = oracle.FIELD_INDEX
    # Listing 1: H_yx with the z shift and SrcHy.
    H = f0[ix["Hyx"]][k, j, i]
    t = co[ix["Hyx"]][k, j, i]
    c = co[12 + ix["Hyx"]][k, j, i]
    S = co[25][k, j, i]
    d = Ex[k, j, i] - Ex[k - 1, j, i]
    R, I = d.real, d.imag
    re = H.real * t.real - H.imag * t.imag + S.real - c.real * R + c.imag * I
    im = H.real * t.imag + H.imag * t.real + S.imag - c.real * I - c.imag * R
    assert abs(f[ix["Hyx"]][k, j, i] - complex(re, im)) <= 1e-14 * abs(complex(re, im))
    # Listing 2: H_zx with the y shift, no source.
    H = f0[ix["Hzx"]][k, j, i]
    t = co[ix["Hzx"]][k, j, i]
    c = co[12 + ix["Hzx"]][k, j, i]
    d = Ex[k, j - 1, i] - Ex[k, j, i]
    R, I = d.real, d.imag
    re = H.real * t.real - H.imag * t.imag - c.real * R + c.imag * I
    im = H.real * t.imag + H.imag * t.real - c.real * I - c.imag * R
    assert abs(f[ix["Hzx"]][k, j, i] - complex(re, im)) <= 1e-14 * abs(complex(re, im))


def test_iteration_is_affine_with_consistent_fixed_point():
    """The one-iteration map x -> M x + b assembled column by column from the
    oracle has (I - M)^-1 b equal to the dense FDFD solution (P1 consistency)."""
    shape = (2, 2, 3)
    rng = np.random.default_rng(4)
    eps, eps_r, omega, tau, sig_mat, sig_star, spe, sph, S = _physical_problem(shape, rng, neg_cells=2)
    co = build_coeffs(eps_r, spe, sph, omega, tau, S=S, sigma_star=sig_star)
    ncell = int(np.prod(shape))
    n = 12 * ncell

    def step(x):
        f = [x[s * ncell:(s + 1) * ncell].reshape(shape).copy() for s in range(12)]
        oracle.iterate(f, co, 1, bc=7)
        return np.concatenate([a.reshape(-1) for a in f])

    b = step(np.zeros(n, np.complex128))
    M = np.zeros((n, n), np.complex128)
    for col in range(n):
        e = np.zeros(n, np.complex128)
        e[col] = 1.0
        M[:, col] = step(e) - b
    x_it = np.linalg.solve(np.eye(n) - M, b)
    sig_e, sig_h = _split_conductivities(shape, sig_mat, sig_star, spe, sph)
    Sfull = {s: S.get(s, np.zeros(shape)) for s in fdfd_ref.SPLITS}
    A, rhs = fdfd_ref.assemble(shape, eps, sig_e, sig_h, omega, tau, Sfull)
    x_ref = np.linalg.solve(A, rhs)
    assert np.linalg.norm(x_it - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
