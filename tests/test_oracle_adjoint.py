"""Pins of the oracle's adjoint (reverse iteration and coefficient gradients).

* Dot-product identity <mu, M v> = <M^H mu, v> for the linear part M of one
  iteration and for three iterations in a row.
* For every one of the 28 coefficient arrays a, one iteration's output is
  exactly linear in a perturbation delta of that array alone, so
  <mu, x'(a + delta) - x'(a)> must equal <g_a, delta> (g_a the accumulated
  gradient) to rounding.
* The permittivity derivatives of the coefficients equal central differences
  of the coefficient builder.
All inner products are <a, b> = sum conj(a) b.
"""
import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs, coeff_eps_derivatives
from workloads import random_coeffs, random_fields


def ip(a, b):
    return sum(np.vdot(x, y) for x, y in zip(a, b))


def _zero_src(co):
    return co[:24] + [np.zeros_like(c) for c in co[24:]]


@pytest.mark.parametrize("bc", [7, 3, 0])
def test_adjoint_dot_product_one_iteration(bc):
    shape = (5, 6, 7)
    nz, ny, nx = shape
    co = _zero_src(random_coeffs(nx, ny, nz, seed=3))
    v = random_fields(nx, ny, nz, seed=4)
    mu = random_fields(nx, ny, nz, seed=5)
    Mv = [a.copy() for a in v]
    oracle.iterate(Mv, co, 1, bc=bc)
    lam = [a.copy() for a in mu]
    grad = [np.zeros(shape, np.complex128) for _ in range(28)]
    oracle.adjoint_step(lam, grad, v, Mv, co, bc=bc)
    lhs, rhs = ip(mu, Mv), ip(lam, v)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_dot_product_three_iterations():
    shape = (6, 5, 9)
    nz, ny, nx = shape
    co = _zero_src(random_coeffs(nx, ny, nz, seed=8))
    states = [random_fields(nx, ny, nz, seed=9)]
    for _ in range(3):
        nxt = [a.copy() for a in states[-1]]
        oracle.iterate(nxt, co, 1, bc=3)
        states.append(nxt)
    mu = random_fields(nx, ny, nz, seed=10)
    lam = [a.copy() for a in mu]
    grad = [np.zeros(shape, np.complex128) for _ in range(28)]
    for n in (2, 1, 0):
        oracle.adjoint_step(lam, grad, states[n], states[n + 1], co, bc=3)
    lhs, rhs = ip(mu, states[3]), ip(lam, states[0])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("bc", [3, 4])
def test_coefficient_gradients_match_exact_linear_response(bc):
    shape = (4, 5, 6)
    nz, ny, nx = shape
    co = random_coeffs(nx, ny, nz, seed=11)
    x = random_fields(nx, ny, nz, seed=12)
    x1 = [a.copy() for a in x]
    oracle.iterate(x1, co, 1, bc=bc)
    mu = random_fields(nx, ny, nz, seed=13)
    lam = [a.copy() for a in mu]
    grad = [np.zeros(shape, np.complex128) for _ in range(28)]
    oracle.adjoint_step(lam, grad, x, x1, co, bc=bc)
    rng = np.random.default_rng(14)
    for a in range(28):
        delta = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        co2 = list(co)
        co2[a] = co[a] + delta
        x2 = [b.copy() for b in x]
        oracle.iterate(x2, co2, 1, bc=bc)
        lhs = ip(mu, [p - q for p, q in zip(x2, x1)])
        rhs = np.vdot(grad[a], delta)
        assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1e-300), (oracle.COEFF_NAMES[a], lhs, rhs)


def test_permittivity_derivatives_match_central_differences():
    from workloads import LayeredStack
    st = LayeredStack(4, 3, 32, lam=20.0, seed=2)
    eps = st.eps()
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau)
    d = coeff_eps_derivatives(eps, st.sigma_pml_e(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    h = 1e-6
    cp = build_coeffs(eps + h, *args, tfsf=(st.k_s, 1.0))
    cm = build_coeffs(eps - h, *args, tfsf=(st.k_s, 1.0))
    for a in range(28):
        fd = (cp[a] - cm[a]) / (2 * h)
        an = d.get(a, np.zeros_like(fd))
        scale = max(np.max(np.abs(fd)), 1e-12)
        assert np.max(np.abs(fd - an)) <= 1e-7 * scale, oracle.COEFF_NAMES[a]
