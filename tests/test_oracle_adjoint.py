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


# ---- steady-state adjoint ------------------------------------------------------

def _affine_map(co, shape, bc):
    """Dense M, b of one oracle iteration x' = M x + b on a tiny grid (x = the 12
    splits flattened in order)."""
    n = int(np.prod(shape))
    zero_src = co[:24] + [np.zeros(shape, np.complex128) for _ in range(4)]
    M = np.empty((12 * n, 12 * n), np.complex128)
    for col in range(12 * n):
        v = [np.zeros(shape, np.complex128) for _ in range(12)]
        v[col // n].flat[col % n] = 1.0
        oracle.iterate(v, zero_src, 1, bc=bc)
        M[:, col] = np.concatenate([a.ravel() for a in v])
    b = [np.zeros(shape, np.complex128) for _ in range(12)]
    oracle.iterate(b, co, 1, bc=bc)
    return M, np.concatenate([a.ravel() for a in b])


def _steady_problem():
    shape = (3, 4, 5)
    nz, ny, nx = shape
    rng = np.random.default_rng(21)
    eps = rng.uniform(1.5, 3.0, shape) + 1j * rng.uniform(0.2, 0.6, shape)
    S = {n: rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for n in ("Hxy", "Hyx", "Exy", "Eyx")}
    co = build_coeffs(eps, np.zeros(nz), np.zeros(nz), 2 * np.pi / 6, 0.5, S=S)
    sigma = rng.uniform(0.5, 1.5, shape)
    return shape, co, sigma


def _J_and_g(x, sigma):
    """J = 1/2 sum sigma |E|^2 and g = 2 dJ/dconj(x) (sigma E on both splits of each E component)."""
    J, g = 0.0, [np.zeros_like(x[0]) for _ in range(12)]
    for comp in (3, 4, 5):
        e = x[2 * comp] + x[2 * comp + 1]
        J += 0.5 * float(np.sum(sigma * np.abs(e) ** 2))
        g[2 * comp] = sigma * e
        g[2 * comp + 1] = sigma * e
    return J, g


def test_steady_adjoint_matches_dense_solves_and_finite_differences():
    """The oracle's steady adjoint (reverse iteration summed at the fixed point)
    against dense linear algebra: lam* = (I - M^H)^{-1} g, and its coefficient
    gradient against central differences of J at the exact fixed point
    x* = (I - M)^{-1} b for perturbations of t, c and Src entries."""
    bc = 3
    shape, co, sigma = _steady_problem()
    n = int(np.prod(shape))

    def fixed_point(cc):
        M, b = _affine_map(cc, shape, bc)
        xs = np.linalg.solve(np.eye(12 * n) - M, b)
        return [xs[i * n:(i + 1) * n].reshape(shape) for i in range(12)], M

    x_star, M = fixed_point(co)
    J0, g = _J_and_g(x_star, sigma)
    lam, grad, k, rel = oracle.adjoint_steady(g, x_star, co, bc=bc, max_iters=20000, tol=1e-15)
    assert rel <= 1e-15 and k < 20000
    gv = np.concatenate([a.ravel() for a in g])
    lam_dense = np.linalg.solve(np.eye(12 * n) - M.conj().T, gv)
    lam_v = np.concatenate([a.ravel() for a in lam])
    assert np.linalg.norm(lam_v - lam_dense) <= 1e-10 * np.linalg.norm(lam_dense)

    h = 1e-6
    for a, p, d in [(oracle.COEFF_NAMES.index("tExy"), 7, 1.0), (oracle.COEFF_NAMES.index("cHzx"), 23, 1j),
                    (oracle.COEFF_NAMES.index("cEyz"), 41, 1.0), (oracle.COEFF_NAMES.index("SrcEyx"), 12, 1j),
                    (oracle.COEFF_NAMES.index("tHyx"), 55, 1.0), (oracle.COEFF_NAMES.index("SrcHyx"), 3, 1.0)]:
        Js = []
        for sgn in (1, -1):
            cc = [c.copy() for c in co]
            cc[a].flat[p] += sgn * h * d
            xs, _ = fixed_point(cc)
            Js.append(_J_and_g(xs, sigma)[0])
        fd = (Js[0] - Js[1]) / (2 * h)
        an = float(np.real(np.conj(grad[a].flat[p]) * d))
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3 * J0), (oracle.COEFF_NAMES[a], fd, an)


def test_steady_adjoint_detects_planted_error():
    """Planted: the adjoint sum cut after 5 terms (as if the adjoint fixed point
    were not reached) misses the finite difference that the full sum meets."""
    bc = 3
    shape, co, sigma = _steady_problem()
    n = int(np.prod(shape))

    def J_at(cc):
        M, b = _affine_map(cc, shape, bc)
        xs = np.linalg.solve(np.eye(12 * n) - M, b)
        return _J_and_g([xs[i * n:(i + 1) * n].reshape(shape) for i in range(12)], sigma)

    J0, g = J_at(co)
    M, b = _affine_map(co, shape, bc)
    xs = np.linalg.solve(np.eye(12 * n) - M, b)
    x_star = [xs[i * n:(i + 1) * n].reshape(shape) for i in range(12)]
    _, grad_cut, _, _ = oracle.adjoint_steady(g, x_star, co, bc=bc, max_iters=5)
    a, p, h = oracle.COEFF_NAMES.index("tExy"), 7, 1e-6
    cp, cm = [c.copy() for c in co], [c.copy() for c in co]
    cp[a].flat[p] += h
    cm[a].flat[p] -= h
    fd = (J_at(cp)[0] - J_at(cm)[0]) / (2 * h)
    an = float(np.real(grad_cut[a].flat[p]))
    assert not (abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3 * J0))
