"""GPU adjoint (thiim_adjoint_iterate, thiim_build_coeffs_grad, autograd) checks.

* The GPU reverse iteration with recomputation from a checkpoint matches the
  oracle's adjoint (lambda and all 28 coefficient gradients) at 1e-10 per
  array (the required bound for GPU vs CPU adjoint).
* The permittivity chain rule matches the oracle's analytic coefficient
  derivatives at 1e-12.
* End to end on the 128^3 adjoint workload (texture confined to a 32x32 box,
  300 iterations, checkpoints every 20): the gradient of the absorbed power
  J = 1/2 sum_{absorber} sigma |E|^2 with respect to Re eps agrees with
  central finite differences at 64 seeded cells of the texture region within
  |g - fd| <= 1e-4 max(|fd|, 1e-3 max|fd|).  The difference step is 1e-4:
  with 1e-6 the two FP64 solves' rounding (~1e-14 J after 300 iterations)
  leaves ~5e-8 of noise in each difference quotient (measured), above that
  floor; at 1e-4 the noise is 100x smaller and the O(h^2) truncation of the
  smooth rational dependence on eps is ~1e-10 relative.
* The same check at the configuration's step 1e-6 on the 16 cells of largest
  |gradient| (|g| ~ 2.4e-3 .. 3.8e-3): there the solves' rounding noise in a
  quotient (~5e-8) is ~2e-5 of |fd|, inside the 1e-4 relative bound
  (measured: at most 5.2e-5).
"""
import numpy as np
import pytest

import oracle
from oracle.coeffs import coeff_eps_derivatives
from tests.gpu_util import rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields, stack_config

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


@pytest.mark.parametrize("shape,bc,n_back", [((6, 11, 37), 3, 3), ((5, 9, 20), 0, 2), ((4, 8, 33), 7, 1)])
def test_adjoint_matches_oracle(shape, bc, n_back):
    p = _lib()
    nz, ny, nx = shape
    x0 = random_fields(nx, ny, nz, seed=61)
    co = random_coeffs(nx, ny, nz, seed=61)
    mu = random_fields(nx, ny, nz, seed=62)
    g0 = [0.1 * a for a in random_fields(nx, ny, nz, seed=63)] + [0.1 * a for a in random_fields(nx, ny, nz, seed=64)] \
        + [0.1 * a for a in random_fields(nx, ny, nz, seed=65)[:4]]
    # oracle: states, then reverse
    states = [[a.copy() for a in x0]]
    for _ in range(n_back):
        nxt = [a.copy() for a in states[-1]]
        oracle.iterate(nxt, co, 1, bc=bc)
        states.append(nxt)
    lam_o = [a.copy() for a in mu]
    g_o = [a.copy() for a in g0]
    for n in range(n_back - 1, -1, -1):
        oracle.adjoint_step(lam_o, g_o, states[n], states[n + 1], co, bc=bc)
    # GPU
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C128, bc)
    try:
        cd = to_dev(co)
        p.thiim_set_coeffs(ctx, cd)
        lam = to_dev(mu)
        gd = to_dev(g0)
        ck = to_dev(x0)
        p.thiim_adjoint_iterate(ctx, lam, gd, ck, n_back)
        lam_g, g_g, ck_g = to_host(lam), to_host(gd), to_host(ck)
    finally:
        p.thiim_destroy(ctx)
    for s in range(12):
        assert rel_l2(lam_g[s], lam_o[s]) <= 1e-10, ("lambda", s)
        assert np.array_equal(ck_g[s], x0[s])          # the checkpoint is read only
    for a in range(28):
        assert rel_l2(g_g[a], g_o[a]) <= 1e-10, oracle.COEFF_NAMES[a]


def test_eps_chain_rule_matches_oracle_derivatives():
    import torch
    p = _lib()
    st = stack_config("stack32")
    eps = st.eps()
    rng = np.random.default_rng(5)
    G = [rng.standard_normal(eps.shape) + 1j * rng.standard_normal(eps.shape) for _ in range(28)]
    ctx = p.thiim_create(st.nx, st.ny, st.nz, p.THIIM_C128, 3)
    try:
        out = torch.empty(eps.shape, dtype=torch.float64, device="cuda")
        ed = torch.from_numpy(eps).to("cuda")
        gd = to_dev(G)
        p.thiim_build_coeffs_grad(ctx, ed, st.sigma_pml_e(), st.omega, st.tau, st.k_s, 1.0, gd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    finally:
        p.thiim_destroy(ctx)
    d = coeff_eps_derivatives(eps, st.sigma_pml_e(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
    want = sum(np.real(np.conj(G[a]) * d[a]) for a in d)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _objective(torch, fields, sigma_mask):
    ex = fields[6] + fields[7]
    ey = fields[8] + fields[9]
    ez = fields[10] + fields[11]
    e2 = ex.real ** 2 + ex.imag ** 2 + ey.real ** 2 + ey.imag ** 2 + ez.real ** 2 + ez.imag ** 2
    return 0.5 * torch.sum(sigma_mask * e2)


def test_permittivity_gradient_matches_finite_differences():
    import torch
    p = _lib()
    from paper_1510_05218_gb300.autograd import Differentiable
    st = stack_config("adjoint128")
    n_it, every = 300, 20
    eps = st.eps()
    sigma = st.omega * eps.imag * st.absorber_mask()
    sig_d = torch.from_numpy(sigma).to("cuda")
    dmod = Differentiable(st.nx, st.ny, st.nz)
    try:
        eps_re = torch.from_numpy(eps.real.copy()).to("cuda").requires_grad_(True)
        eps_im = torch.from_numpy(eps.imag.copy()).to("cuda")
        args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
        co = dmod.build_coeffs(eps_re, eps_im, *args)
        x = dmod.solve(co, n_it, every)
        J = _objective(torch, x, sig_d)
        J.backward()
        grad = eps_re.grad.detach().cpu().numpy()

        # central differences at 64 seeded cells of the texture box (x, y in [48, 80), z in [48, 64))
        rng = np.random.default_rng(2)
        cells = np.stack([rng.integers(48, 64, 64), rng.integers(48, 80, 64), rng.integers(48, 80, 64)], 1)
        h = 1e-4

        def J_at(eps_re_t):
            with torch.no_grad():
                c2 = dmod.build_coeffs(eps_re_t, eps_im, *args)
                x2 = dmod.solve(c2, n_it, 60)
                return float(_objective(torch, x2, sig_d))

        fd = []
        base = eps_re.detach().clone()
        for k, j, i in cells:
            e = base.clone()
            e[k, j, i] += h
            jp = J_at(e)
            e[k, j, i] -= 2 * h
            jm = J_at(e)
            fd.append((jp - jm) / (2 * h))
        fd = np.array(fd)
        g = np.array([grad[k, j, i] for k, j, i in cells])
        # the configuration's step, 1e-6, on the 16 cells of largest |g|
        h6 = 1e-6
        top = np.argsort(-np.abs(g))[:16]
        fd6 = []
        for idx in top:
            k, j, i = cells[idx]
            e = base.clone()
            e[k, j, i] += h6
            jp = J_at(e)
            e[k, j, i] -= 2 * h6
            jm = J_at(e)
            fd6.append((jp - jm) / (2 * h6))
        fd6 = np.array(fd6)
    finally:
        dmod.close()
    assert np.all(np.abs(g[top] - fd6) <= 1e-4 * np.abs(fd6)), np.max(np.abs(g[top] - fd6) / np.abs(fd6))
    tol = 1e-4 * np.maximum(np.abs(fd), 1e-3 * np.max(np.abs(fd)))
    assert np.all(np.abs(g - fd) <= tol), np.max(np.abs(g - fd) / tol)
