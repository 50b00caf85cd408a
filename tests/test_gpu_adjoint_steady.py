"""GPU steady-state adjoint (thiim_adjoint_steady, Differentiable.solve_steady).

* Against the oracle's adjoint_steady with a fixed number of terms (25), on a
  lossy grid with ragged tiles: lam* and all 28 coefficient gradients within
  1e-10 relative per array (FP64 on both sides; the oracle sums the
  per-term gradient contributions, the GPU evaluates the gradient once on
  the summed lam*, which differs only in rounding).
* Stopping at a tolerance, for a seed g of an objective of the full E
  components (the case in which the sum converges, see include/thiim.h):
  the GPU and the oracle sum the same number of terms (+-1) and agree to
  1e-8.
* End to end on a textured 8x8x32 stack (10-cell absorbing layers): the gradient of the converged
  absorbed power J = 1/2 sum_{absorber} sigma |E|^2 with respect to Re eps
  (solve_steady + build_coeffs backward) agrees with central differences of
  converged solves at 12 absorber cells within |g - fd| <= 1e-4 max(|fd|,
  1e-3 max|fd|).  Forward solves stop at residual 1e-13; with a step of 1e-4
  the difference quotients carry ~1e-8 relative truncation and rounding.
"""
import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs
from tests.gpu_util import rel_l2, to_dev, to_host
from workloads import random_fields
from workloads.thiim_workloads import LayeredStack

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _lossy(shape, seed=31):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.5, 3.0, shape) + 1j * rng.uniform(0.2, 0.6, shape)
    S = {n: rng.standard_normal(shape) + 1j * rng.standard_normal(shape) for n in ("Hxy", "Hyx", "Exy", "Eyx")}
    return build_coeffs(eps, np.zeros(nz), np.zeros(nz), 2 * np.pi / 6, 0.5, S=S)


def _gpu_steady(p, co, x_star, g, max_iters, check_every, tol):
    nz, ny, nx = co[0].shape
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C128, 3)
    try:
        cd = to_dev(co)
        p.thiim_set_coeffs(ctx, cd)
        lam = to_dev(g)
        gco = to_dev([np.zeros_like(co[0]) for _ in range(28)])
        xs = to_dev(x_star)
        k, rel = p.thiim_adjoint_steady(ctx, lam, gco, xs, max_iters, check_every, tol)
        out = to_host(lam), to_host(gco), k, rel
        assert all(np.array_equal(a, b) for a, b in zip(to_host(xs), x_star))   # x* is read only
        return out
    finally:
        p.thiim_destroy(ctx)


def test_steady_adjoint_matches_oracle_fixed_terms():
    p = _lib()
    shape = (6, 9, 35)
    co = _lossy(shape)
    nz, ny, nx = shape
    x_star = random_fields(nx, ny, nz, seed=32)
    g = random_fields(nx, ny, nz, seed=33)
    lam_g, grad_g, k, _ = _gpu_steady(p, co, x_star, g, 25, 5, 0.0)
    lam_o, grad_o, k_o, _ = oracle.adjoint_steady(g, x_star, co, bc=3, max_iters=25)
    assert k == k_o == 25
    for s in range(12):
        assert rel_l2(lam_g[s], lam_o[s]) <= 1e-10, oracle.SPLITS[s]
    for a in range(28):
        assert rel_l2(grad_g[a], grad_o[a]) <= 1e-10, oracle.COEFF_NAMES[a]


def test_steady_adjoint_stops_at_tolerance_like_the_oracle():
    p = _lib()
    shape = (5, 8, 12)
    co = _lossy(shape, seed=41)
    nz, ny, nx = shape
    x_star = random_fields(nx, ny, nz, seed=42)
    # g of an objective of the full E components: equal on the two splits of
    # each E component, zero on H (the case in which the sum converges)
    r = random_fields(nx, ny, nz, seed=43)
    g = [np.zeros(shape, np.complex128) for _ in range(6)] + [r[c // 2].copy() for c in range(6)]
    lam_g, grad_g, k, rel = _gpu_steady(p, co, x_star, g, 20000, 1, 1e-9)
    lam_o, grad_o, k_o, rel_o = oracle.adjoint_steady(g, x_star, co, bc=3, max_iters=20000, tol=1e-9)
    assert rel <= 1e-9 and rel_o <= 1e-9 and abs(k - k_o) <= 1 and k < 20000
    for s in range(12):
        assert rel_l2(lam_g[s], lam_o[s]) <= 1e-8, oracle.SPLITS[s]
    for a in range(28):
        assert rel_l2(grad_g[a], grad_o[a]) <= 1e-8, oracle.COEFF_NAMES[a]


def test_steady_adjoint_argument_errors():
    p = _lib()
    ctx = p.thiim_create(4, 4, 4, p.THIIM_C64, 3)
    try:
        with pytest.raises(p.ThiimError) as e:      # complex128 only
            p.thiim_adjoint_steady(ctx, [16] * 12, [16] * 28, [16] * 12, 10)
        assert e.value.code == -1
    finally:
        p.thiim_destroy(ctx)
    ctx = p.thiim_create(4, 4, 4, p.THIIM_C128, 3)
    try:
        with pytest.raises(p.ThiimError) as e:      # no coefficients yet
            p.thiim_adjoint_steady(ctx, [16] * 12, [16] * 28, [16] * 12, 10)
        assert e.value.code == -3
        co = to_dev(_lossy((4, 4, 4)))
        p.thiim_set_coeffs(ctx, co)
        for bad in ((0, 1, 0.0), (5, 0, 0.0), (5, 1, -1.0), (5, 1, float("nan"))):
            with pytest.raises(p.ThiimError) as e:
                p.thiim_adjoint_steady(ctx, [16] * 12, [16] * 28, [16] * 12, *bad)
            assert e.value.code == -1
    finally:
        p.thiim_destroy(ctx)


def test_converged_absorption_gradient_matches_finite_differences():
    import torch
    p = _lib()
    from paper_1510_05218_gb300.autograd import Differentiable
    # 10-cell absorbing layers: the residual reaches 1e-13 in ~45k iterations
    # (6-cell layers need >150k: a weakly damped mode between them)
    st = LayeredStack(nx=8, ny=8, nz=32, amp=2.0, seed=11, pml_cells=10)
    eps = st.eps()
    mask = st.absorber_mask()
    sig_d = torch.from_numpy(st.omega * eps.imag * mask).to("cuda")
    args = (st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0)
    tol = 1e-13

    def objective(x):
        e2 = sum((x[2 * c] + x[2 * c + 1]).abs() ** 2 for c in (3, 4, 5))
        return 0.5 * torch.sum(sig_d * e2)

    dmod = Differentiable(st.nx, st.ny, st.nz)
    p.thiim_set_tuning(dmod.ctx, 1, 2)     # 2 planes per CTA: 16 CTAs for this small grid
    try:
        eps_re = torch.from_numpy(eps.real.copy()).to("cuda").requires_grad_(True)
        eps_im = torch.from_numpy(eps.imag.copy()).to("cuda")
        co = dmod.build_coeffs(eps_re, eps_im, *args)
        x = dmod.solve_steady(co, tol=tol, max_iters=200000, check_every=2500)
        J = objective(x)
        J.backward()
        grad = eps_re.grad.detach().cpu().numpy()

        def J_at(e_re):
            with torch.no_grad():
                c2 = dmod.build_coeffs(e_re, eps_im, *args)
                return float(objective(dmod.solve_steady(c2, tol=tol, max_iters=200000, check_every=2500)))

        cells = np.argwhere(mask)
        rng = np.random.default_rng(3)
        cells = cells[rng.choice(len(cells), 12, replace=False)]
        h = 1e-4
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
    finally:
        dmod.close()
    tolv = 1e-4 * np.maximum(np.abs(fd), 1e-3 * np.max(np.abs(fd)))
    assert np.all(np.abs(g - fd) <= tolv), np.max(np.abs(g - fd) / tolv)
