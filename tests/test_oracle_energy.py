"""Pin P6: discrete energy balance at the oracle's fixed point (no GPU).

Away from sources and absorbing layers the fixed point of the iteration
satisfies, with omega_t = 2 sin(omega tau / 2) / tau (Eqs. 3-5 with E and H
stationary),
    i omega_t H = -curl^- E,      (i omega_t eps + sigma e^{+-i omega tau/2}) E = curl^+ H
(the sign of the phase is + where eps > 0, Eq. 3, and - where eps < 0, Eq. 5).
Summing conj(E) . curl^+ H - H . curl^- conj(E) over a slab of whole x-y
planes (periodic in x, y) and summing by parts in z leaves only the two
faces, so
    Re [F(k0) - F(k1 + 1)] = cos(omega tau / 2) * sum_{slab} sigma |E|^2,
    F(k) = sum_{i,j} conj(E_x(k-1)) H_y(k) - conj(E_y(k-1)) H_x(k)
(H plane k sits at z = k - 1/2; the slab holds E and H planes k0 .. k1).
This is an identity of the discrete equations, independent of the oracle's
loops, so the oracle's converged field must satisfy it to the convergence
error; the factor cos(omega tau / 2) (the phase of the loss term) is part of
it, and dropping it fails.  The same identity gives the incident power of the
discrete plane wave, 1/2 Re F = 1/2 |A|^2 sin(kappa) / omega_t per face.
"""
import math

import numpy as np

import oracle
from oracle.coeffs import absorbed_power, build_coeffs, incident_wave
from workloads.thiim_workloads import LayeredStack


def _full(f):
    return [f[2 * c] + f[2 * c + 1] for c in range(6)]


def _solve(st, tfsf, tol=1e-13, chunk=2500, max_iter=300000):
    """Iterate until one iteration changes the full fields by <= tol relative (the
    split parts alone never settle where sigma* = 0)."""
    co = build_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=tfsf)
    f = [np.zeros((st.nz, st.ny, st.nx), np.complex128) for _ in range(12)]
    done = 0
    while done < max_iter:
        oracle.iterate(f, co, chunk - 1, bc=3)
        before = _full(f)
        oracle.iterate(f, co, 1, bc=3)
        done += chunk
        after = _full(f)
        num = sum(float(np.sum(np.abs(a - b) ** 2)) for a, b in zip(after, before))
        den = sum(float(np.sum(np.abs(a) ** 2)) for a in after)
        if math.sqrt(num / den) <= tol:
            return f
    raise AssertionError("oracle did not converge")


def _flux(f, k):
    ex, ey = f[6] + f[7], f[8] + f[9]
    hx, hy = f[0] + f[1], f[2] + f[3]
    return complex(np.sum(np.conj(ex[k - 1]) * hy[k] - np.conj(ey[k - 1]) * hx[k]))


def test_discrete_energy_balance_at_the_fixed_point():
    # 10-cell absorbing layers: E planes 11..21 and H planes 11..21 lie outside
    # both layers and below the source plane (k_s = 8); the slab holds the
    # textured absorber.
    st = LayeredStack(4, 4, 32, amp=2.0, seed=11, pml_cells=10)
    k0, k1 = 11, 21
    assert np.all(st.sigma_pml_e()[k0:k1 + 1] == 0) and np.all(st.sigma_pml_h()[k0:k1 + 1] == 0)
    for tfsf in ((st.k_s, 1.0), (st.k_s, 0.3 - 0.2j, 0.7 + 0.4j)):
        f = _solve(st, tfsf)
        sigma = st.omega * st.eps().imag
        mask = np.zeros(sigma.shape, bool)
        mask[k0:k1 + 1] = True
        loss = 2.0 * absorbed_power(f, sigma * mask)         # sum sigma |E|^2 over the slab
        lhs = (_flux(f, k0) - _flux(f, k1 + 1)).real
        cosf = math.cos(st.omega * st.tau / 2.0)
        assert loss > 0
        assert abs(lhs - cosf * loss) <= 1e-7 * loss, (lhs, cosf * loss)
        # without the phase of the loss term the balance is off by 1 - cos(omega tau / 2)
        assert not (abs(lhs - loss) <= 1e-7 * loss)


def test_incident_flux_of_the_discrete_plane_wave():
    """1/2 Re F of the incident wave equals 1/2 |A|^2 sin(kappa) / omega_t per cell face."""
    omega, tau, k_s, amp = 2 * math.pi / 20, 0.5, 8, 0.6 - 0.3j
    e_inc, h_inc = incident_wave(omega, tau, k_s, amp)
    wt = 2 * math.sin(omega * tau / 2) / tau
    kappa = 2 * math.asin(wt / 2)
    for k in (9, 13, 20):
        flux = (np.conj(e_inc(k - 1)) * h_inc(k)).real
        assert abs(0.5 * flux - 0.5 * abs(amp) ** 2 * math.sin(kappa) / wt) <= 1e-14


def test_spectrum_incident_power_is_the_plane_wave_flux():
    """The spectrum driver's incident power (product code, host arithmetic)
    equals the discrete plane wave's time-averaged flux over a plane of faces."""
    from paper_1510_05218_gb300.spectrum import incident_power
    for lam, tau, amp in ((20.0, 0.5, 1.0), (33.0, 0.4, 0.3 + 0.7j), (80.0, 0.5, 2.0)):
        omega = 2 * math.pi / lam
        e_inc, h_inc = incident_wave(omega, tau, 5, amp)
        flux = 0.5 * (np.conj(e_inc(9)) * h_inc(10)).real          # one face, E plane 9 / H plane 10
        assert abs(incident_power(omega, tau, 7, 3, amp) - 21 * flux) <= 1e-13 * abs(21 * flux)
