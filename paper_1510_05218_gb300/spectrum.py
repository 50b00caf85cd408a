"""Absorption spectrum of one structure: one THIIM solve per wavelength and
polarisation, all advanced together by the batched kernel.

The paper's workload is many runs of the same code: covering the visible
spectrum for one solar-cell configuration takes 80-160 simulations (Sec. V).
Here each (wavelength, polarisation) pair is a solve with its own context;
their coefficients are built on the GPU (thiim_build_coeffs_jones), they
iterate together in thiim_batch_iterate, and each reports its absorbed power
(thiim_absorbed_power).  The absorption is the power dissipated in the
absorber over the incident power, and the unpolarised absorption is the mean
over the x- and y-polarised runs.

Dissipated power: at the fixed point the loss term of Eqs. 3 and 5 carries the
phase e^{+-i omega tau / 2}, so the discrete Poynting balance of a slab reads
Re(flux in - flux out) = cos(omega tau / 2) sum sigma |E|^2 (an identity of
the discrete equations); the power dissipated is cos(omega tau / 2) times
P = 1/2 sum sigma |E|^2.

Incident power: the discrete plane wave E_x(k) = A e^{-i kappa k},
H_y = -dE_x/(i omega_t) (2 sin(kappa/2) = omega_t = 2 sin(omega tau/2)/tau)
carries the time-averaged flux 1/2 Re(E_x conj(H_y)) = |A|^2 sin(kappa) /
(2 omega_t) per unit cell face, which tends to |A|^2 / 2 as the cell
shrinks; over the nx * ny faces of a plane it is the incident power.
"""
from __future__ import annotations

import math

from . import thiim as T

POLARISATIONS = {"x": (1.0, 0.0), "y": (0.0, 1.0)}


def incident_power(omega: float, tau: float, nx: int, ny: int, amp: complex = 1.0) -> float:
    wt = 2.0 * math.sin(omega * tau / 2.0) / tau
    kappa = 2.0 * math.asin(wt / 2.0)
    return 0.5 * abs(amp) ** 2 * math.sin(kappa) / wt * nx * ny


def absorption_spectrum(eps, lambdas, sigma_pml_e, sigma_pml_h, k_s, tau, absorber, precision=T.THIIM_C128_PAIR,
                        max_iters=4000, check_every=50, tol=1e-6, polarisations=("x", "y"), bc=3, stream=None,
                        device=None):
    """Absorption of the cells in `absorber` for every wavelength and polarisation.

    eps:       (nz, ny, nx) complex relative permittivity (physics convention),
               or a callable lam -> such an array (dispersive materials).
    lambdas:   free-space wavelengths in cells (omega = 2 pi / lam).
    absorber:  bool (nz, ny, nx) mask; the absorbed power counts
               sigma = omega Im(eps) on these cells only.
    The solves stop at relative residual `tol` or after `max_iters`
    iterations (thiim_batch_iterate).  Returns a dict with the wavelengths,
    "A" = {polarisation: [absorption per wavelength]}, "A_unpolarised" (the
    mean over the polarisations), and per solve the iterations run and the
    last residual.
    """
    import numpy as np
    import torch

    dev = torch.device(device or "cuda")
    mask = np.asarray(absorber, bool)
    nz, ny, nx = mask.shape
    dt = torch.complex64 if precision == T.THIIM_C64 else torch.complex128
    solves = []
    try:
        for lam in lambdas:
            omega = 2.0 * math.pi / lam
            e = np.asarray(eps(lam) if callable(eps) else eps, np.complex128)
            eps_d = torch.from_numpy(np.ascontiguousarray(e)).to(dev)
            sigma_d = torch.from_numpy(np.ascontiguousarray(omega * e.imag * mask)).to(dev)
            for pol in polarisations:
                ctx = T.thiim_create(nx, ny, nz, precision, bc, stream)
                co = [torch.empty((nz, ny, nx), dtype=dt, device=dev) for _ in range(28)]
                fields = [torch.zeros((nz, ny, nx), dtype=dt, device=dev) for _ in range(12)]
                solves.append({"ctx": ctx, "co": co, "fields": fields, "sigma": sigma_d, "lam": lam,
                               "omega": omega, "pol": pol})
                ax, ay = POLARISATIONS[pol]
                T.thiim_build_coeffs_jones(ctx, eps_d, sigma_pml_e, sigma_pml_h, omega, tau, k_s, ax, ay, co)
                T.thiim_set_coeffs(ctx, co)
                T.thiim_set_fields(ctx, fields)
        iters, res = T.thiim_batch_iterate([s["ctx"] for s in solves], max_iters, check_every, tol)
        out = {"lambdas": list(lambdas), "A": {p: [] for p in polarisations}, "iterations": list(iters),
               "residuals": list(res), "power": []}
        for s in solves:
            p_abs = T.thiim_absorbed_power(s["ctx"], s["sigma"])
            out["power"].append(p_abs)
            dissipated = math.cos(s["omega"] * tau / 2.0) * p_abs
            out["A"][s["pol"]].append(dissipated / incident_power(s["omega"], tau, nx, ny))
        out["A_unpolarised"] = [sum(out["A"][p][i] for p in polarisations) / len(polarisations)
                                for i in range(len(lambdas))]
        return out
    finally:
        for s in solves:
            T.thiim_destroy(s["ctx"])
