"""Oracle coefficient arrays from Eqs. 3-5 (test infrastructure only).

Each split update has the form x <- t x + Src + sign * c * D(F).  Solving the
paper's discrete equations for the new value gives, with tau the pseudo time
step, omega the frequency and e(a) = exp(i a):

  H (Eq. 4):          t = e(-w tau/2) / (e(w tau/2) + tau sig*/mu)
                      c = tau / (mu (e(w tau/2) + tau sig*/mu))
                      Src = tau S_H / (e(w tau/2) + tau sig*/mu)
  E, eps > 0 (Eq. 3): t = e(-w tau) / (1 + tau sig/eps)
                      c = tau e(-w tau/2) / (eps + tau sig)
                      Src = tau e(-w tau) S_E / (1 + tau sig/eps)
  E, eps < 0 (Eq. 5): t = e(+w tau) / (1 - tau sig/eps)
                      c = -tau e(+w tau/2) / (eps - tau sig)
                      Src = -tau S_E / (1 - tau sig/eps)

The curl sign of each split is applied by the sweep, not stored in c.

Split conductivities (Berenger split field, Eqs. 6-7): every E split carries
the material conductivity sig_mat = omega * Im(eps_r) (the permittivity is
given in the physics convention, Im > 0 lossy, while the paper's fields vary
as e^{+i omega t}); the splits whose difference runs along z (Hxy, Hyx, Exy,
Eyx) also carry the absorbing-layer conductivity of their z position (E at k,
H at k - 1/2).  mu = 1; sig*_mat is zero unless given.

Plane-wave source (total-field/scattered-field plane at k_s, normal
incidence): the incident wave solves the discrete equations in air,
E_x(k) = A e(-kappa (k - k_s)) with 2 sin(kappa/2) = omega_t, where
omega_t = 2 sin(omega tau / 2) / tau is the discrete frequency that the fixed
point of Eqs. 3-4 carries, and H_y(k) = -(E_x(k) - E_x(k-1)) / (i omega_t).
H planes with index <= k_s are scattered field, E planes >= k_s are total
field, so H_yx(k_s) reads the incident E_x(k_s) across the plane and
E_xy(k_s) reads the incident H_y(k_s):
  SrcHyx(k_s) = -sign(Hyx) c_Hyx(k_s) E_inc(k_s),
  SrcExy(k_s) = -sign(Exy) c_Exy(k_s) H_inc(k_s).
The y-polarised wave (E_y, H_x) follows from the same curl with the other
two z-difference splits: H_x(k) = +(E_y(k) - E_y(k-1)) / (i omega_t), and
  SrcHxy(k_s) = -sign(Hxy) c_Hxy(k_s) E_y,inc(k_s),
  SrcEyx(k_s) = -sign(Eyx) c_Eyx(k_s) H_x,inc(k_s).
A general polarisation (Jones vector (A_x, A_y)) is the sum of the two.
"""
from __future__ import annotations

import math

import numpy as np

from .thiim_oracle import rule, SPLITS

SRC_SPLITS = {"Hxy": 24, "Hyx": 25, "Exy": 26, "Eyx": 27}


def discrete_omega(omega: float, tau: float) -> float:
    """omega_t = 2 sin(omega tau / 2) / tau."""
    return 2.0 * math.sin(omega * tau / 2.0) / tau


def incident_wave(omega: float, tau: float, k_s: int, amp: complex = 1.0, pol: str = "x"):
    """(E_inc(k), H_inc(k)) callables of the discrete plane wave in air:
    pol "x": (E_x, H_y), H_y = -dE/(i omega_t); pol "y": (E_y, H_x), H_x = +dE/(i omega_t)."""
    wt = discrete_omega(omega, tau)
    kappa = 2.0 * math.asin(wt / 2.0)
    sgn = -1.0 if pol == "x" else 1.0

    def e_inc(k):
        return amp * np.exp(-1j * kappa * (np.asarray(k, dtype=np.float64) - k_s))

    def h_inc(k):
        return sgn * (e_inc(k) - e_inc(np.asarray(k) - 1)) / (1j * wt)

    return e_inc, h_inc


def build_coeffs(eps_r, sigma_pml_e, sigma_pml_h, omega, tau, tfsf=None, S=None, sigma_star=None):
    """28 coefficient arrays (t[12], c[12], SrcHxy, SrcHyx, SrcExy, SrcEyx).

    eps_r: (nz, ny, nx) complex relative permittivity per cell (physics convention).
    sigma_pml_e / sigma_pml_h: (nz,) absorbing conductivity at E / H planes.
    tfsf: optional (k_s, amplitude) of the x-polarised plane-wave source, or
       (k_s, A_x, A_y) for a general polarisation (Jones vector).
    S: optional dict {"Hxy"|"Hyx"|"Exy"|"Eyx": array} of physical sources
       S_H / S_E of Eqs. 3-5 on the four source splits.
    sigma_star: optional (nz, ny, nx) magnetic conductivity of the material
       (Eq. 2), added to every H split; zero by default.
    """
    eps_r = np.asarray(eps_r, np.complex128)
    nz, ny, nx = eps_r.shape
    eps = eps_r.real
    sig_mat = omega * eps_r.imag
    sz_e = np.asarray(sigma_pml_e, np.float64)[:, None, None]
    sz_h = np.asarray(sigma_pml_h, np.float64)[:, None, None]
    ph = lambda a: np.exp(1j * a)  # noqa: E731
    mu = 1.0
    t = [None] * 12
    c = [None] * 12
    src_scale = [None] * 12
    for s in range(12):
        d, _, _, _, _ = rule(s)
        if s < 6:  # H splits, Eq. 4
            sig_star = np.broadcast_to(sz_h if d == 2 else 0.0, eps.shape)
            if sigma_star is not None:
                sig_star = sig_star + np.asarray(sigma_star, np.float64)
            den = ph(omega * tau / 2.0) + tau * sig_star / mu
            t[s] = ph(-omega * tau / 2.0) / den
            c[s] = tau / (mu * den)
            src_scale[s] = tau / den
        else:      # E splits, Eq. 3 or Eq. 5
            sig = sig_mat + (sz_e if d == 2 else 0.0)
            fwd = eps > 0
            t_f = ph(-omega * tau) / (1.0 + tau * sig / eps)
            c_f = tau * ph(-omega * tau / 2.0) / (eps + tau * sig)
            s_f = tau * ph(-omega * tau) / (1.0 + tau * sig / eps)
            t_b = ph(omega * tau) / (1.0 - tau * sig / eps)
            c_b = -tau * ph(omega * tau / 2.0) / (eps - tau * sig)
            s_b = -tau / (1.0 - tau * sig / eps)
            t[s] = np.where(fwd, t_f, t_b)
            c[s] = np.where(fwd, c_f, c_b)
            src_scale[s] = np.where(fwd, s_f, s_b)
    srcs = {name: np.zeros((nz, ny, nx), np.complex128) for name in SRC_SPLITS}
    if S is not None:
        for name, arr in S.items():
            s = SPLITS.index(name)
            srcs[name] = srcs[name] + src_scale[s] * np.asarray(arr, np.complex128)
    if tfsf is not None:
        k_s = tfsf[0]
        amps = {"x": tfsf[1], "y": tfsf[2] if len(tfsf) > 2 else 0.0}
        for pol, h_name, e_name in (("x", "Hyx", "Exy"), ("y", "Hxy", "Eyx")):
            if amps[pol] == 0:
                continue
            e_inc, h_inc = incident_wave(omega, tau, k_s, amps[pol], pol)
            s_h = SPLITS.index(h_name)
            s_e = SPLITS.index(e_name)
            sign_h = rule(s_h)[3]
            sign_e = rule(s_e)[3]
            srcs[h_name][k_s] += -sign_h * c[s_h][k_s] * e_inc(k_s)
            srcs[e_name][k_s] += -sign_e * c[s_e][k_s] * h_inc(k_s)
    out = [np.ascontiguousarray(np.broadcast_to(a, (nz, ny, nx)).astype(np.complex128)) for a in t + c]
    out += [srcs[n] for n in ("Hxy", "Hyx", "Exy", "Eyx")]
    return out


def absorbed_power(fields, sigma):
    """1/2 sum over cells of sigma |E|^2, E = the full E components (split sums)."""
    e2 = sum(np.abs(fields[2 * a] + fields[2 * a + 1]) ** 2 for a in (3, 4, 5))
    return 0.5 * float(np.sum(np.asarray(sigma, np.float64) * e2))


def stack_coeffs(stack):
    """Coefficients of a workloads.LayeredStack with its plane-wave source."""
    return build_coeffs(stack.eps(), stack.sigma_pml_e(), stack.sigma_pml_h(),
                        stack.omega, stack.tau, tfsf=(stack.k_s, 1.0))


def coeff_eps_derivatives(eps_r, sigma_pml_e, omega, tau, tfsf=None):
    """d(coefficient)/d(Re eps) for the arrays that depend on the permittivity.

    Returns {array index: derivative array} for t and c of the six E splits
    and, with a plane-wave source, SrcExy (proportional to c_Exy at k_s).
    Differentiating the E coefficients of Eqs. 3 and 5 with sigma held fixed:
      eps > 0:  dt/deps = e(-w tau) (tau sig / eps^2) / (1 + tau sig/eps)^2
                dc/deps = -tau e(-w tau/2) / (eps + tau sig)^2
      eps < 0:  dt/deps = -e(+w tau) (tau sig / eps^2) / (1 - tau sig/eps)^2
                dc/deps = tau e(+w tau/2) / (eps - tau sig)^2
    """
    eps_r = np.asarray(eps_r, np.complex128)
    eps = eps_r.real
    sig_mat = omega * eps_r.imag
    sz_e = np.asarray(sigma_pml_e, np.float64)[:, None, None]
    ph = lambda a: np.exp(1j * a)  # noqa: E731
    out = {}
    for s in range(6, 12):
        d = rule(s)[0]
        sig = sig_mat + (sz_e if d == 2 else 0.0)
        fwd = eps > 0
        dt_f = ph(-omega * tau) * (tau * sig / eps ** 2) / (1.0 + tau * sig / eps) ** 2
        dc_f = -tau * ph(-omega * tau / 2.0) / (eps + tau * sig) ** 2
        dt_b = -ph(omega * tau) * (tau * sig / eps ** 2) / (1.0 - tau * sig / eps) ** 2
        dc_b = tau * ph(omega * tau / 2.0) / (eps - tau * sig) ** 2
        out[s] = np.where(fwd, dt_f, dt_b)
        out[12 + s] = np.where(fwd, dc_f, dc_b)
    if tfsf is not None:
        k_s, amp = tfsf
        _, h_inc = incident_wave(omega, tau, k_s, amp)
        s_e = SPLITS.index("Exy")
        dsrc = np.zeros(eps.shape, np.complex128)
        dsrc[k_s] = -rule(s_e)[3] * out[12 + s_e][k_s] * h_inc(k_s)
        out[26] = dsrc
    return out
