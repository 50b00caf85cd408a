"""torch.autograd wrappers: differentiable THIIM solves for inverse design.

``build_coeffs(eps_re, eps_im, ...)`` maps a per-cell permittivity to the 28
coefficient arrays (thiim_build_coeffs); its backward is
thiim_build_coeffs_grad (d objective / d Re eps per cell, Im eps held fixed).
``solve(coeffs, n_iters, every)`` runs n_iters THIIM iterations from zero
fields (thiim_iterate) and keeps every `every`-th iterate as a checkpoint; its
backward replays each segment from its checkpoint and reverses it with
thiim_adjoint_iterate, so memory holds N/every checkpoints plus one segment.
``solve_steady(coeffs, tol)`` iterates until the residual reaches tol; its
backward is the steady-state adjoint (thiim_adjoint_steady), the gradient of
the converged solution, with no checkpoints.
All run entirely in libthiim.so kernels; torch only owns the tensors.
Gradients follow torch's complex convention (2 dJ/dconj(z) for complex z).
"""
from __future__ import annotations

import torch

from . import thiim as T


class _BuildCoeffs(torch.autograd.Function):
    @staticmethod
    def forward(fctx, eps_re, eps_im, ctx, sig_e, sig_h, omega, tau, k_s, amp):
        eps = torch.complex(eps_re.detach().to(torch.float64), eps_im.detach().to(torch.float64)).contiguous()
        co = [torch.empty_like(eps) for _ in range(28)]
        T.thiim_build_coeffs(ctx, eps, sig_e, sig_h, omega, tau, k_s, amp, co)
        fctx.save_for_backward(eps)
        fctx.args = (ctx, sig_e, omega, tau, k_s, amp)
        return tuple(co)

    @staticmethod
    def backward(fctx, *grads):
        (eps,) = fctx.saved_tensors
        ctx, sig_e, omega, tau, k_s, amp = fctx.args
        g = [(gi if gi is not None else torch.zeros_like(eps)).contiguous() for gi in grads]
        out = torch.empty(eps.shape, dtype=torch.float64, device=eps.device)
        T.thiim_build_coeffs_grad(ctx, eps, sig_e, omega, tau, k_s, amp, g, out)
        return out, None, None, None, None, None, None, None, None


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, n_iters, every, *coeffs):
        co = [c.detach().contiguous() for c in coeffs]
        T.thiim_set_coeffs(ctx, co)
        x = [torch.zeros_like(co[0]) for _ in range(12)]
        T.thiim_set_fields(ctx, x)
        ckpts, lens = [], []
        done = 0
        while done < n_iters:
            seg = min(every, n_iters - done)
            ckpts.append([t.clone() for t in x])
            lens.append(seg)
            T.thiim_iterate(ctx, seg)
            done += seg
        fctx.ctx, fctx.co, fctx.ckpts, fctx.lens = ctx, co, ckpts, lens
        return tuple(x)

    @staticmethod
    def backward(fctx, *grads):
        ctx, co = fctx.ctx, fctx.co
        T.thiim_set_coeffs(ctx, co)
        lam = [(g if g is not None else torch.zeros_like(co[0])).clone().contiguous() for g in grads]
        gco = [torch.zeros_like(co[0]) for _ in range(28)]
        for ck, n in zip(reversed(fctx.ckpts), reversed(fctx.lens)):
            T.thiim_adjoint_iterate(ctx, lam, gco, ck, n)
        return (None, None, None, *gco)


class _SolveSteady(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, tol, max_iters, check_every, adj_tol, *coeffs):
        co = [c.detach().contiguous() for c in coeffs]
        T.thiim_set_coeffs(ctx, co)
        x = [torch.zeros_like(co[0]) for _ in range(12)]
        T.thiim_set_fields(ctx, x)
        done, res = 0, float("inf")
        while done < max_iters and not res <= tol:
            n = min(check_every, max_iters - done)
            T.thiim_iterate(ctx, n)
            done += n
            res = T.thiim_residual(ctx)
        fctx.ctx, fctx.co, fctx.x = ctx, co, [t.clone() for t in x]
        fctx.args = (max_iters, check_every, adj_tol)
        fctx.info = {"iterations": done, "residual": res}
        return tuple(x)

    @staticmethod
    def backward(fctx, *grads):
        ctx, co = fctx.ctx, fctx.co
        max_iters, check_every, adj_tol = fctx.args
        T.thiim_set_coeffs(ctx, co)
        lam = [(g if g is not None else torch.zeros_like(co[0])).clone().contiguous() for g in grads]
        gco = [torch.zeros_like(co[0]) for _ in range(28)]
        T.thiim_adjoint_steady(ctx, lam, gco, fctx.x, max_iters, check_every, adj_tol)
        return (None, None, None, None, None, *gco)


class Differentiable:
    """A THIIM_C128 context with differentiable coefficient building and solving."""

    def __init__(self, nx, ny, nz, bc=T.THIIM_PERIODIC_X | T.THIIM_PERIODIC_Y, stream=None):
        self.ctx = T.thiim_create(nx, ny, nz, T.THIIM_C128, bc, stream)

    def build_coeffs(self, eps_re, eps_im, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp=1.0):
        return _BuildCoeffs.apply(eps_re, eps_im, self.ctx, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp)

    def solve(self, coeffs, n_iters, every=20):
        if every > 64:
            raise ValueError("checkpoint interval above the library's segment limit (64)")
        return _Solve.apply(self.ctx, int(n_iters), int(every), *coeffs)

    def solve_steady(self, coeffs, tol=1e-10, max_iters=1000000, check_every=500, adjoint_tol=None):
        """Iterate from zero until the residual is <= tol (or max_iters); the backward
        pass is the steady-state adjoint (thiim_adjoint_steady), i.e. the gradient of
        the fixed point, valid once the forward solve has converged."""
        return _SolveSteady.apply(self.ctx, float(tol), int(max_iters), int(check_every),
                                  float(tol if adjoint_tol is None else adjoint_tol), *coeffs)

    def close(self):
        if self.ctx:
            T.thiim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
