"""ctypes front end of the C oracle (test infrastructure only).

Arrays are NumPy complex128, C-contiguous, shape (nz, ny, nx): the layout of
the paper's listings (x fastest).  Updates happen in place.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

SPLITS = ["Hxy", "Hxz", "Hyx", "Hyz", "Hzx", "Hzy", "Exy", "Exz", "Eyx", "Eyz", "Ezx", "Ezy"]
FIELD_INDEX = {n: i for i, n in enumerate(SPLITS)}
COEFF_NAMES = (["t" + s for s in SPLITS] + ["c" + s for s in SPLITS]
               + ["SrcHxy", "SrcHyx", "SrcExy", "SrcEyx"])

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.oracle_iterate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                       pp, pp, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]
        lib.oracle_iterate.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_rule.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip]
        lib.oracle_rule.restype = ctypes.c_int
        lib.oracle_adjoint_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint, pp, pp, pp, pp, pp]
        lib.oracle_adjoint_step.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptrs(arrays, shape):
    out = (ctypes.c_void_p * len(arrays))()
    for n, a in enumerate(arrays):
        if a.dtype != np.complex128 or not a.flags.c_contiguous or a.shape != shape:
            raise ValueError("oracle arrays must be C-contiguous complex128 of shape %s" % (shape,))
        out[n] = a.ctypes.data
    return out


def iterate(fields, coeffs, n: int, bc: int = 3, nthreads: int = 1) -> float:
    """Run n THIIM iterations in place; return ||x^n - x^{n-1}|| / ||x^n|| (FP64).

    bc: bit 0 periodic x, bit 1 periodic y, bit 2 periodic z (else zero outside).
    """
    lib = _load()
    if len(fields) != 12 or len(coeffs) != 28:
        raise ValueError("need 12 field and 28 coefficient arrays")
    shape = fields[0].shape
    nz, ny, nx = shape
    fp = _ptrs(fields, shape)
    cp = _ptrs(coeffs, shape)
    rel = ctypes.c_double(0.0)
    rc = lib.oracle_iterate(nx, ny, nz, bc, fp, cp, int(n), int(nthreads), ctypes.byref(rel))
    if rc != 0:
        raise ValueError("oracle_iterate rejected its arguments")
    return rel.value


def rule(s: int):
    """(direction, src_a, src_b, sign, src_array) of split s: direction 0=x, 1=y, 2=z."""
    lib = _load()
    v = [ctypes.c_int() for _ in range(5)]
    if lib.oracle_rule(s, *[ctypes.byref(x) for x in v]) != 0:
        raise ValueError(s)
    return tuple(x.value for x in v)


def adjoint_step(lam, grad, x_n, x_np1, coeffs, bc: int = 3) -> None:
    """Reverse one iteration in place: lam (12 arrays) goes from the adjoint of
    x^{n+1} to that of x^n; grad (28 arrays) accumulates the coefficient
    gradients.  x_n, x_np1: the forward iterates n and n+1."""
    lib = _load()
    shape = lam[0].shape
    nz, ny, nx = shape
    rc = lib.oracle_adjoint_step(nx, ny, nz, bc, _ptrs(lam, shape), _ptrs(grad, shape), _ptrs(x_n, shape),
                                 _ptrs(x_np1, shape), _ptrs(coeffs, shape))
    if rc != 0:
        raise ValueError("oracle_adjoint_step failed (%d)" % rc)


def adjoint_steady(g, x_star, coeffs, bc: int = 3, max_iters: int = 100000, tol: float = 0.0):
    """Steady-state adjoint at a fixed point x* = F(x*) of the iteration.

    The gradient of J(x*) with respect to the coefficients is (dF/da)^H lam*
    where lam* = M^H lam* + g solves the adjoint fixed point (M the linear
    part of one iteration, g the gradient of J with respect to conj(x*)).
    Written as the reverse iteration of adjoint_step with every state equal
    to x*: lam* = sum_k (M^H)^k g and the gradient is the sum of the per-step
    contributions.  Terms are added until max_iters have been summed or the
    last one is <= tol times the sum (norms over all 12 arrays).
    Returns (lam*, grad (28 arrays), terms summed, |last term| / |lam*|).
    """
    shape = g[0].shape
    lam = [np.array(a, np.complex128) for a in g]
    total = [np.zeros(shape, np.complex128) for _ in range(12)]
    grad = [np.zeros(shape, np.complex128) for _ in range(28)]
    k, rel = 0, float("inf")
    while k < max_iters:
        term = np.sqrt(sum(float(np.vdot(a, a).real) for a in lam))
        for s, a in zip(total, lam):
            s += a
        adjoint_step(lam, grad, x_star, x_star, coeffs, bc)
        k += 1
        tot = np.sqrt(sum(float(np.vdot(a, a).real) for a in total))
        rel = term / tot if tot > 0 else 0.0
        if tol > 0 and rel <= tol:
            break
    return total, grad, k, rel
