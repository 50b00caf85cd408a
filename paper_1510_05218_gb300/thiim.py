"""ctypes binding of the THIIM C ABI (include/thiim.h), same names as the C calls.

Tensors are torch CUDA tensors (complex128 for THIIM_C128, complex64 for
THIIM_C64), contiguous, in the layout (nz, ny, nx) with x fastest.  Only their
data pointers cross the ABI.  Errors raise ThiimError with the library's code.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

THIIM_C128 = 0
THIIM_C64 = 1
THIIM_C128_PAIR = 2
THIIM_PERIODIC_X = 1
THIIM_PERIODIC_Y = 2
THIIM_PERIODIC_Z = 4
THIIM_MAX_MATERIALS = 256
THIIM_INT_ADD = 1
THIIM_INT_MUL = 2
THIIM_INT_SUMS = 4

_HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "thiim.h")
_lib = None


class ThiimError(RuntimeError):
    def __init__(self, call, code):
        self.code = code
        msg = "unknown"
        if _lib is not None:
            msg = _lib.thiim_strerror(code).decode()
        super().__init__("%s failed: %s (%d)" % (call, msg, code))


def lib_path() -> str:
    return os.environ.get("THIIM_LIBRARY") or _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libthiim.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("libthiim.so is not built (%s); run __graft_entry__.build() or "
                               "python paper_1510_05218_gb300/build.py" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    P28 = vp * 28
    P12 = vp * 12
    lib.thiim_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_uint, vp]
    lib.thiim_set_stream.argtypes = [vp, vp]
    lib.thiim_set_tuning.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.thiim_set_fp64_int_ops.argtypes = [vp, ctypes.c_uint]
    lib.thiim_set_fp64_int_ops.restype = ctypes.c_int
    lib.thiim_set_coeffs.argtypes = [vp, P28]
    lib.thiim_set_fields.argtypes = [vp, P12]
    lib.thiim_iterate.argtypes = [vp, ctypes.c_int]
    lib.thiim_residual.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.thiim_build_coeffs.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, P28]
    lib.thiim_step_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                       P12, P12, P28, vp, ctypes.POINTER(ctypes.c_double)]
    lib.thiim_step_noalloc.restype = ctypes.c_int
    lib.thiim_mixed_solve.argtypes = [vp, P28, P12, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.thiim_mixed_solve.restype = ctypes.c_int
    lib.thiim_batch_iterate.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double)]
    lib.thiim_batch_iterate.restype = ctypes.c_int
    lib.thiim_adjoint_iterate.argtypes = [vp, P12, P28, P12, ctypes.c_int]
    lib.thiim_adjoint_iterate.restype = ctypes.c_int
    lib.thiim_adjoint_steady.argtypes = [vp, P12, P28, P12, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.thiim_adjoint_steady.restype = ctypes.c_int
    lib.thiim_build_coeffs_grad.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_double, P28, vp]
    lib.thiim_build_coeffs_grad.restype = ctypes.c_int
    lib.thiim_build_material_table.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, vp, vp]
    lib.thiim_build_coeffs_jones.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             vp, P28]
    lib.thiim_build_coeffs_jones.restype = ctypes.c_int
    lib.thiim_absorbed_power.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.thiim_absorbed_power.restype = ctypes.c_int
    lib.thiim_build_material_table.restype = ctypes.c_int
    lib.thiim_set_material_coeffs.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.thiim_set_material_coeffs.restype = ctypes.c_int
    lib.thiim_fp64_pipe_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.thiim_fp64_pipe_rate.restype = ctypes.c_int
    lib.thiim_destroy.argtypes = [vp]
    lib.thiim_destroy.restype = None
    lib.thiim_strerror.argtypes = [ctypes.c_int]
    lib.thiim_strerror.restype = ctypes.c_char_p
    lib.thiim_version.argtypes = []
    for name in ("thiim_create", "thiim_set_stream", "thiim_set_tuning", "thiim_set_coeffs", "thiim_set_fields", "thiim_iterate",
                 "thiim_residual", "thiim_build_coeffs", "thiim_version"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def declared_symbols():
    """Names of the functions declared in include/thiim.h."""
    text = open(_HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(thiim_\w+)\s*\(", text, re.M)))


def exported_symbols():
    """Names of the thiim_* functions the built library exports."""
    lib = load_library()
    return sorted(n for n in declared_symbols() if hasattr(lib, n))


def _check(call, rc):
    if rc != 0:
        raise ThiimError(call, rc)


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _ptrs(tensors, n, kind):
    if len(tensors) != n:
        raise ValueError("need %d %s arrays, got %d" % (n, kind, len(tensors)))
    arr = (ctypes.c_void_p * n)()
    for i, t in enumerate(tensors):
        if hasattr(t, "is_cuda"):
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("%s array %d must be a contiguous CUDA tensor" % (kind, i))
            arr[i] = t.data_ptr()
        else:
            arr[i] = int(t)
    return arr


def thiim_create(nx, ny, nz, precision=THIIM_C128, bc_flags=THIIM_PERIODIC_X | THIIM_PERIODIC_Y, stream=None):
    lib = load_library()
    h = ctypes.c_void_p()
    _check("thiim_create", lib.thiim_create(ctypes.byref(h), int(nx), int(ny), int(nz), int(precision),
                                            int(bc_flags), _stream_ptr(stream)))
    return h


def thiim_set_stream(ctx, stream=None):
    _check("thiim_set_stream", load_library().thiim_set_stream(ctx, _stream_ptr(stream)))


def thiim_set_tuning(ctx, temporal_block=1, zchunk=0):
    _check("thiim_set_tuning", load_library().thiim_set_tuning(ctx, int(temporal_block), int(zchunk)))


def thiim_set_fp64_int_ops(ctx, ops):
    """Binary64 operations of the THIIM_C128 sweep computed on the integer pipe (bit-identical results)."""
    _check("thiim_set_fp64_int_ops", load_library().thiim_set_fp64_int_ops(ctx, int(ops)))


def thiim_set_coeffs(ctx, coeffs):
    _check("thiim_set_coeffs", load_library().thiim_set_coeffs(ctx, _ptrs(coeffs, 28, "coefficient")))


def thiim_set_fields(ctx, fields):
    _check("thiim_set_fields", load_library().thiim_set_fields(ctx, _ptrs(fields, 12, "field")))


def thiim_iterate(ctx, n_iters):
    _check("thiim_iterate", load_library().thiim_iterate(ctx, int(n_iters)))


def thiim_residual(ctx) -> float:
    r = ctypes.c_double()
    _check("thiim_residual", load_library().thiim_residual(ctx, ctypes.byref(r)))
    return r.value


def thiim_build_coeffs(ctx, eps_r, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp, coeffs):
    import numpy as np
    lib = load_library()
    se = None if sigma_pml_e is None else np.ascontiguousarray(sigma_pml_e, dtype=np.float64)
    sh = None if sigma_pml_h is None else np.ascontiguousarray(sigma_pml_h, dtype=np.float64)
    if not (eps_r.is_cuda and eps_r.is_contiguous()):
        raise ValueError("eps_r must be a contiguous CUDA complex128 tensor")
    amp = complex(amp)
    _check("thiim_build_coeffs", lib.thiim_build_coeffs(
        ctx, ctypes.c_void_p(eps_r.data_ptr()),
        None if se is None else se.ctypes.data_as(ctypes.c_void_p),
        None if sh is None else sh.ctypes.data_as(ctypes.c_void_p),
        float(omega), float(tau), int(k_s), amp.real, amp.imag, _ptrs(coeffs, 28, "coefficient")))


def _jones(amp_x, amp_y):
    ax, ay = complex(amp_x), complex(amp_y)
    return (ctypes.c_double * 4)(ax.real, ax.imag, ay.real, ay.imag)


def _host_profile(a):
    import numpy as np
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.c_void_p)


def thiim_build_coeffs_jones(ctx, eps_r, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp_x, amp_y, coeffs):
    """thiim_build_coeffs for the incident wave E = (amp_x, amp_y, 0)."""
    se, se_p = _host_profile(sigma_pml_e)
    sh, sh_p = _host_profile(sigma_pml_h)
    _check("thiim_build_coeffs_jones", load_library().thiim_build_coeffs_jones(
        ctx, _dev_ptr(eps_r, "eps_r"), se_p, sh_p, float(omega), float(tau), int(k_s), _jones(amp_x, amp_y),
        _ptrs(coeffs, 28, "coefficient")))


def thiim_absorbed_power(ctx, sigma) -> float:
    """1/2 sum sigma |E|^2 over the context's current fields (sigma: float64 CUDA tensor)."""
    out = ctypes.c_double()
    _check("thiim_absorbed_power", load_library().thiim_absorbed_power(ctx, _dev_ptr(sigma, "sigma"),
                                                                       ctypes.byref(out)))
    return out.value


def _dev_ptr(t, what):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


def thiim_build_material_table(ctx, eps_mat, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp, table, amp_y=0.0):
    """Fill `table` (CUDA tensor of n_mat * nz * 28 complex values) for the permittivities eps_mat;
    the plane wave is E = (amp, amp_y, 0)."""
    import numpy as np
    em = np.asarray(eps_mat, dtype=np.complex128).ravel()
    eh = np.ascontiguousarray(np.stack([em.real, em.imag], 1).ravel())
    se, se_p = _host_profile(sigma_pml_e)
    sh, sh_p = _host_profile(sigma_pml_h)
    _check("thiim_build_material_table", load_library().thiim_build_material_table(
        ctx, len(em), eh.ctypes.data_as(ctypes.c_void_p), se_p, sh_p,
        float(omega), float(tau), int(k_s), _jones(amp, amp_y), _dev_ptr(table, "table")))


def thiim_set_material_coeffs(ctx, mat, n_mat, table):
    """Use the uint8 material map `mat` and the table in place of the 28 coefficient arrays."""
    _check("thiim_set_material_coeffs", load_library().thiim_set_material_coeffs(
        ctx, _dev_ptr(mat, "mat"), int(n_mat), _dev_ptr(table, "table")))


def thiim_mixed_solve(ctx, coeffs64, x64, inner_iters=50, max_outer=1, tol=0.0):
    """Defect-correction solve; returns (corrections applied, last FP64 residual)."""
    done = ctypes.c_int()
    r = ctypes.c_double()
    _check("thiim_mixed_solve", load_library().thiim_mixed_solve(
        ctx, _ptrs(coeffs64, 28, "coefficient"), _ptrs(x64, 12, "field"), int(inner_iters), int(max_outer),
        float(tol), ctypes.byref(done), ctypes.byref(r)))
    return done.value, r.value


def thiim_adjoint_iterate(ctx, lam, grad_coeffs, checkpoint, n_back):
    """Reverse n_back iterations in place on `lam`, accumulating into `grad_coeffs`."""
    _check("thiim_adjoint_iterate", load_library().thiim_adjoint_iterate(
        ctx, _ptrs(lam, 12, "lambda"), _ptrs(grad_coeffs, 28, "gradient"), _ptrs(checkpoint, 12, "field"),
        int(n_back)))


def thiim_adjoint_steady(ctx, lam, grad_coeffs, x_star, max_iters, check_every=50, tol=0.0):
    """Steady-state adjoint at the fixed point x_star: lam (in: g, out: lam*), gradient added to
    grad_coeffs; returns (terms summed, |last term| / |lam*|)."""
    k = ctypes.c_int()
    r = ctypes.c_double()
    _check("thiim_adjoint_steady", load_library().thiim_adjoint_steady(
        ctx, _ptrs(lam, 12, "lambda"), _ptrs(grad_coeffs, 28, "gradient"), _ptrs(x_star, 12, "field"),
        int(max_iters), int(check_every), float(tol), ctypes.byref(k), ctypes.byref(r)))
    return k.value, r.value


def thiim_build_coeffs_grad(ctx, eps_r, sigma_pml_e, omega, tau, k_s, amp, grad_coeffs, grad_eps_re):
    """dJ/dRe(eps) per cell into the float64 CUDA tensor grad_eps_re."""
    import numpy as np
    se = None if sigma_pml_e is None else np.ascontiguousarray(sigma_pml_e, dtype=np.float64)
    amp = complex(amp)
    _check("thiim_build_coeffs_grad", load_library().thiim_build_coeffs_grad(
        ctx, ctypes.c_void_p(eps_r.data_ptr()), None if se is None else se.ctypes.data_as(ctypes.c_void_p),
        float(omega), float(tau), int(k_s), amp.real, amp.imag, _ptrs(grad_coeffs, 28, "gradient"),
        ctypes.c_void_p(grad_eps_re.data_ptr())))


def thiim_batch_iterate(ctxs, max_iters, check_every=50, tol=0.0):
    """Advance several solves together; returns (iterations per solve, residual per solve)."""
    n = len(ctxs)
    arr = (ctypes.c_void_p * n)(*[c.value if hasattr(c, "value") else c for c in ctxs])
    iters = (ctypes.c_int * n)()
    res = (ctypes.c_double * n)()
    _check("thiim_batch_iterate", load_library().thiim_batch_iterate(arr, n, int(max_iters), int(check_every),
                                                                      float(tol), iters, res))
    return list(iters), list(res)


def thiim_step_noalloc(nx, ny, nz, precision, bc_flags, src, dst, coeffs, stream=None, want_residual=True):
    """One iteration src -> dst without any allocation; returns the residual or None."""
    r = ctypes.c_double()
    rc = load_library().thiim_step_noalloc(int(nx), int(ny), int(nz), int(precision), int(bc_flags),
                                           _ptrs(src, 12, "field"), _ptrs(dst, 12, "field"),
                                           _ptrs(coeffs, 28, "coefficient"), _stream_ptr(stream),
                                           ctypes.byref(r) if want_residual else None)
    _check("thiim_step_noalloc", rc)
    return r.value if want_residual else None


def thiim_fp64_pipe_rate(stream=None) -> float:
    """Measured FP64 FMA instructions per second of the current device."""
    r = ctypes.c_double()
    _check("thiim_fp64_pipe_rate", load_library().thiim_fp64_pipe_rate(_stream_ptr(stream), ctypes.byref(r)))
    return r.value


def thiim_destroy(ctx):
    if ctx:
        load_library().thiim_destroy(ctx)


def thiim_strerror(code) -> str:
    return load_library().thiim_strerror(int(code)).decode()


def thiim_version() -> int:
    return load_library().thiim_version()


class Solver:
    """Owns the torch tensors of one THIIM problem and a library context.

    fields: 12 tensors, coeffs: 28 tensors, shape (nz, ny, nx), complex128 or
    complex64 on the current CUDA device.
    """

    def __init__(self, nx, ny, nz, precision=THIIM_C128, bc=THIIM_PERIODIC_X | THIIM_PERIODIC_Y,
                 stream=None, device=None):
        import torch
        self.nx, self.ny, self.nz = nx, ny, nz
        self.precision = precision
        self.dtype = torch.complex64 if precision == THIIM_C64 else torch.complex128
        self.device = torch.device(device or "cuda")
        self.ctx = thiim_create(nx, ny, nz, precision, bc, stream)
        self.fields = None
        self.coeffs = None

    def _empty(self, n):
        import torch
        return [torch.zeros((self.nz, self.ny, self.nx), dtype=self.dtype, device=self.device) for _ in range(n)]

    def set_coeffs(self, coeffs):
        self.coeffs = list(coeffs)
        thiim_set_coeffs(self.ctx, self.coeffs)

    def set_fields(self, fields=None):
        self.fields = list(fields) if fields is not None else self._empty(12)
        thiim_set_fields(self.ctx, self.fields)

    def build_coeffs(self, eps_r, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp=1.0):
        coeffs = self.coeffs if self.coeffs is not None else self._empty(28)
        thiim_build_coeffs(self.ctx, eps_r, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp, coeffs)
        self.set_coeffs(coeffs)

    def set_material_coeffs(self, mat, table, n_mat):
        """Material-table coefficients; the tensors are kept alive here."""
        self.mat, self.table = mat, table
        thiim_set_material_coeffs(self.ctx, mat, n_mat, table)

    def build_material_table(self, eps_mat, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp=1.0):
        """A new table for the permittivities eps_mat (one per material id)."""
        import torch
        table = torch.empty(len(eps_mat) * self.nz * 28, dtype=self.dtype, device=self.device)
        thiim_build_material_table(self.ctx, eps_mat, sigma_pml_e, sigma_pml_h, omega, tau, k_s, amp, table)
        return table

    def iterate(self, n):
        thiim_iterate(self.ctx, n)

    def residual(self) -> float:
        return thiim_residual(self.ctx)

    def close(self):
        if self.ctx:
            thiim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
