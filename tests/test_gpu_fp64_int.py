"""The FP64 sweep with binary64 operations on the integer pipe is bit-identical.

thiim_set_fp64_int_ops moves the sweep's additions (THIIM_INT_ADD) and the
leading products of its updates (THIIM_INT_MUL) from the FP64 pipe to exact
integer arithmetic.  Each operation keeps its IEEE 754 result and the order of
operations does not change, so fields and residuals must equal those of the
pure FP64-pipe sweep bit for bit — on random data, and on data salted with
zeros of both signs, subnormals and values near the ends of the exponent
range (whose products overflow to Inf and NaN; NaN results compare as NaN).
The integer-pipe sweep also matches the oracle at 1e-12 per split.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_util import rel_l2, to_dev, to_host
from workloads import random_coeffs, random_fields

pytestmark = pytest.mark.gpu

SHAPES = [(9, 13, 70), (5, 17, 33), (40, 9, 31), (1, 5, 7)]
MODES = [0, 1, 3, 4]


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


def _salt(arrays, seed):
    """Replace ~3 % of the entries by zeros, -0, subnormals and extreme magnitudes."""
    rng = np.random.default_rng(seed)
    specials = np.array([0.0, -0.0, 5e-310, -2.5e-320, 1e-300, -3e-290, 1e250, -7e200])
    out = []
    for a in arrays:
        a = a.copy()
        for part in ("real", "imag"):
            v = getattr(a, part).copy()
            m = rng.random(v.shape) < 0.03
            v[m] = rng.choice(specials, size=int(m.sum()))
            if part == "real":
                a = v + 1j * a.imag
            else:
                a = a.real + 1j * v
        out.append(a)
    return out


def _bits(t):
    """Bit patterns of the real and imaginary parts; every NaN maps to one
    value (IEEE 754 leaves the sign and payload of a propagated NaN open)."""
    import torch
    r = torch.view_as_real(t).contiguous()
    b = r.view(torch.int64).clone()
    b[torch.isnan(r)] = -1
    return b


def _run(p, f, c, n, bc, ops):
    import torch
    nz, ny, nx = f[0].shape
    fd, cd = to_dev(f), to_dev(c)
    ctx = p.thiim_create(nx, ny, nz, p.THIIM_C128, bc)
    try:
        p.thiim_set_fp64_int_ops(ctx, ops)
        p.thiim_set_coeffs(ctx, cd)
        p.thiim_set_fields(ctx, fd)
        p.thiim_iterate(ctx, n)
        try:
            r = p.thiim_residual(ctx)
        except p.ThiimError as e:      # extreme salt values may overflow to Inf / NaN
            assert e.code == -6
            r = float("nan")
    finally:
        p.thiim_destroy(ctx)
    torch.cuda.synchronize()
    return [_bits(t).cpu() for t in fd], r, fd


@pytest.mark.parametrize("salted", [False, True])
@pytest.mark.parametrize("bc", [3, 7, 0])
@pytest.mark.parametrize("shape", SHAPES)
def test_integer_pipe_modes_are_bit_identical(shape, bc, salted):
    import torch
    p = _lib()
    nz, ny, nx = shape
    f = random_fields(nx, ny, nz, seed=21)
    c = random_coeffs(nx, ny, nz, seed=21)
    if salted:
        f, c = _salt(f, 1), _salt(c, 2)
    runs = {ops: _run(p, f, c, 3, bc, ops) for ops in MODES}
    ref_bits, ref_r, _ = runs[0]
    for ops in (1, 3, 4):
        bits, r, _ = runs[ops]
        assert r == ref_r or (np.isnan(r) and np.isnan(ref_r))
        for s in range(12):
            assert torch.equal(bits[s], ref_bits[s]), (ops, s)


def test_integer_pipe_sweep_matches_oracle():
    p = _lib()
    nz, ny, nx = 9, 13, 70
    f = random_fields(nx, ny, nz, seed=22)
    c = random_coeffs(nx, ny, nz, seed=22)
    _, _, fd = _run(p, f, c, 4, 3, 3)
    got = to_host(fd)
    o = [a.copy() for a in f]
    oracle.iterate(o, c, 4, bc=3)
    for s in range(12):
        assert rel_l2(got[s], o[s]) <= 1e-12


def test_set_fp64_int_ops_arguments():
    p = _lib()
    ctx = p.thiim_create(8, 8, 8, p.THIIM_C64, 3)
    try:
        with pytest.raises(p.ThiimError):
            p.thiim_set_fp64_int_ops(ctx, 1)
    finally:
        p.thiim_destroy(ctx)
    ctx = p.thiim_create(8, 8, 8, p.THIIM_C128, 3)
    try:
        for bad in (2, 5, 7):
            with pytest.raises(p.ThiimError):
                p.thiim_set_fp64_int_ops(ctx, bad)
        for good in (0, 1, 3, 4):
            p.thiim_set_fp64_int_ops(ctx, good)
    finally:
        p.thiim_destroy(ctx)


def test_fp64_pipe_rate_is_plausible():
    """thiim_fp64_pipe_rate (the FP64 roofline's denominator) reports a device-wide
    FMA rate between 1/4 and 4x of GB300's 152 SMs x 2 FMA/clk x ~2 GHz."""
    p = _lib()
    r = p.thiim_fp64_pipe_rate()
    assert 1.5e11 <= r <= 2.5e12, r
