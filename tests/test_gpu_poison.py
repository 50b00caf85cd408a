"""Out-of-bounds check by poison fill (the in-pool stand-in for a memory checker).

Every caller array a kernel reads or writes is carved out of one large device
buffer filled with NaN (material ids: 0xFF, an id beyond every table), with a
guard of more than one z-plane between consecutive arrays and at both ends.
A kernel that reads one element outside its array picks up a NaN (or an id
whose table row is NaN), which spreads into the result; one that writes
outside overwrites a guard.  So each run must (1) match the oracle at the
tolerance of its precision, (2) contain no NaN, and (3) leave every guard
element NaN (0xFF).  Ragged shapes under Dirichlet-everywhere (bc 0) and
periodic-everywhere (bc 7) boundaries, for complex128, FP32 pairs and
complex64, the material-table variant, the batched launch, the two-iteration
temporal-blocked kernel and the allocation-free entry point.

Tolerances: 1e-12 relative per split for complex128 and pairs; 5e-6 for
complex64 over 3 iterations (the bound derived in test_gpu_sweep).
"""
import numpy as np
import pytest

import oracle
from oracle.coeffs import build_coeffs as oracle_coeffs
from tests.gpu_util import rel_l2, to_host
from workloads import random_coeffs, random_fields
from workloads.thiim_workloads import LayeredStack

pytestmark = pytest.mark.gpu

SHAPES = [(7, 13, 70), (5, 9, 33), (10, 1, 3)]   # (nz, ny, nx)


def _lib():
    import paper_1510_05218_gb300 as p
    p.load_library()
    return p


class Poisoned:
    """n arrays of `shape` carved from one NaN-filled buffer with guards."""

    def __init__(self, n, shape, dtype, fill=None):
        import torch
        self.count = int(np.prod(shape))
        plane = shape[-1] * (shape[-2] if len(shape) > 1 else 1)
        self.guard = plane + 4096
        self.stride = self.count + self.guard
        total = self.guard + n * self.stride
        if fill is None:
            fill = complex(float("nan"), float("nan"))
        self.buf = torch.full((total,), fill, dtype=dtype, device="cuda")
        self.views = [self.buf[self.guard + i * self.stride: self.guard + i * self.stride + self.count].view(shape)
                      for i in range(n)]

    def load(self, host_arrays):
        import torch
        for v, a in zip(self.views, host_arrays):
            v.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(v.dtype))

    def guards_intact(self):
        import torch
        mask = torch.ones(self.buf.numel(), dtype=torch.bool, device="cuda")
        for i in range(len(self.views)):
            s = self.guard + i * self.stride
            mask[s: s + self.count] = False
        g = self.buf[mask]
        if g.dtype == torch.uint8:
            return bool(torch.all(g == 0xFF))
        return bool(torch.all(torch.isnan(g.real) & torch.isnan(g.imag)))


def _dtype(precision):
    import torch
    return torch.complex64 if precision == 1 else torch.complex128


def _check(got, want, tol):
    for s in range(12):
        assert np.all(np.isfinite(got[s])), s
        assert rel_l2(got[s], want[s]) <= tol, (s, rel_l2(got[s], want[s]))


def _inputs(shape, seed, precision):
    nz, ny, nx = shape
    f = random_fields(nx, ny, nz, seed=seed)
    c = random_coeffs(nx, ny, nz, seed=seed)
    if precision == 1:   # the oracle runs on the complex64-rounded inputs
        f = [a.astype(np.complex64).astype(np.complex128) for a in f]
        c = [a.astype(np.complex64).astype(np.complex128) for a in c]
    return f, c


@pytest.mark.parametrize("precision,tol,temporal", [(0, 1e-12, 1), (2, 1e-12, 1), (1, 5e-6, 1), (1, 5e-6, 2)])
@pytest.mark.parametrize("bc", [0, 7])
@pytest.mark.parametrize("shape", SHAPES)
def test_sweep_reads_and_writes_only_its_arrays(shape, bc, precision, tol, temporal):
    p = _lib()
    nz, ny, nx = shape
    f, c = _inputs(shape, 11, precision)
    fp = Poisoned(12, shape, _dtype(precision))
    cp = Poisoned(28, shape, _dtype(precision))
    fp.load(f)
    cp.load(c)
    n = 3
    ctx = p.thiim_create(nx, ny, nz, precision, bc)
    try:
        if temporal != 1:
            p.thiim_set_tuning(ctx, temporal, 0)
        p.thiim_set_coeffs(ctx, cp.views)
        p.thiim_set_fields(ctx, fp.views)
        p.thiim_iterate(ctx, n)
        r = p.thiim_residual(ctx)
    finally:
        p.thiim_destroy(ctx)
    got = to_host(fp.views)
    o = [a.copy() for a in f]
    oracle.iterate(o, c, n, bc=bc)
    _check(got, o, tol)
    assert np.isfinite(r)
    assert fp.guards_intact() and cp.guards_intact()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-12), (1, 5e-6)])
@pytest.mark.parametrize("bc", [0, 7])
def test_table_variant_reads_only_its_map_and_table(precision, tol, bc):
    import torch
    p = _lib()
    st = LayeredStack(nx=40, ny=20, nz=24, seed=3)
    shape = (st.nz, st.ny, st.nx)
    em = st.material_eps()
    ids = st.material_ids()
    mp = Poisoned(1, shape, torch.uint8, fill=0xFF)
    mp.views[0].copy_(torch.from_numpy(ids))
    tp = Poisoned(1, (len(em) * st.nz * 28,), _dtype(precision))
    f0 = random_fields(st.nx, st.ny, st.nz, seed=4)
    if precision == 1:
        f0 = [a.astype(np.complex64).astype(np.complex128) for a in f0]
    fp = Poisoned(12, shape, _dtype(precision))
    fp.load(f0)
    n = 3
    ctx = p.thiim_create(st.nx, st.ny, st.nz, precision, bc)
    try:
        p.thiim_build_material_table(ctx, em, st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, st.k_s, 1.0,
                                     tp.views[0])
        table = to_host(tp.views)[0].reshape(len(em), st.nz, 28)
        p.thiim_set_material_coeffs(ctx, mp.views[0], len(em), tp.views[0])
        p.thiim_set_fields(ctx, fp.views)
        p.thiim_iterate(ctx, n)
    finally:
        p.thiim_destroy(ctx)
    got = to_host(fp.views)
    # the oracle iterates the same (device-built) coefficients expanded through the map
    k = np.arange(st.nz)[:, None, None]
    co = [table[ids, k, i] for i in range(28)]
    if precision != 1:   # the table itself equals the oracle's builder (test_gpu_material pins 1e-14)
        oc = oracle_coeffs(st.eps(), st.sigma_pml_e(), st.sigma_pml_h(), st.omega, st.tau, tfsf=(st.k_s, 1.0))
        for i in range(28):
            assert rel_l2(co[i], oc[i]) <= 1e-14
    o = [a.copy() for a in f0]
    oracle.iterate(o, co, n, bc=bc)
    _check(got, o, tol)
    assert fp.guards_intact() and tp.guards_intact() and mp.guards_intact()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-12)])
def test_batch_reads_and_writes_only_its_arrays(precision, tol):
    p = _lib()
    shapes, bcs = [(7, 13, 70), (10, 1, 3), (5, 9, 33)], [0, 7, 3]
    made = []
    for i, (shape, bc) in enumerate(zip(shapes, bcs)):
        nz, ny, nx = shape
        f, c = _inputs(shape, 60 + i, precision)
        fp = Poisoned(12, shape, _dtype(precision))
        cp = Poisoned(28, shape, _dtype(precision))
        fp.load(f)
        cp.load(c)
        ctx = p.thiim_create(nx, ny, nz, precision, bc)
        p.thiim_set_coeffs(ctx, cp.views)
        p.thiim_set_fields(ctx, fp.views)
        made.append((ctx, f, c, fp, cp, bc))
    n = 5
    try:
        iters, res = p.thiim_batch_iterate([m[0] for m in made], n, 2, 0.0)
    finally:
        for m in made:
            p.thiim_destroy(m[0])
    assert iters == [n] * len(made)
    for ctx, f, c, fp, cp, bc in made:
        o = [a.copy() for a in f]
        oracle.iterate(o, c, n, bc=bc)
        _check(to_host(fp.views), o, tol)
        assert fp.guards_intact() and cp.guards_intact()
    assert all(np.isfinite(res))


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 5e-6)])
def test_noalloc_step_reads_and_writes_only_its_arrays(precision, tol):
    p = _lib()
    shape = (7, 13, 70)
    nz, ny, nx = shape
    f, c = _inputs(shape, 12, precision)
    sp = Poisoned(12, shape, _dtype(precision))
    dp = Poisoned(12, shape, _dtype(precision))
    cp = Poisoned(28, shape, _dtype(precision))
    sp.load(f)
    cp.load(c)
    r = p.thiim_step_noalloc(nx, ny, nz, precision, 0, sp.views, dp.views, cp.views)
    o = [a.copy() for a in f]
    oracle.iterate(o, c, 1, bc=0)
    _check(to_host(dp.views), o, tol)
    assert np.isfinite(r)
    assert sp.guards_intact() and dp.guards_intact() and cp.guards_intact()
