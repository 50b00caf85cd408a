"""Seeded synthetic inputs shaped like the paper's solar-cell workload.

The paper simulates a textured thin-film tandem cell (Fig. 1, Sec. I-A) whose
interface heights come from atomic-force-microscopy scans and whose materials
are mapped to the grid by FIT.  Neither the scans nor the meshes exist here, so
a seeded stand-in is generated instead:

* z (outer dimension, k) carries the layer stack: an absorbing layer (PML) in
  air at the top, air, a textured absorber (a-Si:H-like, eps = 16 + 0.5i), a
  glass-like layer (eps = 2.1) and an Ag-like back contact (eps = -20 + 1.0i)
  that also hosts the bottom absorbing layer.  Permittivities are given in the
  physics convention (Im > 0 means lossy).
* The absorber's top interface is z_top(x, y) = base + sum_m a_m sin(2 pi
  (p_m x / Nx + q_m y / Ny) + phi_m), periodic in x and y.
* A unit, x-polarised, normally incident plane wave enters at the plane k_s.

All lengths are given for Nz = 32 and scale with Nz / 32.  Every array uses the
layout of the paper's listings (Sec. III, Listings 1-2): shape (Nz, Ny, Nx), x
fastest, complex128.

Nothing here performs a step of the iteration: permittivity maps, absorbing
layer conductivity profiles and random numbers are inputs that both the GPU
path and the oracle consume.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N_FIELDS = 12   # split field components (Sec. I-A, Eqs. 6-7)
N_COEFFS = 28   # 4*3 + 8*2 coefficient arrays (Sec. III)

# Relative permittivities of the stack's layers, physics convention (Im > 0 lossy).
MATERIALS = {
    "air": 1.0 + 0.0j,
    "asi": 16.0 + 0.5j,
    "glass": 2.1 + 0.0j,
    "ag": -20.0 + 1.0j,
}


def _scaled(v: float, s: float) -> int:
    return int(round(v * s))


@dataclass
class LayeredStack:
    """A textured thin-film stack on an (nx, ny, nz) grid.

    Geometry for nz = 32 (scale s = nz/32 multiplies every z length):
      absorbing layers: k in [0, 6) at the top and the last 6 planes at the bottom;
      plane-wave source plane k_s = 8;
      absorber (a-Si:H-like) from z_top(i, j) (base 14, |texture| <= amp) to k < 22;
      glass-like for 22 <= k < 24; Ag-like for k >= 24.
    ``lam`` is the free-space wavelength in cells, ``tau`` the pseudo time step.
    ``eps_scale`` multiplies every non-air permittivity (dispersion of the
    spectrum sweep).  ``texture_box`` optionally confines the texture to
    x, y in [x0, x1) (flat interface at the base height elsewhere).
    """

    nx: int
    ny: int
    nz: int
    lam: float = 20.0
    tau: float = 0.5
    n_sin: int = 4
    amp: float = 4.0
    seed: int = 0
    eps_scale: float = 1.0
    pml_cells: int | None = None
    texture_box: tuple | None = None
    # derived
    s: float = field(init=False)
    omega: float = field(init=False)
    k_s: int = field(init=False)
    L: int = field(init=False)
    z_base: float = field(init=False)
    z_asi_end: int = field(init=False)
    z_glass_end: int = field(init=False)
    sigma_max: float = field(init=False)
    tex_a: np.ndarray = field(init=False, repr=False)
    tex_p: np.ndarray = field(init=False, repr=False)
    tex_q: np.ndarray = field(init=False, repr=False)
    tex_phi: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self.s = self.nz / 32.0
        self.omega = 2.0 * math.pi / self.lam
        self.L = self.pml_cells if self.pml_cells is not None else max(1, _scaled(6, self.s))
        self.k_s = _scaled(8, self.s)
        self.z_base = 14.0 * self.s
        self.z_asi_end = _scaled(22, self.s)
        self.z_glass_end = _scaled(24, self.s)
        # Quadratic absorbing profile sigma(d) = sigma_max (d/L)^2 with a
        # nominal normal-incidence reflection of 1e-6.
        self.sigma_max = -3.0 * math.log(1e-6) / (2.0 * self.L)
        rng = np.random.default_rng(self.seed)
        raw = rng.uniform(0.2, 1.0, self.n_sin)
        self.tex_a = raw / raw.sum() * self.amp          # sum |a_m| == amp
        self.tex_p = rng.integers(1, 4, self.n_sin)      # p, q in {1, 2, 3}
        self.tex_q = rng.integers(1, 4, self.n_sin)
        self.tex_phi = rng.uniform(0.0, 2.0 * math.pi, self.n_sin)

    # --- geometry -----------------------------------------------------------
    def z_top(self) -> np.ndarray:
        """Absorber top interface height at the cell centres (i+1/2, j+1/2), shape (ny, nx)."""
        x = (np.arange(self.nx) + 0.5)[None, :]
        y = (np.arange(self.ny) + 0.5)[:, None]
        z = np.full((self.ny, self.nx), self.z_base)
        tex = np.zeros((self.ny, self.nx))
        for a, p, q, ph in zip(self.tex_a, self.tex_p, self.tex_q, self.tex_phi):
            tex = tex + a * np.sin(2.0 * math.pi * (p * x / self.nx + q * y / self.ny) + ph)
        if self.texture_box is not None:
            x0, x1, y0, y1 = self.texture_box
            mask = np.zeros((self.ny, self.nx), bool)
            mask[y0:y1, x0:x1] = True
            tex = np.where(mask, tex, 0.0)
        return z + tex

    def material(self, name: str) -> complex:
        e = MATERIALS[name]
        return e if name == "air" else e * self.eps_scale

    def eps_planes(self, k0: int, k1: int) -> np.ndarray:
        """Relative permittivity (physics convention) of cells k0 <= k < k1, shape (k1-k0, ny, nx)."""
        zt = self.z_top()
        out = np.empty((k1 - k0, self.ny, self.nx), np.complex128)
        for idx, k in enumerate(range(k0, k1)):
            plane = np.full((self.ny, self.nx), self.material("air"), np.complex128)
            if k >= self.z_glass_end:
                plane[:] = self.material("ag")
            elif k >= self.z_asi_end:
                plane[:] = self.material("glass")
            else:
                plane[k >= zt] = self.material("asi")
            out[idx] = plane
        return out

    def eps(self) -> np.ndarray:
        return self.eps_planes(0, self.nz)

    # material order of the ids below
    MATERIAL_ORDER = ("air", "asi", "glass", "ag")

    def material_eps(self) -> np.ndarray:
        """Permittivity of material id m = 0..3 (order MATERIAL_ORDER)."""
        return np.array([self.material(n) for n in self.MATERIAL_ORDER], np.complex128)

    def material_id_planes(self, k0: int, k1: int) -> np.ndarray:
        """Material id (uint8) of cells k0 <= k < k1; material_eps()[ids] == eps_planes(k0, k1)."""
        zt = self.z_top()
        out = np.zeros((k1 - k0, self.ny, self.nx), np.uint8)
        for idx, k in enumerate(range(k0, k1)):
            if k >= self.z_glass_end:
                out[idx] = 3
            elif k >= self.z_asi_end:
                out[idx] = 2
            else:
                out[idx][k >= zt] = 1
        return out

    def material_ids(self) -> np.ndarray:
        return self.material_id_planes(0, self.nz)

    def absorber_mask(self) -> np.ndarray:
        """Cells of the a-Si:H-like absorber (bool, shape (nz, ny, nx))."""
        zt = self.z_top()
        k = np.arange(self.nz)[:, None, None]
        return (k >= zt[None]) & (k < self.z_asi_end)

    # --- absorbing layers -----------------------------------------------------
    def _sigma_at(self, p: np.ndarray) -> np.ndarray:
        d_top = np.maximum(0.0, self.L - p)
        d_bot = np.maximum(0.0, p - (self.nz - 1 - self.L))
        d = np.maximum(d_top, d_bot)
        return self.sigma_max * (d / self.L) ** 2

    def sigma_pml_e(self) -> np.ndarray:
        """Absorbing-layer conductivity at the E planes (z = k), shape (nz,)."""
        return self._sigma_at(np.arange(self.nz, dtype=np.float64))

    def sigma_pml_h(self) -> np.ndarray:
        """Absorbing-layer conductivity at the H planes (z = k - 1/2), shape (nz,)."""
        return self._sigma_at(np.arange(self.nz, dtype=np.float64) - 0.5)

    def describe(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, lam=self.lam, tau=self.tau,
                    omega=self.omega, k_s=self.k_s, pml=self.L, sigma_max=self.sigma_max,
                    n_sin=self.n_sin, amp=self.amp, seed=self.seed, eps_scale=self.eps_scale)


def stack_config(name: str) -> LayeredStack:
    """The named layered-stack workloads.

    stack32     32^3, 4 sinusoids, amplitude <= 4, lambda = 20 cells.
    stack512    512^3, everything scaled by 16: 16 sinusoids, amplitude <= 64,
                lambda = 320, absorbing layers 96 cells.
    stack256    the stack512 structure at 256^3 (scale 8).
    adjoint128  128^3, scale 4, texture confined to x, y in [48, 80).
    stackN      any other N: the 32^3 stack scaled by N/32.
    """
    if name == "stack32":
        return LayeredStack(32, 32, 32, lam=20.0, n_sin=4, amp=4.0, seed=0)
    if name == "stack512":
        return LayeredStack(512, 512, 512, lam=320.0, n_sin=16, amp=64.0, seed=0)
    if name == "stack256":
        return LayeredStack(256, 256, 256, lam=160.0, n_sin=16, amp=32.0, seed=0)
    if name == "stack128":
        return LayeredStack(128, 128, 128, lam=80.0, n_sin=16, amp=16.0, seed=0)
    if name == "adjoint128":
        return LayeredStack(128, 128, 128, lam=80.0, n_sin=4, amp=16.0, seed=0,
                            texture_box=(48, 80, 48, 80))
    if name.startswith("stack") and name[5:].isdigit():
        # stackN: the 32^3 stack scaled to N^3 (wavelength and every z length x N/32)
        n = int(name[5:])
        return LayeredStack(n, n, n, lam=20.0 * n / 32.0, n_sin=16 if n >= 256 else 4,
                            amp=4.0 * n / 32.0, seed=0)
    raise KeyError(name)


def batch_configs(n: int = 32, seed: int = 1):
    """The spectrum-sweep batch: ``n`` solves with seeded uneven grids.

    Nx = Ny drawn from {64, 80, ..., 192}, Nz from {96, 128, ..., 256}; the
    wavelength of solve b is 20 + 40 b / (n - 1) cells and every non-air
    permittivity is scaled by 0.8 + 0.4 (lambda - 20) / 40 (linear dispersion
    between -20 % and +20 %).
    """
    rng = np.random.default_rng(seed)
    nxy = rng.choice(np.arange(64, 193, 16), n)
    nzs = rng.choice(np.arange(96, 257, 32), n)
    out = []
    for b in range(n):
        lam = 20.0 + 40.0 * b / max(1, n - 1)
        scale = 0.8 + 0.4 * (lam - 20.0) / 40.0
        nz = int(nzs[b])
        out.append(LayeredStack(int(nxy[b]), int(nxy[b]), nz, lam=lam, n_sin=4,
                                amp=4.0 * nz / 32.0, seed=seed * 1000 + b, eps_scale=scale))
    return out


# --- seeded random arrays ------------------------------------------------------

# Magnitude ranges of the random coefficient arrays, chosen like the physical
# ones: |t| <= 1 and |c| in the range tau/|eps| takes for the stack's materials.
_T_RANGE = (0.70, 1.0)
_C_RANGE = (0.025, 0.25)


def random_plane(seed: int, array_id: int, k: int, ny: int, nx: int, kind: str) -> np.ndarray:
    """One z-plane of a seeded random complex array, independent of every other plane.

    The generator for (seed, array_id, k) is NumPy's default bit generator
    seeded with that triple, so any plane can be regenerated on its own.
    kind: 'field' (complex normal), 't' (|t| in [0.7, 1), uniform phase),
    'c' (|c| in [0.025, 0.25), uniform phase), 'src' (0.1 x complex normal).
    """
    rng = np.random.default_rng([seed, array_id, k])
    if kind == "field":
        v = rng.standard_normal((ny, nx, 2))
        return v[..., 0] + 1j * v[..., 1]
    if kind == "src":
        v = rng.standard_normal((ny, nx, 2)) * 0.1
        return v[..., 0] + 1j * v[..., 1]
    lo, hi = _T_RANGE if kind == "t" else _C_RANGE
    mag = rng.uniform(lo, hi, (ny, nx))
    ph = rng.uniform(0.0, 2.0 * math.pi, (ny, nx))
    return mag * np.exp(1j * ph)


def _coeff_kind(idx: int) -> str:
    return "t" if idx < 12 else ("c" if idx < 24 else "src")


def random_fields(nx, ny, nz, seed, k0=0, k1=None):
    """12 random field arrays (planes k0..k1-1), list of (k1-k0, ny, nx) complex128."""
    k1 = nz if k1 is None else k1
    return [np.stack([random_plane(seed, a, k, ny, nx, "field") for k in range(k0, k1)])
            for a in range(N_FIELDS)]


def random_coeffs(nx, ny, nz, seed, k0=0, k1=None):
    """28 random coefficient arrays (t[12], c[12], 4 source arrays), planes k0..k1-1."""
    k1 = nz if k1 is None else k1
    return [np.stack([random_plane(seed, 100 + a, k, ny, nx, _coeff_kind(a)) for k in range(k0, k1)])
            for a in range(N_COEFFS)]


def random_sweep_inputs(nx, ny, nz, seed=0):
    return random_fields(nx, ny, nz, seed), random_coeffs(nx, ny, nz, seed)


# Named workloads for the benchmark and the tests.
WORKLOADS = {
    "stack32": dict(kind="stack", stack="stack32", iters=20, dtype="c128"),
    "stack512": dict(kind="stack", stack="stack512", iters=200, dtype="c128"),
}
