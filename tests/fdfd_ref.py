"""Dense FDFD systems written straight from the paper's equations (pins).

These assemble, for small grids, the linear system that a fixed point of the
THIIM iteration must satisfy: Eqs. 3-5 with E^{n+1} = E^n and
H^{n+1/2} = H^{n-1/2}, split per Eqs. 6-7.  They use the physical parameters
(eps, sigma, sigma*, S) and the curl written out from Maxwell's equations, not
the update coefficients or the split table of the oracle, so a wrong sign,
index, phase or coefficient in the oracle shows up as a mismatch.

Split naming follows the listings (Sec. III): split F_ab of component a reads
component b of the other field.  For the cyclic triple (a, b, c):
  (curl H)_a  = d_b H_c - d_c H_b  ->  E_ac gets +d_b H_c, E_ab gets -d_c H_b
  (-curl E)_a = d_c E_b - d_b E_c  ->  H_ab gets +d_c E_b, H_ac gets -d_b E_c
H differences look backward (H index k sits between E planes k-1 and k),
E differences look forward (Fig. 3).
"""
import cmath

import numpy as np

COMP = "xyz"
SPLITS = ["Hxy", "Hxz", "Hyx", "Hyz", "Hzx", "Hzy", "Exy", "Exz", "Eyx", "Eyz", "Ezx", "Ezy"]


def split_terms():
    """{split: (sign, derivative axis, component read)} from the curl formulas."""
    terms = {}
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        A, B, C = COMP[a], COMP[b], COMP[c]
        terms["E" + A + C] = (+1, b, C)
        terms["E" + A + B] = (-1, c, B)
        terms["H" + A + B] = (+1, c, B)
        terms["H" + A + C] = (-1, b, C)
    return terms


def assemble(shape, eps, sig_e, sig_h, omega, tau, S, bc=(True, True, True)):
    """Dense matrix A and right-hand side b with A x = b at the fixed point.

    shape = (nz, ny, nx); eps (real), sig_e[split] and sig_h[split] are
    per-cell arrays (conductivity of each split), S[split] per-cell physical
    sources (zero arrays where absent).  bc: periodic flags (x, y, z).
    Unknown ordering: split-major, then the cell index (k*ny + j)*nx + i.
    """
    nz, ny, nx = shape
    ncell = nx * ny * nz
    n = 12 * ncell
    A = np.zeros((n, n), np.complex128)
    b = np.zeros(n, np.complex128)
    terms = split_terms()
    e = lambda a: cmath.exp(1j * a)  # noqa: E731
    w_e = (e(omega * tau) - 1.0) / tau              # E: (e^{iwt} - 1)/tau
    w_h = (e(omega * tau / 2) - e(-omega * tau / 2)) / tau   # H, Eq. 4
    per = {0: bc[0], 1: bc[1], 2: bc[2]}
    dims = {0: nx, 1: ny, 2: nz}

    def cell(i, j, k):
        return (k * ny + j) * nx + i

    def shifted(i, j, k, axis, off):
        q = [i, j, k]
        q[axis] += off
        if q[axis] < 0 or q[axis] >= dims[axis]:
            if not per[axis]:
                return None
            q[axis] %= dims[axis]
        return cell(*q)

    for s_idx, s in enumerate(SPLITS):
        sign, axis, comp = terms[s]
        field = s[0]
        other = "E" if field == "H" else "H"
        reads = [SPLITS.index(other + comp + z) for z in COMP if z != comp]
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    p = cell(i, j, k)
                    row = s_idx * ncell + p
                    if field == "H":
                        # w_h x = sign/mu D^- F - sig*/mu x + S
                        A[row, row] += w_h + sig_h[s][k, j, i]
                        here, nb = p, shifted(i, j, k, axis, -1)
                        coef = sign * 1.0
                        b[row] += S[s][k, j, i]
                        for r in reads:
                            A[row, r * ncell + here] -= coef
                            if nb is not None:
                                A[row, r * ncell + nb] += coef
                    else:
                        ep = eps[k, j, i]
                        sg = sig_e[s][k, j, i]
                        if ep > 0:   # Eq. 3
                            A[row, row] += w_e + sg / ep * e(omega * tau)
                        else:        # Eq. 5
                            A[row, row] += w_e + sg / ep
                        coef = sign * e(omega * tau / 2) / ep
                        b[row] += S[s][k, j, i]
                        here, nb = p, shifted(i, j, k, axis, +1)
                        for r in reads:
                            A[row, r * ncell + here] += coef
                            if nb is not None:
                                A[row, r * ncell + nb] -= coef
    return A, b


def to_fields(x, shape):
    ncell = int(np.prod(shape))
    return [x[s * ncell:(s + 1) * ncell].reshape(shape) for s in range(12)]
