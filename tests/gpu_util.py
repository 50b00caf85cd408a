"""Helpers shared by the GPU tests: host<->device copies and error norms."""
import math

import numpy as np


def to_dev(arrays, dtype="complex128"):
    import torch
    td = torch.complex128 if dtype == "complex128" else torch.complex64
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=td) for a in arrays]


def to_host(tensors):
    import torch
    torch.cuda.synchronize()
    return [t.to(torch.complex128).cpu().numpy() for t in tensors]


def rel_l2(a, b):
    """||a - b|| / ||b|| (0 when both are zero)."""
    den = float(np.sum(np.abs(b) ** 2))
    num = float(np.sum(np.abs(a - b) ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return math.sqrt(num / den)


def full_fields(f):
    """Full components (Hx, Hy, Hz, Ex, Ey, Ez) from the 12 splits."""
    return [f[2 * a] + f[2 * a + 1] for a in range(6)]
