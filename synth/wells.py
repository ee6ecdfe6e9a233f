"""Well source fields f (source density per unit volume), shape (nz, ny, nx).

Wells are vertical columns of cells modelled as volumetric sources/sinks, as in
the paper's 5-spot setup (Sec. "Numerical setup").  Each well's total rate is
split evenly over its column cells; the rates sum to zero so that a problem
with no-flow walls is compatible.
"""
from __future__ import annotations

import numpy as np


def _column(f, i, j, rate, cell_volume):
    nz = f.shape[0]
    f[:, j, i] += rate / (nz * cell_volume)


def corner_wells(nx, ny, nz, h=(1.0, 1.0, 1.0)):
    """Unit injector in column (0, 0) and unit producer in column (nx-1, ny-1)."""
    vol = h[0] * h[1] * h[2]
    f = np.zeros((nz, ny, nx), dtype=np.float64)
    _column(f, 0, 0, +1.0, vol)
    _column(f, nx - 1, ny - 1, -1.0, vol)
    return f


def five_spot_wells(nx, ny, nz, h=(1.0, 1.0, 1.0)):
    """Central injector (+1) and four corner producers (-1/4 each)."""
    vol = h[0] * h[1] * h[2]
    f = np.zeros((nz, ny, nx), dtype=np.float64)
    _column(f, nx // 2, ny // 2, +1.0, vol)
    for (i, j) in ((0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)):
        _column(f, i, j, -0.25, vol)
    return f
