"""Log-normal anisotropic permeability fields (stand-ins for the SPE10 data).

The paper's experiments use the SPE10 permeability (Sec. "Numerical setup"),
which is not available here.  These generators produce seeded synthetic fields
with the same kind of statistics: a zero-mean Gaussian field g with exponential
covariance sigma^2 * exp(-r / lam) (r in cell units), and K = exp(g).

Sampling is by circulant embedding: the covariance is laid out on a periodic
grid of twice the field's size along every axis (so every in-window distance is
represented exactly), its FFT gives the circulant's eigenvalues, negative ones
are clipped to zero (their mass is reported), and the field is
C^{1/2} w for white noise w drawn from numpy's PCG64 with the given seed.
"""
from __future__ import annotations

import numpy as np


def _embedding_eigs(pshape, sigma, lam, dtype):
    """Eigenvalues (real FFT layout) of the periodic exponential covariance."""
    axes = []
    for n in pshape:
        d = np.arange(n, dtype=np.float64)
        axes.append(np.minimum(d, n - d))
    grids = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    c = (sigma * sigma) * np.exp(-r / lam)
    eig = np.fft.rfftn(c.astype(dtype), axes=tuple(range(len(pshape)))).real
    return eig


def gaussian_field(shape, sigma, lam, seed, return_clipped=False):
    """Zero-mean stationary Gaussian field of the given (nz, ny, nx) or (ny, nx) shape.

    Covariance sigma^2 exp(-|x-y|/lam), |.| Euclidean in cell units.  The field is
    exact up to the clipping of negative embedding eigenvalues, whose relative
    mass is returned when ``return_clipped`` is set.
    """
    shape = tuple(int(s) for s in shape)
    pshape = tuple(2 * s for s in shape)
    big = np.prod(pshape) > 64 * 1024 * 1024
    dtype = np.float32 if big else np.float64
    eig = _embedding_eigs(pshape, sigma, lam, dtype)
    neg = eig < 0
    clipped = float(-eig[neg].sum() / np.abs(eig).sum()) if neg.any() else 0.0
    eig[neg] = 0
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(pshape, dtype=dtype)
    axes = tuple(range(len(pshape)))
    g = np.fft.irfftn(np.sqrt(eig) * np.fft.rfftn(w, axes=axes), s=pshape, axes=axes)
    sl = tuple(slice(0, s) for s in shape)
    g = np.ascontiguousarray(g[sl], dtype=np.float64)
    if return_clipped:
        return g, clipped
    return g


def lognormal_K(shape, sigma, lam, kz_ratio, seed, h=(1.0, 1.0, 1.0)):
    """Diagonal K as a (3, nz, ny, nx) float64 array: Kx = Ky = exp(g), Kz = kz_ratio * Kx.

    ``h`` is accepted for symmetry with other generators; correlation lengths are
    always in cells.
    """
    g = gaussian_field(shape, sigma, lam, seed)
    kx = np.exp(g)
    K = np.empty((3,) + tuple(shape), dtype=np.float64)
    K[0] = kx
    K[1] = kx
    K[2] = kz_ratio * kx
    return K


def layered_field(shape, sigma, lam_range, kz_ratio_range, seed):
    """Layered log-normal K, (3, nz, ny, nx): each z-layer an independent 2-D field.

    Per layer: correlation length ~ U[lam_range], Kz/Kx log-uniform in
    kz_ratio_range.  This mimics the layered, high-contrast character of the
    SPE10 model the paper uses (60x220x85 cells), with sigma as given.
    """
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    lams = rng.uniform(lam_range[0], lam_range[1], size=nz)
    lo, hi = np.log(kz_ratio_range[0]), np.log(kz_ratio_range[1])
    ratios = np.exp(rng.uniform(lo, hi, size=nz))
    layer_seeds = rng.integers(0, 2**62, size=nz)
    K = np.empty((3, nz, ny, nx), dtype=np.float64)
    for k in range(nz):
        g = gaussian_field((ny, nx), sigma, float(lams[k]), int(layer_seeds[k]))
        kx = np.exp(g)
        K[0, k] = kx
        K[1, k] = kx
        K[2, k] = ratios[k] * kx
    return K
