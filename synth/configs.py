"""Named synthetic workloads shaped like the paper's experiments.

A workload fixes the grid, the per-axis subdomain edge lists, the interface
patch sizes, the Robin parameter mode and the recipe for K and f.  Nothing
here computes anything of the method; edge lists and patch sizes are inputs.

Patch sizes are given per face orientation as ``patch[a] = (p1, p2)``: for
faces normal to axis ``a`` the two tangential axes are taken in increasing
order and ``p1``/``p2`` count fine faces along the first/second of them;
0 means "the whole face".
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from .fields import layered_field, lognormal_K
from .wells import corner_wells, five_spot_wells

BETA_CONST = 0
BETA_ALPHA_H_OVER_K = 1


def uniform_edges(n, e):
    assert n % e == 0, (n, e)
    return [e] * (n // e)


def random_edges(n, choices, rng):
    """Edges drawn from ``choices`` until they cover n; the last one is truncated."""
    out = []
    tot = 0
    while tot < n:
        e = int(rng.choice(choices))
        e = min(e, n - tot)
        out.append(e)
        tot += e
    return out


@dataclasses.dataclass
class Workload:
    name: str
    n: tuple                      # (nx, ny, nz)
    edges: tuple                  # (list_x, list_y, list_z) subdomain edges in cells
    patch: tuple                  # ((p1,p2) for x-faces, y-faces, z-faces)
    beta_mode: int = BETA_CONST
    alpha: float = 1.0
    beta_const: float = 1.0
    h: tuple = (1.0, 1.0, 1.0)
    make_K: Optional[Callable] = None
    make_f: Optional[Callable] = None
    note: str = ""

    @property
    def cells(self):
        return int(np.prod(self.n))

    @property
    def n_sub(self):
        return len(self.edges[0]) * len(self.edges[1]) * len(self.edges[2])

    def K(self):
        return self.make_K()

    def f(self):
        return self.make_f()


def _c1():
    nx, ny, nz = 40, 40, 8
    return Workload(
        name="mrcm_40x40x8_sub10x10x4_patch5x2",
        n=(nx, ny, nz),
        edges=(uniform_edges(nx, 10), uniform_edges(ny, 10), uniform_edges(nz, 4)),
        # x-faces are 10(y) x 4(z): 5 along y, 2 along z; same for y-faces (x, z);
        # z-faces are 10(x) x 10(y): 5 along x, 2 along y.
        patch=((5, 2), (5, 2), (5, 2)),
        beta_mode=BETA_CONST, beta_const=1.0,
        make_K=lambda: lognormal_K((nz, ny, nx), 2.0, 8.0, 0.1, seed=0),
        make_f=lambda: corner_wells(nx, ny, nz),
        note="40x40x8 cells, 4x4x2 subdomains of 10x10x4, 5x2-face patches, beta=1, "
             "sigma=2 lambda=8 Kz=0.1Kx seed 0, corner injector/producer",
    )


def _c2(beta_mode=BETA_CONST):
    nx, ny, nz = 60, 220, 85
    return Workload(
        name="mrcm_60x220x85_sub10x10x5_patch5x5" + ("_betaHK" if beta_mode else ""),
        n=(nx, ny, nz),
        edges=(uniform_edges(nx, 10), uniform_edges(ny, 10), uniform_edges(nz, 5)),
        patch=((5, 5), (5, 5), (5, 5)),
        beta_mode=beta_mode, alpha=1.0, beta_const=1.0,
        make_K=lambda: layered_field((nz, ny, nx), 3.0, (4.0, 20.0), (1e-3, 0.1), seed=0),
        make_f=lambda: five_spot_wells(nx, ny, nz),
        note="60x220x85 cells (SPE10 shape), 6x22x17=2244 subdomains of 10x10x5, 5x5 patches, "
             "layered sigma=3, per-layer lambda U[4,20], Kz/Kx log-U[1e-3,0.1], seed 0, 5-spot",
    )


def _c3():
    nx, ny, nz = 256, 256, 128
    rng = np.random.Generator(np.random.PCG64(0))
    ex = random_edges(nx, [8, 12, 16], rng)
    ey = random_edges(ny, [8, 12, 16], rng)
    ez = random_edges(nz, [8, 12, 16], rng)
    return Workload(
        name="mrcm_256x256x128_uneven_8_12_16",
        n=(nx, ny, nz), edges=(ex, ey, ez),
        patch=((0, 0), (0, 0), (0, 0)),
        beta_mode=BETA_CONST, beta_const=1.0,
        make_K=lambda: lognormal_K((nz, ny, nx), 2.5, 8.0, 0.1, seed=0),
        make_f=lambda: five_spot_wells(nx, ny, nz),
        note="256x256x128 cells, per-axis edges from {8,12,16} (seed 0, last truncated), "
             "whole-face patches, sigma=2.5 lambda=8 Kz=0.1Kx",
    )


def _c5():
    nx, ny, nz = 512, 512, 256
    return Workload(
        name="mrcm_512x512x256_sub16x16x8",
        n=(nx, ny, nz),
        edges=(uniform_edges(nx, 16), uniform_edges(ny, 16), uniform_edges(nz, 8)),
        patch=((0, 0), (0, 0), (0, 0)),
        beta_mode=BETA_CONST, beta_const=1.0,
        make_K=lambda: lognormal_K((nz, ny, nx), 3.0, 8.0, 0.05, seed=0),
        make_f=lambda: five_spot_wells(nx, ny, nz),
        note="512x512x256 cells, 32768 subdomains of 16x16x8, whole-face patches, "
             "sigma=3 lambda=8 Kz=0.05Kx",
    )


def _c5_slab():
    """A 128 x 256 x 128 slab of the C5 layout (2048 subdomains of 16 x 16 x 8):
    the same kernels and block shapes at a size a full profiler capture handles."""
    nx, ny, nz = 128, 256, 128
    return Workload(
        name="mrcm_128x256x128_sub16x16x8",
        n=(nx, ny, nz),
        edges=(uniform_edges(nx, 16), uniform_edges(ny, 16), uniform_edges(nz, 8)),
        patch=((0, 0), (0, 0), (0, 0)),
        beta_mode=BETA_CONST, beta_const=1.0,
        make_K=lambda: lognormal_K((nz, ny, nx), 3.0, 8.0, 0.05, seed=0),
        make_f=lambda: five_spot_wells(nx, ny, nz),
        note="128x256x128 cells, 2048 subdomains of 16x16x8, whole-face patches, "
             "sigma=3 lambda=8 Kz=0.05Kx",
    )


def small(n=(8, 8, 4), edges=None, patch=((0, 0), (0, 0), (0, 0)), sigma=1.0, lam=3.0,
          kz_ratio=0.3, seed=1, beta_mode=BETA_CONST, beta_const=1.0, alpha=1.0,
          wells="corner", h=(1.0, 1.0, 1.0)):
    """A small seeded workload for tests (several tiles, ragged edges allowed)."""
    nx, ny, nz = n
    if edges is None:
        edges = ([nx // 2, nx - nx // 2], [ny // 2, ny - ny // 2], [nz])
    mk = corner_wells if wells == "corner" else five_spot_wells
    return Workload(
        name=f"small_{nx}x{ny}x{nz}", n=(nx, ny, nz), edges=tuple(list(e) for e in edges),
        patch=patch, beta_mode=beta_mode, alpha=alpha, beta_const=beta_const, h=h,
        make_K=lambda: lognormal_K((nz, ny, nx), sigma, lam, kz_ratio, seed=seed),
        make_f=lambda: mk(nx, ny, nz, h),
    )


WORKLOADS = {
    "c1": _c1,
    "c2": _c2,
    "c2_betaHK": lambda: _c2(BETA_ALPHA_H_OVER_K),
    "c3": _c3,
    "c5": _c5,
    "c5_slab": _c5_slab,
}


def workload(name):
    return WORKLOADS[name]()


# Settings of the timed mixed-precision solve per workload: FP64 refinement
# sweeps after the first FP32 solve, the per-column stop ||r|| <= tol ||b||,
# the memory budget of the local block factors per wave (GB, 0 = one wave),
# and the FP64 refinement steps of the interface solve (-1 = none: the
# interface LDL^T with its exactly emulated trailing updates already meets
# the oracle to 1e-10 at C2, and the step costs 0.8 ms there).  The benchmark
# times these and the full-size parity tests check them.
BENCH_SETTINGS = {
    "c1": dict(ir_sweeps=3, ir_tol=1e-9, wave_gb=0.0, interface_refine=-1),
    "c2": dict(ir_sweeps=5, ir_tol=1e-9, wave_gb=0.0, interface_refine=-1),
    "c2_betaHK": dict(ir_sweeps=5, ir_tol=1e-9, wave_gb=0.0, interface_refine=-1),
    "c3": dict(ir_sweeps=4, ir_tol=1e-9, wave_gb=0.0, interface_refine=-1),
    "c5": dict(ir_sweeps=7, ir_tol=1e-9, wave_gb=16.0, interface_refine=-1),
    "c5_slab": dict(ir_sweeps=6, ir_tol=1e-9, wave_gb=0.0, interface_refine=-1),
}
