"""Problem description and the interface space V_H (ORACLE - test infrastructure only).

This package is the plain CPU FP64 reference that the CUDA path is checked
against.  Only tests, the package smoke check and the bench's CPU-baseline leg
may import it; the product path never does.

Geometry follows Sec. "Domain decomposition and Darcy solvers" of the paper:
a Cartesian grid of nx x ny x nz cells of size (hx, hy, hz), cut into
non-overlapping box subdomains by per-axis edge lists.  Cells are numbered
c = i + nx*(j + ny*k) (x fastest); subdomains l = ix + Nx*(iy + Ny*iz).
Because numbering is lexicographic, the lower-indexed side of every interface
is the side with the lower coordinate, so n_hat = n^{min(l,l')} is always the
+axis direction.

The interface space V_H (Sec. "A domain decomposition Multiscale Mixed
method", Fig. "decomposition_h_H") consists of indicator functions of patches:
on every interface Gamma_{l,l'} normal to axis a, the fine faces are grouped
into rectangles of p1 x p2 faces along the two tangential axes (taken in
increasing axis order), tiled from the interface's lower corner, with the last
rectangle truncated when p does not divide the edge.  Basis functions are
numbered by normal axis, then by lower subdomain index, then by patch
(second tangential axis slow, first fast).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NOFLOW = 0
DIRICHLET = 1


@dataclasses.dataclass
class Problem:
    n: tuple                 # (nx, ny, nz)
    h: tuple                 # (hx, hy, hz)
    edges: tuple             # per-axis subdomain edge lists (cells)
    patch: tuple             # ((p1, p2) per normal axis); 0 = whole face
    K: np.ndarray            # (3, nz, ny, nx) diagonal permeability
    f: np.ndarray            # (nz, ny, nx) source density (div u = f)
    beta_mode: int = 0       # 0: beta = beta_const; 1: beta = alpha * H_a / K_a (Eq. Robin_par)
    alpha: float = 1.0
    beta_const: float = 1.0
    bc_type: tuple = ((NOFLOW, NOFLOW),) * 3     # per axis (low wall, high wall)
    bc_value: tuple = ((0.0, 0.0),) * 3          # Dirichlet pressure per wall

    # ---- derived geometry -------------------------------------------------
    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        self.h = tuple(float(v) for v in self.h)
        self.edges = tuple(tuple(int(e) for e in ed) for ed in self.edges)
        for a in range(3):
            assert sum(self.edges[a]) == self.n[a], (a, self.edges[a], self.n[a])
        self.Nd = tuple(len(e) for e in self.edges)
        self.starts = tuple(np.concatenate([[0], np.cumsum(e)]).astype(int) for e in self.edges)
        self.K = np.asarray(self.K, dtype=np.float64)
        self.f = np.asarray(self.f, dtype=np.float64)
        nx, ny, nz = self.n
        assert self.K.shape == (3, nz, ny, nx)
        assert self.f.shape == (nz, ny, nx)

    @property
    def ncells(self):
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def nsub(self):
        return self.Nd[0] * self.Nd[1] * self.Nd[2]

    @property
    def cell_volume(self):
        return self.h[0] * self.h[1] * self.h[2]

    def face_area(self, a):
        return float(np.prod([self.h[b] for b in range(3) if b != a]))

    def has_dirichlet(self):
        return any(t == DIRICHLET for pair in self.bc_type for t in pair)

    def cell(self, i, j, k):
        nx, ny, _ = self.n
        return i + nx * (j + ny * k)

    def sub_coords(self, l):
        Nx, Ny, _ = self.Nd
        return [l % Nx, (l // Nx) % Ny, l // (Nx * Ny)]

    def sub_index(self, idx):
        Nx, Ny, _ = self.Nd
        return idx[0] + Nx * (idx[1] + Ny * idx[2])

    def sub_box(self, l):
        idx = self.sub_coords(l)
        lo = [int(self.starts[a][idx[a]]) for a in range(3)]
        size = [int(self.edges[a][idx[a]]) for a in range(3)]
        return lo, size

    def sub_of_cell(self):
        """(nz, ny, nx) array of subdomain indices."""
        ids = []
        for a in range(3):
            ids.append(np.repeat(np.arange(self.Nd[a]), self.edges[a]))
        Nx, Ny, _ = self.Nd
        return ids[0][None, None, :] + Nx * (ids[1][None, :, None] + Ny * ids[2][:, None, None])


def from_workload(w, K=None, f=None, **overrides):
    """Build a Problem from a synth.Workload (K and f drawn if not given)."""
    kw = dict(n=w.n, h=w.h, edges=w.edges, patch=w.patch,
              K=w.K() if K is None else K, f=w.f() if f is None else f,
              beta_mode=w.beta_mode, alpha=w.alpha, beta_const=w.beta_const)
    kw.update(overrides)
    return Problem(**kw)


@dataclasses.dataclass
class Basis:
    axis: int
    lo: int                 # lower-side subdomain (s = +1)
    hi: int                 # upper-side subdomain (s = -1)
    faces: list             # [(cell_lo, cell_hi)] fine faces in the patch


def build_bases(prob: Problem):
    """Enumerate the patch basis functions phi_k of V_H in canonical order.

    Returns (bases, sub_bases, face_basis) where sub_bases[l] is the sorted list
    I^l of basis indices supported on the boundary of subdomain l and
    face_basis maps (axis, cell_lo) -> basis index for every fine Gamma face.
    """
    bases = []
    sub_bases = [[] for _ in range(prob.nsub)]
    face_basis = {}
    for a in range(3):
        t1, t2 = [b for b in range(3) if b != a]
        for l in range(prob.nsub):
            idx = prob.sub_coords(l)
            if idx[a] == prob.Nd[a] - 1:
                continue
            idx2 = list(idx)
            idx2[a] += 1
            l2 = prob.sub_index(idx2)
            lo1, E1 = int(prob.starts[t1][idx[t1]]), int(prob.edges[t1][idx[t1]])
            lo2, E2 = int(prob.starts[t2][idx[t2]]), int(prob.edges[t2][idx[t2]])
            p1, p2 = prob.patch[a]
            p1 = E1 if p1 == 0 else min(p1, E1)
            p2 = E2 if p2 == 0 else min(p2, E2)
            n1, n2 = math.ceil(E1 / p1), math.ceil(E2 / p2)
            xa = int(prob.starts[a][idx[a] + 1])
            for q2 in range(n2):
                for q1 in range(n1):
                    faces = []
                    for c2 in range(lo2 + q2 * p2, min(lo2 + (q2 + 1) * p2, lo2 + E2)):
                        for c1 in range(lo1 + q1 * p1, min(lo1 + (q1 + 1) * p1, lo1 + E1)):
                            co = [0, 0, 0]
                            co[a], co[t1], co[t2] = xa - 1, c1, c2
                            clo = prob.cell(*co)
                            co[a] = xa
                            chi = prob.cell(*co)
                            faces.append((clo, chi))
                    k = len(bases)
                    bases.append(Basis(a, l, l2, faces))
                    sub_bases[l].append(k)
                    sub_bases[l2].append(k)
                    for (clo, _) in faces:
                        face_basis[(a, clo)] = k
    for l in range(prob.nsub):
        sub_bases[l].sort()
    return bases, sub_bases, face_basis


def count_interface_dofs(Nd, H_over_Hbar):
    """#{phi_j} of Eq. dof_PH for a uniform decomposition.

    Nd = (N_d1, N_d2, N_d3) subdomains per axis; H_over_Hbar = (H1/Hbar1, H2/Hbar2,
    H3/Hbar3).  Interfaces normal to axis a number (N_da - 1) * prod(other N_d),
    each carrying the product of the two tangential ratios.
    """
    total = 0
    for a in range(3):
        t1, t2 = [b for b in range(3) if b != a]
        total += (Nd[a] - 1) * Nd[t1] * Nd[t2] * H_over_Hbar[t1] * H_over_Hbar[t2]
    return total


def interior_rhs_count(per_face_dofs):
    """Right-hand sides of one interior subdomain: 2|I^l| MBFs plus the particular one.

    ``per_face_dofs[a]`` is the number of basis functions on each face normal to a
    (Sec. "A domain decomposition Multiscale Mixed method": an interior subdomain
    has two faces per axis).
    """
    return 2 * sum(2 * d for d in per_face_dofs) + 1
