"""Staged MRCM: local problems, interface system, reconstruction (ORACLE).

Test infrastructure only: the product path never imports this module.

Follows the paper's Alg. MRCM step by step:

1. For each subdomain l (Alg. MRCM, first loop): assemble the local TPFA
   matrix A^H_l with Robin conditions on the faces lying on Gamma
   (Eq. localomegapar / Eq. localomegaint) and solve Eq. multiscale_functions
   and Eq. particular_problem_discrete: one P-MBF and one U-MBF per basis
   function k in I^l, plus the particular solution.
2. Assemble the interface system of Eq. interface_problem from the MBF flux
   traces and solve it (second stage).
3. Reconstruct p and u in each subdomain from the MBFs (reconstruction
   option 1; option 2, the re-solve, is also provided as a cross-check).

Robin faces.  On a Gamma face f of subdomain l with normal axis a, the
condition -beta u.n^l + p = g (g the Robin data) together with the half-cell
two-point flux u.n^l = 2 K_a (p_c - p_f) / h_a gives the integrated outward
flux q_f = T_R (p_c - g), T_R = A_f / (h_a / (2 K_a) + beta).  This is what the
lowest-order Raviart-Thomas element with trapezoidal quadrature produces.

Robin data of the MBFs (Eq. localomegaint): g = P_H - beta s U_H with
s = n_hat . n^l = +1 on the lower side of the interface and -1 on the upper
side.  P-MBF k: g = phi_k; U-MBF k: g = -beta s phi_k; particular: g = 0 with
the well sources.

beta (Eq. Robin_par): either a constant, or beta = alpha H_a / K_a with H_a the
subdomain's edge length along the face normal and K_a the normal permeability
of the subdomain's own cell next to the face (so beta differs on the two sides).

Interface rows (Eq. weakcont_f, Eq. weakcont_p, with the integrals over a
patch becoming sums over its fine faces):
  F row i:  sum_l sum_{f in phi_i} q_f^l                                 = 0
  U row i:  sum_l sum_{f in phi_i} beta_f^l (s_l q_f^l - A_f U_H(f))     = 0
Writing q^l = sum_j pi^p_j q^l[P_j] + pi^u_j q^l[U_j] + qbar^l gives
A^PP, A^PU, A^UP, A^UU and b^P = -sum qbar, b^U = -sum beta s qbar
(Eq. sec2-int-APP, Eq. sec2-int-AUU, Eq. sec2-int-bU; the garbled A^UP and the
missing sign of b^P are read this way).

Null space.  With no-flow walls everywhere, adding a constant to every pi^p
shifts every subdomain's pressure by that constant and leaves all fluxes
unchanged, so A^int is singular; the sum of the F rows is the (zero) total
source.  F row 0 is then replaced by pi^p_0 = 0 and the pressure is shifted to
zero mean.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .problem import DIRICHLET, Problem, build_bases
from .tpfa import harmonic, normalise_pressure


@dataclasses.dataclass
class RobinFace:
    local_cell: int
    axis: int
    s: int            # +1 if l is the lower side of the interface, -1 otherwise
    T_R: float
    beta: float
    area: float
    basis: int        # global basis index
    col: int          # position of the basis in I^l


@dataclasses.dataclass
class LocalProblem:
    l: int
    lo: list
    size: list
    cells: np.ndarray           # global cell index of each local cell (x fastest in the box)
    A: sp.csr_matrix            # local TPFA + Robin matrix A^H_l
    rhs_part: np.ndarray        # particular right-hand side f V (+ Dirichlet wall terms)
    faces: list                 # RobinFace list
    I: list                     # I^l, sorted global basis indices
    interior: list              # (local a, local b, axis, T) interior faces


def _beta(prob: Problem, l, a, Kc):
    if prob.beta_mode == 0:
        return prob.beta_const
    _, size = prob.sub_box(l)
    return prob.alpha * size[a] * prob.h[a] / Kc


def local_problem(prob: Problem, l, sub_bases, face_basis) -> LocalProblem:
    """Assemble A^H_l and its particular right-hand side (Alg. MRCM, Assembly)."""
    lo, size = prob.sub_box(l)
    sx, sy, sz = size
    n = sx * sy * sz
    kk, jj, ii = np.meshgrid(np.arange(sz), np.arange(sy), np.arange(sx), indexing="ij")
    gi, gj, gk = (ii + lo[0]).ravel(), (jj + lo[1]).ravel(), (kk + lo[2]).ravel()
    cells = prob.cell(gi, gj, gk)
    Kflat = prob.K.reshape(3, -1)
    I = sub_bases[l]
    col_of = {b: c for c, b in enumerate(I)}
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    rhs = prob.f.ravel()[cells] * prob.cell_volume
    interior = []
    faces = []
    local = lambda i, j, k: i + sx * (j + sy * k)
    for a in range(3):
        A_f = prob.face_area(a)
        for k in range(sz):
            for j in range(sy):
                for i in range(sx):
                    c = local(i, j, k)
                    pos = [i, j, k]
                    # interior face towards +a
                    if pos[a] + 1 < size[a]:
                        q = list(pos)
                        q[a] += 1
                        d = local(*q)
                        T = A_f * harmonic(Kflat[a, cells[c]], Kflat[a, cells[d]]) / prob.h[a]
                        rows += [c, d]
                        cols += [d, c]
                        vals += [-T, -T]
                        diag[c] += T
                        diag[d] += T
                        interior.append((c, d, a, T))
                    # the two box faces normal to a
                    for side in (0, 1):
                        if (side == 0 and pos[a] != 0) or (side == 1 and pos[a] != size[a] - 1):
                            continue
                        g = [gi[c], gj[c], gk[c]]
                        wall = (side == 0 and g[a] == 0) or (side == 1 and g[a] == prob.n[a] - 1)
                        Kc = Kflat[a, cells[c]]
                        if wall:
                            if prob.bc_type[a][side] == DIRICHLET:
                                TD = A_f * 2.0 * Kc / prob.h[a]
                                diag[c] += TD
                                rhs[c] += TD * prob.bc_value[a][side]
                            continue
                        if side == 1:
                            clo, s = cells[c], +1
                        else:
                            clo, s = cells[c] - (prob.n[0] if a == 1 else 1 if a == 0 else prob.n[0] * prob.n[1]), -1
                        b = face_basis[(a, clo)]
                        beta = _beta(prob, l, a, Kc)
                        T_R = A_f / (prob.h[a] / (2.0 * Kc) + beta)
                        diag[c] += T_R
                        faces.append(RobinFace(c, a, s, T_R, beta, A_f, b, col_of[b]))
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    rows = np.concatenate([np.atleast_1d(np.asarray(r)) for r in rows])
    cols = np.concatenate([np.atleast_1d(np.asarray(r)) for r in cols])
    vals = np.concatenate([np.atleast_1d(np.asarray(r, dtype=float)) for r in vals])
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return LocalProblem(l, lo, size, cells, A, rhs, faces, I, interior)


def robin_data(lp: LocalProblem):
    """Robin data g_f for every face (rows) and every local column (cols).

    Columns: [P-MBF for k in I^l] + [U-MBF for k in I^l] + [particular].
    """
    m = len(lp.I)
    G = np.zeros((len(lp.faces), 2 * m + 1))
    for r, fc in enumerate(lp.faces):
        G[r, fc.col] = 1.0
        G[r, m + fc.col] = -fc.beta * fc.s
    return G


def mbf_rhs(lp: LocalProblem):
    """Right-hand sides f^H_{l,k;P}, f^H_{l,k;U} and f^H_{l;gamma} as an (n, 2|I|+1) block."""
    n = lp.A.shape[0]
    G = robin_data(lp)
    B = np.zeros((n, G.shape[1]))
    for r, fc in enumerate(lp.faces):
        B[fc.local_cell] += fc.T_R * G[r]
    B[:, -1] += lp.rhs_part
    return B


def solve_local(lp: LocalProblem):
    """LocalSolver: all MBFs and the particular solution of one subdomain, (n, 2|I|+1)."""
    B = mbf_rhs(lp)
    lu = spla.splu(lp.A.tocsc())
    return lu.solve(B)


def traces(lp: LocalProblem, X):
    """Integrated outward Robin fluxes q_f = T_R (p_c - g_f), (faces, columns)."""
    G = robin_data(lp)
    Q = np.zeros_like(G)
    for r, fc in enumerate(lp.faces):
        Q[r] = fc.T_R * (X[fc.local_cell] - G[r])
    return Q


@dataclasses.dataclass
class MRCMResult:
    p: np.ndarray           # (ncells,) pressure, global cell order
    u: np.ndarray           # (6, nz, ny, nx) per-cell face velocities (+axis component)
    X: np.ndarray           # (2 NV,) interface unknowns (pi^p, pi^u)
    A_int: sp.csr_matrix    # interface matrix (after pinning when singular)
    b_int: np.ndarray
    A_int_raw: sp.csr_matrix  # interface matrix before pinning
    b_int_raw: np.ndarray
    locals: list
    mbfs: list              # per subdomain (n_l, 2|I^l|+1)
    traces: list
    mass_residual_max: float


def interface_entries(NV, lp: LocalProblem, Q):
    """One subdomain's block of A^int and b^int (Eq. sec2-int-APP, sec2-int-AUU, sec2-int-bU).

    The faces' traces are summed over each basis function's faces into the
    subdomain's local interface block E (2|I^l| x 2|I^l|, rows and columns
    ordered [P of I^l, U of I^l]) and right-hand side e; returned as COO
    triplets (rows, cols, vals) and (b_rows, b_vals) in global numbering.  The
    interface system is the sum of these blocks over all subdomains.
    """
    m = len(lp.I)
    E = np.zeros((2 * m, 2 * m))
    e = np.zeros(2 * m)
    for r, fc in enumerate(lp.faces):
        k = fc.col
        E[k, :] += Q[r, :2 * m]                          # F row: sum of fluxes
        E[m + k, :] += fc.beta * fc.s * Q[r, :2 * m]     # U row: sum of beta s fluxes
        E[m + k, m + k] -= fc.beta * fc.area             # U row: - beta A_f pi^u
        e[k] -= Q[r, -1]
        e[m + k] -= fc.beta * fc.s * Q[r, -1]
    I = np.asarray(lp.I, dtype=np.int64)
    g = np.concatenate([I, NV + I])
    return np.repeat(g, 2 * m), np.tile(g, 2 * m), E.ravel(), g, e


def assemble_interface(prob: Problem, bases, locs, Qs, entries=None):
    """A^int and b^int of Eq. interface_problem (before any pinning).

    ``entries`` may hold the subdomains' ``interface_entries`` already computed
    (by a worker pool); they are summed in subdomain order either way.
    """
    NV = len(bases)
    if entries is None:
        entries = [interface_entries(NV, lp, Q) for lp, Q in zip(locs, Qs)]
    b = np.zeros(2 * NV)
    for (_, _, _, br, bv) in entries:
        np.add.at(b, br, bv)
    if entries:
        rows = np.concatenate([x[0] for x in entries])
        cols = np.concatenate([x[1] for x in entries])
        vals = np.concatenate([x[2] for x in entries])
    else:
        rows = cols = np.zeros(0, dtype=np.int64)
        vals = np.zeros(0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(2 * NV, 2 * NV))
    A.sum_duplicates()
    return A, b


def pin_interface(prob: Problem, A, b):
    """Replace F row 0 by pi^p_0 = 0 when the walls leave p free up to a constant."""
    if prob.has_dirichlet() or A.shape[0] == 0:
        return A, b
    A = A.tolil()
    A[0, :] = 0.0
    A[0, 0] = 1.0
    b = b.copy()
    b[0] = 0.0
    return A.tocsr(), b


def solve_interface(A, b, refine=2):
    """InterfaceSolver: sparse direct LU plus a few FP64 refinement steps."""
    if A.shape[0] == 0:
        return np.zeros(0)
    lu = spla.splu(A.tocsc())
    x = lu.solve(b)
    for _ in range(refine):
        x = x + lu.solve(b - A @ x)
    return x


def robin_data_final(lp: LocalProblem, X, NV):
    """g_f = P_H(f) - beta s U_H(f) on every Robin face of the subdomain."""
    return np.array([X[fc.basis] - fc.beta * fc.s * X[NV + fc.basis] for fc in lp.faces])


def reconstruct_local(lp: LocalProblem, Xmbf, X, NV):
    """ReconstructMscSolution, option 1: p^l = sum pi^p p(phi,0) + pi^u p(0,phi) + pbar."""
    coef = np.concatenate([X[lp.I], X[NV + np.asarray(lp.I, dtype=int)], [1.0]]) if lp.I else np.array([1.0])
    return Xmbf @ coef


def reconstruct_local_resolve(lp: LocalProblem, X, NV):
    """Option 2: re-solve the local problem with the final Robin data."""
    g = robin_data_final(lp, X, NV)
    rhs = lp.rhs_part.copy()
    for r, fc in enumerate(lp.faces):
        rhs[fc.local_cell] += fc.T_R * g[r]
    return spla.splu(lp.A.tocsc()).solve(rhs)


def local_velocity_entries(prob: Problem, lp: LocalProblem, p_loc, X, NV):
    """The per-cell face velocities of subdomain l as (row, flat cell, value) triplets.

    Interior faces by Eq. two_point; Gamma faces by the Robin flux with the final
    Robin data, each side keeping its own value; walls 0 or the Dirichlet flux.
    Rows index the six faces (x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) of a cell.
    """
    rows, cells, vals = [], [], []
    for (c, d, a, T) in lp.interior:
        vel = T * (p_loc[c] - p_loc[d]) / prob.face_area(a)
        rows += [2 * a + 1, 2 * a]
        cells += [lp.cells[c], lp.cells[d]]
        vals += [vel, vel]
    g = robin_data_final(lp, X, NV) if lp.faces else []
    for r, fc in enumerate(lp.faces):
        q_out = fc.T_R * (p_loc[fc.local_cell] - g[r])
        vel = q_out / fc.area
        if fc.s == +1:   # outward of l is +axis: the cell's high face
            rows.append(2 * fc.axis + 1)
            vals.append(vel)
        else:            # outward of l is -axis: the cell's low face
            rows.append(2 * fc.axis)
            vals.append(-vel)
        cells.append(lp.cells[fc.local_cell])
    # Dirichlet walls
    nx, ny, nz = prob.n
    Kflat = prob.K.reshape(3, -1)
    for a in range(3):
        for side in (0, 1):
            if prob.bc_type[a][side] != DIRICHLET:
                continue
            gval = prob.bc_value[a][side]
            for c, gc in enumerate(lp.cells):
                co = [gc % nx, (gc // nx) % ny, gc // (nx * ny)]
                if (side == 0 and co[a] == 0):
                    rows.append(2 * a)
                    cells.append(gc)
                    vals.append(-2.0 * Kflat[a, gc] * (p_loc[c] - gval) / prob.h[a])
                if (side == 1 and co[a] == prob.n[a] - 1):
                    rows.append(2 * a + 1)
                    cells.append(gc)
                    vals.append(-2.0 * Kflat[a, gc] * (gval - p_loc[c]) / prob.h[a])
    return np.asarray(rows, dtype=np.int64), np.asarray(cells, dtype=np.int64), np.asarray(vals, dtype=float)


def local_velocities(prob: Problem, lp: LocalProblem, p_loc, X, NV, u):
    """Fill the per-cell face velocities of subdomain l into u (6, nz, ny, nx)."""
    rows, cells, vals = local_velocity_entries(prob, lp, p_loc, X, NV)
    u.reshape(6, -1)[rows, cells] = vals


def mass_residual(prob: Problem, u):
    """Per-cell sum of outward integrated fluxes minus f V (zero for a conservative field)."""
    div = np.zeros(prob.f.shape)
    for a in range(3):
        div += (u[2 * a + 1] - u[2 * a]) * prob.face_area(a)
    return div - prob.f * prob.cell_volume


# ---- worker pool (Sec. 8(d) oracle timing: subdomains are independent, one process per core)
_POOL_STATE = {}


def _pool_init(prob, sub_bases, face_basis, NV):
    _POOL_STATE.update(prob=prob, sub_bases=sub_bases, face_basis=face_basis, NV=NV)


def _pool_local(ls):
    """Local stage of a chunk of subdomains: A^H_l, all MBF columns, traces, interface block."""
    st = _POOL_STATE
    out = []
    for l in ls:
        lp = local_problem(st["prob"], l, st["sub_bases"], st["face_basis"])
        Xl = solve_local(lp)
        Q = traces(lp, Xl)
        out.append((lp if st.get("keep_locals") else None, Xl, Q, interface_entries(st["NV"], lp, Q)))
    return out


def _pool_reconstruct(task):
    """Reconstruction of a chunk of subdomains (the local problem is re-assembled
    where it was not kept): p^l and the face-velocity triplets."""
    items, X, option = task
    st = _POOL_STATE
    out = []
    for l, lp, Xl in items:
        if lp is None:
            lp = local_problem(st["prob"], l, st["sub_bases"], st["face_basis"])
        pl = reconstruct_local(lp, Xl, X, st["NV"]) if option == 1 else reconstruct_local_resolve(lp, X, st["NV"])
        out.append((lp.cells, pl, local_velocity_entries(st["prob"], lp, pl, X, st["NV"])))
    return out


def _chunks(seq, n):
    return [seq[i:i + n] for i in range(0, len(seq), n)]


def make_pool(prob: Problem, processes):
    """A pool of ``processes`` spawned workers holding ``prob`` (one BLAS thread each).

    Pass it to ``solve_mrcm(pool=...)`` to reuse it over several solves of the
    same problem; close it with ``pool.close(); pool.join()``.
    """
    import multiprocessing as mp
    import os
    bases, sub_bases, face_basis = build_bases(prob)
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    try:
        pool = mp.get_context("spawn").Pool(processes, initializer=_pool_init,
                                            initargs=(prob, sub_bases, face_basis, len(bases)))
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    pool.n_procs = processes
    return pool


def solve_mrcm(prob: Problem, option=1, keep=True, processes=None, pool=None) -> MRCMResult:
    """Run Alg. MRCM end to end on the CPU in FP64.

    ``processes`` > 1 runs the per-subdomain work (local problems, MBFs,
    traces, interface blocks, reconstruction) in a pool of that many spawned
    processes, one BLAS thread each (or ``pool``, from ``make_pool`` for this
    problem); the arithmetic and the order of every sum are the same as with
    one process.  The pool does not ship the local problems back (the
    reconstruction re-assembles them), so the result's ``locals`` is empty
    then.
    """
    bases, sub_bases, face_basis = build_bases(prob)
    NV = len(bases)
    locs, mbfs, Qs, entries = [], [], [], []
    own_pool = False
    if pool is None and processes and processes > 1 and prob.nsub > 1:
        pool = make_pool(prob, processes)
        own_pool = True
    nproc = getattr(pool, "n_procs", 1) if pool else 1
    try:
        chunk = max(1, prob.nsub // (4 * nproc)) if pool else prob.nsub
        if pool:
            parts = pool.map(_pool_local, _chunks(list(range(prob.nsub)), chunk))
        else:
            _pool_init(prob, sub_bases, face_basis, NV)
            _POOL_STATE["keep_locals"] = True
            parts = [_pool_local(list(range(prob.nsub)))]
        for part in parts:
            for lp, Xl, Q, ent in part:
                if lp is not None:
                    locs.append(lp)
                mbfs.append(Xl)
                Qs.append(Q)
                entries.append(ent)
        A_raw, b_raw = assemble_interface(prob, bases, locs, Qs, entries)
        A, b = pin_interface(prob, A_raw, b_raw)
        X = solve_interface(A, b)
        p = np.zeros(prob.ncells)
        u = np.zeros((6,) + prob.f.shape)
        items = [(l, locs[l] if locs else None, mbfs[l]) for l in range(prob.nsub)]
        tasks = [(c, X, option) for c in _chunks(items, chunk)]
        rparts = pool.map(_pool_reconstruct, tasks) if pool else [_pool_reconstruct(t) for t in tasks]
        uf = u.reshape(6, -1)
        for part in rparts:
            for cells_l, pl, (rows, cells, vals) in part:
                p[cells_l] = pl
                uf[rows, cells] = vals
    finally:
        if own_pool:
            pool.close()
            pool.join()
        if not pool:
            _POOL_STATE.clear()
    shift = 0.0 if prob.has_dirichlet() else p.mean()
    p = p - shift
    res = mass_residual(prob, u)
    return MRCMResult(p, u, X, A, b, A_raw, b_raw, locs if keep else [], mbfs if keep else [],
                      Qs if keep else [], float(np.abs(res).max()))


def relative_errors(prob: Problem, p, u, p_ref, u_ref):
    """Relative L2 pressure error and K^{-1}-weighted velocity error (Sec. "Numerical setup").

    The velocity norm integrates K^{-1}|v|^2 with the trapezoidal rule on each
    cell: sum over cells and over the cell's six faces of (V/2) u_f^2 / K_a,
    each cell using its own face values.
    """
    V = prob.cell_volume
    ep = np.sqrt(np.sum(V * (p - p_ref) ** 2)) / max(np.sqrt(np.sum(V * p_ref ** 2)), 1e-300)
    num = den = 0.0
    for a in range(3):
        w = 0.5 * V / prob.K[a]
        for side in (0, 1):
            num += np.sum(w * (u[2 * a + side] - u_ref[2 * a + side]) ** 2)
            den += np.sum(w * u_ref[2 * a + side] ** 2)
    ev = np.sqrt(num) / max(np.sqrt(den), 1e-300)
    return float(ep), float(ev)
