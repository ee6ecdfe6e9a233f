"""Algorithmic cost of the paper's local direct solver (ORACLE - test infrastructure only).

The product path never imports this module.

The paper factors each local TPFA matrix with a sparse direct LDL^T under a
fill-reducing ordering (MUMPS with AMD, Sec. "MBFs: LocalSolver()").  The
algorithmic flop count of the local stage is that factorisation's, from the
elimination of the local matrix graph (the 7-point stencil of the
subdomain's box; Robin terms touch only the diagonal).  Reading: exact
minimum degree stands in for AMD, ties broken by the lowest cell index in
box-lexicographic order (x fastest).  Eliminating a vertex makes its current
neighbours a clique; the neighbour count c_j at elimination is the number of
below-diagonal entries of column j of L.  Flops of column j: c_j(c_j + 1)
for the rank-1 update of the trailing matrix (c_j(c_j+1)/2 multiply-adds)
plus 2 c_j for l = a / d and d l, i.e. c_j (c_j + 3).  A solve with one
right-hand side costs 4 nnz(L) flops (forward and backward, a multiply and
an add per entry), nnz(L) counting the below-diagonal entries.
"""
from __future__ import annotations


def box_graph(sx, sy, sz):
    """Adjacency sets of the 7-point stencil on an sx x sy x sz box (x fastest)."""
    n = sx * sy * sz
    adj = [set() for _ in range(n)]
    for k in range(sz):
        for j in range(sy):
            for i in range(sx):
                c = i + sx * (j + sy * k)
                if i + 1 < sx:
                    adj[c].add(c + 1)
                    adj[c + 1].add(c)
                if j + 1 < sy:
                    adj[c].add(c + sx)
                    adj[c + sx].add(c)
                if k + 1 < sz:
                    adj[c].add(c + sx * sy)
                    adj[c + sx * sy].add(c)
    return adj


def min_degree_counts(adj):
    """Column counts of L under exact minimum degree (ties: lowest index)."""
    G = [set(a) for a in adj]
    alive = set(range(len(G)))
    counts = []
    for _ in range(len(G)):
        v = min(alive, key=lambda x: (len(G[x]), x))
        nb = G[v]
        counts.append(len(nb))
        for a in nb:
            G[a] |= nb
            G[a].discard(a)
            G[a].discard(v)
        alive.remove(v)
        G[v] = set()
    return counts


def ldl_cost(sx, sy, sz):
    """(factor flops, nnz(L) below the diagonal) of one box's local matrix."""
    c = min_degree_counts(box_graph(sx, sy, sz))
    return float(sum(x * (x + 3) for x in c)), int(sum(c))
