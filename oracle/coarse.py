"""Coarse space V^H and its nodal interpolation into V^h.

Oracle (test infrastructure only).  Section 2.3: the fine partition J_h is a
uniform refinement of the coarse partition J_H, so V^H is a subspace of V^h;
the matrix P (n x n_H) holds, in column c, the fine nodal values of the c-th
coarse basis function.  The coarse matrices of Section 3 are then the
Galerkin products K_H = P^T K P and M_H = P^T M P.

Coarse elements are the same kind as the fine ones on the subdomain grid
(m = n_d / S_d fine cells per coarse cell, equal on every axis so that the
diagonals of the simplicial splits line up and the spaces are nested).  A fine
node at offset r = (r_x, r_y[, r_z]) in {0..m-1}^d inside coarse cell
(I_x, I_y[, I_z]) takes the coarse basis values
  p1_2d, r_x >= r_y : corner (0,0): (m - r_x)/m, (1,0): (r_x - r_y)/m, (1,1): r_y/m
  p1_2d, r_x <  r_y : corner (0,0): (m - r_y)/m, (1,1): r_x/m,        (0,1): (r_y - r_x)/m
  p1_3d (Kuhn)      : with the offsets sorted r_a >= r_b >= r_c:
                      0: (m - r_a)/m, e_a: (r_a - r_b)/m, e_a+e_b: (r_b - r_c)/m, 1: r_c/m
  q1_3d             : prod_d (m - r_d or r_d) / m^3
(barycentric / trilinear coordinates, each an integer divided by m or m^3).
Coarse boundary nodes are dropped (Dirichlet), as are exact zeros.
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def _coarse_index(C, S):
    """Interior coarse node (C_x, C_y[, C_z]) -> coarse dof, x fastest; -1 on the boundary."""
    idx, stride = 0, 1
    for d, c in enumerate(C):
        if c <= 0 or c >= S[d]:
            return -1
        idx += (c - 1) * stride
        stride *= S[d] - 1
    return idx


def _weights(kind, r, m):
    """List of (corner offset tuple, integer numerator, denominator power)."""
    dim = len(r)
    if kind == "p1_2d":
        rx, ry = r
        if rx >= ry:
            return [((0, 0), m - rx, 1), ((1, 0), rx - ry, 1), ((1, 1), ry, 1)]
        return [((0, 0), m - ry, 1), ((1, 1), rx, 1), ((0, 1), ry - rx, 1)]
    if kind == "p1_3d":
        order = sorted(range(3), key=lambda a: -r[a])          # descending offsets
        a, b, c = order
        e = lambda *axes: tuple(1 if q in axes else 0 for q in range(3))
        return [((0, 0, 0), m - r[a], 1), (e(a), r[a] - r[b], 1),
                (e(a, b), r[b] - r[c], 1), ((1, 1, 1), r[c], 1)]
    if kind == "q1_3d":
        out = []
        for corner in itertools.product((0, 1), repeat=dim):
            num = 1
            for d in range(dim):
                num *= r[d] if corner[d] else (m - r[d])
            out.append((corner, num, dim))
        return out
    raise ValueError(kind)


def prolongation(spec) -> sp.csr_matrix:
    """P (n x n_H) as canonical CSR, float64 (for morley_2d the intergrid transfer of
    ``oracle.morley.prolongation``)."""
    if spec.kind == "morley_2d":
        from . import morley
        return morley.prolongation(spec.n[0], spec.nsub[0])
    if spec.kind == "bfs_2d":
        from . import bfs
        return bfs.prolongation(spec.n[0], spec.nsub[0])
    if spec.kind == "q1_lshape":
        from dataclasses import replace
        from .fem import lshape3_map
        Pbox = prolongation(replace(spec, kind="q1_3d"))
        rows = np.flatnonzero(lshape3_map(*spec.n) >= 0)
        cols = np.flatnonzero(lshape3_map(*spec.nsub) >= 0)
        P = Pbox[rows][:, cols].tocsr()
        P.sort_indices()
        return P
    if spec.kind == "p1_lshape":
        # the square's nodal interpolation, rows and columns restricted to the interior
        # nodes of the fine and coarse L-shapes (coarse functions vanish on its boundary)
        from dataclasses import replace
        from .fem import lshape_map
        Psq = prolongation(replace(spec, kind="p1_2d"))
        rows = np.flatnonzero(lshape_map(spec.n[0]) >= 0)
        cols = np.flatnonzero(lshape_map(spec.nsub[0]) >= 0)
        P = Psq[rows][:, cols].tocsr()
        P.sort_indices()
        return P
    n, S, dim = spec.n, spec.nsub, spec.dim
    ms = [n[d] // S[d] for d in range(dim)]
    if len(set(ms)) != 1:
        raise ValueError("coarse cells must have the same number of fine cells on every axis")
    m = ms[0]
    rows, cols, vals = [], [], []
    inner = [q - 1 for q in n]
    for node in itertools.product(*[range(1, n[d]) for d in reversed(range(dim))]):
        node = tuple(reversed(node))                       # (i, j[, l]) with x fastest order
        g, stride = 0, 1
        for d in range(dim):
            g += (node[d] - 1) * stride
            stride *= inner[d]
        cell = [min(node[d] // m, S[d] - 1) for d in range(dim)]
        r = [node[d] - cell[d] * m for d in range(dim)]
        for corner, num, pw in _weights(spec.kind, r, m):
            if num == 0:
                continue
            c = _coarse_index([cell[d] + corner[d] for d in range(dim)], S)
            if c < 0:
                continue
            rows.append(g)
            cols.append(c)
            vals.append(num / float(m ** pw))
    P = sp.csr_matrix((vals, (rows, cols)), shape=(spec.n_dofs, spec.n_coarse))
    P.sum_duplicates()
    P.sort_indices()
    return P
