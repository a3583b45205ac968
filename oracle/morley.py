"""Morley element for the clamped plate (the fourth-order model problem, m = 2).

Oracle (test infrastructure only).

Section 2.1: Delta^2 u = lambda u in Omega with u = du/dn = 0 on the boundary,
a(u, v) = int Delta u Delta v on H^2_0(Omega), which there equals
int D^2 u : D^2 v (two integrations by parts).  The paper discretises this
problem with BFS elements; this module uses Morley's nonconforming quadratic
triangle with the element-wise (broken) Hessian form
    a_h(u, v) = sum_T int_T D^2 u : D^2 v,        b(u, v) = int u v,
the broken form for which the Morley element is consistent.

Mesh: the square [0, L]^2 cut into n x n squares, each split along its SW->NE
diagonal (as for p1_2d).  The Morley degrees of freedom sit on the half-grid
of points (X h/2, Y h/2), X, Y = 0..2n, one per point:
    X, Y both even     vertex value                       u
    X odd,  Y even     horizontal edge midpoint           h du/dy
    X even, Y odd      vertical edge midpoint             h du/dx
    X, Y both odd      diagonal edge midpoint             h (du/dx - du/dy)
i.e. normal derivatives with fixed global normals (+y, +x, (1, -1)/sqrt 2),
scaled by h, h and h sqrt 2 so that every element quantity is a rational
number times a power of h.  The clamped conditions remove exactly the
half-grid points on the boundary: the dofs are the interior half-grid points,
numbered (Y - 1)(2n - 1) + (X - 1) (x fastest).  Simply supported conditions
(u = 0 on the boundary only) keep the boundary edge midpoints.

The coarse space is conforming: BFS bicubics on the subdomain grid, brought into
V^h by the Morley interpolant (their values at fine vertices and scaled normal
derivatives at fine edge midpoints); its Galerkin eigenvalues lie within a few
tenths of a percent of the fine ones, where an averaging transfer from a coarse
Morley space gives a coarse pencil 1.7 to 30 times too stiff.

All rational work uses ``fractions.Fraction``; floats appear only when the
element matrices are scaled by h and when the transfer matrix is returned.
"""

from __future__ import annotations

from fractions import Fraction as F
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

# monomials xi^p eta^q of the element's scaled coordinates (xi, eta) = (x - x_SW, y - y_SW) / h
MONO = ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2))

# reference elements of the unit square: (xi, eta, functional) per local dof
_REF_DOFS = {
    "lower": ((0, 0, "v"), (1, 0, "v"), (1, 1, "v"),                   # SW, SE, NE
              (F(1, 2), 0, "dy"), (1, F(1, 2), "dx"), (F(1, 2), F(1, 2), "dd")),
    "upper": ((0, 0, "v"), (1, 1, "v"), (0, 1, "v"),                   # SW, NE, NW
              (F(1, 2), F(1, 2), "dd"), (F(1, 2), 1, "dy"), (0, F(1, 2), "dx")),
}


def half_grid_kind(X: int, Y: int) -> str:
    """Functional attached to half-grid point (X, Y)."""
    return {(0, 0): "v", (1, 0): "dy", (0, 1): "dx", (1, 1): "dd"}[(X % 2, Y % 2)]


def _mono_value(p, q, x, y):
    return F(x) ** p * F(y) ** q


def _mono_dxi(p, q, x, y):
    return p * F(x) ** (p - 1) * F(y) ** q if p > 0 else F(0)


def _mono_deta(p, q, x, y):
    return q * F(x) ** p * F(y) ** (q - 1) if q > 0 else F(0)


def functional(kind, p, q, x, y):
    """The (scaled) dof functional applied to the monomial xi^p eta^q at (x, y):
    value, d/deta (= h d/dy), d/dxi (= h d/dx) or d/dxi - d/deta."""
    if kind == "v":
        return _mono_value(p, q, x, y)
    if kind == "dy":
        return _mono_deta(p, q, x, y)
    if kind == "dx":
        return _mono_dxi(p, q, x, y)
    if kind == "dd":
        return _mono_dxi(p, q, x, y) - _mono_deta(p, q, x, y)
    raise ValueError(kind)


def _inverse(A):
    """Gauss-Jordan inverse of a small square matrix of Fractions."""
    n = len(A)
    M = [list(row) + [F(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:] for row in M]


@lru_cache(maxsize=None)
def reference_basis(shape: str):
    """Coefficients C[m][a] of the Morley basis of the reference triangle: basis a =
    sum_m C[m][a] xi^p_m eta^q_m, dual to the six dof functionals (unisolvence)."""
    V = [[functional(kind, p, q, x, y) for (p, q) in MONO] for (x, y, kind) in _REF_DOFS[shape]]
    return _inverse(V)


def _tri_integral(shape, p, q):
    """int xi^p eta^q over the reference triangle: lower = {0 <= eta <= xi <= 1},
    upper = {0 <= xi <= eta <= 1}."""
    if shape == "lower":
        return F(1, (q + 1) * (p + q + 2))
    return F(1, (p + 1) * (p + q + 2))


@lru_cache(maxsize=None)
def reference_matrices(shape: str):
    """Element stiffness and mass of the reference triangle with h = 1, as Fractions.
    Stiffness: area (1/2) times the Frobenius product of the constant Hessians
    [[2 c_xx, c_xy], [c_xy, 2 c_yy]]; mass: exact integral of the basis products.
    For cell size h the element matrices are S / h^2 and R h^2."""
    C = reference_basis(shape)
    S = [[F(0)] * 6 for _ in range(6)]
    R = [[F(0)] * 6 for _ in range(6)]
    for a in range(6):
        for b in range(6):
            hxx = 4 * C[3][a] * C[3][b]
            hxy = 2 * C[4][a] * C[4][b]
            hyy = 4 * C[5][a] * C[5][b]
            S[a][b] = F(1, 2) * (hxx + hxy + hyy)
            acc = F(0)
            for m1, (p1, q1) in enumerate(MONO):
                for m2, (p2, q2) in enumerate(MONO):
                    acc += C[m1][a] * C[m2][b] * _tri_integral(shape, p1 + p2, q1 + q2)
            R[a][b] = acc
    return S, R


def _local_offsets(shape):
    return [(int(2 * x), int(2 * y)) for (x, y, _) in _REF_DOFS[shape]]


def assemble_full(n: int, L: float = 1.0):
    """K, M over ALL half-grid points (boundary included), point id Y (2n + 1) + X."""
    h = L / n
    side = 2 * n + 1
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    conns, Kes, Mes = [], [], []
    for shape in ("lower", "upper"):
        S, R = reference_matrices(shape)
        Ks = np.array([[float(v) for v in row] for row in S]) / (h * h)
        Ms = np.array([[float(v) for v in row] for row in R]) * (h * h)
        offs = _local_offsets(shape)
        conn = np.stack([(2 * jj + oy) * side + (2 * ii + ox) for (ox, oy) in offs], -1).reshape(-1, 6)
        conns.append(conn)
        Kes.append(np.broadcast_to(Ks, (conn.shape[0], 6, 6)))
        Mes.append(np.broadcast_to(Ms, (conn.shape[0], 6, 6)))
    conn = np.concatenate(conns)
    Ke = np.concatenate(Kes)
    Me = np.concatenate(Mes)
    rows = np.repeat(conn, 6, axis=1).ravel()
    cols = np.tile(conn, (1, 6)).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(side * side,) * 2).tocsr()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(side * side,) * 2).tocsr()
    for A in (K, M):
        A.sum_duplicates()
        A.sort_indices()
    return K, M


def dof_points(n: int, bc: str = "clamped"):
    """Half-grid point ids (Y (2n + 1) + X) of the dofs, in dof order."""
    side = 2 * n + 1
    Y, X = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    inside = (X > 0) & (X < 2 * n) & (Y > 0) & (Y < 2 * n)
    if bc == "clamped":
        keep = inside
    elif bc == "simply_supported":
        on_vertex = (X % 2 == 0) & (Y % 2 == 0)
        keep = inside | ~on_vertex          # boundary edge midpoints stay free
    else:
        raise ValueError(bc)
    return np.flatnonzero(keep)


def assemble(n: int, L: float = 1.0, bc: str = "clamped"):
    """Stiffness K and mass M on the dofs of the given boundary condition (canonical CSR)."""
    Kf, Mf = assemble_full(n, L)
    keep = dof_points(n, bc)
    K = Kf[keep][:, keep].tocsr()
    M = Mf[keep][:, keep].tocsr()
    for A in (K, M):
        A.sum_duplicates()
        A.sort_indices()
    return K, M


def transfer_full(n: int, S: int):
    """The transfer V^H -> V^h over all half-grid points, as a dict
    {(fine point, coarse dof): Fraction}.  V^H is the conforming BFS space (C^1
    bicubic Hermite functions, ``oracle.bfs``) on the S x S subdomain grid, coarse
    dofs 4 (J (S + 1) + I) + a + 2 b for node (I, J) with x / y derivative orders a, b
    (derivatives scaled by H); a fine dof takes its Morley functional (value or scaled
    normal derivative at its point) of the coarse function, which is C^1, so every
    coarse cell holding the point gives the same value; the lowest-indexed one is used."""
    if n % S != 0:
        raise ValueError("n must be a multiple of S")
    m = n // S
    side, cside = 2 * n + 1, S + 1
    out = {}
    for Y in range(side):
        for X in range(side):
            I, J = min(X // (2 * m), S - 1), min(Y // (2 * m), S - 1)
            for a, b, val in _cell_values(m, X - 2 * m * I, Y - 2 * m * J, half_grid_kind(X, Y)):
                c = 4 * ((J + (b >> 1)) * cside + I + (a >> 1)) + (a & 1) + 2 * (b & 1)
                key = (Y * side + X, c)
                out[key] = out.get(key, F(0)) + val
    return out


@lru_cache(maxsize=None)
def _cell_values(m: int, tx: int, ty: int, kind: str):
    """The fine functional `kind` of the 16 coarse bicubic Hermite basis functions of a
    coarse cell at local position (tx, ty) / (2 m): tuples (a, b, value), nonzero only;
    a / b = local x / y dof (node offset a >> 1, derivative order a & 1)."""
    from .bfs import hermite_basis
    C = hermite_basis()

    def herm(s):
        v = [sum(C[p][a] * s ** p for p in range(4)) for a in range(4)]
        d = [sum(p * C[p][a] * s ** (p - 1) for p in range(1, 4)) for a in range(4)]
        return v, d

    vx, dx = herm(F(tx, 2 * m))
    vy, dy = herm(F(ty, 2 * m))
    res = []
    for b in range(4):
        for a in range(4):
            u = vx[a] * vy[b]
            ux = dx[a] * vy[b] / m              # fine h d/dx = (h / H) d/ds
            uy = vx[a] * dy[b] / m
            val = {"v": u, "dy": uy, "dx": ux, "dd": ux - uy}[kind]
            if val != 0:
                res.append((a, b, val))
    return tuple(res)


def prolongation(n: int, S: int) -> sp.csr_matrix:
    """P (n_dofs x n_H) between the clamped spaces: rows = fine interior half-grid points,
    columns = the four dofs of the interior coarse nodes (node-major), exact zeros
    dropped, each entry the correctly rounded value of its rational."""
    side, cside = 2 * n + 1, S + 1
    fine = -np.ones(side * side, dtype=np.int64)
    fine[dof_points(n)] = np.arange((2 * n - 1) ** 2)
    coarse = -np.ones(4 * cside * cside, dtype=np.int64)
    for J in range(1, S):
        for I in range(1, S):
            for c in range(4):
                coarse[4 * (J * cside + I) + c] = 4 * ((J - 1) * (S - 1) + (I - 1)) + c
    rows, cols, vals = [], [], []
    for (f, c), v in transfer_full(n, S).items():
        if v == 0 or fine[f] < 0 or coarse[c] < 0:
            continue
        rows.append(fine[f])
        cols.append(coarse[c])
        vals.append(float(v))
    P = sp.csr_matrix((vals, (rows, cols)), shape=((2 * n - 1) ** 2, 4 * (S - 1) ** 2))
    P.sum_duplicates()
    P.sort_indices()
    return P
