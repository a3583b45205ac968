"""Bogner-Fox-Schmit (BFS) elements for the clamped plate (the paper's element for m = 2).

Oracle (test infrastructure only).

Section 2.1 and Section 2.2: Delta^2 u = lambda u in Omega, u = du/dn = 0 on the
boundary, a(u, v) = int Delta u Delta v on H^2_0, discretised with the conforming
BFS space: C^1 piecewise bicubics on a square grid, i.e. tensor products of 1-D
cubic Hermite functions.  On H^2_0 the form equals int D^2 u : D^2 v, so with the
1-D element matrices
    M0 = int phi psi,   K1 = int phi' psi',   K2 = int phi'' psi''
the element stiffness is K2 (x) M0 + 2 K1 (x) K1 + M0 (x) K2 and the mass M0 (x) M0.

Square [0, L]^2, n x n cells of side h.  Each grid node carries four dofs
    c = 0: u,   c = 1: h du/dx,   c = 2: h du/dy,   c = 3: h^2 d^2u/dxdy
(derivatives scaled by h so that every element quantity is a rational number times a
power of h).  Clamped data remove every dof of the boundary nodes; dof numbering is
node-major: 4 ((j - 1)(n - 1) + (i - 1)) + c for interior node (i, j).

The coarse space is BFS on the subdomain grid; it is nested (V^H in V^h), and P
holds the fine dofs of the coarse basis functions (exact rationals, rounded once).
"""

from __future__ import annotations

from fractions import Fraction as F
from functools import lru_cache

import numpy as np
import scipy.sparse as sp


@lru_cache(maxsize=None)
def hermite_basis():
    """Coefficients of the cubic Hermite basis on [0, 1] (monomials 1, s, s^2, s^3):
    basis 0/1 = value / derivative at s = 0, basis 2/3 = value / derivative at s = 1."""
    # rows: functional (value at 0, derivative at 0, value at 1, derivative at 1) of s^p
    V = [[F(1), F(0), F(0), F(0)],
         [F(0), F(1), F(0), F(0)],
         [F(1), F(1), F(1), F(1)],
         [F(0), F(1), F(2), F(3)]]
    n = 4
    A = [row[:] + [F(int(i == j)) for j in range(n)] for i, row in enumerate(V)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        inv = 1 / A[c][c]
        A[c] = [v * inv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [row[n:] for row in A]           # C[p][a]: coefficient of s^p in basis a


def _poly_mul_integral(p, q):
    """int_0^1 p(s) q(s) ds for coefficient lists."""
    return sum(a * b / (i + j + 1) for i, a in enumerate(p) for j, b in enumerate(q))


def _deriv(p):
    return [i * a for i, a in enumerate(p)][1:] or [F(0)]


@lru_cache(maxsize=None)
def element_matrices_1d():
    """1-D element matrices on the unit cell (h = 1) as Fractions: M0, K1, K2.  For cell
    size h with derivative dofs scaled by h they become M0 h, K1 / h, K2 / h^3."""
    C = hermite_basis()
    basis = [[C[p][a] for p in range(4)] for a in range(4)]
    M0 = [[_poly_mul_integral(basis[a], basis[b]) for b in range(4)] for a in range(4)]
    K1 = [[_poly_mul_integral(_deriv(basis[a]), _deriv(basis[b])) for b in range(4)] for a in range(4)]
    K2 = [[_poly_mul_integral(_deriv(_deriv(basis[a])), _deriv(_deriv(basis[b]))) for b in range(4)]
          for a in range(4)]
    return M0, K1, K2


def _global_1d(n: int, L: float, interior: bool):
    """Assembled 1-D matrices (M0, K1, K2) over node dofs (value, h derivative), node-major;
    interior=True drops both dofs of the two end nodes."""
    h = L / n
    M0, K1, K2 = element_matrices_1d()
    mats = []
    for E, scale in ((M0, h), (K1, 1.0 / h), (K2, 1.0 / h ** 3)):
        Ef = np.array([[float(v) for v in row] for row in E]) * scale
        nd = 2 * (n + 1)
        A = np.zeros((nd, nd))
        for e in range(n):
            idx = [2 * e, 2 * e + 1, 2 * e + 2, 2 * e + 3]
            A[np.ix_(idx, idx)] += Ef
        if interior:
            A = A[2:-2, 2:-2]
        mats.append(A)
    return mats


def assemble(n: int, L: float = 1.0, interior: bool = True):
    """K, M of the clamped plate (interior=True) or over all nodes (interior=False),
    node-major CSR with the pattern of dof pairs sharing a cell.  Entry
    ((i, j, a, b), (i', j', a', b')) = M0y K2x + 2 (K1y K1x) + K2y M0x (the Kronecker
    products of the 1-D matrices, y factor first), evaluated on that pattern only."""
    M0, K1, K2 = _global_1d(n, L, interior)
    m = (n - 1) if interior else (n + 1)
    dof = np.arange(4 * m * m)
    node, c = dof // 4, dof % 4
    ni, nj = node % m, node // m
    rows, cols = [], []
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            ok = (ni + di >= 0) & (ni + di < m) & (nj + dj >= 0) & (nj + dj < m)
            r = dof[ok]
            q = (nj[ok] + dj) * m + (ni[ok] + di)
            for c2 in range(4):
                rows.append(r)
                cols.append(4 * q + c2)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    rx, ry = 2 * ni[rows] + (c[rows] & 1), 2 * nj[rows] + (c[rows] >> 1)
    cn, cc = cols // 4, cols % 4
    cx, cy = 2 * (cn % m) + (cc & 1), 2 * (cn // m) + (cc >> 1)
    kv = (M0[ry, cy] * K2[rx, cx] + 2.0 * (K1[ry, cy] * K1[rx, cx])) + K2[ry, cy] * M0[rx, cx]
    mv = M0[ry, cy] * M0[rx, cx]
    K = sp.csr_matrix((kv, (rows, cols)), shape=(4 * m * m, 4 * m * m))
    M = sp.csr_matrix((mv, (rows, cols)), shape=(4 * m * m, 4 * m * m))
    for A in (K, M):
        A.sort_indices()
    return K, M


def _transfer_1d(n: int, S: int):
    """1-D transfer: fine node dofs (value, h_f derivative) of the coarse Hermite cubic,
    as a dict {(fine dof, coarse dof): Fraction} over all nodes."""
    m = n // S
    C = hermite_basis()
    out = {}
    for f in range(n + 1):
        cell = min(f // m, S - 1)
        s = F(f - cell * m, m)                      # position in the coarse cell
        for a in range(4):                          # coarse local dofs: node cell (a < 2) or cell + 1
            cnode = cell + (a >> 1)
            cdof = 2 * cnode + (a & 1)
            coef = [C[p][a] for p in range(4)]
            val = sum(c * s ** p for p, c in enumerate(coef))
            der = sum(p * c * s ** (p - 1) for p, c in enumerate(coef) if p > 0)
            # fine h_f d/dx = (h_f / H) d/ds = d/ds / m
            for fd, v in ((2 * f, val), (2 * f + 1, der / m)):
                if v != 0:
                    out[(fd, cdof)] = out.get((fd, cdof), F(0)) + v
    return out


def transfer_full(n: int, S: int):
    """The 2-D transfer over all nodes (node-major on both sides), {(fine, coarse): Fraction}."""
    if n % S != 0:
        raise ValueError("n must be a multiple of S")
    T1 = _transfer_1d(n, S)
    rows_by_fine = {}
    for (f, c), v in T1.items():
        rows_by_fine.setdefault(f, []).append((c, v))
    out = {}
    mf, mc = n + 1, S + 1
    for fy in range(2 * mf):
        for fx in range(2 * mf):
            jf, b = divmod(fy, 2)
            i_f, a = divmod(fx, 2)
            fine = 4 * (jf * mf + i_f) + a + 2 * b
            for cy, vy in rows_by_fine.get(fy, []):
                for cx, vx in rows_by_fine.get(fx, []):
                    jc, bc = divmod(cy, 2)
                    ic, ac = divmod(cx, 2)
                    coarse = 4 * (jc * mc + ic) + ac + 2 * bc
                    out[(fine, coarse)] = out.get((fine, coarse), F(0)) + vx * vy
    return out


def prolongation(n: int, S: int) -> sp.csr_matrix:
    """P between the clamped spaces (interior nodes on both grids), exact zeros dropped."""
    mf, mc = n + 1, S + 1

    def interior_map(m_all, m_in):
        out = -np.ones(4 * m_all * m_all, dtype=np.int64)
        for j in range(1, m_all - 1):
            for i in range(1, m_all - 1):
                for c in range(4):
                    out[4 * (j * m_all + i) + c] = 4 * ((j - 1) * m_in + (i - 1)) + c
        return out

    fmap = interior_map(mf, n - 1)
    cmap = interior_map(mc, S - 1)
    rows, cols, vals = [], [], []
    for (f, c), v in transfer_full(n, S).items():
        if v == 0 or fmap[f] < 0 or cmap[c] < 0:
            continue
        rows.append(fmap[f])
        cols.append(cmap[c])
        vals.append(float(v))
    P = sp.csr_matrix((vals, (rows, cols)), shape=(4 * (n - 1) ** 2, 4 * (S - 1) ** 2))
    P.sum_duplicates()
    P.sort_indices()
    return P
