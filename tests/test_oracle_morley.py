"""Pins of the oracle's Morley discretisation of the clamped plate (Section 2.1, m = 2).

The paper prints no fourth-order numbers, so the Morley assembly, its intergrid
transfer and partition are pinned against what the mathematics fixes:

* element matrices against an independent symbolic construction (sympy: basis
  solved in physical coordinates, exact integration over the triangle);
* exactness on quadratics: the Morley space contains P2, so the assembled forms
  of a global quadratic equal its exact integrals;
* the coarse space (BFS bicubics, Morley-interpolated): the transfer maps the BFS
  dofs of any bicubic to its fine Morley functionals exactly, each row touches one
  coarse cell, and the Galerkin eigenvalues bound the fine ones from above;
* eigenvalue limits: the simply supported plate has the closed form
  pi^4 (i^2 + j^2)^2, and the first clamped eigenvalue of the unit square is
  1294.9339795917 (Bjorstad and Tjostheim, BIT 39 (1999), high-accuracy
  spectral computation), approached from below at O(h^2) (Morley eigenvalues
  are asymptotic lower bounds);
* the partition rule against the geometry of the overlapping boxes;
* the BPJD iteration on a Morley problem against a dense generalised eigensolve.
"""

from fractions import Fraction as F

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse.linalg as sla

from oracle import bpjd, metrics, morley, partition, problem
from workloads import config_small_morley

CLAMPED_LAMBDA1 = 1294.9339795917


def _sym_basis(verts, dofs, x, y):
    """Morley basis in physical coordinates, solved symbolically."""
    import sympy
    c = sympy.symbols("c0:6")
    mons = [1, x, y, x * x, x * y, y * y]
    out = []
    for a in range(6):
        p = sum(ci * mi for ci, mi in zip(c, mons))
        eqs = [f(p) - (1 if r == a else 0) for r, f in enumerate(dofs)]
        sol = sympy.solve(eqs, c, dict=True)[0]
        out.append(sympy.expand(p.subs(sol)))
    return out


@pytest.mark.parametrize("shape", ["lower", "upper"])
def test_element_matrices_match_symbolic_integration(shape):
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    h = sympy.Rational(1, 8)
    x0, y0 = 3 * h, 5 * h
    R = sympy.Rational
    if shape == "lower":
        pts = [(x0, y0), (x0 + h, y0), (x0 + h, y0 + h)]
        mids = [((x0 + h / 2, y0), "dy"), ((x0 + h, y0 + h / 2), "dx"), ((x0 + h / 2, y0 + h / 2), "dd")]
    else:
        pts = [(x0, y0), (x0 + h, y0 + h), (x0, y0 + h)]
        mids = [((x0 + h / 2, y0 + h / 2), "dd"), ((x0 + h / 2, y0 + h), "dy"), ((x0, y0 + h / 2), "dx")]
    dofs = [(lambda p, a=a, b=b: p.subs({x: a, y: b})) for (a, b) in pts]
    for (a, b), kind in mids:
        if kind == "dy":
            dofs.append(lambda p, a=a, b=b: h * sympy.diff(p, y).subs({x: a, y: b}))
        elif kind == "dx":
            dofs.append(lambda p, a=a, b=b: h * sympy.diff(p, x).subs({x: a, y: b}))
        else:
            dofs.append(lambda p, a=a, b=b: h * (sympy.diff(p, x) - sympy.diff(p, y)).subs({x: a, y: b}))
    phi = _sym_basis(pts, dofs, x, y)

    def integrate(f):
        if shape == "lower":   # y0 <= y <= y0 + (x - x0)
            return sympy.integrate(f, (y, y0, y0 + (x - x0)), (x, x0, x0 + h))
        return sympy.integrate(f, (x, x0, x0 + (y - y0)), (y, y0, y0 + h))

    S, Rm = morley.reference_matrices(shape)
    hf = 1.0 / 8.0
    for a in range(6):
        for b in range(a, 6):
            hess = lambda p: (sympy.diff(p, x, 2), sympy.diff(p, x, y), sympy.diff(p, y, 2))
            ha, hb = hess(phi[a]), hess(phi[b])
            k_ab = integrate(ha[0] * hb[0] + 2 * ha[1] * hb[1] + ha[2] * hb[2])
            m_ab = integrate(phi[a] * phi[b])
            assert float(k_ab) == pytest.approx(float(S[a][b]) / hf ** 2, rel=1e-13, abs=1e-9)
            assert float(m_ab) == pytest.approx(float(Rm[a][b]) * hf ** 2, rel=1e-13, abs=1e-18)


def _quadratic_dofs(coef, n, L):
    """Dof values (all half-grid points, id Y (2n+1) + X) of q = c0 + c1 x + c2 y + c3 x^2
    + c4 x y + c5 y^2 with Fraction coefficients: values at vertices and the scaled
    normal derivatives of the module docstring at edge midpoints."""
    c0, c1, c2, c3, c4, c5 = coef
    h = F(L) / n
    out = []
    for Y in range(2 * n + 1):
        for X in range(2 * n + 1):
            px, py = X * h / 2, Y * h / 2
            qx = c1 + 2 * c3 * px + c4 * py
            qy = c2 + c4 * px + 2 * c5 * py
            kind = morley.half_grid_kind(X, Y)
            out.append({"v": c0 + c1 * px + c2 * py + c3 * px * px + c4 * px * py + c5 * py * py,
                        "dy": h * qy, "dx": h * qx, "dd": h * (qx - qy)}[kind])
    return out


def _square_integral(a, b, L):
    return L ** (a + b + 2) / ((a + 1) * (b + 1))


def test_assembled_forms_exact_on_quadratics():
    rng = np.random.default_rng(3)
    n, L = 6, 1.0
    Kf, Mf = morley.assemble_full(n, L)
    c1 = [F(int(v), 7) for v in rng.integers(-9, 10, 6)]
    c2 = [F(int(v), 5) for v in rng.integers(-9, 10, 6)]
    q1 = np.array([float(v) for v in _quadratic_dofs(c1, n, L)])
    q2 = np.array([float(v) for v in _quadratic_dofs(c2, n, L)])
    # a(q1, q2) = area * (q1_xx q2_xx + 2 q1_xy q2_xy + q1_yy q2_yy), constant Hessians
    a_exact = L * L * float(2 * c1[3] * 2 * c2[3] + 2 * c1[4] * c2[4] + 2 * c1[5] * 2 * c2[5])
    assert q1 @ (Kf @ q2) == pytest.approx(a_exact, rel=1e-12)
    mons = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    b_exact = sum(float(c1[i] * c2[j]) * _square_integral(mons[i][0] + mons[j][0], mons[i][1] + mons[j][1], L)
                  for i in range(6) for j in range(6))
    assert q1 @ (Mf @ q2) == pytest.approx(b_exact, rel=1e-12)


def _bfs_coarse_dofs(coef, S, L):
    """BFS node dofs (u, H u_x, H u_y, H^2 u_xy) of the bicubic q = sum coef[r][p] x^p y^r at
    the (S+1)^2 coarse nodes, node-major."""
    H = F(L) / S
    out = []
    for J in range(S + 1):
        for I in range(S + 1):
            x, y = I * H, J * H
            u = ux = uy = uxy = F(0)
            for r in range(4):
                for p in range(4):
                    c = coef[r][p]
                    u += c * x ** p * y ** r
                    if p:
                        ux += c * p * x ** (p - 1) * y ** r
                    if r:
                        uy += c * r * x ** p * y ** (r - 1)
                    if p and r:
                        uxy += c * p * r * x ** (p - 1) * y ** (r - 1)
            out += [u, H * ux, H * uy, H * H * uxy]
    return out


def _morley_functionals(coef, n, L):
    """Fine Morley dofs (all half-grid points) of the bicubic q: values at vertices and the
    scaled normal derivatives of the module docstring at edge midpoints."""
    h = F(L) / n
    out = []
    for Y in range(2 * n + 1):
        for X in range(2 * n + 1):
            x, y = X * h / 2, Y * h / 2
            u = ux = uy = F(0)
            for r in range(4):
                for p in range(4):
                    c = coef[r][p]
                    u += c * x ** p * y ** r
                    if p:
                        ux += c * p * x ** (p - 1) * y ** r
                    if r:
                        uy += c * r * x ** p * y ** (r - 1)
            out.append({"v": u, "dy": h * uy, "dx": h * ux, "dd": h * (ux - uy)}[morley.half_grid_kind(X, Y)])
    return out


def test_transfer_reproduces_coarse_bicubics_exactly():
    """P maps the BFS dofs of any bicubic (one piece of the coarse space) to its Morley
    functionals on the fine grid; each row only touches the 16 dofs of one coarse cell that
    holds the row's point (the coarse function is C^1, so any holding cell gives the same)."""
    rng = np.random.default_rng(5)
    n, S = 12, 3
    m = n // S
    T = morley.transfer_full(n, S)
    for trial in range(2):
        coef = [[F(int(v), 5) for v in rng.integers(-5, 6, 4)] for _ in range(4)]
        fine = _morley_functionals(coef, n, 1)
        coarse = _bfs_coarse_dofs(coef, S, 1)
        got = [F(0)] * len(fine)
        for (f, c), v in T.items():
            got[f] += v * coarse[c]
        assert got == fine
    side = 2 * n + 1
    for (f, c), v in T.items():
        Y, X = divmod(f, side)
        J, I = divmod(c // 4, S + 1)
        # the coarse node (I, J) is a corner of a coarse cell whose closure holds the point
        assert 2 * m * (I - 1) <= X <= 2 * m * (I + 1) and 2 * m * (J - 1) <= Y <= 2 * m * (J + 1)


def test_coarse_pencil_bounds_fine_spectrum_from_above():
    """range(P) is a subspace of the Morley space, so the Galerkin eigenvalues are upper bounds
    of the fine ones (Courant-Fischer); the conforming coarse space keeps them close."""
    n, S, k = 32, 4, 6
    K, M = morley.assemble(n)
    P = morley.prolongation(n, S)
    lh = la.eigh((P.T @ K @ P).toarray(), (P.T @ M @ P).toarray(), eigvals_only=True)[:k]
    w = la.eigh(K.toarray(), M.toarray(), eigvals_only=True)[:k]
    assert np.all(lh >= w * (1 - 1e-12))
    assert np.all(lh <= 1.1 * w)


def _lowest(K, M, k):
    if K.shape[0] <= 1100:
        return la.eigh(K.toarray(), M.toarray(), eigvals_only=True)[:k]
    return np.sort(sla.eigsh(K.tocsc(), k, M.tocsc(), v0=np.random.default_rng(0).standard_normal(K.shape[0]), sigma=0, which="LM")[0])


def test_simply_supported_plate_converges_to_closed_form():
    want = np.array([4.0, 25.0, 25.0, 64.0])           # (i^2 + j^2)^2, lowest four
    errs = []
    for n in (16, 32):
        w = _lowest(*morley.assemble(n, 1.0, "simply_supported"), 4) / np.pi ** 4
        errs.append(np.abs(w - want))
    assert np.all(errs[1] < 1.5e-2 * want)
    ratio = errs[0] / errs[1]
    assert np.all((ratio > 3.5) & (ratio < 4.6)), ratio


def test_clamped_plate_first_eigenvalue_from_below():
    lam = [_lowest(*morley.assemble(n), 1)[0] for n in (16, 32, 64)]
    assert lam[0] < lam[1] < lam[2] < CLAMPED_LAMBDA1
    e = [CLAMPED_LAMBDA1 - v for v in lam]
    assert 3.5 < e[1] / e[2] < 4.5
    richardson = (4 * lam[2] - lam[1]) / 3
    assert abs(richardson - CLAMPED_LAMBDA1) < 0.25


def test_partition_matches_box_geometry():
    spec = config_small_morley(n=24, ns=4, delta=2)
    ptr, dofs, col, nc = partition.box_partition(spec)
    n, S, m, d = 24, 4, 6, 2
    inner = 2 * n - 1
    Xs = dofs % inner + 1
    Ys = dofs // inner + 1
    for sy in range(S):
        for sx in range(S):
            l = sx + S * sy
            box = []
            for s in (sx, sy):
                lo = 0.0 if s == 0 else (s * m - d) / n
                hi = 1.0 if s == S - 1 else ((s + 1) * m + d) / n
                box.append((lo, hi))
            X = np.arange(1, 2 * n)
            px = X / (2.0 * n)
            inside_x = X[(px > box[0][0]) & (px < box[0][1])]
            inside_y = X[(px > box[1][0]) & (px < box[1][1])]
            want = np.sort(((inside_y[:, None] - 1) * inner + (inside_x[None, :] - 1)).ravel())
            np.testing.assert_array_equal(dofs[ptr[l]:ptr[l + 1]], want)
            assert col[l] == (sx % 2) + 2 * (sy % 2)
    for c in range(nc):
        members = [dofs[ptr[l]:ptr[l + 1]] for l in range(S * S) if col[l] == c]
        allm = np.concatenate(members)
        assert len(np.unique(allm)) == len(allm)
    assert np.all(Xs >= 1) and np.all(Ys >= 1)


def test_bpjd_on_clamped_plate_matches_dense_eigensolve():
    spec = config_small_morley(n=32, ns=8, delta=1, k=8)
    pb = problem.build(spec)
    res = bpjd.solve(pb.setup(), tol=1e-8, subspace="3s")
    assert res.converged
    w, V = la.eigh(pb.K.toarray(), pb.M.toarray())
    k = spec.k
    np.testing.assert_allclose(res.lam, w[:k], rtol=1e-10)
    for a, b in metrics.clusters(w[:k + 1]):
        if b <= k:
            assert metrics.gap_b(res.X[:, a:b], V[:, a:b], pb.M) <= 1e-6
    assert metrics.rel_residuals(pb.K, pb.M, res.lam, res.X).max() <= 1e-8
