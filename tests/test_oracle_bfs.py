"""Pins of the oracle's BFS (Bogner-Fox-Schmit) discretisation of the clamped plate
(Section 2.1 and Section 2.2, m = 2).

* 1-D Hermite element matrices against an independent symbolic construction (sympy);
* exactness on bicubics: the assembled forms of a bicubic equal its exact integrals,
  and the coarse-to-fine transfer reproduces a bicubic exactly;
* nestedness V^H in V^h: P^T K P and P^T M P equal the coarse-grid assembly;
* the first clamped eigenvalue of the unit square, 1294.9339795917 (Bjorstad and
  Tjostheim, BIT 39 (1999)), approached from above (conforming element, Section 2.2)
  at O(h^4), and the exact double eigenvalues of the square's symmetry;
* the partition rule against the geometry, and the BPJD iteration against a dense
  generalised eigensolve.
"""

from fractions import Fraction as F

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse.linalg as sla

from oracle import bfs, bpjd, metrics, partition, problem
from workloads import config_small_bfs

CLAMPED_LAMBDA1 = 1294.9339795917


def test_hermite_element_matrices_match_symbolic_integration():
    sympy = pytest.importorskip("sympy")
    s = sympy.symbols("s")
    c = sympy.symbols("c0:4")
    p = sum(ci * s ** i for i, ci in enumerate(c))
    conds = [p.subs(s, 0), sympy.diff(p, s).subs(s, 0), p.subs(s, 1), sympy.diff(p, s).subs(s, 1)]
    basis = []
    for a in range(4):
        sol = sympy.solve([cond - (1 if r == a else 0) for r, cond in enumerate(conds)], c, dict=True)[0]
        basis.append(sympy.expand(p.subs(sol)))
    M0, K1, K2 = bfs.element_matrices_1d()
    for a in range(4):
        for b in range(4):
            assert sympy.integrate(basis[a] * basis[b], (s, 0, 1)) == sympy.Rational(M0[a][b].numerator,
                                                                                    M0[a][b].denominator)
            d1 = sympy.integrate(sympy.diff(basis[a], s) * sympy.diff(basis[b], s), (s, 0, 1))
            assert d1 == sympy.Rational(K1[a][b].numerator, K1[a][b].denominator)
            d2 = sympy.integrate(sympy.diff(basis[a], s, 2) * sympy.diff(basis[b], s, 2), (s, 0, 1))
            assert d2 == sympy.Rational(K2[a][b].numerator, K2[a][b].denominator)


def _bicubic_dofs(coef, n, L):
    """Node-major dofs (u, h u_x, h u_y, h^2 u_xy) of q = sum_{p,r<=3} coef[r][p] x^p y^r
    at all (n+1)^2 nodes."""
    h = F(L) / n
    out = []
    for j in range(n + 1):
        for i in range(n + 1):
            x, y = i * h, j * h
            u = ux = uy = uxy = F(0)
            for r in range(4):
                for p in range(4):
                    cf = coef[r][p]
                    u += cf * x ** p * y ** r
                    if p:
                        ux += cf * p * x ** (p - 1) * y ** r
                    if r:
                        uy += cf * r * x ** p * y ** (r - 1)
                    if p and r:
                        uxy += cf * p * r * x ** (p - 1) * y ** (r - 1)
            out += [u, h * ux, h * uy, h * h * uxy]
    return out


def test_assembled_forms_exact_on_bicubics():
    rng = np.random.default_rng(4)
    n, L = 5, 1.0
    K, M = bfs.assemble(n, L, interior=False)
    c1 = [[F(int(v), 7) for v in rng.integers(-5, 6, 4)] for _ in range(4)]
    c2 = [[F(int(v), 3) for v in rng.integers(-5, 6, 4)] for _ in range(4)]
    q1 = np.array([float(v) for v in _bicubic_dofs(c1, n, L)])
    q2 = np.array([float(v) for v in _bicubic_dofs(c2, n, L)])

    def integral(f):   # int over the unit square of sum f[(p, r)] x^p y^r
        return sum(float(v) / ((p + 1) * (r + 1)) for (p, r), v in f.items())

    def product(a, b):
        out = {}
        for (p1, r1), v1 in a.items():
            for (p2, r2), v2 in b.items():
                out[(p1 + p2, r1 + r2)] = out.get((p1 + p2, r1 + r2), 0) + v1 * v2
        return out

    def poly(cf):
        return {(p, r): cf[r][p] for r in range(4) for p in range(4)}

    def dx(f):
        return {(p - 1, r): p * v for (p, r), v in f.items() if p}

    def dy(f):
        return {(p, r - 1): r * v for (p, r), v in f.items() if r}

    a, b = poly(c1), poly(c2)
    hess = integral(product(dx(dx(a)), dx(dx(b)))) + 2 * integral(product(dx(dy(a)), dx(dy(b)))) + \
        integral(product(dy(dy(a)), dy(dy(b))))
    assert q1 @ (K @ q2) == pytest.approx(hess, rel=1e-11)
    assert q1 @ (M @ q2) == pytest.approx(integral(product(a, b)), rel=1e-11)


def test_transfer_reproduces_bicubics_exactly():
    rng = np.random.default_rng(6)
    n, S = 12, 3
    T = bfs.transfer_full(n, S)
    coef = [[F(int(v), 5) for v in rng.integers(-5, 6, 4)] for _ in range(4)]
    fine = _bicubic_dofs(coef, n, 1)
    coarse = _bicubic_dofs(coef, S, 1)
    got = [F(0)] * len(fine)
    for (f, c), v in T.items():
        got[f] += v * coarse[c]
    assert got == fine


def test_coarse_space_is_nested():
    n, S = 16, 4
    K, M = bfs.assemble(n)
    KH, MH = bfs.assemble(S)
    P = bfs.prolongation(n, S)
    for A, AH in ((K, KH), (M, MH)):
        G = (P.T @ A @ P).toarray()
        np.testing.assert_allclose(G, AH.toarray(), rtol=0, atol=1e-12 * np.abs(AH.toarray()).max())


def _lowest(K, M, k):
    if K.shape[0] <= 1000:
        return la.eigh(K.toarray(), M.toarray(), eigvals_only=True)[:k]
    return np.sort(sla.eigsh(K.tocsc(), k, M.tocsc(), v0=np.random.default_rng(0).standard_normal(K.shape[0]), sigma=0, which="LM")[0])


def test_clamped_plate_eigenvalues_from_above_fourth_order():
    lam = [_lowest(*bfs.assemble(n), 3) for n in (8, 16, 32)]
    l1 = [v[0] for v in lam]
    assert l1[0] > l1[1] > l1[2] > CLAMPED_LAMBDA1
    e = [v - CLAMPED_LAMBDA1 for v in l1]
    assert 12.0 < e[0] / e[1] < 17.0 and 12.0 < e[1] / e[2] < 17.0
    for v in lam:          # the (1,2)/(2,1) pair is exactly double on the square
        assert abs(v[1] - v[2]) <= 1e-10 * v[2]


def test_partition_nodes_carry_four_dofs():
    spec = config_small_bfs(n=24, ns=4, delta=2)
    ptr, dofs, col, nc = partition.box_partition(spec)
    n, S, m, d = 24, 4, 6, 2
    for sy in range(S):
        for sx in range(S):
            l = sx + S * sy
            box = []
            for s in (sx, sy):
                lo = 0 if s == 0 else s * m - d
                hi = n if s == S - 1 else (s + 1) * m + d
                box.append(np.arange(max(lo, 0) + 1, min(hi, n)))
            nodes = ((box[1][:, None] - 1) * (n - 1) + (box[0][None, :] - 1)).ravel()
            want = np.sort((4 * nodes[:, None] + np.arange(4)).ravel())
            np.testing.assert_array_equal(dofs[ptr[l]:ptr[l + 1]], want)
            assert col[l] == (sx % 2) + 2 * (sy % 2)


def test_bpjd_on_bfs_plate_matches_dense_eigensolve():
    spec = config_small_bfs(n=32, ns=4, delta=2, k=4)
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
