"""Pins of the oracle's L-shaped domains (Section 6, Examples 6.2 and 6.4).

* Table 3 and Table 7, first columns: the 20 printed eigenvalues (8 decimals) of the
  oracle's assembly, by a shift-invert Lanczos solve (scipy eigsh);
* the restriction of the square's matrices equals an assembly over the L-shape's own
  triangles (every triangle of the removed quadrant has all its vertices on the
  Dirichlet boundary);
* the coarse interpolation is nested: the Galerkin products P^T K P and P^T M P equal
  the assembly on the coarse grid of the same L-shape;
* the partition keeps the boxes of the domain (192 for the paper's H = pi / 8);
* the BPJD iteration on a small L-shape against a dense generalised eigensolve.
"""

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from conftest import golden
from oracle import bpjd, fem, metrics, partition, problem
from dataclasses import replace

from workloads import config_small_lshape, config_table3_col1, config_table7_col1


@pytest.mark.parametrize("col,n,dofs", [(0, 128, 12033), (1, 256, 48641)])
def test_table3_columns(col, n, dofs):
    spec = replace(config_table3_col1(), n=(n, n))
    K, M = fem.assemble(spec)
    assert K.shape[0] == dofs
    w = np.sort(sla.eigsh(K.tocsc(), 20, M.tocsc(), v0=np.random.default_rng(0).standard_normal(K.shape[0]), sigma=0.0, which="LM", tol=1e-14)[0])
    want = np.array([r[col] for r in golden("table3.txt")])
    np.testing.assert_allclose(w, want, rtol=0, atol=6e-9)


def test_restriction_equals_direct_assembly_on_the_lshape():
    """Assemble only the triangles of the L-shape (node ids of the full grid), then drop
    every boundary node of the L-shape: the same matrices as the restricted square."""
    n, a = 16, 2 * np.pi
    h = a / n
    nn = n + 1
    tri = []
    for j in range(n):
        for i in range(n):
            if i >= n // 2 and j < n // 2:
                continue                                  # cell in the removed quadrant
            sw, se, ne, nw = j * nn + i, j * nn + i + 1, (j + 1) * nn + i + 1, (j + 1) * nn + i
            tri += [[sw, se, ne], [sw, ne, nw]]
    tri = np.array(tri)
    xy = np.stack([(tri % nn) * h, (tri // nn) * h], -1)
    rows, cols, kv, mv = [], [], [], []
    for t, X in zip(tri, xy):
        B = np.array([X[1] - X[0], X[2] - X[0]])
        area = abs(np.linalg.det(B)) / 2
        G = np.linalg.solve(B, np.array([[-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]]))   # gradients (2 x 3)
        for p in range(3):
            for q in range(3):
                rows.append(t[p])
                cols.append(t[q])
                kv.append(area * G[:, p] @ G[:, q])
                mv.append(area / 12 * (2 if p == q else 1))
    Kd = sp.csr_matrix((kv, (rows, cols)), shape=(nn * nn, nn * nn))
    Md = sp.csr_matrix((mv, (rows, cols)), shape=(nn * nn, nn * nn))
    i, j = np.meshgrid(np.arange(nn), np.arange(nn), indexing="xy")
    i, j = i.ravel(), j.ravel()
    interior = (i > 0) & (i < n) & (j > 0) & (j < n) & ~((i >= n // 2) & (j <= n // 2))
    keep = np.flatnonzero(interior)
    K, M = fem.assemble(config_small_lshape(n=n))
    np.testing.assert_allclose(K.toarray(), Kd[keep][:, keep].toarray(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(M.toarray(), Md[keep][:, keep].toarray(), rtol=0, atol=1e-15)


def test_coarse_interpolation_is_nested():
    """P K-Galerkin equals the coarse-grid assembly of the same L-shape (nested P1 spaces)."""
    spec = config_small_lshape(n=32, ns=4)
    pb = problem.build(spec)
    Kc, Mc = fem.assemble(config_small_lshape(n=4, ns=2))
    np.testing.assert_allclose((pb.P.T @ pb.K @ pb.P).toarray(), Kc.toarray(), rtol=0, atol=1e-12)
    np.testing.assert_allclose((pb.P.T @ pb.M @ pb.P).toarray(), Mc.toarray(), rtol=0, atol=1e-13)


def test_partition_keeps_the_domain_boxes():
    spec = config_table3_col1()
    ptr, dofs, col, nc = partition.box_partition(spec)
    assert len(ptr) - 1 == 192                       # 256 boxes minus the removed quadrant's 64
    lm = fem.lshape_map(spec.n[0])
    assert dofs.max() < lm.max() + 1
    covered = np.zeros(lm.max() + 1, dtype=bool)
    covered[dofs] = True
    assert covered.all()                             # every dof lies in some subdomain
    for c in range(nc):
        members = np.concatenate([dofs[ptr[l]:ptr[l + 1]] for l in range(len(ptr) - 1) if col[l] == c])
        assert len(np.unique(members)) == len(members)


def test_bpjd_on_lshape_matches_dense_eigensolve():
    spec = config_small_lshape(n=32, ns=8, delta=1, k=4)
    pb = problem.build(spec)
    res = bpjd.solve(pb.setup(), tol=1e-8, subspace="3s")
    assert res.converged
    w, V = la.eigh(pb.K.toarray(), pb.M.toarray())
    k = spec.k
    np.testing.assert_allclose(res.lam, w[:k], rtol=1e-10)
    for a, b in metrics.clusters(w[:k + 1]):
        if b <= k:
            assert metrics.gap_b(res.X[:, a:b], V[:, a:b], pb.M) <= 1e-6


def test_table7_first_column():
    spec = config_table7_col1()
    K, M = fem.assemble(spec)
    assert K.shape[0] == 10575
    w = np.sort(sla.eigsh(K.tocsc(), 20, M.tocsc(), v0=np.random.default_rng(0).standard_normal(K.shape[0]), sigma=0.0, which="LM", tol=1e-14)[0])
    want = np.array([r[0] for r in golden("table7.txt")])
    np.testing.assert_allclose(w, want, rtol=0, atol=6e-9)


def test_prism_coarse_space_is_nested_and_partition_has_the_papers_n():
    spec = config_table7_col1()
    small = replace(spec, n=(16, 16, 8), nsub=(8, 8, 4))
    pb = problem.build(small)
    Kc, Mc = fem.assemble(replace(small, n=(8, 8, 4)))
    np.testing.assert_allclose((pb.P.T @ pb.K @ pb.P).toarray(), Kc.toarray(), rtol=0, atol=1e-12)
    np.testing.assert_allclose((pb.P.T @ pb.M @ pb.P).toarray(), Mc.toarray(), rtol=0, atol=1e-13)
    ptr, dofs, col, nc = partition.box_partition(spec)
    assert len(ptr) - 1 == 1536                      # the paper's N
    covered = np.zeros(spec.n_dofs, dtype=bool)
    covered[dofs] = True
    assert covered.all()
