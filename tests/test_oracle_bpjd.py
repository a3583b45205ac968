"""Pins of the oracle's BPJD iteration (Section 3, Algorithm 3.1, Eq. (3.3)).

The iteration converges to the lowest k eigenpairs of the pencil (K, M), a
result with a plain definition: a dense generalised eigensolve.  Its pieces
are pinned against textbook special cases (a single subdomain covering the
domain reduces the preconditioner to a shifted solve; the spectral coarse
solve equals a direct solve on the complement of the wanted coarse
eigenvectors) and against the invariants the paper proves (Eq. (4.1)
monotonicity, b-orthonormality, mesh-independent iteration counts).
"""

from dataclasses import replace

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from conftest import golden
from oracle import bpjd, metrics, problem
from workloads import ProblemSpec, config_c1, config_small_2d, config_small_3d, config_table1_col1


@pytest.fixture(scope="module")
def c1():
    pb = problem.build(config_c1())
    S = pb.setup()
    res = bpjd.solve(S, tol=1e-8)
    w, V = la.eigh(pb.K.toarray(), pb.M.toarray())
    return pb, S, res, w, V


def test_c1_matches_dense_eigensolve(c1):
    pb, S, res, w, V = c1
    k = pb.spec.k
    assert res.converged
    np.testing.assert_allclose(res.lam, w[:k], rtol=1e-10)
    # published C1 spectrum in units of pi^2 (unit square, h = 1/32)
    np.testing.assert_allclose(res.lam / np.pi ** 2,
                               [2.00482122, 5.02072060, 5.03235583, 8.07692593, 10.09492161, 10.09545111],
                               atol=6e-9)
    for a, b in metrics.clusters(w[:k]):
        assert metrics.gap_b(res.X[:, a:b], V[:, a:b], pb.M) <= 1e-6
    assert metrics.rel_residuals(pb.K, pb.M, res.lam, res.X).max() <= 1e-8
    G = res.X.T @ (pb.M @ res.X)
    np.testing.assert_allclose(G, np.eye(k), atol=1e-12)


def test_ritz_values_monotone_and_above_discrete(c1):
    """Eq. (4.1): lambda_i^h <= lambda_i^{k+1} <= lambda_i^k (Courant-Fischer), and the trace
    functional of Remark 3.4 decreases."""
    pb, S, res, w, V = c1
    k = pb.spec.k
    H = np.array(res.history_lam)
    assert np.all(np.diff(H, axis=0) <= 1e-12 * H[:-1])
    assert np.all(H >= w[None, :k] * (1 - 1e-12))
    tr = H.sum(axis=1)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])


def test_single_subdomain_reduces_to_shifted_solve():
    """With one subdomain covering Omega and no coarse term, Eq. (3.3) is (K - lambda_i M)^{-1}."""
    spec = ProblemSpec("p1_2d", (16, 12), (1.0, 0.75), (1, 1), 0, 3)
    pb = problem.build(replace(spec, nsub=(4, 3)))
    ptr = np.array([0, spec.n_dofs], dtype=np.int64)
    dofs = np.arange(spec.n_dofs, dtype=np.int32)
    S = bpjd.setup(pb.K, pb.M, pb.P, ptr, dofs, 3)
    rng = np.random.default_rng(0)
    rho = rng.standard_normal((spec.n_dofs, 3))
    lam = np.array([5.0, 12.0, 20.0])           # below lambda_1 ~ 27.4, so K - lambda M is SPD
    Z = bpjd.apply_preconditioner(S, rho, lam, coarse=False)
    for i in range(3):
        zi = sla.spsolve((pb.K - lam[i] * pb.M).tocsc(), rho[:, i])
        np.testing.assert_allclose(Z[:, i], zi, rtol=1e-10, atol=1e-12 * np.abs(zi).max())


def test_coarse_term_equals_direct_solve_on_complement(c1):
    """(B_0)^{-1} Q_{s+1}^H Q^H in matrix form: q = M_H^{-1} P^T rho, remove the M_H-projection
    onto the first s coarse eigenvectors, then solve (K_H - lambda M_H) w = M_H q'."""
    pb, S, res, w, V = c1
    k = pb.spec.k
    rng = np.random.default_rng(2)
    rho = rng.standard_normal((S.n, k))
    lam = np.linspace(15.0, 60.0, k)
    Z = bpjd.coarse_correction(S, rho, lam)
    for i in range(k):
        q = np.linalg.solve(S.MH, S.P.T @ rho[:, i])
        Ub = S.Phi[:, :k]
        q2 = q - Ub @ (Ub.T @ (S.MH @ q))
        wH = np.linalg.solve(S.KH - lam[i] * S.MH, S.MH @ q2)
        np.testing.assert_allclose(Z[:, i], S.P @ wH, rtol=1e-9, atol=1e-11 * np.abs(S.P @ wH).max())


def test_preconditioner_is_symmetric(c1):
    """For a common shift the operator rho -> z of Eq. (3.3) is a symmetric matrix."""
    pb, S, res, w, V = c1
    rng = np.random.default_rng(4)
    u = rng.standard_normal((S.n, 1))
    v = rng.standard_normal((S.n, 1))
    lam = np.array([40.0])
    Zu = bpjd.apply_preconditioner(S, u, lam)
    Zv = bpjd.apply_preconditioner(S, v, lam)
    assert (v.T @ Zu).item() == pytest.approx((u.T @ Zv).item(), rel=1e-11)


def test_projection_is_b_orthogonal(c1):
    pb, S, res, w, V = c1
    X, AX, MX, lam = bpjd.initial_guess(S)
    Z = np.random.default_rng(5).standard_normal(X.shape)
    T = bpjd.project_out(X, MX, Z)
    assert np.abs(MX.T @ T).max() <= 1e-12 * np.abs(Z).max()


def test_initial_guess_is_coarse_eigenpairs(c1):
    """Step 1: X^0 = P0 Phi~, b-orthonormal, lambda_i^0 = Rq = the coarse eigenvalues."""
    pb, S, res, w, V = c1
    X, AX, MX, lam = bpjd.initial_guess(S)
    np.testing.assert_allclose(X.T @ MX, np.eye(pb.spec.k), atol=1e-12)
    np.testing.assert_allclose(lam, S.lam0H[:pb.spec.k], rtol=1e-12)


@pytest.mark.parametrize("spec", [config_small_2d(), config_small_3d(), config_small_3d(kind="q1_3d")],
                         ids=lambda s: s.name)
def test_other_problems_converge(spec):
    pb = problem.build(spec)
    S = pb.setup()
    res = bpjd.solve(S, tol=1e-8, subspace="3s")
    assert res.converged
    w, V = la.eigh(pb.K.toarray(), pb.M.toarray())
    np.testing.assert_allclose(res.lam, w[:spec.k], rtol=1e-10)
    for a, b in metrics.clusters(w[:spec.k]):
        assert metrics.gap_b(res.X[:, a:b], V[:, a:b], pb.M) <= 1e-6


def test_subspace_variants_agree(c1):
    pb, S, res, w, V = c1
    r3 = bpjd.solve(S, tol=1e-8, subspace="3s")
    assert r3.converged and r3.iterations < res.iterations
    np.testing.assert_allclose(r3.lam, res.lam, rtol=1e-10)


def test_growing_space_is_nested_and_converges(c1):
    """Algorithm 3.1's own search space, W^0 = U^0 and W^{k+1} = W^k + span{t_i}: the spaces are
    nested, so by Courant-Fischer no Ritz value rises from one step to the next; the basis stays
    b-orthonormal, and the result is the dense generalised eigensolve's.  The step count is
    pinned against drift (the 2s and 3s spaces of Remark 3.1 take 54 and 21)."""
    pb, S, res, w, V = c1
    k = S.k
    r = bpjd.solve(S, tol=1e-8, subspace="grow")
    assert r.converged and r.restarts == 0
    H = np.array(r.history_lam)
    assert np.all(np.diff(H, axis=0) <= 1e-12 * np.abs(H[:-1])), np.diff(H, axis=0).max()
    np.testing.assert_allclose(r.lam, w[:k], rtol=1e-10)
    for a, b in metrics.clusters(w[:k]):
        assert metrics.gap_b(r.X[:, a:b], V[:, a:b], pb.M) <= 1e-6
    assert metrics.rel_residuals(pb.K, pb.M, r.lam, r.X).max() <= 1e-8
    assert r.iterations == 18, r.iterations


def test_growing_space_restarted_at_3s_is_the_3s_space(c1):
    """Restarted whenever it would exceed 3s columns, the growing space is U^{k-1} + U^k +
    span{t_i} at every step (step 1: W^1 = U^0 + span{t} contains U^1 and U^0; later steps restart
    to U^k + U^{k-1} before the append), i.e. Remark 3.1's 3s space in another basis: the same
    Ritz values at every step and the same step count."""
    pb, S, res, w, V = c1
    k = S.k
    r3 = bpjd.solve(S, tol=1e-8, subspace="3s")
    rg = bpjd.solve(S, tol=1e-8, subspace="grow", max_dim=3 * k)
    assert rg.converged and rg.iterations == r3.iterations
    assert rg.restarts == rg.iterations - 2
    np.testing.assert_allclose(np.array(rg.history_lam), np.array(r3.history_lam), rtol=1e-9)


@pytest.mark.slow
def test_paper_iteration_count_with_the_growing_space():
    """Table 1, first column, with the search space of Algorithm 3.1 as printed (W^{k+1} = W^k +
    span{t}, up to 19 x 22 columns): on the paper's partition (2 and 3 rings of fine triangles)
    the counts bracket the printed 21 as the 3s space's do (22 and 20), one step fewer with 3
    rings; restarted at 5s columns it takes the 3s counts."""
    from oracle import partition
    spec = replace(config_table1_col1(), nsub=(16, 16), delta=2)
    pb = problem.build(spec)
    its, its5 = {}, {}
    for layers in (2, 3):
        ptr, dofs, col, nc = partition.triangle_partition(128, 16, layers)
        S = bpjd.setup(pb.K, pb.M, pb.P, ptr, dofs, 19)
        res = bpjd.solve(S, tol=1e-10, stop="dlambda", subspace="grow", max_iter=60)
        assert res.converged and res.restarts == 0
        its[layers] = res.iterations
        if layers == 3:
            want = np.array([r[0] for r in golden("table1.txt")])
            np.testing.assert_allclose(res.lam, want, rtol=0, atol=6e-9)
        res5 = bpjd.solve(S, tol=1e-10, stop="dlambda", subspace="grow", max_dim=5 * 19, max_iter=60)
        its5[layers] = res5.iterations
    assert its[3] <= 21 <= its[2], its
    assert its == {2: 22, 3: 19}, its
    assert its5 == {2: 22, 3: 20}, its5


@pytest.mark.slow
def test_iteration_count_is_mesh_independent():
    """Theorem 5.1 / Table 1: with H and delta/H fixed, the iteration count of the paper's stop
    rule sum |lambda^{k+1} - lambda^k| < 1e-10 does not grow as h -> 0."""
    counts = []
    for n in (32, 64, 128):
        spec = ProblemSpec("p1_2d", (n, n), (np.pi, np.pi), (8, 8), n // 32, 6)
        pb = problem.build(spec)
        res = bpjd.solve(pb.setup(), tol=1e-10, stop="dlambda", subspace="3s")
        assert res.converged
        counts.append(res.iterations)
    assert max(counts) - min(counts) <= 2, counts


def test_local_indefinite_detected():
    """Eq. (3.1) requires lambda_i below the local Dirichlet spectrum; C1 with the initial
    guess on J_H itself (tau = 0) violates it in the first iteration."""
    pb = problem.build(replace(config_c1(), tau=0))
    S = pb.setup()
    with pytest.raises(bpjd.LocalIndefinite):
        bpjd.solve(S, tol=1e-8, max_iter=2)


def test_paper_triangle_partition_is_a_coloured_cover():
    """Example 6.1's partition J_H: 512 coarse triangles of the 16 x 16 grid of (0, pi)^2, each
    enlarged by rings of fine triangles; every dof is covered and same-coloured subdomains are
    disjoint (Assumption 2)."""
    from oracle import partition
    for layers in (2, 3):
        ptr, dofs, col, nc = partition.triangle_partition(128, 16, layers)
        assert len(ptr) - 1 == 512 and nc == 8
        covered = np.zeros(127 * 127, dtype=bool)
        covered[dofs] = True
        assert covered.all()
        for c in range(nc):
            members = np.concatenate([dofs[ptr[l]:ptr[l + 1]] for l in range(512) if col[l] == c])
            assert len(np.unique(members)) == len(members)
    # enlargements that would make same-coloured subdomains overlap are rejected
    with pytest.raises(ValueError):
        partition.triangle_partition(128, 16, 4)
    with pytest.raises(ValueError):
        partition.triangle_partition(100, 16, 1)


def test_paper_iteration_count_with_its_partition():
    """Section 6, Table 1, first column: 21 iterations to sum |lambda^{k+1} - lambda^k| < 1e-10
    with N = 512 triangles and delta / H = 1/4.  delta = H/4 = sqrt(2) pi / 64 is 2.83 fine steps
    (h = pi / 128); with the enlargement by 3 and by 2 rings of fine triangles, the W^{k+1} =
    U^{k-1} + U^k + span{t} space (Remark 3.1) and the paper's stop rule, the oracle's counts
    bracket the printed 21."""
    from oracle import partition
    spec = replace(config_table1_col1(), nsub=(16, 16), delta=2)      # coarse P1 on the 16 x 16 grid
    pb = problem.build(spec)
    its = {}
    for layers in (2, 3):
        ptr, dofs, col, nc = partition.triangle_partition(128, 16, layers)
        S = bpjd.setup(pb.K, pb.M, pb.P, ptr, dofs, 19)
        res = bpjd.solve(S, tol=1e-10, stop="dlambda", subspace="3s", max_iter=60)
        assert res.converged
        its[layers] = res.iterations
    # against the paper: the two enlargements bracket the printed count
    assert its[3] <= 21 <= its[2], its
    assert its[2] - its[3] <= 3, its
    # against drift of the configuration or the arithmetic: the oracle's own counts
    assert its == {2: 22, 3: 20}, its
