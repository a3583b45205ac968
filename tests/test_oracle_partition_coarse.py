"""Pins of the oracle's subdomain partition (Section 2.3, Assumption 2) and of the
coarse interpolation P (Section 2.3, V^H subset of V^h)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import coarse, fem, partition
from workloads import ProblemSpec, config_c1, config_small_2d, config_small_3d


def _sets(ptr, dofs):
    return [set(dofs[ptr[l]:ptr[l + 1]].tolist()) for l in range(len(ptr) - 1)]


def test_c1_partition_by_hand():
    """C1: 4 x 4 boxes of 8 cells grown by 2 layers.  Along an axis the open index
    intervals are (0,10), (6,18), (14,26), (22,32): 9, 11, 11, 9 interior nodes."""
    spec = config_c1()
    ptr, dofs, col, nc = partition.box_partition(spec)
    sizes = np.diff(ptr).reshape(4, 4)              # [s_y, s_x]
    per_axis = np.array([9, 11, 11, 9])
    np.testing.assert_array_equal(sizes, per_axis[:, None] * per_axis[None, :])
    # subdomain 0 = nodes i, j in 1..9 ; dof = (j-1)*31 + (i-1)
    want0 = sorted((j - 1) * 31 + (i - 1) for j in range(1, 10) for i in range(1, 10))
    assert dofs[ptr[0]:ptr[1]].tolist() == want0
    # subdomain 5 = (s_x, s_y) = (1, 1): nodes 7..17 on both axes
    want5 = sorted((j - 1) * 31 + (i - 1) for j in range(7, 18) for i in range(7, 18))
    assert dofs[ptr[5]:ptr[6]].tolist() == want5
    assert nc == 4
    assert col.reshape(4, 4).tolist() == [[0, 1, 0, 1], [2, 3, 2, 3], [0, 1, 0, 1], [2, 3, 2, 3]]


@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_3d(),
                                  config_small_3d(n=16, ns=4, delta=2)],
                         ids=lambda s: s.name)
def test_partition_invariants(spec):
    ptr, dofs, col, nc = partition.box_partition(spec)
    sets = _sets(ptr, dofs)
    n = spec.n_dofs
    # ascending lists, valid ids, every dof covered, at most 2^dim owners
    for l in range(len(sets)):
        d = dofs[ptr[l]:ptr[l + 1]]
        assert np.all(np.diff(d) > 0) and d.min() >= 0 and d.max() < n
    count = np.zeros(n, int)
    for s in sets:
        count[list(s)] += 1
    assert count.min() >= 1 and count.max() <= 2 ** spec.dim
    # Assumption 2: same-coloured subdomains are disjoint
    for a in range(len(sets)):
        for b in range(a + 1, len(sets)):
            if col[a] == col[b]:
                assert not (sets[a] & sets[b])
    # overlap: two neighbouring boxes share exactly 2*delta - 1 node layers
    m = spec.n[0] // spec.nsub[0]
    if spec.delta > 0:
        shared = sets[0] & sets[1]
        xs = {g % (spec.n[0] - 1) for g in shared}
        assert len(xs) == 2 * spec.delta - 1
    assert 2 * spec.delta <= m


def _brute_coarse_value_2d(spec, c, x, y):
    """Evaluate the c-th coarse P1 hat function at (x, y) by locating the coarse triangle
    that contains the point and solving for its barycentric coordinates."""
    S = spec.nsub
    Hx, Hy = spec.length[0] / S[0], spec.length[1] / S[1]
    CI, CJ = c % (S[0] - 1) + 1, c // (S[0] - 1) + 1
    best = 0.0
    for J in range(S[1]):
        for I in range(S[0]):
            sw = (I * Hx, J * Hy)
            tris = [[(I, J), (I + 1, J), (I + 1, J + 1)], [(I, J), (I + 1, J + 1), (I, J + 1)]]
            for tri in tris:
                V = np.array([[a * Hx, b * Hy] for a, b in tri])
                A = np.vstack([V.T, np.ones(3)])
                lam = np.linalg.solve(A, np.array([x, y, 1.0]))
                if lam.min() >= -1e-12:
                    for q, (a, b) in enumerate(tri):
                        if (a, b) == (CI, CJ):
                            return lam[q]
                    return 0.0
    return best


def test_prolongation_matches_pointwise_evaluation_2d():
    spec = config_small_2d()
    P = coarse.prolongation(spec).toarray()
    nx, ny = spec.n
    hx, hy = spec.h
    rng = np.random.default_rng(1)
    for g in rng.choice(spec.n_dofs, 60, replace=False):
        i, j = g % (nx - 1) + 1, g // (nx - 1) + 1
        for c in range(spec.n_coarse):
            assert P[g, c] == pytest.approx(_brute_coarse_value_2d(spec, c, i * hx, j * hy), abs=1e-12)


@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_3d(),
                                  config_small_3d(kind="q1_3d")], ids=lambda s: s.name)
def test_galerkin_equals_direct_coarse_assembly(spec):
    """V^H is a subspace of V^h, so P^T K P and P^T M P equal the matrices assembled
    directly on J_H (for kappa constant on each coarse cell; here kappa = 1)."""
    from dataclasses import replace
    spec = replace(spec, kappa=None)
    K, M = fem.assemble(spec)
    P = coarse.prolongation(spec)
    cspec = replace(spec, n=spec.nsub, nsub=(1,) * spec.dim)
    KH, MH = fem.assemble(cspec)
    np.testing.assert_allclose((P.T @ K @ P).toarray(), KH.toarray(), atol=1e-12 * abs(KH).max())
    np.testing.assert_allclose((P.T @ M @ P).toarray(), MH.toarray(), atol=1e-12 * abs(MH).max())


def test_prolongation_partition_of_unity_interior():
    """Away from the coarse boundary layer the coarse hat functions sum to one."""
    spec = config_small_3d(n=16, ns=4, kind="p1_3d")
    P = coarse.prolongation(spec)
    m = spec.n[0] // spec.nsub[0]
    rows = P.sum(axis=1).A1
    N = spec.n[0] - 1
    for g in range(spec.n_dofs):
        i, j, l = g % N + 1, (g // N) % N + 1, g // (N * N) + 1
        if all(m <= q <= spec.n[0] - m for q in (i, j, l)):
            assert rows[g] == pytest.approx(1.0, abs=1e-14)
