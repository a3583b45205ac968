"""Pins of oracle.metrics: the gap of Definition 2.1 (and Remark 2.2), the
relative residual of the stop test, and the eigenvalue clusters.  Every expected
value below is worked out by hand from the definitions or reduces to a library
routine on a transformed problem; none is produced by the functions under test.
"""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import metrics


def _rot(theta):
    """Columns: e1 and the unit vector at angle theta from e1 in the (e1, e2) plane (R^3)."""
    return np.array([[1.0], [0.0], [0.0]]), np.array([[np.cos(theta)], [np.sin(theta)], [0.0]])


@pytest.mark.parametrize("theta", [0.0, 1e-7, 0.3, 1.0, np.pi / 2 - 1e-3])
def test_line_rotated_by_theta_euclidean(theta):
    """Two lines at angle theta (M = I): both directed sines and the gap are sin(theta)."""
    u, v = _rot(theta)
    M = np.eye(3)
    assert metrics.sin_b(u, v, M) == pytest.approx(np.sin(theta), abs=1e-14)
    assert metrics.sin_b(v, u, M) == pytest.approx(np.sin(theta), abs=1e-14)
    assert metrics.gap_b(u, v, M) == pytest.approx(np.sin(theta), abs=1e-14)


def test_line_angle_in_a_diagonal_b_product():
    """M = diag(4, 1, 9), u = e1, v = (1, 2, 0).  In the b-product
    cos = u^T M v / (|u|_b |v|_b) = 4 / (2 sqrt(8)), so sin = 1 / sqrt(2); the
    Euclidean angle (sin = 2 / sqrt(5)) is different, so a metric that ignored M
    fails here."""
    M = np.diag([4.0, 1.0, 9.0])
    u = np.array([[1.0], [0.0], [0.0]])
    v = np.array([[1.0], [2.0], [0.0]])
    assert metrics.gap_b(u, v, M) == pytest.approx(1 / np.sqrt(2), abs=1e-14)
    assert metrics.gap_b(u, v, np.eye(3)) == pytest.approx(2 / np.sqrt(5), abs=1e-14)


def test_plane_pair_known_principal_angles():
    """span{e1, e2} against span{e1, cos(t) e2 + sin(t) e3} (M = I): principal
    angles 0 and t, so the gap is sin(t); scaling and mixing the basis vectors
    does not change it (it depends on the spans only)."""
    t = 0.2
    U = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0], [0.0, 0.0]])
    V = np.array([[1.0, 0.0], [0.0, np.cos(t)], [0.0, np.sin(t)], [0.0, 0.0]])
    M = np.eye(4)
    assert metrics.gap_b(U, V, M) == pytest.approx(np.sin(t), abs=1e-14)
    mix = np.array([[3.0, 1.0], [-2.0, 5.0]])
    assert metrics.gap_b(U @ mix, V @ mix.T, M) == pytest.approx(np.sin(t), abs=1e-13)


def test_general_spd_product_reduces_to_euclidean_principal_angles():
    """With M = R^T R, the b-product of u, v is the Euclidean product of R u, R v, so
    the b-gap of equal-dimensional spans is the sine of the largest Euclidean
    principal angle between span(R U) and span(R V) (scipy.linalg.subspace_angles)."""
    rng = np.random.default_rng(7)
    n = 9
    A = rng.standard_normal((n, n))
    M = A @ A.T + n * np.eye(n)
    R = np.linalg.cholesky(M).T
    for p in (1, 2, 4):
        U = rng.standard_normal((n, p))
        V = U + 0.05 * rng.standard_normal((n, p))
        ref = np.sin(sla.subspace_angles(R @ U, R @ V).max())
        assert metrics.gap_b(U, V, M) == pytest.approx(ref, rel=1e-10, abs=1e-14)
        assert metrics.sin_b(U, V, M) == pytest.approx(ref, rel=1e-10, abs=1e-14)
        assert metrics.sin_b(V, U, M) == pytest.approx(ref, rel=1e-10, abs=1e-14)


def test_directed_sines_of_unequal_dimensions():
    """Definition 2.1 takes the larger of the two directed sines.  For a line inside
    a plane, sin{line; plane} = 0 but sin{plane; line} = 1 (some unit vector of the
    plane is b-orthogonal to the line), so the gap is 1.  A line at angle t off the
    plane: sin{line; plane} = sin(t), and still sin{plane; line} = 1."""
    M = np.diag([1.0, 2.0, 5.0])
    line = np.array([[1.0], [1.0], [0.0]])
    plane = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    assert metrics.sin_b(line, plane, M) == pytest.approx(0.0, abs=1e-14)
    assert metrics.sin_b(plane, line, M) == pytest.approx(1.0, abs=1e-14)
    assert metrics.gap_b(line, plane, M) == pytest.approx(1.0, abs=1e-14)
    assert metrics.gap_b(plane, line, M) == pytest.approx(1.0, abs=1e-14)
    # line (1, 0, c): b-norm^2 = 1 + 5 c^2, its b-projection onto the plane is (1, 0, 0);
    # the residual (0, 0, c) has b-norm sqrt(5) |c|, so sin = sqrt(5) c / sqrt(1 + 5 c^2)
    c = 0.1
    tilted = np.array([[1.0], [0.0], [c]])
    want = np.sqrt(5.0) * c / np.sqrt(1 + 5 * c * c)
    assert metrics.sin_b(tilted, plane, M) == pytest.approx(want, abs=1e-14)
    assert metrics.gap_b(tilted, plane, M) == pytest.approx(1.0, abs=1e-14)


def test_residual_of_exact_and_perturbed_pairs():
    """K = diag(2, 12), M = diag(1, 4): eigenpairs (2, e1) and (3, e2).  Exact pairs
    give 0.  x = (1, 1/4) with lambda = 2: K x - 2 M x = (0, 12/4 - 8/4) = (0, 1),
    M x = (1, 1), so the relative residual is 1 / (2 sqrt(2)); with x = (1/4, 1) and
    lambda = 3: K x - 3 M x = (2/4 - 3/4, 0) = (-1/4, 0), M x = (1/4, 4), giving
    (1/4) / (3 sqrt(1/16 + 16))."""
    K = np.diag([2.0, 12.0])
    M = np.diag([1.0, 4.0])
    X = np.eye(2)
    lam = np.array([2.0, 3.0])
    np.testing.assert_allclose(metrics.rel_residuals(K, M, lam, X), [0.0, 0.0], atol=0)
    Xp = np.array([[1.0, 0.25], [0.25, 1.0]])
    got = metrics.rel_residuals(K, M, lam, Xp)
    np.testing.assert_allclose(got, [1 / (2 * np.sqrt(2)), 0.25 / (3 * np.sqrt(1 / 16 + 16))], rtol=1e-14)
    # the same with sparse matrices (the form the tests pass)
    import scipy.sparse as sp
    got_sp = metrics.rel_residuals(sp.csr_matrix(K), sp.csr_matrix(M), lam, Xp)
    np.testing.assert_allclose(got_sp, got, rtol=1e-15)


def test_residual_is_scale_invariant_and_sign_free():
    """The relative residual does not change when x is scaled (or negated)."""
    K = np.diag([2.0, 12.0])
    M = np.diag([1.0, 4.0])
    lam = np.array([2.0])
    x = np.array([[1.0], [0.25]])
    r1 = metrics.rel_residuals(K, M, lam, x)
    r2 = metrics.rel_residuals(K, M, lam, -7.5 * x)
    np.testing.assert_allclose(r1, r2, rtol=1e-15)


def test_clusters_on_a_hand_made_spectrum():
    """A pair, a triple and two singletons at relative spacing threshold 1e-2."""
    lam = np.array([1.0, 1.001, 2.0, 2.0001, 2.0002, 5.0, 10.0])
    assert metrics.clusters(lam) == [(0, 2), (2, 5), (5, 6), (6, 7)]
    # a finer threshold separates the pair (spacing 1e-3 relative to 1.001)
    assert metrics.clusters(lam, rel_gap=1e-4) == [(0, 1), (1, 2), (2, 5), (5, 6), (6, 7)]
    # the spacing is measured relative to the upper eigenvalue: (1.02 - 1) / 1.02 < 2e-2
    assert metrics.clusters(np.array([1.0, 1.02]), rel_gap=2e-2) == [(0, 2)]
    assert metrics.clusters(np.array([1.0, 1.03]), rel_gap=2e-2) == [(0, 1), (1, 2)]
    assert metrics.clusters(np.array([3.0])) == [(0, 1)]
    # clusters partition the index range
    groups = metrics.clusters(lam)
    assert groups[0][0] == 0 and groups[-1][1] == len(lam)
    assert all(a[1] == b[0] for a, b in zip(groups, groups[1:]))
