"""Accuracy measures used to compare eigen-solutions.

Oracle (test infrastructure only).

* ``gap_b``: the gap theta_b(W1, W2) of Definition 2.1 in the b-inner product
  (the M-inner product in coefficient space); for equal finite dimensions it
  equals sin{W1; W2} (Remark 2.2), the sine of the largest principal angle.
* ``rel_residuals``: ||K x_i - lambda_i M x_i||_2 / (|lambda_i| ||M x_i||_2).
* ``clusters``: groups of adjacent eigenvalues whose relative spacing is below
  a threshold; eigenvectors are compared cluster by cluster because a basis of
  a (nearly) multiple eigenspace is not unique.

Pinned by tests/test_oracle_metrics.py: lines at a known angle (Euclidean and in
a diagonal b-product), planes with known principal angles, a general SPD
b-product reduced to Euclidean principal angles (scipy) of the Cholesky-
transformed spans, unequal dimensions (the max of Definition 2.1), residuals of
exact and perturbed eigenpairs worked out by hand, and a hand-made spectrum
with a pair and a triple.
"""

from __future__ import annotations

import numpy as np


def _m_orthonormal(U, M):
    G = U.T @ (M @ U)
    G = 0.5 * (G + G.T)
    L = np.linalg.cholesky(G)
    return np.linalg.solve(L, U.T).T          # U L^{-T}


def sin_b(U, V, M) -> float:
    """sin{span U; span V} = sup_{u in U, |u|_b=1} inf_{v in V} |u - v|_b."""
    Uo = _m_orthonormal(np.asarray(U, float), M)
    Vo = _m_orthonormal(np.asarray(V, float), M)
    # b-orthogonal projection of each u onto span V, residual R = Uo - Vo (Vo^T M Uo)
    R = Uo - Vo @ (Vo.T @ (M @ Uo))
    S = R.T @ (M @ R)
    S = 0.5 * (S + S.T)
    return float(np.sqrt(max(np.linalg.eigvalsh(S).max(), 0.0)))


def gap_b(U, V, M) -> float:
    """theta_b(span U, span V) = max(sin{U;V}, sin{V;U})  (Definition 2.1)."""
    return max(sin_b(U, V, M), sin_b(V, U, M))


def rel_residuals(K, M, lam, X):
    KX = K @ X
    MX = M @ X
    R = KX - MX * lam[None, :]
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MX, axis=0))


def clusters(lam, rel_gap: float = 1e-2):
    """Index groups [a, b) of ascending eigenvalues; a new group starts where
    (lam[i] - lam[i-1]) / |lam[i]| >= rel_gap."""
    out, start = [], 0
    for i in range(1, len(lam)):
        if (lam[i] - lam[i - 1]) / abs(lam[i]) >= rel_gap:
            out.append((start, i))
            start = i
    out.append((start, len(lam)))
    return out
