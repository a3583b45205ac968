"""The two-level block preconditioned Jacobi-Davidson method, plain FP64.

Oracle (test infrastructure only).  Notation follows Section 3: s wanted
eigenpairs (called k here, columns of X), iterate u_i^k (column i of X) with
Ritz value lambda_i^k, residual r_i^k = lambda_i^k u_i^k - A^h u_i^k, and the
preconditioner of Eq. (3.3)

    (B_i^k)^{-1} = (B_{0,i}^k)^{-1} Q_{s+1}^H Q^H + sum_l (B_{l,i}^k)^{-1} Q^(l),

with B_{0,i}^k = A^H - lambda_i^k and B_{l,i}^k = A^(l) - lambda_i^k.

Coefficient-space (matrix) form used throughout, with K, M the stiffness and
mass matrices on V^h:
  * the residual enters as the dual vector rho_i = lambda_i M x_i - K x_i
    (= M times the coefficients of r_i);
  * Q^(l) followed by (B_{l,i})^{-1}: w = (K_l - lambda_i M_l)^{-1} R_l rho_i,
    with K_l, M_l the principal submatrices of K, M on the dofs of V^(l)
    (the local Dirichlet matrices, V^(l) having zero trace on the boundary
    of Omega_l'), added back through R_l^T;
  * Q^H, Q_{s+1}^H and (B_{0,i})^{-1} in the basis Phi of M_H-orthonormal
    eigenvectors of (K_H, M_H): with c = P^T rho_i, the coarse part is
    P sum_{j > s} phi_j (phi_j^T c) / (lambda_j^H - lambda_i)
    (Q^H q is M_H^{-1} P^T rho = Phi Phi^T P^T rho; Q_{s+1}^H keeps j > s;
    A^H is diagonal in Phi; Eq. (3.2) makes this well defined);
  * I - Q_{U^k} is I - X X^T M (Remark 3.2), so t_i = z_i - X (M X)^T z_i
    (Eq. (3.5), the inner sum read as running over j with u_j^k, x_j).

Algorithm 3.1:
  Step 1  coarse eigenproblem on the grid H~ = H / 2^tau (interpolation P0):
          X^0 = P0 Phi~_{1..s}, lambda_i^0 = Rq(x_i^0).  Remark 3.3 notes that
          tau = 0 usually suffices; a larger tau also keeps lambda_i^0 below the
          smallest local Dirichlet eigenvalue when the coarse grid is very coarse.
  Step 2  t_i = (I - Q_U) (B_i)^{-1} r_i for every column.
  Step 3  Rayleigh-Ritz for the lowest s pairs in W^{k+1}; by Remark 3.1 the
          default search space is W^{k+1} = U^k + span{t_i} (dimension <= 2s);
          "3s" uses U^{k-1} + U^k + span{t_i} (the previous iterate is made
          b-orthogonal to U^k first); "grow" is the space of Algorithm 3.1
          itself, W^0 = U^0 and W^{k+1} = W^k + span{t_i}, kept as a
          b-orthonormal basis (each new block b-orthogonalised against the
          basis twice, then orthonormalised within itself, dependent
          directions dropped), optionally restarted to U^k + U^{k-1} (the
          choice V^k of Remark 3.1) when it would exceed max_dim.
  Step 4  stop: "dlambda" is the paper's rule sum_i |lambda_i^{k+1} - lambda_i^k|
          < tol; "residual" stops when every relative residual
          ||K x_i - lambda_i M x_i||_2 / (|lambda_i| ||M x_i||_2) <= tol.

The Rayleigh-Ritz step b-orthonormalises W explicitly: T columns are scaled
to unit M-norm, the Gram matrix G = W^T M W is diagonalised, directions with
eigenvalue below drop_tol * max are dropped (near-dependent corrections of
converged columns), and the projected pencil is reduced to a standard
symmetric eigenproblem.  The k lowest Ritz pairs are kept.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


class LocalIndefinite(RuntimeError):
    """A shifted local matrix K_l - lambda_i M_l is not positive definite (Eq. (3.1) violated)."""


class CoarseGap(RuntimeError):
    """lambda_s^H and lambda_{s+1}^H coincide (Assumption 1 fails on the coarse space)."""


@dataclass
class Setup:
    K: sp.csr_matrix
    M: sp.csr_matrix
    P: sp.csr_matrix
    sub_ptr: np.ndarray
    sub_dofs: np.ndarray
    k: int
    K_loc: List[np.ndarray]
    M_loc: List[np.ndarray]
    lamH: np.ndarray
    Phi: np.ndarray
    KH: np.ndarray
    MH: np.ndarray
    P0: sp.csr_matrix
    lam0H: np.ndarray
    Phi0: np.ndarray

    @property
    def n(self) -> int:
        return self.K.shape[0]

    def dofs(self, l: int) -> np.ndarray:
        return self.sub_dofs[self.sub_ptr[l]:self.sub_ptr[l + 1]]


def _coarse_pencil(K, M, P, k, gap_rtol):
    KH = (P.T @ (K @ P)).toarray()
    MH = (P.T @ (M @ P)).toarray()
    KH = 0.5 * (KH + KH.T)
    MH = 0.5 * (MH + MH.T)
    if not k < KH.shape[0]:
        raise ValueError("s must be smaller than dim V^H")
    lamH, Phi = sla.eigh(KH, MH)
    if (lamH[k] - lamH[k - 1]) <= gap_rtol * abs(lamH[k]):
        raise CoarseGap(f"coarse eigenvalues {k} and {k + 1} coincide")
    return KH, MH, lamH, Phi


def setup(K, M, P, sub_ptr, sub_dofs, k: int, P0=None, gap_rtol: float = 1e-8) -> Setup:
    """Local Dirichlet matrices, the coarse Galerkin pencil and its eigen-decomposition.

    P0 interpolates from the grid H~ of Algorithm 3.1 Step 1 (None: H~ = H)."""
    K = sp.csr_matrix(K)
    M = sp.csr_matrix(M)
    P = sp.csr_matrix(P)
    sub_ptr = np.asarray(sub_ptr, dtype=np.int64)
    sub_dofs = np.asarray(sub_dofs, dtype=np.int64)
    K_loc, M_loc = [], []
    for l in range(len(sub_ptr) - 1):
        d = sub_dofs[sub_ptr[l]:sub_ptr[l + 1]]
        K_loc.append(K[d][:, d].toarray())
        M_loc.append(M[d][:, d].toarray())
    KH, MH, lamH, Phi = _coarse_pencil(K, M, P, k, gap_rtol)
    if P0 is None:
        P0, lam0H, Phi0 = P, lamH, Phi
    else:
        P0 = sp.csr_matrix(P0)
        _, _, lam0H, Phi0 = _coarse_pencil(K, M, P0, k, gap_rtol)
    return Setup(K, M, P, sub_ptr, sub_dofs, k, K_loc, M_loc, lamH, Phi, KH, MH, P0, lam0H, Phi0)


def initial_guess(S: Setup):
    """Algorithm 3.1 Step 1: x_i^0 = P0 phi~_i from the grid H~, lambda_i^0 = Rq(x_i^0)."""
    X = S.P0 @ S.Phi0[:, :S.k]
    AX = S.K @ X
    MX = S.M @ X
    lam = np.einsum("ij,ij->j", X, AX) / np.einsum("ij,ij->j", X, MX)
    return X, AX, MX, lam


def coarse_correction(S: Setup, rho: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """(B_{0,i})^{-1} Q_{s+1}^H Q^H r_i for every column i, mapped into V^h by P."""
    c = S.P.T @ rho                        # n_H x k
    a = S.Phi.T @ c                        # coordinates in the coarse eigenbasis
    a[:S.k, :] = 0.0                       # Q_{s+1}^H: drop U_s^H
    for i in range(rho.shape[1]):
        a[S.k:, i] /= (S.lamH[S.k:] - lam[i])
    return S.P @ (S.Phi @ a)


def local_corrections(S: Setup, rho: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """sum_l R_l^T (K_l - lambda_i M_l)^{-1} R_l rho_i for every column i, l in order."""
    Z = np.zeros_like(rho)
    for l in range(len(S.K_loc)):
        d = S.dofs(l)
        for i in range(rho.shape[1]):
            B = S.K_loc[l] - lam[i] * S.M_loc[l]
            try:
                cf = sla.cho_factor(B, lower=True)
            except np.linalg.LinAlgError as e:
                raise LocalIndefinite(f"subdomain {l}, column {i}") from e
            Z[d, i] += sla.cho_solve(cf, rho[d, i])
    return Z


def apply_preconditioner(S: Setup, rho: np.ndarray, lam: np.ndarray, coarse: bool = True) -> np.ndarray:
    """Eq. (3.3) applied to every column: coarse term first, then subdomains l = 0..N-1."""
    Z = coarse_correction(S, rho, lam) if coarse else np.zeros_like(rho)
    return Z + local_corrections(S, rho, lam)


def residual(AX, MX, lam):
    """rho_i = lambda_i M x_i - K x_i and the relative residual norms."""
    rho = MX * lam[None, :] - AX
    rel = np.linalg.norm(rho, axis=0) / (np.abs(lam) * np.linalg.norm(MX, axis=0))
    return rho, rel


def project_out(X, MX, Z):
    """Eq. (3.5) in matrix form: T = (I - X X^T M) Z."""
    return Z - X @ (MX.T @ Z)


def rayleigh_ritz(W, AW, MW, k: int, n_fixed: int, drop_tol: float = 1e-10):
    """Lowest k Ritz pairs of (K, M) in span W (Eq. (3.6)).

    The first ``n_fixed`` columns of W are the current (b-orthonormal) Ritz
    vectors; the others are scaled to unit M-norm (zero columns dropped).
    Returns (theta[:k], C) with W C the new b-orthonormal Ritz vectors.
    """
    m = W.shape[1]
    G = W.T @ MW
    H = W.T @ AW
    G = 0.5 * (G + G.T)
    H = 0.5 * (H + H.T)
    s = np.ones(m)
    for j in range(n_fixed, m):
        s[j] = 1.0 / np.sqrt(G[j, j]) if G[j, j] > 0 else 0.0
    Gs = G * s[:, None] * s[None, :]
    Hs = H * s[:, None] * s[None, :]
    g, Q = np.linalg.eigh(Gs)
    keep = g > drop_tol * g.max()
    B = Q[:, keep] / np.sqrt(g[keep])[None, :]
    Hr = B.T @ Hs @ B
    Hr = 0.5 * (Hr + Hr.T)
    theta, Y = np.linalg.eigh(Hr)
    C = s[:, None] * (B @ Y[:, :k])
    return theta[:k], C


@dataclass
class Result:
    lam: np.ndarray
    X: np.ndarray
    iterations: int
    converged: bool
    history_lam: List[np.ndarray] = field(default_factory=list)
    history_res: List[float] = field(default_factory=list)
    history_dlam: List[float] = field(default_factory=list)
    restarts: int = 0


def extend_orthonormal(K, M, V, KV, MV, T, drop_tol: float = 1e-10):
    """Append span(T) to the b-orthonormal basis V (growing space of Algorithm 3.1).

    T is b-orthogonalised against V twice (classical Gram-Schmidt in the M-inner
    product, repeated), then orthonormalised within itself through the eigen-
    decomposition of its Gram matrix, directions below drop_tol * max dropped.
    The products K V, M V of the new columns are formed from the columns
    themselves (near convergence a new direction is a small difference of large
    terms, whose products by linear combination would carry that cancellation).
    Returns the extended (V, KV, MV) and the number of columns added.
    """
    for _ in range(2):
        T = T - V @ (MV.T @ T)
    MT = M @ T
    G = T.T @ MT
    G = 0.5 * (G + G.T)
    g, Q = np.linalg.eigh(G)
    keep = g > drop_tol * max(g.max(), 0.0) if g.max() > 0 else np.zeros_like(g, dtype=bool)
    Tn = T @ (Q[:, keep] / np.sqrt(g[keep])[None, :])
    return (np.hstack([V, Tn]), np.hstack([KV, K @ Tn]), np.hstack([MV, M @ Tn]), int(keep.sum()))


def sign_normalise(X):
    """Flip each column so its largest-magnitude entry is positive (lowest index wins ties)."""
    X = X.copy()
    for i in range(X.shape[1]):
        j = int(np.argmax(np.abs(X[:, i])))
        if X[j, i] < 0:
            X[:, i] = -X[:, i]
    return X


def solve(S: Setup, tol: float = 1e-8, max_iter: int = 200, stop: str = "residual",
          subspace: str = "2s", drop_tol: float = 1e-10, coarse: bool = True,
          callback=None, max_dim: Optional[int] = None) -> Result:
    """Algorithm 3.1 until the stop rule holds or max_iter Rayleigh-Ritz steps were taken.

    max_dim (subspace "grow" only): restart the growing space to U^k + U^{k-1}
    when appending the next block would make it larger than max_dim columns.
    """
    k = S.k
    X, AX, MX, lam = initial_guess(S)
    res = Result(lam.copy(), X, 0, False)
    res.history_lam.append(lam.copy())
    Xprev = AXprev = MXprev = None
    # growing space: b-orthonormal basis of W^k and its products (W^0 = U^0)
    Vg, KVg, MVg = X, AX, MX
    res.restarts = 0
    for it in range(max_iter + 1):
        rho, rel = residual(AX, MX, lam)
        res.history_res.append(float(rel.max()))
        if stop == "residual" and rel.max() <= tol:
            res.converged = True
            break
        if it == max_iter:
            break
        Z = apply_preconditioner(S, rho, lam, coarse=coarse)
        T = project_out(X, MX, Z)
        AT = S.K @ T
        MT = S.M @ T
        if subspace == "2s":
            W, AW, MW = np.hstack([X, T]), np.hstack([AX, AT]), np.hstack([MX, MT])
        elif subspace == "3s":
            if Xprev is None:
                W, AW, MW = np.hstack([X, T]), np.hstack([AX, AT]), np.hstack([MX, MT])
            else:
                # previous iterate, made b-orthogonal to X so the first k columns stay fixed
                Pp = Xprev - X @ (MX.T @ Xprev)
                W = np.hstack([X, Pp, T])
                AW = np.hstack([AX, S.K @ Pp, AT])
                MW = np.hstack([MX, S.M @ Pp, MT])
        elif subspace == "grow":
            if max_dim is not None and Vg.shape[1] + k > max_dim:
                # restart inside Remark 3.1: V^k = U^k + U^{k-1}
                Vg, KVg, MVg = X, AX, MX
                if Xprev is not None:
                    Vg, KVg, MVg, _ = extend_orthonormal(S.K, S.M, Vg, KVg, MVg, Xprev, drop_tol)
                res.restarts += 1
            Vg, KVg, MVg, _ = extend_orthonormal(S.K, S.M, Vg, KVg, MVg, T, drop_tol)
            Hg = Vg.T @ KVg
            Hg = 0.5 * (Hg + Hg.T)
            theta_all, Y = np.linalg.eigh(Hg)
            theta, C = theta_all[:k], Y[:, :k]
            W, AW, MW = Vg, KVg, MVg
        else:
            raise ValueError(subspace)
        if subspace != "grow":
            theta, C = rayleigh_ritz(W, AW, MW, k, k, drop_tol)
        Xprev, AXprev, MXprev = X, AX, MX
        X = W @ C
        AX = S.K @ X
        MX = S.M @ X
        dl = float(np.abs(theta - lam).sum())
        lam = theta
        res.iterations = it + 1
        res.history_lam.append(lam.copy())
        res.history_dlam.append(dl)
        if callback is not None:
            callback(it + 1, lam, X)
        if stop == "dlambda" and dl < tol:
            res.converged = True
            break
    res.lam = lam
    res.X = sign_normalise(X)
    return res
