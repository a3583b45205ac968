// Host dense symmetric-definite eigensolver for the coarse pencil (K_H, M_H)
// of Section 3 (n_H is a few hundred at most).  Used once per setup.
//
// Method (textbook, Golub & Van Loan, "Matrix Computations", Sections 8.3):
//   M_H = L L^T (Cholesky); C = L^{-1} K_H L^{-T}; Householder reduction of C
//   to tridiagonal form with the orthogonal factor accumulated; implicit
//   symmetric QR steps with Wilkinson shifts on the tridiagonal matrix; the
//   eigenvectors of the pencil are L^{-T} Q, which are M_H-orthonormal.

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "bpjd_internal.h"

namespace bpjd {

namespace {

// A: n x n row-major symmetric (overwritten).  On return d, e hold the
// tridiagonal (e[i] couples i and i+1) and Q the accumulated orthogonal factor
// with A_in = Q T Q^T.
void householder_tridiag(int n, std::vector<double>& A, std::vector<double>& d, std::vector<double>& e,
                         std::vector<double>& Q) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the reflected part, rows k+1..n-1
    double xnorm2 = 0;
    for (int i = 0; i < m; ++i) {
      double x = A[(size_t)(k + 1 + i) * n + k];
      v[i] = x;
      xnorm2 += x * x;
    }
    double xnorm = std::sqrt(xnorm2);
    if (xnorm == 0.0) continue;
    double alpha = (v[0] > 0) ? -xnorm : xnorm;
    v[0] -= alpha;
    double vtv = 0;
    for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) continue;
    double beta = 2.0 / vtv;
    // p = beta * A_sub v
    for (int i = 0; i < m; ++i) {
      double s = 0;
      const double* row = &A[(size_t)(k + 1 + i) * n + (k + 1)];
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      p[i] = beta * s;
    }
    double ptv = 0;
    for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
    double Kc = 0.5 * beta * ptv;
    for (int i = 0; i < m; ++i) w[i] = p[i] - Kc * v[i];
    for (int i = 0; i < m; ++i) {
      double* row = &A[(size_t)(k + 1 + i) * n + (k + 1)];
      for (int j = 0; j < m; ++j) row[j] -= v[i] * w[j] + w[i] * v[j];
    }
    A[(size_t)(k + 1) * n + k] = alpha;
    A[(size_t)k * n + (k + 1)] = alpha;
    for (int i = 1; i < m; ++i) {
      A[(size_t)(k + 1 + i) * n + k] = 0.0;
      A[(size_t)k * n + (k + 1 + i)] = 0.0;
    }
    // Q <- Q (I - beta v v^T) on columns k+1..n-1
    for (int r = 0; r < n; ++r) {
      double* row = &Q[(size_t)r * n + (k + 1)];
      double s = 0;
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      s *= beta;
      for (int j = 0; j < m; ++j) row[j] -= s * v[j];
    }
  }
  d.resize(n);
  e.assign(n > 0 ? n - 1 : 0, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
}

// Implicit symmetric tridiagonal QR with Wilkinson shifts.  Zc (n x n, stored
// column-major: column k contiguous) accumulates the rotations from the right.
// Returns false if it fails to converge.
bool tridiag_qr(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Zc) {
  const double eps = 2.220446049250313e-16;
  int iter = 0;
  const int max_iter = 60 * std::max(n, 1);
  int hi = n - 1;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (++iter > max_iter) return false;
    // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
    double a = d[hi - 1], b = e[hi - 1], c = d[hi];
    double dd = 0.5 * (a - c);
    double den = dd + std::copysign(std::hypot(dd, b), dd == 0.0 ? 1.0 : dd);
    double mu = c - b * b / den;
    double x = d[lo] - mu, z = e[lo];
    double bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      if (k > lo) {
        x = e[k - 1];
        z = bulge;
      }
      double r = std::hypot(x, z);
      double cs, sn;
      if (r == 0.0) {
        cs = 1.0;
        sn = 0.0;
      } else {
        cs = x / r;
        sn = -z / r;
      }
      if (k > lo) e[k - 1] = r;
      // G^T T G on the 2x2 block (k, k+1), G = [[c, s], [-s, c]]
      double ak = d[k], bk = e[k], ck = d[k + 1];
      d[k] = cs * cs * ak - 2 * cs * sn * bk + sn * sn * ck;
      d[k + 1] = sn * sn * ak + 2 * cs * sn * bk + cs * cs * ck;
      e[k] = cs * sn * (ak - ck) + (cs * cs - sn * sn) * bk;
      if (k + 1 < hi) {
        bulge = -sn * e[k + 1];
        e[k + 1] = cs * e[k + 1];
      }
      double* zk = &Zc[(size_t)k * n];
      double* zk1 = &Zc[(size_t)(k + 1) * n];
      for (int i = 0; i < n; ++i) {
        const double a = zk[i], b = zk1[i];
        zk[i] = cs * a - sn * b;
        zk1[i] = sn * a + cs * b;
      }
    }
  }
  return true;
}

}  // namespace

int sym_eig_host(int n, std::vector<double> A, std::vector<double>& lam, std::vector<double>& V) {
  std::vector<double> d, e, Q;
  householder_tridiag(n, A, d, e, Q);
  // column-major copy of Q for the rotations
  std::vector<double> Qc((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Qc[(size_t)j * n + i] = Q[(size_t)i * n + j];
  if (!tridiag_qr(n, d, e, Qc)) return BPJD_ERR_BREAKDOWN;
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
  lam.resize(n);
  V.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    lam[j] = d[ord[j]];
    for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = Qc[(size_t)ord[j] * n + i];
  }
  return BPJD_OK;
}

int gen_eig_host(int n, const std::vector<double>& K, const std::vector<double>& M, std::vector<double>& lam,
                 std::vector<double>& Phi) {
  // Cholesky M = L L^T (lower, row-major)
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double s = M[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) s -= L[(size_t)j * n + p] * L[(size_t)j * n + p];
    if (!(s > 0.0)) return BPJD_ERR_BREAKDOWN;
    double ljj = std::sqrt(s);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = M[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) t -= L[(size_t)i * n + p] * L[(size_t)j * n + p];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  // Y = L^{-1} K  (forward substitution, row by row)
  std::vector<double> Y(K);
  for (int i = 0; i < n; ++i) {
    double* yi = &Y[(size_t)i * n];
    for (int p = 0; p < i; ++p) {
      const double lip = L[(size_t)i * n + p];
      const double* yp = &Y[(size_t)p * n];
      for (int c = 0; c < n; ++c) yi[c] -= lip * yp[c];
    }
    const double inv = 1.0 / L[(size_t)i * n + i];
    for (int c = 0; c < n; ++c) yi[c] *= inv;
  }
  // C = Y L^{-T} = (L^{-1} Y^T)^T
  std::vector<double> C((size_t)n * n);
  for (int r = 0; r < n; ++r)
    for (int i = 0; i < n; ++i) {
      double t = Y[(size_t)r * n + i];
      for (int p = 0; p < i; ++p) t -= L[(size_t)i * n + p] * C[(size_t)r * n + p];
      C[(size_t)r * n + i] = t / L[(size_t)i * n + i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
    }
  std::vector<double> Qv;
  int rc = sym_eig_host(n, C, lam, Qv);
  if (rc != BPJD_OK) return rc;
  // Phi = L^{-T} Q  (backward substitution, row by row)
  Phi = Qv;
  for (int i = n - 1; i >= 0; --i) {
    double* fi = &Phi[(size_t)i * n];
    for (int p = i + 1; p < n; ++p) {
      const double lpi = L[(size_t)p * n + i];
      const double* fp = &Phi[(size_t)p * n];
      for (int c = 0; c < n; ++c) fi[c] -= lpi * fp[c];
    }
    const double inv = 1.0 / L[(size_t)i * n + i];
    for (int c = 0; c < n; ++c) fi[c] *= inv;
  }
  return BPJD_OK;
}

}  // namespace bpjd
