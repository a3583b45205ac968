// Host dense symmetric-definite eigensolver for the coarse pencil (K_H, M_H)
// of Section 3 (n_H is a few hundred at most).  Used once per setup, on a
// host thread that overlaps the device-side setup.
//
// Method (textbook, Golub & Van Loan, "Matrix Computations", Sections 8.3):
//   M_H = L L^T (Cholesky); C = L^{-1} K_H L^{-T}; Householder reduction of C
//   to tridiagonal form T = Q^T C Q (reflectors kept, Q not formed); implicit
//   symmetric QR steps with Wilkinson shifts on T, the Givens rotations
//   recorded; the eigenvectors of T are the rotations applied to the identity
//   (row ranges independently), those of C are Q times them, and those of the
//   pencil are L^{-T} times those, which are M_H-orthonormal.
// The O(n^3) stages that act on independent rows or columns run on up to 16
// host threads; every element sees the same operations in the same order
// whatever the thread count, so the result is bit-reproducible.

#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

#include "bpjd_internal.h"

namespace bpjd {

namespace {

// body(lo, hi) over [0, n) split into contiguous ranges, one per thread (at most 16)
template <typename F>
void parallel_ranges(int n, F body) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int T = std::max(1, std::min<int>({(int)hw, 16, n / 16}));
  if (T <= 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T - 1);
  const int step = (n + T - 1) / T;
  for (int t = 1; t < T; ++t) {
    const int lo = t * step, hi = std::min(n, lo + step);
    if (lo < hi) th.emplace_back(body, lo, hi);
  }
  body(0, std::min(n, step));
  for (auto& x : th) x.join();
}

struct Reflectors {
  std::vector<std::vector<double>> v;  // v[k] acts on indices k+1 .. n-1
  std::vector<double> beta;
};

// A: n x n row-major symmetric; only its lower triangle is read and updated
// (overwritten).  On return d, e hold the tridiagonal (e[i] couples i and i+1)
// and R the reflectors H_k = I - beta v v^T with A_in = Q T Q^T,
// Q = H_0 H_1 ... H_{n-3}.
void householder_tridiag(int n, std::vector<double>& A, std::vector<double>& d, std::vector<double>& e,
                         Reflectors& R) {
  R.v.assign(std::max(0, n - 2), {});
  R.beta.assign(std::max(0, n - 2), 0.0);
  std::vector<double> p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the reflected part, rows k+1..n-1
    const int o = k + 1;
    std::vector<double>& v = R.v[k];
    v.resize(m);
    double xnorm2 = 0;
    for (int i = 0; i < m; ++i) {
      const double x = A[(size_t)(o + i) * n + k];
      v[i] = x;
      xnorm2 += x * x;
    }
    const double xnorm = std::sqrt(xnorm2);
    const double alpha = (v[0] > 0) ? -xnorm : xnorm;
    if (xnorm == 0.0) {
      A[(size_t)o * n + k] = 0.0;
      continue;
    }
    v[0] -= alpha;
    double vtv = 0;
    for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) continue;
    const double beta = 2.0 / vtv;
    R.beta[k] = beta;
    // p = beta * A_sub v from the lower triangle: row i contributes A_ij v_j to p_i
    // and A_ij v_i to p_j for j < i
    std::fill(p.begin(), p.begin() + m, 0.0);
    for (int i = 0; i < m; ++i) {
      const double* row = &A[(size_t)(o + i) * n + o];
      const double vi = v[i];
      double si = 0;
      for (int j = 0; j < i; ++j) {
        si += row[j] * v[j];
        p[j] += row[j] * vi;
      }
      p[i] += si + row[i] * vi;
    }
    for (int i = 0; i < m; ++i) p[i] *= beta;
    double ptv = 0;
    for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
    const double Kc = 0.5 * beta * ptv;
    for (int i = 0; i < m; ++i) w[i] = p[i] - Kc * v[i];
    // rank-2 update of the lower triangle
    for (int i = 0; i < m; ++i) {
      double* row = &A[(size_t)(o + i) * n + o];
      const double vi = v[i], wi = w[i];
      for (int j = 0; j <= i; ++j) row[j] -= vi * w[j] + wi * v[j];
    }
    A[(size_t)o * n + k] = alpha;
  }
  d.resize(n);
  e.assign(n > 0 ? n - 1 : 0, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
}

struct Rot {
  int k;
  double c, s;
};

// Implicit symmetric tridiagonal QR with Wilkinson shifts.  The rotation
// acting on columns (k, k+1) of the eigenvector matrix is recorded in order.
// Returns false if it fails to converge.
bool tridiag_qr(int n, std::vector<double>& d, std::vector<double>& e, std::vector<Rot>& rots) {
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
    const double a = d[hi - 1], b = e[hi - 1], c = d[hi];
    const double dd = 0.5 * (a - c);
    const double den = dd + std::copysign(std::hypot(dd, b), dd == 0.0 ? 1.0 : dd);
    const double mu = c - b * b / den;
    double x = d[lo] - mu, z = e[lo];
    double bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      if (k > lo) {
        x = e[k - 1];
        z = bulge;
      }
      const double r = std::sqrt(x * x + z * z);
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
      const double ak = d[k], bk = e[k], ck = d[k + 1];
      d[k] = cs * cs * ak - 2 * cs * sn * bk + sn * sn * ck;
      d[k + 1] = sn * sn * ak + 2 * cs * sn * bk + cs * cs * ck;
      e[k] = cs * sn * (ak - ck) + (cs * cs - sn * sn) * bk;
      if (k + 1 < hi) {
        bulge = -sn * e[k + 1];
        e[k + 1] = cs * e[k + 1];
      }
      rots.push_back({k, cs, sn});
    }
  }
  return true;
}

// Zc (n x n, column-major: column j contiguous) <- Q Zc with Q = H_0 ... H_{n-3},
// for the columns [c0, c1): reflectors applied in reverse order.
void apply_q(int n, const Reflectors& R, std::vector<double>& Zc, int c0, int c1) {
  for (int j = c0; j < c1; ++j) {
    double* z = &Zc[(size_t)j * n];
    for (int k = n - 3; k >= 0; --k) {
      const double beta = R.beta[k];
      if (beta == 0.0) continue;
      const double* v = R.v[k].data();
      const int m = n - k - 1;
      double* zz = z + k + 1;
      double s = 0;
      for (int i = 0; i < m; ++i) s += v[i] * zz[i];
      s *= beta;
      for (int i = 0; i < m; ++i) zz[i] -= s * v[i];
    }
  }
}

}  // namespace

int sym_eig_host(int n, std::vector<double> A, std::vector<double>& lam, std::vector<double>& V) {
  std::vector<double> d, e;
  Reflectors R;
  householder_tridiag(n, A, d, e, R);
  std::vector<Rot> rots;
  rots.reserve((size_t)2 * n * n);
  if (!tridiag_qr(n, d, e, rots)) return BPJD_ERR_BREAKDOWN;
  // eigenvectors of T: the rotations applied to the identity (Zc column-major;
  // each thread updates its own range of rows of every column pair)
  std::vector<double> Zc((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Zc[(size_t)i * n + i] = 1.0;
  parallel_ranges(n, [&](int r0, int r1) {
    for (const Rot& g : rots) {
      double* zk = &Zc[(size_t)g.k * n];
      double* zk1 = &Zc[(size_t)(g.k + 1) * n];
      for (int i = r0; i < r1; ++i) {
        const double a = zk[i], b = zk1[i];
        zk[i] = g.c * a - g.s * b;
        zk1[i] = g.s * a + g.c * b;
      }
    }
  });
  parallel_ranges(n, [&](int c0, int c1) { apply_q(n, R, Zc, c0, c1); });
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
  lam.resize(n);
  V.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) lam[j] = d[ord[j]];
  for (int j = 0; j < n; ++j) {
    const double* z = &Zc[(size_t)ord[j] * n];
    for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = z[i];
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
    const double ljj = std::sqrt(s);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = M[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) t -= L[(size_t)i * n + p] * L[(size_t)j * n + p];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  // Y = L^{-1} K  (forward substitution, row by row, on a column range)
  std::vector<double> Y(K);
  parallel_ranges(n, [&](int c0, int c1) {
    for (int i = 0; i < n; ++i) {
      double* yi = &Y[(size_t)i * n];
      for (int p = 0; p < i; ++p) {
        const double lip = L[(size_t)i * n + p];
        const double* yp = &Y[(size_t)p * n];
        for (int c = c0; c < c1; ++c) yi[c] -= lip * yp[c];
      }
      const double inv = 1.0 / L[(size_t)i * n + i];
      for (int c = c0; c < c1; ++c) yi[c] *= inv;
    }
  });
  // C = Y L^{-T} = (L^{-1} Y^T)^T, row by row
  std::vector<double> C((size_t)n * n);
  parallel_ranges(n, [&](int r0, int r1) {
    for (int r = r0; r < r1; ++r)
      for (int i = 0; i < n; ++i) {
        double t = Y[(size_t)r * n + i];
        for (int p = 0; p < i; ++p) t -= L[(size_t)i * n + p] * C[(size_t)r * n + p];
        C[(size_t)r * n + i] = t / L[(size_t)i * n + i];
      }
  });
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
    }
  std::vector<double> Qv;
  const int rc = sym_eig_host(n, std::move(C), lam, Qv);
  if (rc != BPJD_OK) return rc;
  // Phi = L^{-T} Q  (backward substitution, row by row, on a column range)
  Phi = std::move(Qv);
  parallel_ranges(n, [&](int c0, int c1) {
    for (int i = n - 1; i >= 0; --i) {
      double* fi = &Phi[(size_t)i * n];
      for (int p = i + 1; p < n; ++p) {
        const double lpi = L[(size_t)p * n + i];
        const double* fp = &Phi[(size_t)p * n];
        for (int c = c0; c < c1; ++c) fi[c] -= lpi * fp[c];
      }
      const double inv = 1.0 / L[(size_t)i * n + i];
      for (int c = c0; c < c1; ++c) fi[c] *= inv;
    }
  });
  return BPJD_OK;
}

}  // namespace bpjd
