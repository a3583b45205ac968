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
#include <cstdint>
#include <numeric>
#include <atomic>
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

// The same reduction on T host threads (for n in the hundreds and more): per
// step, thread 0 forms the reflector, the matrix-vector product runs over
// fixed chunks of 32 rows with one partial vector per chunk (summed in chunk
// order, so the result does not depend on T), and the rank-2 update is split
// by chunks.  Threads meet at a spinning barrier five times per step.
struct SpinBarrier {
  std::atomic<int> count{0}, gen{0};
  int n;
  explicit SpinBarrier(int n_) : n(n_) {}
  void wait() {
    const int g = gen.load(std::memory_order_acquire);
    if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
      count.store(0, std::memory_order_relaxed);
      gen.fetch_add(1, std::memory_order_release);
    } else {
      while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
    }
  }
};

void householder_tridiag_threads(int n, std::vector<double>& A, std::vector<double>& d, std::vector<double>& e,
                                 Reflectors& R, int T) {
  constexpr int CH = 32;
  R.v.assign(std::max(0, n - 2), {});
  R.beta.assign(std::max(0, n - 2), 0.0);
  const int nch_max = (n + CH - 1) / CH;
  std::vector<double> part((size_t)nch_max * n), p(n), w(n);
  SpinBarrier bar(T);
  double alpha_s = 0, beta_s = 0;
  int skip = 0;
  auto body = [&](int tid) {
    for (int k = 0; k + 2 < n; ++k) {
      const int m = n - k - 1, o = k + 1;
      std::vector<double>& v = R.v[k];
      if (tid == 0) {
        v.resize(m);
        double xnorm2 = 0;
        for (int i = 0; i < m; ++i) {
          const double x = A[(size_t)(o + i) * n + k];
          v[i] = x;
          xnorm2 += x * x;
        }
        const double xnorm = std::sqrt(xnorm2);
        alpha_s = (v[0] > 0) ? -xnorm : xnorm;
        skip = 0;
        if (xnorm == 0.0) {
          A[(size_t)o * n + k] = 0.0;
          skip = 1;
        } else {
          v[0] -= alpha_s;
          double vtv = 0;
          for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
          if (vtv == 0.0) {
            skip = 1;
          } else {
            beta_s = 2.0 / vtv;
            R.beta[k] = beta_s;
          }
        }
      }
      bar.wait();
      if (skip) continue;
      const int nch = (m + CH - 1) / CH;
      // partial products, one vector per chunk of rows (entries 0 .. last row of the chunk)
      for (int c = tid; c < nch; c += T) {
        const int i0 = c * CH, i1 = std::min(m, i0 + CH);
        double* pc = &part[(size_t)c * n];
        std::fill(pc, pc + i1, 0.0);
        for (int i = i0; i < i1; ++i) {
          const double* row = &A[(size_t)(o + i) * n + o];
          const double vi = v[i];
          double si = 0;
          for (int j = 0; j < i; ++j) {
            si += row[j] * v[j];
            pc[j] += row[j] * vi;
          }
          pc[i] += si + row[i] * vi;
        }
      }
      bar.wait();
      // p_j = beta * sum over the chunks that reach row j, in chunk order
      for (int j0 = tid * CH; j0 < m; j0 += T * CH) {
        const int j1 = std::min(m, j0 + CH);
        for (int j = j0; j < j1; ++j) {
          double sj = 0;
          for (int c = j / CH; c < nch; ++c) sj += part[(size_t)c * n + j];
          p[j] = beta_s * sj;
        }
      }
      bar.wait();
      if (tid == 0) {
        double ptv = 0;
        for (int i = 0; i < m; ++i) ptv += p[i] * v[i];
        const double Kc = 0.5 * beta_s * ptv;
        for (int i = 0; i < m; ++i) w[i] = p[i] - Kc * v[i];
      }
      bar.wait();
      for (int c = tid; c < nch; c += T) {
        const int i0 = c * CH, i1 = std::min(m, i0 + CH);
        for (int i = i0; i < i1; ++i) {
          double* row = &A[(size_t)(o + i) * n + o];
          const double vi = v[i], wi = w[i];
          for (int j = 0; j <= i; ++j) row[j] -= vi * w[j] + wi * v[j];
        }
      }
      bar.wait();
      if (tid == 0) A[(size_t)o * n + k] = alpha_s;
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(body, t);
  body(0);
  for (auto& x : th) x.join();
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
// acting on columns (k, k+1) of the eigenvector matrix is recorded in order
// (when rots is not NULL).
// Returns false if it fails to converge.
bool tridiag_qr(int n, std::vector<double>& d, std::vector<double>& e, std::vector<Rot>* rots) {
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
      if (rots) rots->push_back({k, cs, sn});
    }
  }
  return true;
}

// The rotation sequence applied to nr rows (row stride ldz) starting at z0.  A
// QR sweep records rotations on consecutive column pairs (k, k+1), (k+1, k+2),
// ...; along such a run the new entry k+1 of one rotation is the entry k of the
// next, so every row carries it in a register (one load and one store per
// rotation and row instead of two of each, the same arithmetic).  NR > 0 fixes
// the row count.
template <int NR>
void rotate_rows(const std::vector<Rot>& rots, double* z0, int ldz, int nr) {
  constexpr int kMax = 8;
  const int cnt = NR > 0 ? NR : nr;
  const size_t nrot = rots.size();
  for (size_t r0 = 0; r0 < nrot;) {
    size_t r1 = r0 + 1;
    while (r1 < nrot && rots[r1].k == rots[r1 - 1].k + 1) ++r1;
    // the run r0 .. r1 - 1 acts on columns rots[r0].k .. rots[r1 - 1].k + 1
    double carry[kMax];
    const int k0 = rots[r0].k;
#pragma GCC unroll 8
    for (int i = 0; i < cnt; ++i) carry[i] = z0[(size_t)i * ldz + k0];
    for (size_t q = r0; q < r1; ++q) {
      const Rot& g = rots[q];
      double* z = z0 + g.k;
#pragma GCC unroll 8
      for (int i = 0; i < cnt; ++i) {
        const double a = carry[i], b = z[(size_t)i * ldz + 1];
        z[(size_t)i * ldz] = g.c * a - g.s * b;
        carry[i] = g.s * a + g.c * b;
      }
    }
    const int kl = rots[r1 - 1].k + 1;
#pragma GCC unroll 8
    for (int i = 0; i < cnt; ++i) z0[(size_t)i * ldz + kl] = carry[i];
    r0 = r1;
  }
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

// Eigenvectors of the symmetric tridiagonal T (diagonal d, off-diagonal e) for
// the given ascending eigenvalues mu[0..nv), by inverse iteration (Wilkinson,
// "The Algebraic Eigenvalue Problem", Ch. 5): (T - mu I) is factorised by
// Gaussian elimination with partial pivoting, three solves from a fixed start
// vector, each followed by Gram-Schmidt (twice) against the vectors of
// eigenvalues closer than 1e-3 ||T|| (a cluster), and normalisation.
// Z: n x nv, column-major.
void tridiag_inverse_iteration(int n, const std::vector<double>& d, const std::vector<double>& e,
                               const std::vector<double>& mu, int nv, std::vector<double>& Z) {
  double tn = 0;
  for (int i = 0; i < n; ++i) tn = std::max(tn, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) +
                                                     (i + 1 < n ? std::fabs(e[i]) : 0.0));
  const double tiny = 1e-15 * std::max(tn, 1e-300);
  Z.assign((size_t)n * nv, 0.0);
  std::vector<double> u0(n), u1(n), u2(n), lm(n), x(n);
  std::vector<char> piv(n);
  for (int j = 0; j < nv; ++j) {
    const double m = mu[j];
    // factorisation of T - m I with row interchanges: U has three diagonals
    double a0 = d[0] - m, a1 = (n > 1) ? e[0] : 0.0, a2 = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
      const double sub = e[i], dn = d[i + 1] - m, up = (i + 2 < n) ? e[i + 1] : 0.0;
      if (std::fabs(sub) > std::fabs(a0)) {
        const double f = a0 / sub;
        u0[i] = sub;
        u1[i] = dn;
        u2[i] = up;
        lm[i] = f;
        piv[i] = 1;
        a0 = a1 - f * dn;
        a1 = a2 - f * up;
        a2 = 0.0;
      } else {
        if (std::fabs(a0) < tiny) a0 = tiny;
        const double f = sub / a0;
        u0[i] = a0;
        u1[i] = a1;
        u2[i] = a2;
        lm[i] = f;
        piv[i] = 0;
        a0 = dn - f * a1;
        a1 = up - f * a2;
        a2 = 0.0;
      }
    }
    if (std::fabs(a0) < tiny) a0 = tiny;
    u0[n - 1] = a0;
    u1[n - 1] = u2[n - 1] = 0.0;
    for (int i = 0; i < n; ++i) x[i] = 1.0 + 0.1 * std::sin(0.7 * i + 0.3 * j);  // fixed start vector
    for (int it = 0; it < 3; ++it) {
      for (int i = 0; i + 1 < n; ++i) {
        if (piv[i]) std::swap(x[i], x[i + 1]);
        x[i + 1] -= lm[i] * x[i];
      }
      x[n - 1] /= u0[n - 1];
      if (n > 1) x[n - 2] = (x[n - 2] - u1[n - 2] * x[n - 1]) / u0[n - 2];
      for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - u1[i] * x[i + 1] - u2[i] * x[i + 2]) / u0[i];
      for (int pass = 0; pass < 2; ++pass)
        for (int q = j - 1; q >= 0 && mu[j] - mu[q] < 1e-3 * tn; --q) {
          const double* zq = &Z[(size_t)q * n];
          double dot = 0;
          for (int i = 0; i < n; ++i) dot += zq[i] * x[i];
          for (int i = 0; i < n; ++i) x[i] -= dot * zq[i];
        }
      double nrm = 0;
      for (int i = 0; i < n; ++i) nrm += x[i] * x[i];
      nrm = std::sqrt(nrm);
      if (!(nrm > 0)) nrm = 1.0;
      for (int i = 0; i < n; ++i) x[i] /= nrm;
    }
    std::copy(x.begin(), x.end(), Z.begin() + (size_t)j * n);
  }
}

}  // namespace

int sym_eig_host(int n, std::vector<double> A, std::vector<double>& lam, std::vector<double>& V, int nvec) {
  std::vector<double> d, e;
  Reflectors R;
  const int T = std::min<int>(16, (int)std::max(1u, std::thread::hardware_concurrency()));
  if (n >= 384 && T > 1)
    householder_tridiag_threads(n, A, d, e, R, T);
  else
    householder_tridiag(n, A, d, e, R);
  if (nvec < 0 || nvec > n) nvec = n;
  if (nvec < n) {
    // eigenvalues by QR without vectors, eigenvectors of the lowest nvec by
    // inverse iteration, back-transformed by the reflectors
    std::vector<double> dq(d), eq(e);
    if (!tridiag_qr(n, dq, eq, nullptr)) return BPJD_ERR_BREAKDOWN;
    std::sort(dq.begin(), dq.end());
    std::vector<double> Zc;
    tridiag_inverse_iteration(n, d, e, dq, nvec, Zc);
    parallel_ranges(nvec, [&](int c0, int c1) { apply_q(n, R, Zc, c0, c1); });
    lam = dq;
    V.assign((size_t)n * n, 0.0);
    for (int j = 0; j < nvec; ++j)
      for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = Zc[(size_t)j * n + i];
    return BPJD_OK;
  }
  std::vector<Rot> rots;
  rots.reserve((size_t)2 * n * n);
  if (!tridiag_qr(n, d, e, &rots)) return BPJD_ERR_BREAKDOWN;
  // eigenvectors of T: the rotations applied to the identity.  Rows are
  // independent (a rotation mixes two columns within each row), so each thread
  // takes a range of rows of a row-major copy (rows padded to whole cache lines,
  // so no two threads write the same line) and applies the whole rotation
  // sequence to eight rows at a time; then the result is transposed into the
  // column-major Zc of the reflector back-transformation.
  const int ldz = (n + 7) & ~7;
  std::vector<double> zbuf((size_t)n * ldz + 8, 0.0);
  double* Zr = zbuf.data() + ((8 - ((reinterpret_cast<uintptr_t>(zbuf.data()) / sizeof(double)) & 7)) & 7);
  for (int i = 0; i < n; ++i) Zr[(size_t)i * ldz + i] = 1.0;
  parallel_ranges(n, [&](int r0, int r1) {
    for (int i0 = r0; i0 < r1; i0 += 8) {
      const int nr = std::min(8, r1 - i0);
      double* z0 = Zr + (size_t)i0 * ldz;
      if (nr == 8)
        rotate_rows<8>(rots, z0, ldz, 8);
      else
        rotate_rows<0>(rots, z0, ldz, nr);
    }
  });
  std::vector<double> Zc((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Zc[(size_t)j * n + i] = Zr[(size_t)i * ldz + j];
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
                 std::vector<double>& Phi, int nvec) {
  if (nvec < 0 || nvec > n) nvec = n;
  // Cholesky M = L L^T (lower, row-major), column by column; for large n the
  // rows below the diagonal of a column are shared among threads
  std::vector<double> L((size_t)n * n, 0.0);
  const int T = std::min<int>(16, (int)std::max(1u, std::thread::hardware_concurrency()));
  bool spd = true;
  auto col_rows = [&](int j, int i0, int i1) {
    const double ljj = L[(size_t)j * n + j];
    const double* lj = &L[(size_t)j * n];
    for (int i = i0; i < i1; ++i) {
      const double* li = &L[(size_t)i * n];
      double t = M[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) t -= li[p] * lj[p];
      L[(size_t)i * n + j] = t / ljj;
    }
  };
  auto diag = [&](int j) {
    double s = M[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) s -= L[(size_t)j * n + p] * L[(size_t)j * n + p];
    if (!(s > 0.0)) {
      spd = false;
      s = 1.0;
    }
    L[(size_t)j * n + j] = std::sqrt(s);
  };
  if (n >= 384 && T > 1) {
    SpinBarrier bar(T);
    auto body = [&](int tid) {
      for (int j = 0; j < n; ++j) {
        if (tid == 0) diag(j);
        bar.wait();
        const int rows = n - j - 1, per = (rows + T - 1) / T;
        const int i0 = j + 1 + tid * per, i1 = std::min(n, i0 + per);
        if (i0 < i1) col_rows(j, i0, i1);
        bar.wait();
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back(body, t);
    body(0);
    for (auto& x : th) x.join();
  } else {
    for (int j = 0; j < n; ++j) {
      diag(j);
      col_rows(j, j + 1, n);
    }
  }
  if (!spd) return BPJD_ERR_BREAKDOWN;
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
  const int rc = sym_eig_host(n, std::move(C), lam, Qv, nvec);
  if (rc != BPJD_OK) return rc;
  // Phi = L^{-T} Q  (backward substitution, row by row, on a column range)
  Phi = std::move(Qv);
  parallel_ranges(nvec, [&](int c0, int c1) {
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
