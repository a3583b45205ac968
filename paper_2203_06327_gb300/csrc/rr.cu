// Rayleigh-Ritz step of Algorithm 3.1 (Step 3, Eq. (3.6)) on the small
// projected pencil: one CTA per call.  Split out of kernels.cu so that the
// two large translation units compile in parallel.

#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bpjd_internal.h"
#include "dword.cuh"

namespace bpjd {

namespace {
// ---------------------------------------------------------------------------
// Rayleigh-Ritz in W (one block, FP64).  Parallel cyclic Jacobi (round-robin
// ordering) for the two small symmetric eigenproblems.
// ---------------------------------------------------------------------------
constexpr int kRRMax = 64;
// leading dimension of the reduced matrices in shared memory: one more than the
// size, so that column accesses fall into distinct banks
constexpr int kRRLd = kRRMax + 1;

// Symmetric eigen-decomposition of A (m x m, leading dimension ld = kRRLd) in
// shared memory; V receives the eigenvectors (columns), A's diagonal the
// eigenvalues.  mp = m rounded up to even (the extra index is a zero row/column
// that never rotates).  Uses all threads of the block.
__device__ void jacobi_eig(double* A, double* V, int m, double* cs, double* sn, int* pp, int* qq) {
  const int mp = m + (m & 1);
  const int ld = kRRLd;
  const int tid = threadIdx.x;
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    int r = t / ld, c = t % ld;
    V[t] = (r == c) ? 1.0 : 0.0;
    if ((r >= m || c >= m) && c < mp) A[t] = 0.0;
  }
  __syncthreads();
  const int half = mp / 2;
  __shared__ int done;
  __shared__ double amax;
  if (tid == 0) {
    double a = 0;
    for (int j = 0; j < m; ++j) a = fmax(a, fabs(A[j * ld + j]));
    amax = a;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) done = 1;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      if (tid < half) {
        // circle method: position 0 fixed, the others rotate
        int e0 = 0, e1;
        auto ring = [&](int pos) { return ((pos + round) % (mp - 1)) + 1; };
        if (tid == 0) {
          e1 = ring(0);
        } else {
          e0 = ring(tid);
          e1 = ring(mp - 1 - tid);
        }
        int p = min(e0, e1), q = max(e0, e1);
        double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300 && fabs(apq) > 1e-17 * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-30 * amax) {
          double tau = (aqq - app) / (2.0 * apq);
          double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
          done = 0;
        }
        cs[tid] = c;
        sn[tid] = s;
        pp[tid] = p;
        qq[tid] = q;
      }
      __syncthreads();
      // A <- A J and V <- V J (columns p, q of every pair)
      for (int t = tid; t < half * mp; t += blockDim.x) {
        int pr = t / mp, r = t % mp;
        int p = pp[pr], q = qq[pr];
        double c = cs[pr], s = sn[pr];
        double ap = A[r * ld + p], aq = A[r * ld + q];
        A[r * ld + p] = c * ap - s * aq;
        A[r * ld + q] = s * ap + c * aq;
        double vp = V[r * ld + p], vq = V[r * ld + q];
        V[r * ld + p] = c * vp - s * vq;
        V[r * ld + q] = s * vp + c * vq;
      }
      __syncthreads();
      // A <- J^T A (rows p, q of every pair)
      for (int t = tid; t < half * mp; t += blockDim.x) {
        int pr = t / mp, col = t % mp;
        int p = pp[pr], q = qq[pr];
        double c = cs[pr], s = sn[pr];
        double ap = A[p * ld + col], aq = A[q * ld + col];
        A[p * ld + col] = c * ap - s * aq;
        A[q * ld + col] = s * ap + c * aq;
      }
      __syncthreads();
    }
    if (done) break;
    __syncthreads();
  }
}

// Strict total order for ranking eigenvalues: NaN counts as +infinity and ties
// go by index, so the ranks always form a permutation (the ranks index shared
// memory, whatever the data).
__device__ __forceinline__ bool order_before(double a, int ia, double b, int ib) {
  a = isnan(a) ? CUDART_INF : a;
  b = isnan(b) ? CUDART_INF : b;
  return a < b || (a == b && ia < ib);
}

// Ascending order of diag(A)[0..m): ord[rank] = index (ties by index).
__device__ void sort_diag(const double* A, int m, int* ord) {
  const int ld = kRRLd;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double dj = A[j * ld + j];
    int rank = 0;
    for (int i = 0; i < m; ++i) {
      if (order_before(A[i * ld + i], i, dj, j)) ++rank;
    }
    ord[rank] = j;
  }
  __syncthreads();
}

// G, H: m x m (row-major, ld m).  scale_all = 0: the first k columns of W are
// M-orthonormal Ritz vectors and stay as they are, the rest are scaled to unit
// M-norm; scale_all = 1: every column is scaled.  Output C (m x k, ld k),
// lam_new (k), hist row, status.
__device__ void rayleigh_ritz_eig(int m, int k, const double* __restrict__ G, const double* __restrict__ H,
                                  double drop_tol, const double* __restrict__ lam_old, double* C, double* lam_new,
                                  double* hist_row, int stop_rule, double tol, DevStatus* st, double* rr,
                                  int scale_all) {
  const int ld = kRRLd;
  double* A = rr;                  // ld x ld
  double* V = A + ld * ld;         // ld x ld
  double* Bm = V + ld * ld;        // ld x ld : basis of the kept directions (m x r)
  double* Hs = Bm + ld * ld;       // ld x ld : scaled H
  double* sc = Hs + ld * ld;       // ld     : column scaling
  double* cs = sc + ld;            // ld/2
  double* sn = cs + ld;
  int* pp = reinterpret_cast<int*>(sn + ld);
  int* qq = pp + ld;
  int* ord = qq + ld;
  __shared__ int r_keep;
  const int tid = threadIdx.x;
  for (int j = tid; j < m; j += blockDim.x) {
    double g = G[j * m + j];
    sc[j] = (j < k && !scale_all) ? 1.0 : (g > 0 ? 1.0 / sqrt(g) : 0.0);
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) {
    int a = t / m, b = t % m;
    double gs = 0.5 * (G[a * m + b] + G[b * m + a]) * sc[a] * sc[b];
    double hs = 0.5 * (H[a * m + b] + H[b * m + a]) * sc[a] * sc[b];
    A[a * ld + b] = gs;
    Hs[a * ld + b] = hs;
  }
  __syncthreads();
  jacobi_eig(A, V, m, cs, sn, pp, qq);
  sort_diag(A, m, ord);
  // keep eigen-directions of the scaled Gram matrix above drop_tol * max
  if (tid == 0) {
    double gmax = A[ord[m - 1] * ld + ord[m - 1]];
    int r = 0;
    for (int t = 0; t < m; ++t)
      if (A[ord[t] * ld + ord[t]] > drop_tol * gmax) ++r;
    r_keep = r;
  }
  __syncthreads();
  const int r = r_keep;
  const int first = m - r;  // kept = ord[first .. m)
  // Bm[:, c] = V[:, ord[first + c]] / sqrt(g)
  for (int t = tid; t < m * r; t += blockDim.x) {
    int a = t / r, c = t % r;
    int j = ord[first + c];
    Bm[a * ld + c] = V[a * ld + j] / sqrt(A[j * ld + j]);
  }
  __syncthreads();
  // V <- Hs Bm (m x r), then A <- Bm^T V (r x r)
  for (int t = tid; t < m * r; t += blockDim.x) {
    int a = t / r, c = t % r;
    double s = 0;
    for (int e = 0; e < m; ++e) s = fma(Hs[a * ld + e], Bm[e * ld + c], s);
    V[a * ld + c] = s;
  }
  __syncthreads();
  for (int t = tid; t < r * r; t += blockDim.x) {
    int a = t / r, c = t % r;
    double s = 0;
    for (int e = 0; e < m; ++e) s = fma(Bm[e * ld + a], V[e * ld + c], s);
    A[a * ld + c] = s;
  }
  __syncthreads();
  for (int t = tid; t < r * r; t += blockDim.x) {
    int a = t / r, c = t % r;
    if (a < c) {
      double s = 0.5 * (A[a * ld + c] + A[c * ld + a]);
      A[a * ld + c] = s;
      A[c * ld + a] = s;
    }
  }
  __syncthreads();
  jacobi_eig(A, V, r, cs, sn, pp, qq);
  sort_diag(A, r, ord);
  // C = diag(sc) Bm Y[:, 0..k)
  const int kk = min(k, r);
  for (int t = tid; t < m * k; t += blockDim.x) {
    int a = t / k, c = t % k;
    double s = 0;
    if (c < kk) {
      int j = ord[c];
      for (int e = 0; e < r; ++e) s = fma(Bm[a * ld + e], V[e * ld + j], s);
    }
    C[a * k + c] = sc[a] * s;
  }
  __syncthreads();
  if (tid == 0) {
    double dl = 0;
    for (int c = 0; c < k; ++c) {
      double th = (c < kk) ? A[ord[c] * ld + ord[c]] : lam_old[c];
      dl += fabs(th - lam_old[c]);
      lam_new[c] = th;
      if (hist_row) hist_row[c] = th;
    }
    st->sum_dl = dl;
    st->kept = r;
    if (r < k) st->err_breakdown = 1;
    if (stop_rule == BPJD_STOP_DLAMBDA) st->converged = (dl < tol) ? 1 : 0;
  }
}

// Parallel cyclic Jacobi, one pass per round: with the round's disjoint
// rotations J, A' = J^T A J is formed element-wise from the old A (4 terms per
// entry, lower triangle mirrored) into a second buffer, and V' = V J.
// A, A2, V, V2 have leading dimension kRRLd; returns (via the buffers that end
// up holding the result) pointers in *Aout / *Vout.
__device__ int jacobi_eig_sym(double* A, double* A2, double* V, double* V2, int m, double** Aout, double** Vout,
                              double* fr, double* gr, int* partner) {
  const int mp = m + (m & 1);
  const int ld = kRRLd;
  const int tid = threadIdx.x;
  __shared__ int done;
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    int r = t / ld, c = t % ld;
    V[t] = (r == c) ? 1.0 : 0.0;
    if ((r >= m || c >= m) && c < mp) A[t] = 0.0;
  }
  __syncthreads();
  const int half = mp / 2;
  // lower-triangle index list (r >= c)
  __shared__ unsigned char tri_r[kRRMax * (kRRMax + 1) / 2], tri_c[kRRMax * (kRRMax + 1) / 2];
  if (tid == 0) {
    int t = 0;
    for (int r = 0; r < mp; ++r)
      for (int c = 0; c <= r; ++c) {
        tri_r[t] = (unsigned char)r;
        tri_c[t] = (unsigned char)c;
        ++t;
      }
  }
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    if (tid == 0) done = 1;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      if (tid < half) {
        int e0 = 0, e1;
        auto ring = [&](int pos) { return ((pos + round) % (mp - 1)) + 1; };
        if (tid == 0) {
          e1 = ring(0);
        } else {
          e0 = ring(tid);
          e1 = ring(mp - 1 - tid);
        }
        const int p = min(e0, e1), q = max(e0, e1);
        const double apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300 && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
          const double tau = (aqq - app) / (2.0 * apq);
          const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
          done = 0;
        }
        // J[p][p] = c, J[q][p] = -s, J[p][q] = s, J[q][q] = c
        fr[p] = c;
        gr[p] = -s;
        partner[p] = q;
        fr[q] = c;
        gr[q] = s;
        partner[q] = p;
      }
      __syncthreads();
      for (int t = tid; t < mp * (mp + 1) / 2; t += blockDim.x) {
        const int r = tri_r[t], c = tri_c[t];
        const int rb = partner[r], cb = partner[c];
        const double v = fr[r] * (fr[c] * A[r * ld + c] + gr[c] * A[r * ld + cb]) +
                         gr[r] * (fr[c] * A[rb * ld + c] + gr[c] * A[rb * ld + cb]);
        A2[r * ld + c] = v;
        A2[c * ld + r] = v;
      }
      for (int t = tid; t < mp * mp; t += blockDim.x) {
        const int x = t / mp, r = t % mp;
        V2[x * ld + r] = V[x * ld + r] * fr[r] + V[x * ld + partner[r]] * gr[r];
      }
      __syncthreads();
      double* tA = A;
      A = A2;
      A2 = tA;
      double* tV = V;
      V = V2;
      V2 = tV;
    }
    if (done) break;
    __syncthreads();
  }
  *Aout = A;
  *Vout = V;
  return sweep + 1;
}

// Parallel cyclic Jacobi in double-word arithmetic (planes *h, *l of hi/lo
// floats, leading dimension kRRLd).  The rotation angle of a pair is chosen
// in FP32 (t = tan of the angle); c = 1 / sqrt(1 + t^2) and s = t c are then
// formed in double-word precision (one Newton step on the FP32 estimate), so
// every rotation is orthogonal to double-word accuracy and only its
// annihilation of a_pq is approximate (relative 2^-24), which the next sweep
// removes.  The two-sided update of a round is formed element-wise from the
// old matrix (Dot2 accumulations) into the second buffer.  Returns sweeps.
__device__ __forceinline__ dw dw_renorm(float s, float c) {
  dw r;
  fast_two_sum(s, c, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dw dw_lin2(dw f1, float x1h, float x1l, dw f2, float x2h, float x2l) {
  dot2 a;
  a.zero();
  a.mac(f1.hi, f1.lo, x1h, x1l);
  a.mac(f2.hi, f2.lo, x2h, x2l);
  return dw_renorm(a.s, a.c);
}

// Round-robin pairings of the parallel cyclic Jacobi (circle method), for
// mp (even) indices: round r pairs index 0 with ring(0) and ring(i) with
// ring(mp - 1 - i), ring(x) = (x + r) mod (mp - 1) + 1.  Written once per
// solve into tp/tq[r half + i], i < half = mp / 2.
__device__ void jacobi_pair_tables(int mp, unsigned char* tp, unsigned char* tq) {
  const int half = mp / 2;
  for (int t = threadIdx.x; t < (mp - 1) * half; t += blockDim.x) {
    const int round = t / half, i = t % half;
    auto ring = [&](int pos) { return ((pos + round) % (mp - 1)) + 1; };
    const int e0 = (i == 0) ? 0 : ring(i);
    const int e1 = (i == 0) ? ring(0) : ring(mp - 1 - i);
    tp[t] = (unsigned char)min(e0, e1);
    tq[t] = (unsigned char)max(e0, e1);
  }
}

// Entry (r, c), c <= r, of the lower triangle with linear index t = r (r + 1) / 2 + c.
__device__ __forceinline__ void tri_entry(int t, int& r, int& c) {
  int rr = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (rr * (rr + 1) / 2 > t) --rr;
  while ((rr + 1) * (rr + 2) / 2 <= t) ++rr;
  r = rr;
  c = t - rr * (rr + 1) / 2;
}

__device__ int jacobi_eig_dw(float* Ah, float* Al, float* A2h, float* A2l, float* Vh, float* Vl, float* V2h,
                             float* V2l, int m, float** Aoh, float** Aol, float** Voh, float** Vol, dw* fr, dw* gr,
                             int* partner) {
  const int mp = m + (m & 1);
  const int ld = kRRLd;
  const int tid = threadIdx.x;
  __shared__ int done;
  __shared__ unsigned char tp[kRRMax * kRRMax / 2], tq[kRRMax * kRRMax / 2];
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    const int r = t / ld, c = t % ld;
    Vh[t] = (r == c) ? 1.f : 0.f;
    Vl[t] = 0.f;
    if ((r >= m || c >= m) && c < mp) {
      Ah[t] = 0.f;
      Al[t] = 0.f;
    }
  }
  jacobi_pair_tables(mp, tp, tq);
  // this thread's entries (the kernel runs 1024 threads): lower-triangle entries
  // tid + u blockDim.x of A, entries tid + u blockDim.x of V
  const int ntri = mp * (mp + 1) / 2;
  int ar[3], ac[3];  // 3 x 1024 threads cover the 2080 entries of mp = 64
  for (int u = 0; u < 3; ++u) {
    const int t = tid + u * (int)blockDim.x;
    if (t < ntri)
      tri_entry(t, ar[u], ac[u]);
    else
      ar[u] = ac[u] = -1;
  }
  // rotation parameters of the current sweep (double-word), kept in the second V buffer
  float* rcs = V2h;
  float* rsn = V2l;
  __shared__ float amax_d;
  if (tid == 0) {
    float a = 0.f;
    for (int j = 0; j < m; ++j) a = fmaxf(a, fabsf(Ah[j * ld + j]));
    amax_d = a;
  }
  __syncthreads();
  // below the double-word noise of the largest diagonal entry an off-diagonal
  // entry is left (its effect on the eigenpairs is below that noise)
  const float abs_floor = 1e-14f * amax_d;
  const int half = mp / 2;
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    // a sweep runs only while some off-diagonal entry passes the rotation test
    if (tid == 0) done = 1;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (ar[u] < 0 || ar[u] == ac[u]) continue;
      const float apq = Ah[ar[u] * ld + ac[u]] + Al[ar[u] * ld + ac[u]];
      if (fabsf(apq) > abs_floor &&
          fabsf(apq) > 1e-15f * __fsqrt_rn(fabsf(Ah[ar[u] * ld + ar[u]] * Ah[ac[u] * ld + ac[u]])))
        done = 0;
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < mp - 1; ++round) {
      if (tid < half) {
        const int p = tp[round * half + tid], q = tq[round * half + tid];
        const float apq = Ah[p * ld + q] + Al[p * ld + q];
        const float app = Ah[p * ld + p], aqq = Ah[q * ld + q];
        dw c = {1.f, 0.f}, s = {0.f, 0.f};
        if (fabsf(apq) > abs_floor && fabsf(apq) > 1e-15f * __fsqrt_rn(fabsf(app * aqq))) {
          // the angle may be approximate; c and s below are orthogonal to double-word accuracy
          const float tau = __fdividef(aqq - app, 2.f * apq);
          const float t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + __fsqrt_rn(1.f + tau * tau));
          // u = 1 + t^2 exactly in double-word
          float ph, pe, uh, ue;
          two_prod(t, t, ph, pe);
          two_sum(1.f, ph, uh, ue);
          dw u = dw_renorm(uh, __fadd_rn(ue, pe));
          // c = u^{-1/2}: c0 = rsqrt(u.hi), r = 1 - u c0^2 (double-word), c = c0 + c0 r / 2
          const float c0 = rsqrtf(u.hi);
          float q1, q1e;
          two_prod(c0, c0, q1, q1e);  // c0^2 = q1 + q1e exactly
          dot2 acc;
          acc.zero();
          acc.add(1.f, 0.f);
          acc.mac(-u.hi, -u.lo, q1, q1e);
          const float r = acc.s + acc.c;
          c = dw_renorm(c0, 0.5f * c0 * r);
          // s = t c
          float sh, se;
          two_prod(t, c.hi, sh, se);
          s = dw_renorm(sh, __fmaf_rn(t, c.lo, se));
        }
        fr[p] = c;
        gr[p] = dw{-s.hi, -s.lo};
        partner[p] = q;
        fr[q] = c;
        gr[q] = s;
        partner[q] = p;
        const int ri = round * half + tid;  // for the update of V after the sweep
        rcs[2 * ri] = c.hi;
        rcs[2 * ri + 1] = c.lo;
        rsn[2 * ri] = s.hi;
        rsn[2 * ri + 1] = s.lo;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (ar[u] < 0) continue;
        const int r = ar[u], c = ac[u];
        const int rb = partner[r], cb = partner[c];
        const dw i1 = dw_lin2(fr[c], Ah[r * ld + c], Al[r * ld + c], gr[c], Ah[r * ld + cb], Al[r * ld + cb]);
        const dw i2 = dw_lin2(fr[c], Ah[rb * ld + c], Al[rb * ld + c], gr[c], Ah[rb * ld + cb], Al[rb * ld + cb]);
        const dw v = dw_lin2(fr[r], i1.hi, i1.lo, gr[r], i2.hi, i2.lo);
        A2h[r * ld + c] = v.hi;
        A2l[r * ld + c] = v.lo;
        A2h[c * ld + r] = v.hi;
        A2l[c * ld + r] = v.lo;
      }
      __syncthreads();
      float* t0 = Ah;
      Ah = A2h;
      A2h = t0;
      t0 = Al;
      Al = A2l;
      A2l = t0;
    }
    // V <- V J_1 ... J_{mp-1}: a warp per row of V, one lane per rotation of a
    // round (disjoint columns), rounds in order
    for (int x = tid >> 5; x < mp; x += (int)blockDim.x >> 5) {
      const int lane = tid & 31;
      for (int round = 0; round < mp - 1; ++round) {
        if (lane < half) {
          const int ri = round * half + lane;
          const int p = tp[ri], q = tq[ri];
          const dw c = {rcs[2 * ri], rcs[2 * ri + 1]}, sn = {rsn[2 * ri], rsn[2 * ri + 1]};
          const dw msn = {-sn.hi, -sn.lo};
          const float vph = Vh[x * ld + p], vpl = Vl[x * ld + p], vqh = Vh[x * ld + q], vql = Vl[x * ld + q];
          const dw np = dw_lin2(c, vph, vpl, msn, vqh, vql);
          const dw nq = dw_lin2(c, vqh, vql, sn, vph, vpl);
          Vh[x * ld + p] = np.hi;
          Vl[x * ld + p] = np.lo;
          Vh[x * ld + q] = nq.hi;
          Vl[x * ld + q] = nq.lo;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  *Aoh = Ah;
  *Aol = Al;
  *Voh = Vh;
  *Vol = Vl;
  return sweep;
}

// ---------------------------------------------------------------------------
// Mixed-precision Rayleigh-Ritz solve of the scaled pencil (H', G') (FP64 in
// Gd, Hd, leading dimension kRRLd):
//  phase A (FP32): G' = L L^T, B = L^{-T}, Jacobi on B^T H' B, Q = B V
//                  -- an approximate G'-orthonormal eigenbasis;
//  phase B (double-word): G2 = Q^T G' Q = I + E, S = I - E/2 + 3E^2/8
//                  ((I + E)^{-1/2} to O(E^3)), Q' = Q S, H3 = S^T Q^T H' Q S,
//                  double-word Jacobi on the nearly diagonal H3 (Y), and the
//                  Ritz basis Q' Y.
// Returns false (nothing written) when the FP32 Cholesky fails or the Gram
// matrix is too ill-conditioned for the series; the caller then takes the
// eigen-based path.  Output: theta (ascending, m values) and the basis Ritz
// vectors as FP64 in Cout (m x m, column j = j-th Ritz vector).
// ---------------------------------------------------------------------------
constexpr int kL = kRRMax * kRRLd;

// C = op(A) * op(B) for m x m double-word matrices (hi/lo planes, ld kRRLd);
// ta / tb: use the transpose.  B may be an FP32 matrix (Bl == nullptr).
__device__ void dw_gemm(int m, const float* Ah, const float* Al, bool ta, const float* Bh, const float* Bl, bool tb,
                        float* Ch, float* Cl) {
  const int ld = kRRLd;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t / m, j = t % m;
    dot2 acc;
    acc.zero();
    for (int p = 0; p < m; ++p) {
      const int ia = ta ? p * ld + i : i * ld + p;
      const int ib = tb ? j * ld + p : p * ld + j;
      acc.mac(Ah[ia], Al ? Al[ia] : 0.f, Bh[ib], Bl ? Bl[ib] : 0.f);
    }
    dw r;
    fast_two_sum(acc.s, acc.c, r.hi, r.lo);
    Ch[i * ld + j] = r.hi;
    Cl[i * ld + j] = r.lo;
  }
  __syncthreads();
}

// FP32 parallel cyclic Jacobi (same ordering as the double-word version).
__device__ int jacobi_f32(float* A, float* A2, float* V, float* V2, int m, float** Aout, float** Vout, float* fr,
                          float* gr, int* partner, float off_tol) {
  const int mp = m + (m & 1);
  const int ld = kRRLd;
  const int tid = threadIdx.x;
  __shared__ int done;
  __shared__ unsigned char tp[kRRMax * kRRMax / 2], tq[kRRMax * kRRMax / 2];
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    const int r = t / ld, c = t % ld;
    V[t] = (r == c) ? 1.f : 0.f;
    if ((r >= m || c >= m) && c < mp) A[t] = 0.f;
  }
  jacobi_pair_tables(mp, tp, tq);
  const int ntri = mp * (mp + 1) / 2;
  int ar[3], ac[3];  // 3 x 1024 threads cover the 2080 entries of mp = 64
  for (int u = 0; u < 3; ++u) {
    const int t = tid + u * (int)blockDim.x;
    if (t < ntri)
      tri_entry(t, ar[u], ac[u]);
    else
      ar[u] = ac[u] = -1;
  }
  // rotation parameters of the current sweep, kept in the second V buffer
  float* rc = V2;
  float* rs = V2 + kRRMax * kRRMax / 2;
  __syncthreads();
  const int half = mp / 2;
  __shared__ float amax_f;
  if (tid == 0) {
    float a = 0.f;
    for (int j = 0; j < m; ++j) a = fmaxf(a, fabsf(A[j * ld + j]));
    amax_f = a;
  }
  __syncthreads();
  // off-diagonal entries below the FP32 noise of the largest diagonal entry are left
  const float abs_floor = 1e-6f * amax_f;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    // a sweep runs only while some off-diagonal entry passes the rotation test
    if (tid == 0) done = 1;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (ar[u] < 0 || ar[u] == ac[u]) continue;
      const float apq = A[ar[u] * ld + ac[u]];
      if (fabsf(apq) > abs_floor &&
          fabsf(apq) > off_tol * __fsqrt_rn(fabsf(A[ar[u] * ld + ar[u]] * A[ac[u] * ld + ac[u]])))
        done = 0;
    }
    __syncthreads();
    if (done) break;
    for (int round = 0; round < mp - 1; ++round) {
      if (tid < half) {
        const int p = tp[round * half + tid], q = tq[round * half + tid];
        const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > abs_floor && fabsf(apq) > off_tol * __fsqrt_rn(fabsf(app * aqq))) {
          // approximate angle (fast intrinsics): phase B restores exact orthogonality
          const float tau = __fdividef(aqq - app, 2.f * apq);
          const float t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + __fsqrt_rn(1.f + tau * tau));
          c = rsqrtf(1.f + t * t);
          s = t * c;
        }
        fr[p] = c;
        gr[p] = -s;
        partner[p] = q;
        fr[q] = c;
        gr[q] = s;
        partner[q] = p;
        rc[round * half + tid] = c;  // for the update of V after the sweep
        rs[round * half + tid] = s;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (ar[u] < 0) continue;
        const int r = ar[u], c = ac[u];
        const int rb = partner[r], cb = partner[c];
        const float v = fr[r] * (fr[c] * A[r * ld + c] + gr[c] * A[r * ld + cb]) +
                        gr[r] * (fr[c] * A[rb * ld + c] + gr[c] * A[rb * ld + cb]);
        A2[r * ld + c] = v;
        A2[c * ld + r] = v;
      }
      __syncthreads();
      float* tA = A;
      A = A2;
      A2 = tA;
    }
    // V <- V J_1 ... J_{mp-1}: a warp per row of V, one lane per rotation of a
    // round (disjoint columns), rounds in order
    for (int x = tid >> 5; x < mp; x += (int)blockDim.x >> 5) {
      const int lane = tid & 31;
      for (int round = 0; round < mp - 1; ++round) {
        if (lane < half) {
          const int p = tp[round * half + lane], q = tq[round * half + lane];
          const float c = rc[round * half + lane], sn = rs[round * half + lane];
          const float vp = V[x * ld + p], vq = V[x * ld + q];
          V[x * ld + p] = c * vp - sn * vq;
          V[x * ld + q] = sn * vp + c * vq;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  *Aout = A;
  *Vout = V;
  return sweep;
}

// G, H: the unscaled Gram matrices (FP64, m x m, ld m); sc: column scaling.
// pool: 12 slots of kL floats.  theta: kRRMax doubles (ascending Ritz values on
// return); fr/gr/partner/ord: kRRMax entries each (fr, gr 8 bytes per entry).
// Writes C = diag(sc) Q' Y[:, lowest k] (m x k, ld k).  Returns the number of
// double-word Jacobi sweeps, or -1 (nothing written).
__device__ int rr_mixed_solve(int m, int k, const double* __restrict__ G, const double* __restrict__ H,
                              const double* sc, float* pool, double* theta, double* C, double* fr, double* gr,
                              int* partner, int* ord, double drop_tol, long long* cyc) {
  const int ld = kRRLd;
  const int tid = threadIdx.x;
  float* s[12];
  for (int i = 0; i < 12; ++i) s[i] = pool + (size_t)i * kL;
  __shared__ int ok;
  float *Gh = s[0], *Gl = s[1], *Hh = s[2], *Hl = s[3];
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    const double gs = 0.5 * (G[a * m + b] + G[b * m + a]) * sc[a] * sc[b];
    const double hs = 0.5 * (H[a * m + b] + H[b * m + a]) * sc[a] * sc[b];
    const dw g = split_f64(gs), hh = split_f64(hs);
    Gh[a * ld + b] = g.hi;
    Gl[a * ld + b] = g.lo;
    Hh[a * ld + b] = hh.hi;
    Hl[a * ld + b] = hh.lo;
  }
  if (tid == 0) ok = 1;
  __syncthreads();
  long long t0 = clock64();
  // ---- phase A (FP32)
  float *L = s[4], *Li = s[5], *T32 = s[6];
  for (int t = tid; t < m * m; t += blockDim.x) L[(t / m) * ld + (t % m)] = Gh[(t / m) * ld + (t % m)];
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const float d = L[j * ld + j];
      if (!(d > 0.f)) ok = 0;
      L[j * ld + j] = (d > 0.f) ? sqrtf(d) : 1.f;
    }
    __syncthreads();
    const float ljj = L[j * ld + j];
    for (int i = j + 1 + tid; i < m; i += blockDim.x) L[i * ld + j] /= ljj;
    __syncthreads();
    const int rem = m - j - 1;
    for (int t = tid; t < rem * rem; t += blockDim.x) {
      const int i = j + 1 + t / rem, c = j + 1 + t % rem;
      if (c <= i) L[i * ld + c] -= L[i * ld + j] * L[c * ld + j];
    }
    __syncthreads();
  }
  for (int c = tid; c < m; c += blockDim.x)
    for (int i = 0; i < m; ++i) {
      float v = 0.f;
      if (i >= c) {
        v = (i == c) ? 1.f : 0.f;
        for (int t = c; t < i; ++t) v -= L[i * ld + t] * Li[t * ld + c];
        v /= L[i * ld + i];
      }
      Li[i * ld + c] = v;
    }
  __syncthreads();
  if (tid == 0) {
    float f = 0.f, tr = 0.f;
    for (int i = 0; i < m; ++i) {
      tr += Gh[i * ld + i];
      for (int c = 0; c <= i; ++c) f += Li[i * ld + c] * Li[i * ld + c];
    }
    // 1 / ||L^{-1}||_F^2 <= lambda_min(G'): keep a margin over the drop threshold
    // (so the eigen-based basis would drop nothing) and over the conditioning
    // that the FP32 basis and the series of phase B resolve
    if (!(1.f / f > (float)(drop_tol * 10.0) * tr) || !(1.f / f > 1e-4f * tr)) ok = 0;
  }
  __syncthreads();
  if (!ok) return -1;
  long long t1 = clock64();
  float* A = s[7];
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    float v = 0.f;
    for (int c = 0; c <= b; ++c) v += Hh[a * ld + c] * Li[b * ld + c];
    T32[a * ld + b] = v;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    float v = 0.f;
    for (int c = 0; c <= a; ++c) v += Li[a * ld + c] * T32[c * ld + b];
    A[a * ld + b] = v;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    if (a < b) {
      const float v = 0.5f * (A[a * ld + b] + A[b * ld + a]);
      A[a * ld + b] = v;
      A[b * ld + a] = v;
    }
  }
  __syncthreads();
  float *Ar, *Vr;
  const int sw32 = jacobi_f32(A, s[8], s[9], s[10], m, &Ar, &Vr, reinterpret_cast<float*>(fr),
                             reinterpret_cast<float*>(gr), partner, 1e-5f);
  long long t2 = clock64();
  float* Q = s[11];
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    float v = 0.f;
    for (int c = a; c < m; ++c) v += Li[c * ld + a] * Vr[c * ld + b];
    Q[a * ld + b] = v;
  }
  __syncthreads();
  // ---- phase B (double-word)
  float *T1h = s[4], *T1l = s[5], *G2h = s[6], *G2l = s[7], *H2h = s[8], *H2l = s[9];
  dw_gemm(m, Gh, Gl, false, Q, nullptr, false, T1h, T1l);   // G' Q
  dw_gemm(m, Q, nullptr, true, T1h, T1l, false, G2h, G2l);  // Q^T G' Q
  dw_gemm(m, Hh, Hl, false, Q, nullptr, false, T1h, T1l);   // H' Q
  dw_gemm(m, Q, nullptr, true, T1h, T1l, false, H2h, H2l);  // Q^T H' Q
  for (int t = tid; t < m; t += blockDim.x) {              // E = G2 - I
    float hi, lo;
    two_sum(G2h[t * ld + t], -1.f, hi, lo);
    const dw e = dw_renorm(hi, __fadd_rn(lo, G2l[t * ld + t]));
    G2h[t * ld + t] = e.hi;
    G2l[t * ld + t] = e.lo;
  }
  __syncthreads();
  dw_gemm(m, G2h, G2l, false, G2h, G2l, false, T1h, T1l);  // E^2
  float *Sh = s[0], *Sl = s[1];
  for (int t = tid; t < m * m; t += blockDim.x) {         // S = I - E/2 + 3 E^2 / 8
    const int a = t / m, b = t % m;
    dot2 acc;
    acc.zero();
    if (a == b) acc.add(1.f, 0.f);
    acc.mac(-0.5f, 0.f, G2h[a * ld + b], G2l[a * ld + b]);
    acc.mac(0.375f, 0.f, T1h[a * ld + b], T1l[a * ld + b]);
    const dw r = dw_renorm(acc.s, acc.c);
    Sh[a * ld + b] = r.hi;
    Sl[a * ld + b] = r.lo;
  }
  __syncthreads();
  dw_gemm(m, H2h, H2l, false, Sh, Sl, false, T1h, T1l);    // H2 S
  float *H3h = s[2], *H3l = s[3];
  dw_gemm(m, Sh, Sl, true, T1h, T1l, false, H3h, H3l);     // S^T H2 S
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    if (a < b) {
      dot2 acc;
      acc.zero();
      acc.add(H3h[a * ld + b], H3l[a * ld + b]);
      acc.add(H3h[b * ld + a], H3l[b * ld + a]);
      const dw r = dw_renorm(0.5f * acc.s, 0.5f * acc.c);
      H3h[a * ld + b] = r.hi;
      H3l[a * ld + b] = r.lo;
      H3h[b * ld + a] = r.hi;
      H3l[b * ld + a] = r.lo;
    }
  }
  __syncthreads();
  float *Qph = s[6], *Qpl = s[7];
  dw_gemm(m, Q, nullptr, false, Sh, Sl, false, Qph, Qpl);  // Q' = Q S
  long long t3 = clock64();
  float *Arh, *Arl, *Vrh, *Vrl;
  const int sw = jacobi_eig_dw(H3h, H3l, s[8], s[9], s[4], s[5], s[0], s[1], m, &Arh, &Arl, &Vrh, &Vrl,
                               reinterpret_cast<dw*>(fr), reinterpret_cast<dw*>(gr), partner);
  __syncthreads();
  long long t4 = clock64();
  for (int j = tid; j < m; j += blockDim.x) theta[j] = dw_to_f64(Arh[j * ld + j], Arl[j * ld + j]);
  __syncthreads();
  for (int j = tid; j < m; j += blockDim.x) {
    const double tj = theta[j];
    int rank = 0;
    for (int i2 = 0; i2 < m; ++i2) {
      rank += order_before(theta[i2], i2, tj, j) ? 1 : 0;
    }
    ord[rank] = j;
  }
  __syncthreads();
  for (int t = tid; t < m * k; t += blockDim.x) {
    const int a = t / k, c = t % k;
    const int j = ord[c];
    dot2 acc;
    acc.zero();
    for (int p = 0; p < m; ++p) acc.mac(Qph[a * ld + p], Qpl[a * ld + p], Vrh[p * ld + j], Vrl[p * ld + j]);
    C[a * k + c] = sc[a] * acc.value();
  }
  __syncthreads();
  if (tid == 0 && cyc) {
    const long long t5 = clock64();
    cyc[0] = t1 - t0;
    cyc[1] = t2 - t1;
    cyc[2] = t3 - t2;
    cyc[3] = t4 - t3;
    cyc[4] = t5 - t4;
    cyc[5] = sw32 * 1000;
  }
  return sw;
}

// Rayleigh-Ritz (Eq. (3.6)) with a Cholesky orthonormalisation of the scaled
// Gram matrix G' = L L^T.  When the lower bound 1 / ||L^{-1}||_F^2 of the
// smallest eigenvalue of G' exceeds drop_tol * trace(G') >= drop_tol * lambda_max,
// the eigen-based basis of k_rayleigh_ritz would keep every direction, so both
// produce the Ritz pairs of the same space; the reduced matrix
// H'' = L^{-1} H' L^{-T} is diagonalised by one symmetric Jacobi.  Otherwise the
// eigen-based path with dropping runs.
__global__ void k_rayleigh_ritz_chol(int m, int k, const double* __restrict__ G, const double* __restrict__ H,
                                     double drop_tol, const double* __restrict__ lam_old, double* C,
                                     double* lam_new, double* hist, int hist_rows, int row_host,
                                     const int32_t* d_row, int stop_rule, double tol, DevStatus* st, int dword) {
  const int row = d_row ? *d_row + 1 : row_host;
  double* hist_row = (hist && row >= 0 && row < hist_rows) ? hist + (size_t)row * k : nullptr;
  extern __shared__ double rr[];
  const int ld = kRRLd;
  const int LL = ld * ld;
  double* B0 = rr;
  double* B1 = B0 + LL;
  double* B2 = B1 + LL;
  double* B3 = B2 + LL;
  double* B4 = B3 + LL;
  double* sc = B4 + 2 * LL;  // B5 (one more slot) belongs to the mixed-precision pool
  double* fr = sc + ld;
  double* gr = fr + ld;
  int* partner = reinterpret_cast<int*>(gr + ld);
  int* ord = partner + ld;
  __shared__ int ok;
  __shared__ double crit_lhs, crit_rhs;
  const int tid = threadIdx.x;
  long long tcl[8];
  tcl[0] = clock64();
  for (int j = tid; j < m; j += blockDim.x) {
    const double g = G[j * m + j];
    // the FP64 path keeps the first k columns (the iterate, M-orthonormal) as they
    // are; the mixed path scales every column, its iterate block being the last
    sc[j] = (j < k && !dword) ? 1.0 : (g > 0 ? 1.0 / sqrt(g) : 0.0);
  }
  if (tid == 0) ok = 1;
  __syncthreads();
  if (dword) {
    double* theta = sc + ld;  // fr and gr are workspace of the solve
    __shared__ double th_s[kRRMax];
    const int sw = rr_mixed_solve(m, k, G, H, sc, reinterpret_cast<float*>(rr), th_s, C, fr, gr, partner, ord,
                                  drop_tol, st->rr_cycles);
    (void)theta;
    if (sw >= 0) {
      if (tid == 0) {
        double dl = 0;
        for (int c = 0; c < k; ++c) {
          const double th = th_s[ord[c]];
          dl += fabs(th - lam_old[c]);
          lam_new[c] = th;
          if (hist_row) hist_row[c] = th;
        }
        st->sum_dl = dl;
        st->kept = m;
        st->sweeps = sw;
        if (stop_rule == BPJD_STOP_DLAMBDA) st->converged = (dl < tol) ? 1 : 0;
        st->rr_cycles[6] = clock64() - tcl[0];  // the whole kernel body
      }
      return;
    }
    // ill-conditioned: eigen-based orthonormalisation with dropping
    rayleigh_ritz_eig(m, k, G, H, drop_tol, lam_old, C, lam_new, hist_row, stop_rule, tol, st, rr, dword);
    return;
  }
  // B0 = G' (becomes L), B1 = H'
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    B0[a * ld + b] = 0.5 * (G[a * m + b] + G[b * m + a]) * sc[a] * sc[b];
    B1[a * ld + b] = 0.5 * (H[a * m + b] + H[b * m + a]) * sc[a] * sc[b];
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0;
    for (int j = 0; j < m; ++j) tr += B0[j * ld + j];
    crit_rhs = drop_tol * tr;
  }
  tcl[1] = clock64();
  // right-looking Cholesky in place (lower triangle)
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      const double d = B0[j * ld + j];
      if (!(d > 0.0)) ok = 0;
      B0[j * ld + j] = (d > 0.0) ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double ljj = B0[j * ld + j];
    for (int i = j + 1 + tid; i < m; i += blockDim.x) B0[i * ld + j] /= ljj;
    __syncthreads();
    const int rem = m - j - 1;
    for (int t = tid; t < rem * rem; t += blockDim.x) {
      const int i = j + 1 + t / rem, c = j + 1 + t % rem;
      if (c <= i) B0[i * ld + c] -= B0[i * ld + j] * B0[c * ld + j];
    }
    __syncthreads();
  }
  tcl[2] = clock64();
  // B2 = L^{-1}: row i of L^{-1} from rows < i, all columns of a row in parallel;
  // the dot products run as double-word Dot2 sums (FP64 dependency chains are
  // long-latency on this GPU)
  {
    double* dinv = B3;  // reciprocal diagonal of L
    for (int i = tid; i < m; i += blockDim.x) dinv[i] = 1.0 / B0[i * ld + i];
    __syncthreads();
    for (int i = 0; i < m; ++i) {
      for (int c = tid; c < m; c += blockDim.x) {
        double v = 0.0;
        if (c == i) {
          v = dinv[i];
        } else if (c < i) {
          dot2 acc;
          acc.zero();
          for (int t = c; t < i; ++t) {
            const dw l = split_f64(B0[i * ld + t]);
            const dw x = split_f64(B2[t * ld + c]);
            acc.mac(l.hi, l.lo, x.hi, x.lo);
          }
          v = -acc.value() * dinv[i];
        }
        B2[i * ld + c] = v;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    double f = 0;
    for (int i = 0; i < m; ++i)
      for (int c = 0; c <= i; ++c) f += B2[i * ld + c] * B2[i * ld + c];
    crit_lhs = 1.0 / f;
    if (!(crit_lhs > crit_rhs)) ok = 0;
  }
  __syncthreads();
  if (!ok) {
    // ill-conditioned basis: eigen-based orthonormalisation with dropping
    rayleigh_ritz_eig(m, k, G, H, drop_tol, lam_old, C, lam_new, hist_row, stop_rule, tol, st, rr, dword);
    return;
  }
  tcl[3] = clock64();
  // B3 = H' L^{-T};  B4 = L^{-1} B3  (= H'')
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    double s = 0;
    for (int c = 0; c <= b; ++c) s = fma(B1[a * ld + c], B2[b * ld + c], s);
    B3[a * ld + b] = s;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    if (a < b) continue;
    double s = 0;
    for (int c = 0; c <= a; ++c) s = fma(B2[a * ld + c], B3[c * ld + b], s);
    B4[a * ld + b] = s;
  }
  __syncthreads();
  for (int t = tid; t < m * m; t += blockDim.x) {
    const int a = t / m, b = t % m;
    if (a < b) B4[a * ld + b] = B4[b * ld + a];
  }
  __syncthreads();
  tcl[4] = clock64();
  int nsweeps = 0;
  const double* Vd = nullptr;  // FP64 eigenvectors (native path)
  float *Vrh = nullptr, *Vrl = nullptr;
  if (!dword) {
    double* Ar;
    double* Vr;
    nsweeps = jacobi_eig_sym(B4, B0, B1, B3, m, &Ar, &Vr, fr, gr, partner);
    for (int j = tid; j < m; j += blockDim.x) fr[j] = Ar[j * ld + j];
    Vd = Vr;
  } else {
    // double-word Jacobi: A planes in B0, A2 in B1, V in B3, V2 in B4 (after
    // H'' has been split out of B4); B2 = L^{-1} is kept
    float* Ah = reinterpret_cast<float*>(B0);
    float* Al = Ah + LL;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int a = t / m, b = t % m;
      const dw sp = split_f64(B4[a * ld + b]);
      Ah[a * ld + b] = sp.hi;
      Al[a * ld + b] = sp.lo;
    }
    __syncthreads();
    float *Arh, *Arl;
    nsweeps = jacobi_eig_dw(Ah, Al, reinterpret_cast<float*>(B1), reinterpret_cast<float*>(B1) + LL,
                            reinterpret_cast<float*>(B3), reinterpret_cast<float*>(B3) + LL,
                            reinterpret_cast<float*>(B4), reinterpret_cast<float*>(B4) + LL, m, &Arh, &Arl, &Vrh,
                            &Vrl, reinterpret_cast<dw*>(fr), reinterpret_cast<dw*>(gr), partner);
    __syncthreads();
    for (int j = tid; j < m; j += blockDim.x) fr[j] = dw_to_f64(Arh[j * ld + j], Arl[j * ld + j]);
  }
  tcl[5] = clock64();
  __syncthreads();
  // ascending order of the eigenvalues (ties by index), one rank per thread
  for (int j = tid; j < m; j += blockDim.x) {
    const double fj = fr[j];
    int rank = 0;
    for (int i2 = 0; i2 < m; ++i2) {
      rank += order_before(fr[i2], i2, fj, j) ? 1 : 0;
    }
    ord[rank] = j;
  }
  __syncthreads();
  auto yv = [&](int b, int j) -> double {
    return Vd ? Vd[b * ld + j] : dw_to_f64(Vrh[b * ld + j], Vrl[b * ld + j]);
  };
  // C = diag(sc) L^{-T} Y[:, 0..k)
  for (int t = tid; t < m * k; t += blockDim.x) {
    const int a = t / k, c = t % k;
    const int j = ord[c];
    double s = 0;
    for (int b = a; b < m; ++b) s = fma(B2[b * ld + a], yv(b, j), s);
    C[a * k + c] = sc[a] * s;
  }
  __syncthreads();
  if (tid == 0) {
    double dl = 0;
    for (int c = 0; c < k; ++c) {
      const double th = fr[ord[c]];
      dl += fabs(th - lam_old[c]);
      lam_new[c] = th;
      if (hist_row) hist_row[c] = th;
    }
    st->sum_dl = dl;
    st->kept = m;
    st->sweeps = nsweeps;
    tcl[6] = clock64();
    for (int q = 0; q < 6; ++q) st->rr_cycles[q] = tcl[q + 1] - tcl[q];
    if (stop_rule == BPJD_STOP_DLAMBDA) st->converged = (dl < tol) ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz of the mixed-precision path (Eq. (3.6)), refined form.
//
// Input: the Gram matrices G = W^T M W and H = W^T K W (FP64, m x m) of the
// search space W; every column of W is scaled to unit M-norm.  Output: the k
// lowest Ritz values and C (m x k) with W C the b-orthonormal Ritz vectors.
//
//  phase A (FP32): G' = L L^T (Cholesky), A = L^{-1} H' L^{-T}, parallel cyclic
//    Jacobi on A to FP32 accuracy (V), Q = L^{-T} V: an approximate
//    G'-orthonormal eigenbasis of the whole pencil;
//  phase B (double-word): refinement of the whole basis by first-order
//    corrections (Ogita & Aishima, "Iterative refinement for symmetric
//    eigenvalue decomposition", Japan J. Indust. Appl. Math. 35 (2018),
//    here for the definite pencil (H', G')): with R = Q^T G' Q and
//    S = Q^T H' Q, theta_i = s_ii / r_ii and Q <- Q (I + E),
//      E_ii = (1 - r_ii) / 2,
//      E_ij = (s_ij - theta_j r_ij) / (theta_j - theta_i)  (i != j),
//    which makes Q^T G' Q = I and Q^T H' Q diagonal to first order; the error
//    squares from one step to the next.  A pair whose correction would not be
//    small (|theta_j - theta_i| <= 100 |s_ij - theta_j r_ij|: nearly equal
//    Ritz values) is only made G'-orthogonal (E_ij = -r_ij / 2); after the last
//    step such pairs, closed under transitivity, form clusters whose blocks of
//    Q^T H' Q are diagonalised by a small FP64 Jacobi.
// Steps run until the largest correction is below 1e-9 (at most four): the
// Ritz values are the Rayleigh quotients of the last step, accurate to the
// square of that.  Shared-memory slots of mp x ld floats (mp = m rounded up to
// even, ld = mp + 1) hold every matrix; m <= kRFMax.
// Returns false (nothing written) when phase A fails (Cholesky breakdown, or a
// Gram matrix too ill-conditioned for an FP32 basis): the caller then takes
// the eigen-based path with dropping.
// ---------------------------------------------------------------------------
constexpr int kRFThreads = 512;
constexpr int kRFMax = 60;
constexpr int kRFSlots = 14;

struct RFRot {
  float c, g;
  int partner, pad;
};

__device__ __forceinline__ size_t rf_slot_floats(int m) {
  const int mp = m + (m & 1);
  return (((size_t)mp * (mp + 1)) + 3) & ~(size_t)3;
}

// Entry (r, c) of J^T A J for the disjoint rotations of one round (rot: c, g and
// partner per index): the same arithmetic everywhere it is evaluated, so that
// the pivots recomputed for the next round equal the stored entries bit for bit.
__device__ __forceinline__ float rf_rotated(const float* A, int ld, const RFRot* rot, int r, int c) {
  const RFRot rr = rot[r], rc = rot[c];
  const float x = __fmaf_rn(rc.c, A[r * ld + c], __fmul_rn(rc.g, A[r * ld + rc.partner]));
  const float y = __fmaf_rn(rc.c, A[rr.partner * ld + c], __fmul_rn(rc.g, A[rr.partner * ld + rc.partner]));
  return __fmaf_rn(rr.c, x, __fmul_rn(rr.g, y));
}

// The same entry from the four entries of A at rows {r, partner(r)} x columns
// {c, partner(c)} held in registers (v_rc = a_{r,c}, v_rp = a_{r,pc}, v_pc = a_{pr,c},
// v_pp = a_{pr,pc}) and the rotations (cr, gr) of r and (cc, gc) of c.
__device__ __forceinline__ float rf_rot4(float cr, float gr, float cc, float gc, float v_rc, float v_rp, float v_pc,
                                         float v_pp) {
  const float x = __fmaf_rn(cc, v_rc, __fmul_rn(gc, v_rp));
  const float y = __fmaf_rn(cc, v_pc, __fmul_rn(gc, v_pp));
  return __fmaf_rn(cr, x, __fmul_rn(gr, y));
}

// Rotation annihilating a_pq (FP32; the angle need not be exact, phase B
// refines the basis).  Returns false for an identity rotation.
__device__ __forceinline__ bool rf_rotation(float app, float aqq, float apq, float floor_abs, float off_tol,
                                            float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (!(fabsf(apq) > floor_abs && fabsf(apq) > off_tol * sqrtf(fabsf(app * aqq)))) return false;
  const float tau = __fdividef(aqq - app, 2.f * apq);
  const float t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + sqrtf(__fmaf_rn(tau, tau, 1.f)));
  c = rsqrtf(__fmaf_rn(t, t, 1.f));
  s = t * c;
  return true;
}

__device__ __forceinline__ void rf_set_pair(RFRot* rot, int p, int q, float c, float s) {
  rot[p] = RFRot{c, -s, q, 0};
  rot[q] = RFRot{c, s, p, 0};
}

// dword helpers of phase B
__device__ __forceinline__ dw dw_from_sum(const dot2& a) {
  dw r;
  fast_two_sum(a.s, a.c, r.hi, r.lo);
  return r;
}
// (ah + al) - x (b_h + b_l), x a float: double-word
__device__ __forceinline__ dw dw_sub_scaled(float ah, float al, float xh, float xl, float bh, float bl) {
  dot2 acc;
  acc.zero();
  acc.add(ah, al);
  acc.mac(-xh, -xl, bh, bl);
  return dw_from_sum(acc);
}

__device__ bool rr_refined_solve(int m, int k, const double* __restrict__ G, const double* __restrict__ H,
                                 const double* __restrict__ sc, float* pool, double drop_tol, double* C,
                                 double* theta_out, int* ord, DevStatus* st, int* sweeps_out) {
  const int tid = threadIdx.x;
  const int mp = m + (m & 1);
  const int ld = mp + 1;
  const size_t SL = rf_slot_floats(m);
  float* slot[kRFSlots];
  for (int i = 0; i < kRFSlots; ++i) slot[i] = pool + (size_t)i * SL;
  float *Gh = slot[0], *Gl = slot[1], *Hh = slot[2], *Hl = slot[3];
  float *Qh = slot[4], *Ql = slot[5];
  __shared__ RFRot rot[2][kRFMax];
  __shared__ unsigned char tp[kRFMax * kRFMax / 2], tq[kRFMax * kRFMax / 2];
  __shared__ float colf[kRFMax];
  __shared__ float emax_s;
  __shared__ double th_s[kRFMax];
  __shared__ float thh[kRFMax], thl[kRFMax];
  __shared__ unsigned long long cmask[kRFMax];
  __shared__ int fail_s, anyclus_s;
  long long t0 = clock64();
  // scaled, symmetrised pencil in double-word planes; pad row / column zero
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    const int a = t / ld, b = t % ld;
    float gh = 0.f, gl = 0.f, hh = 0.f, hl = 0.f;
    if (a < m && b < m) {
      const double gs = 0.5 * (G[a * m + b] + G[b * m + a]) * sc[a] * sc[b];
      const double hs = 0.5 * (H[a * m + b] + H[b * m + a]) * sc[a] * sc[b];
      const dw g = split_f64(gs), h = split_f64(hs);
      gh = g.hi;
      gl = g.lo;
      hh = h.hi;
      hl = h.lo;
    } else if (a == b && a < mp) {
      gh = 1.f;  // the pad index is a decoupled unit direction
    }
    Gh[t] = gh;
    Gl[t] = gl;
    Hh[t] = hh;
    Hl[t] = hl;
  }
  if (tid == 0) {
    fail_s = 0;
    anyclus_s = 0;
  }
  __syncthreads();
  // ---- phase A: FP32 Cholesky G' = L L^T (column j of L to slot 6, the
  // trailing matrix updated in slot 7)
  float *L = slot[6], *Wk = slot[7];
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    Wk[t] = Gh[t];
    L[t] = 0.f;
  }
  __syncthreads();
  bool fail = false;
  for (int j = 0; j < mp; ++j) {
    const float d = Wk[j * ld + j];
    if (!(d > 0.f)) fail = true;
    const float inv = rsqrtf(d > 0.f ? d : 1.f);
    const int rem = mp - j;
    for (int t = tid; t < rem; t += blockDim.x) L[(j + t) * ld + j] = Wk[(j + t) * ld + j] * inv;
    const int tr = rem - 1;
    for (int t = tid; t < tr * tr; t += blockDim.x) {
      const int i = j + 1 + t / tr, c = j + 1 + t % tr;
      if (c <= i) Wk[i * ld + c] = __fmaf_rn(-(Wk[i * ld + j] * inv), Wk[c * ld + j] * inv, Wk[i * ld + c]);
    }
    __syncthreads();
  }
  if (__syncthreads_or(fail ? 1 : 0)) return false;
  const long long tchol = clock64();
  // Li = L^{-1} (slot 7), one column per thread; condition check as in the
  // eigen-based path: 1 / ||L^{-1}||_F^2 <= lambda_min(G')
  float* Li = slot[7];
  for (int t = tid; t < mp * ld; t += blockDim.x) Li[t] = 0.f;
  __syncthreads();
  for (int c = tid; c < mp; c += blockDim.x) {
    float f = 0.f;
    for (int i = c; i < mp; ++i) {
      float s0 = (i == c) ? 1.f : 0.f, s1 = 0.f;
      int t = c;
      for (; t + 1 < i; t += 2) {
        s0 = __fmaf_rn(-L[i * ld + t], Li[t * ld + c], s0);
        s1 = __fmaf_rn(-L[i * ld + t + 1], Li[(t + 1) * ld + c], s1);
      }
      if (t < i) s0 = __fmaf_rn(-L[i * ld + t], Li[t * ld + c], s0);
      const float v = (s0 + s1) / L[i * ld + i];
      Li[i * ld + c] = v;
      f = __fmaf_rn(v, v, f);
    }
    colf[c] = f;
  }
  __syncthreads();
  if (tid == 0) {
    float f = 0.f, tr = 0.f;
    for (int i = 0; i < m; ++i) {
      f += colf[i];
      tr += Gh[i * ld + i];
    }
    if (!(1.f / f > (float)(drop_tol * 10.0) * tr) || !(1.f / f > 1e-4f * tr)) fail_s = 1;
  }
  __syncthreads();
  if (fail_s) return false;
  // A = Li H' Li^T (slot 8), via T = H' Li^T (slot 9)
  float *A = slot[8], *A2 = slot[9], *V = slot[10], *V2 = slot[11];
  for (int t = tid; t < mp * mp; t += blockDim.x) {
    const int a = t / mp, b = t % mp;
    float s0 = 0.f, s1 = 0.f;
    int c = 0;
    for (; c + 1 <= b; c += 2) {
      s0 = __fmaf_rn(Hh[a * ld + c], Li[b * ld + c], s0);
      s1 = __fmaf_rn(Hh[a * ld + c + 1], Li[b * ld + c + 1], s1);
    }
    if (c <= b) s0 = __fmaf_rn(Hh[a * ld + c], Li[b * ld + c], s0);
    A2[a * ld + b] = s0 + s1;
  }
  __syncthreads();
  for (int t = tid; t < mp * mp; t += blockDim.x) {
    const int a = t / mp, b = t % mp;
    if (a < b) continue;
    float s0 = 0.f, s1 = 0.f;
    int c = 0;
    for (; c + 1 <= a; c += 2) {
      s0 = __fmaf_rn(Li[a * ld + c], A2[c * ld + b], s0);
      s1 = __fmaf_rn(Li[a * ld + c + 1], A2[(c + 1) * ld + b], s1);
    }
    if (c <= a) s0 = __fmaf_rn(Li[a * ld + c], A2[c * ld + b], s0);
    const float v = (a < m && b < m) ? s0 + s1 : ((a == b) ? 0.f : 0.f);
    A[a * ld + b] = v;
    A[b * ld + a] = v;
  }
  for (int t = tid; t < mp * ld; t += blockDim.x) V[t] = ((t / ld) == (t % ld)) ? 1.f : 0.f;
  jacobi_pair_tables(mp, tp, tq);
  __syncthreads();
  long long t1 = clock64();
  // ---- FP32 parallel cyclic Jacobi, one barrier per round.  Warp 0 forms the
  // rotations of the next round (its pivots evaluated from the current matrix
  // and the current rotations) while warps 1.. apply the current round to A and
  // V; a round whose rotations are all identities changes nothing and is skipped.
  const int half = mp / 2, rounds = mp - 1;
  const int ntri = mp * (mp + 1) / 2;
  float amax = 0.f;
  for (int j = 0; j < m; ++j) amax = fmaxf(amax, fabsf(A[j * ld + j]));
  const float floor_abs = 1e-7f * amax, off_tol = 1e-6f;
  const int wid = tid >> 5, lane = tid & 31;
  const int ut = tid - 32, nut = (int)blockDim.x - 32;  // update threads (warps 1..)
  // Update items of warps 1.. for a round whose rotations pair (p_a, q_a), a < half:
  //  * the 2 x 2 block of A at rows {p_a, q_a} x columns {p_b, q_b}, a >= b (code a << 8 | b):
  //    its four entries are the only inputs of its four rotated entries, so each entry of A
  //    is read once per round;
  //  * rows x0 .. x0 + 3 of V at columns {p_b, q_b} (code 1 << 16 | x0 << 8 | b).
  const int nblk = half * (half + 1) / 2, nvg = ((mp + 3) / 4) * half;
  constexpr int kNI = ((kRFMax / 2) * (kRFMax / 2 + 1) / 2 + (kRFMax / 4) * (kRFMax / 2) + (kRFThreads - 32) - 1) /
                      (kRFThreads - 32);
  int item[kNI];
#pragma unroll
  for (int u = 0; u < kNI; ++u) {
    const int t = ut + u * nut;
    int code = -1;
    if (ut >= 0 && t < nblk) {
      int a = 0, b = 0;
      tri_entry(t, a, b);
      code = (a << 8) | b;
    } else if (ut >= 0 && t < nblk + nvg) {
      const int w = t - nblk;
      code = (1 << 16) | ((4 * (w / half)) << 8) | (w % half);
    }
    item[u] = code;
  }
  __shared__ int rany[2];
  int sweeps = 0;
  for (; sweeps < 30; ++sweeps) {
    // any off-diagonal entry above the thresholds?  (warp 0: rotations of round 0)
    int need = 0;
    for (int t = tid; t < ntri; t += blockDim.x) {
      int r = 0, c = 0;
      tri_entry(t, r, c);
      if (r != c) {
        float cc, ss;
        need |= rf_rotation(A[r * ld + r], A[c * ld + c], A[r * ld + c], floor_abs, off_tol, cc, ss) ? 1 : 0;
      }
    }
    if (wid == 0) {
      bool rot_on = false;
      if (lane < half) {
        const int p = tp[lane], q = tq[lane];
        float cc, ss;
        rot_on = rf_rotation(A[p * ld + p], A[q * ld + q], A[p * ld + q], floor_abs, off_tol, cc, ss);
        rf_set_pair(rot[0], p, q, cc, ss);
      }
      const bool any = __any_sync(0xffffffffu, rot_on);
      if (lane == 0) rany[0] = any ? 1 : 0;
    }
    if (!__syncthreads_or(need)) break;
    for (int round = 0; round < rounds; ++round) {
      const RFRot* rc = rot[round & 1];
      const int act = rany[round & 1];
      if (wid == 0) {
        if (round + 1 < rounds) {
          bool rot_on = false;
          if (lane < half) {
            const int ri = (round + 1) * half + lane;
            const int p = tp[ri], q = tq[ri];
            // with identity rotations rf_rotated returns the stored entries unchanged
            const float app = rf_rotated(A, ld, rc, p, p), aqq = rf_rotated(A, ld, rc, q, q);
            const float apq = rf_rotated(A, ld, rc, q, p);  // stored lower entry (q > p)
            float cc, ss;
            rot_on = rf_rotation(app, aqq, apq, floor_abs, off_tol, cc, ss);
            rf_set_pair(rot[(round + 1) & 1], p, q, cc, ss);
          }
          const bool any = __any_sync(0xffffffffu, rot_on);
          if (lane == 0) rany[(round + 1) & 1] = any ? 1 : 0;
        }
      } else if (act) {
        const int ri = round * half;
#pragma unroll
        for (int u = 0; u < kNI; ++u) {
          const int it = item[u];
          if (it < 0) continue;
          if (it >> 16) {
            // V <- V J on four rows, columns p, q of pair b (rot[q].g = -rot[p].g)
            const int x0 = (it >> 8) & 255;
            const RFRot rp = rc[tp[ri + (it & 255)]];
            const int pcol = tp[ri + (it & 255)], qcol = rp.partner;
            const float gq = -rp.g;
            const int x1 = min(x0 + 4, mp);
            for (int x = x0; x < x1; ++x) {
              const float vp = V[x * ld + pcol], vq = V[x * ld + qcol];
              V2[x * ld + pcol] = __fmaf_rn(vp, rp.c, __fmul_rn(vq, rp.g));
              V2[x * ld + qcol] = __fmaf_rn(vq, rp.c, __fmul_rn(vp, gq));
            }
          } else {
            const int a = it >> 8, b = it & 255;
            const int P1[2] = {tp[ri + a], tq[ri + a]}, P2[2] = {tp[ri + b], tq[ri + b]};
            const RFRot r1 = rc[P1[0]], r2 = rc[P2[0]];
            const float g1[2] = {r1.g, -r1.g}, g2[2] = {r2.g, -r2.g};
            float w[2][2];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
              for (int j = 0; j < 2; ++j) w[i][j] = A[P1[i] * ld + P2[j]];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                if (a == b && i < j) continue;  // the diagonal block's upper entry is its lower one
                const int R = P1[i], Cc = P2[j];
                // the entry is formed in the orientation row >= column, as rf_rotated does
                const float v = (R >= Cc)
                                    ? rf_rot4(r1.c, g1[i], r2.c, g2[j], w[i][j], w[i][1 - j], w[1 - i][j], w[1 - i][1 - j])
                                    : rf_rot4(r2.c, g2[j], r1.c, g1[i], w[i][j], w[1 - i][j], w[i][1 - j], w[1 - i][1 - j]);
                A2[R * ld + Cc] = v;
                A2[Cc * ld + R] = v;
              }
          }
        }
      }
      __syncthreads();
      if (act) {
        float* tA = A;
        A = A2;
        A2 = tA;
        float* tV = V;
        V = V2;
        V2 = tV;
      }
    }
  }
  *sweeps_out = sweeps;
  long long t2 = clock64();
  // Q = Li^T V (FP32), lo planes zero
  for (int t = tid; t < mp * ld; t += blockDim.x) {
    const int a = t / ld, b = t % ld;
    float v = 0.f;
    if (a < mp && b < mp) {
      float s0 = 0.f, s1 = 0.f;
      int c = a;
      for (; c + 1 < mp; c += 2) {
        s0 = __fmaf_rn(Li[c * ld + a], V[c * ld + b], s0);
        s1 = __fmaf_rn(Li[(c + 1) * ld + a], V[(c + 1) * ld + b], s1);
      }
      if (c < mp) s0 = __fmaf_rn(Li[c * ld + a], V[c * ld + b], s0);
      v = s0 + s1;
    }
    Qh[t] = v;
    Ql[t] = 0.f;
  }
  __syncthreads();
  long long t3 = clock64();
  // ---- phase B: refinement in double-word arithmetic
  float *GQh = slot[6], *GQl = slot[7], *HQh = slot[8], *HQl = slot[9];
  float *Rh = slot[10], *Rl = slot[11], *Sh = slot[12], *Sl = slot[13];
  float* E = slot[8];                  // after R and S are formed
  float *Q2h = slot[6], *Q2l = slot[7];  // updated basis
  int step = 0;
  bool last = false;
  for (; !last; ++step) {
    // GQ = G' Q, HQ = H' Q, a 2 x 2 tile of outputs per thread (each output sums
    // over c in ascending order, as one output at a time would); with m odd the
    // tiles reach the pad row / column, whose outputs are not stored
    const int hm = (m + 1) / 2;
    for (int t = tid; t < hm * hm; t += blockDim.x) {
      const int a0 = 2 * (t / hm), b0 = 2 * (t % hm);
      dot2 g[2][2], h[2][2];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          g[x][y].zero();
          h[x][y].zero();
        }
      for (int c = 0; c < m; ++c) {
        const float qh[2] = {Qh[c * ld + b0], Qh[c * ld + b0 + 1]}, ql[2] = {Ql[c * ld + b0], Ql[c * ld + b0 + 1]};
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const float gh = Gh[(a0 + x) * ld + c], gl = Gl[(a0 + x) * ld + c];
          const float hh = Hh[(a0 + x) * ld + c], hl = Hl[(a0 + x) * ld + c];
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            g[x][y].mac(gh, gl, qh[y], ql[y]);
            h[x][y].mac(hh, hl, qh[y], ql[y]);
          }
        }
      }
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          const int a = a0 + x, b = b0 + y;
          if (a >= m || b >= m) continue;
          const dw gv = dw_from_sum(g[x][y]), hv = dw_from_sum(h[x][y]);
          GQh[a * ld + b] = gv.hi;
          GQl[a * ld + b] = gv.lo;
          HQh[a * ld + b] = hv.hi;
          HQl[a * ld + b] = hv.lo;
        }
    }
    __syncthreads();
    // R = Q^T GQ, S = Q^T HQ on the tiles on or above the diagonal (entries a <= b
    // formed, both triangles written)
    for (int t = tid; t < hm * hm; t += blockDim.x) {
      const int ta = t / hm, tb = t % hm;
      if (ta > tb) continue;
      const int a0 = 2 * ta, b0 = 2 * tb;
      dot2 r[2][2], sacc[2][2];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          r[x][y].zero();
          sacc[x][y].zero();
        }
      for (int c = 0; c < m; ++c) {
        const float qh[2] = {Qh[c * ld + a0], Qh[c * ld + a0 + 1]}, ql[2] = {Ql[c * ld + a0], Ql[c * ld + a0 + 1]};
        const float gh[2] = {GQh[c * ld + b0], GQh[c * ld + b0 + 1]}, gl[2] = {GQl[c * ld + b0], GQl[c * ld + b0 + 1]};
        const float hh[2] = {HQh[c * ld + b0], HQh[c * ld + b0 + 1]}, hl[2] = {HQl[c * ld + b0], HQl[c * ld + b0 + 1]};
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            r[x][y].mac(qh[x], ql[x], gh[y], gl[y]);
            sacc[x][y].mac(qh[x], ql[x], hh[y], hl[y]);
          }
      }
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          const int a = a0 + x, b = b0 + y;
          if (a > b || b >= m) continue;
          const dw rv = dw_from_sum(r[x][y]), sv = dw_from_sum(sacc[x][y]);
          Rh[a * ld + b] = rv.hi;
          Rl[a * ld + b] = rv.lo;
          Sh[a * ld + b] = sv.hi;
          Sl[a * ld + b] = sv.lo;
          Rh[b * ld + a] = rv.hi;
          Rl[b * ld + a] = rv.lo;
          Sh[b * ld + a] = sv.hi;
          Sl[b * ld + a] = sv.lo;
        }
    }
    if (tid == 0) {
      emax_s = 0.f;
      anyclus_s = 0;
    }
    __syncthreads();
    // Rayleigh quotients
    for (int i = tid; i < m; i += blockDim.x) {
      const double r = dw_to_f64(Rh[i * ld + i], Rl[i * ld + i]);
      const double s = dw_to_f64(Sh[i * ld + i], Sl[i * ld + i]);
      if (step == 0 && !(r > 0.5 && r < 1.5)) fail_s = 1;  // the FP32 basis is not usable
      th_s[i] = s / r;
      const dw ts = split_f64(th_s[i]);
      thh[i] = ts.hi;
      thl[i] = ts.lo;
      cmask[i] = 0ull;
    }
    __syncthreads();
    if (fail_s) return false;
    // E (FP32 is enough for a correction), largest off-cluster entry, cluster pairs
    float emax = 0.f;
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int i = t / m, j = t % m;
      float e;
      if (i == j) {
        float hi, lo;
        two_sum(1.f, -Rh[i * ld + i], hi, lo);
        e = 0.5f * (hi + (lo - Rl[i * ld + i]));
      } else {
        const dw tj = {thh[j], thl[j]}, ti = {thh[i], thl[i]};
        // s_ij - theta_j r_ij and s_ji - theta_i r_ji (the test is symmetric in i, j)
        const dw nij = dw_sub_scaled(Sh[i * ld + j], Sl[i * ld + j], tj.hi, tj.lo, Rh[i * ld + j], Rl[i * ld + j]);
        const dw nji = dw_sub_scaled(Sh[j * ld + i], Sl[j * ld + i], ti.hi, ti.lo, Rh[j * ld + i], Rl[j * ld + i]);
        float dh, dl;
        two_sum(tj.hi, -ti.hi, dh, dl);
        const float d = dh + (dl + (tj.lo - ti.lo));
        const float num = nij.hi + nij.lo;
        const float big = fmaxf(fabsf(num), fabsf(nji.hi + nji.lo));
        const float scale = fmaxf(fabsf(tj.hi), fabsf(ti.hi));
        if (fabsf(d) > 100.f * big && fabsf(d) > 1e-13f * scale) {
          e = __fdiv_rn(num, d);
          emax = fmaxf(emax, fabsf(e));
        } else {
          e = -0.5f * (Rh[i * ld + j] + Rl[i * ld + j]);
          atomicOr(&cmask[i], 1ull << j);
          anyclus_s = 1;
        }
      }
      E[i * ld + j] = e;
    }
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 16));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 8));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 4));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 2));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
    if ((tid & 31) == 0) atomicMax(reinterpret_cast<int*>(&emax_s), __float_as_int(emax));
    __syncthreads();
    if (!(emax_s < 1e30f)) return false;  // NaN or overflow: the eigen-based path takes over
    last = (emax_s <= 1e-9f) || step == 3;
    // Q <- Q + Q E (the correction product in FP32, added in double-word)
    for (int t = tid; t < m * m; t += blockDim.x) {
      const int a = t / m, b = t % m;
      float s0 = 0.f, s1 = 0.f;
      int c = 0;
      for (; c + 1 < m; c += 2) {
        s0 = __fmaf_rn(Qh[a * ld + c], E[c * ld + b], s0);
        s1 = __fmaf_rn(Qh[a * ld + c + 1], E[(c + 1) * ld + b], s1);
      }
      if (c < m) s0 = __fmaf_rn(Qh[a * ld + c], E[c * ld + b], s0);
      float hi, lo;
      two_sum(Qh[a * ld + b], s0 + s1, hi, lo);
      const dw q = dw_renorm(hi, lo + Ql[a * ld + b]);
      Q2h[a * ld + b] = q.hi;
      Q2l[a * ld + b] = q.lo;
    }
    __syncthreads();
    for (int t = tid; t < m * ld; t += blockDim.x) {
      Qh[t] = Q2h[t];
      Ql[t] = Q2l[t];
    }
    __syncthreads();
  }
  long long t4 = clock64();
  // ---- clusters of the last step: FP64 Jacobi on their blocks of Q^T H' Q
  if (anyclus_s) {
    // transitive closure of the pair relation (one warp, Warshall)
    if (tid < 32) {
      for (int i = tid; i < m; i += 32) cmask[i] |= 1ull << i;
      __syncwarp();
      for (int p = 0; p < m; ++p) {
        const unsigned long long mp_ = cmask[p];
        __syncwarp();
        for (int i = tid; i < m; i += 32)
          if ((cmask[i] >> p) & 1ull) cmask[i] |= mp_;
        __syncwarp();
      }
    }
    __syncthreads();
    // a cluster of more than eight members (not met in practice) leaves the
    // refined form: the eigen-based path takes over
    int big = 0;
    for (int i = tid; i < m; i += blockDim.x) big |= (__popcll(cmask[i]) > 8) ? 1 : 0;
    if (__syncthreads_or(big)) return false;
    // warp w serves the clusters whose leader (lowest member) is i = w, w + 8, ...
    const int w = tid >> 5, lane = tid & 31;
    for (int i = w; i < m; i += (int)(blockDim.x >> 5)) {
      const unsigned long long mk = cmask[i];
      if ((int)__ffsll((long long)mk) - 1 != i || __popcll(mk) < 2) continue;
      int idx[8];
      int c = 0;
      for (int j = 0; j < m; ++j)
        if ((mk >> j) & 1ull) idx[c++] = j;
      // rows a = lane, lane + 32 of H' Q_C (double-word), then B = Q_C^T H' Q_C
      float hqh[2][8], hql[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          dot2 acc;
          acc.zero();
          if (a < m && v < c)
            for (int b2 = 0; b2 < m; ++b2)
              acc.mac(Hh[a * ld + b2], Hl[a * ld + b2], Qh[b2 * ld + idx[v]], Ql[b2 * ld + idx[v]]);
          const dw r = dw_from_sum(acc);
          hqh[h][v] = r.hi;
          hql[h][v] = r.lo;
        }
      }
      double Bm[8][8], Y[8][8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          Y[u][v] = (u == v) ? 1.0 : 0.0;
          Bm[u][v] = 0.0;
          if (u >= c || v >= c || v < u) continue;
          dot2 acc;
          acc.zero();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int a = lane + 32 * h;
            if (a < m) acc.mac(Qh[a * ld + idx[u]], Ql[a * ld + idx[u]], hqh[h][v], hql[h][v]);
          }
          double val = acc.value();
          for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
          Bm[u][v] = val;
        }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < u; ++v) Bm[u][v] = Bm[v][u];
      // cyclic Jacobi in FP64, every lane redundantly (identical results)
      for (int sw = 0; sw < 12; ++sw) {
        bool rotated = false;
        for (int p = 0; p < c; ++p)
          for (int q = p + 1; q < c; ++q) {
            const double apq = Bm[p][q];
            if (!(fabs(apq) > 1e-15 * sqrt(fabs(Bm[p][p] * Bm[q][q])) && fabs(apq) > 1e-300)) continue;
            rotated = true;
            const double tau = (Bm[q][q] - Bm[p][p]) / (2.0 * apq);
            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
            for (int r = 0; r < c; ++r) {
              const double x = Bm[r][p], y = Bm[r][q];
              Bm[r][p] = cs * x - sn * y;
              Bm[r][q] = sn * x + cs * y;
            }
            for (int r = 0; r < c; ++r) {
              const double x = Bm[p][r], y = Bm[q][r];
              Bm[p][r] = cs * x - sn * y;
              Bm[q][r] = sn * x + cs * y;
            }
            for (int r = 0; r < c; ++r) {
              const double x = Y[r][p], y = Y[r][q];
              Y[r][p] = cs * x - sn * y;
              Y[r][q] = sn * x + cs * y;
            }
          }
        if (!rotated) break;
      }
      __syncwarp();
      // Q_C <- Q_C Y (rows over the lanes), Ritz values of the block
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int a = lane + 32 * h;
        if (a >= m) continue;
        double qrow[8];
        for (int u = 0; u < c; ++u) qrow[u] = dw_to_f64(Qh[a * ld + idx[u]], Ql[a * ld + idx[u]]);
        for (int v = 0; v < c; ++v) {
          double sacc = 0.0;
          for (int u = 0; u < c; ++u) sacc = fma(qrow[u], Y[u][v], sacc);
          const dw q = split_f64(sacc);
          Qh[a * ld + idx[v]] = q.hi;
          Ql[a * ld + idx[v]] = q.lo;
        }
      }
      if (lane == 0)
        for (int u = 0; u < c; ++u) th_s[idx[u]] = Bm[u][u];
    }
    __syncthreads();
  }
  long long t5 = clock64();
  // ascending order, outputs
  for (int j = tid; j < m; j += blockDim.x) {
    const double tj = th_s[j];
    int rank = 0;
    for (int i2 = 0; i2 < m; ++i2) rank += order_before(th_s[i2], i2, tj, j) ? 1 : 0;
    ord[rank] = j;
  }
  __syncthreads();
  for (int j = tid; j < m; j += blockDim.x) theta_out[j] = th_s[j];
  for (int t = tid; t < m * k; t += blockDim.x) {
    const int a = t / k, c = t % k;
    const int j = ord[c];
    C[a * k + c] = sc[a] * dw_to_f64(Qh[a * ld + j], Ql[a * ld + j]);
  }
  __syncthreads();
  if (tid == 0) {
    long long* cyc = st->rr_cycles;
    cyc[0] = t1 - t0;
    cyc[1] = t2 - t1;
    cyc[2] = t3 - t2;
    cyc[3] = t4 - t3;
    cyc[4] = t5 - t4;
    cyc[5] = (long long)step * 1000;
    cyc[7] = tchol - t0;  // of cyc[0]: the pencil's load and the Cholesky
  }
  return true;
}

// Mixed-precision Rayleigh-Ritz launch of the refined form (m <= kRFMax); the
// eigen-based path with dropping when phase A fails.
__global__ void __launch_bounds__(kRFThreads, 1) k_rayleigh_ritz_refined(
    int m, int k, const double* __restrict__ G, const double* __restrict__ H, double drop_tol,
    const double* __restrict__ lam_old, double* C, double* lam_new, double* hist, int hist_rows, int row_host,
    const int32_t* d_row, int stop_rule, double tol, DevStatus* st) {
  // history row: the host's step count, or (captured iterations) the device counter + 1
  const int row = d_row ? *d_row + 1 : row_host;
  double* hist_row = (hist && row >= 0 && row < hist_rows) ? hist + (size_t)row * k : nullptr;
  extern __shared__ __align__(16) double rfsm[];
  __shared__ double sc[kRFMax], theta[kRFMax];
  __shared__ int ord[kRFMax];
  const int tid = threadIdx.x;
  const long long t0 = clock64();
  for (int j = tid; j < m; j += blockDim.x) {
    const double g = G[j * m + j];
    sc[j] = g > 0 ? 1.0 / sqrt(g) : 0.0;
  }
  __syncthreads();
  int sweeps = 0;
  const bool ok = rr_refined_solve(m, k, G, H, sc, reinterpret_cast<float*>(rfsm), drop_tol, C, theta, ord, st,
                                   &sweeps);
  if (!ok) {
    __syncthreads();
    rayleigh_ritz_eig(m, k, G, H, drop_tol, lam_old, C, lam_new, hist_row, stop_rule, tol, st, rfsm, 1);
    return;
  }
  if (tid == 0) {
    double dl = 0;
    for (int c = 0; c < k; ++c) {
      const double th = theta[ord[c]];
      dl += fabs(th - lam_old[c]);
      lam_new[c] = th;
      if (hist_row) hist_row[c] = th;
    }
    st->sum_dl = dl;
    st->kept = m;
    st->sweeps = sweeps;
    if (stop_rule == BPJD_STOP_DLAMBDA) st->converged = (dl < tol) ? 1 : 0;
    st->rr_cycles[6] = clock64() - t0;
  }
}

}  // namespace

int launch_rr(Handle& h, int m, const double* G, const double* Hm, const double* lam_old, double* C,
              double* lam_new, int hist_row, const int32_t* d_row) {
  if (m > kRRMax) return (int)cudaErrorInvalidValue;
  ProfScope ps(h, BPJD_PROF_RR);
  h.launches += 1;
  if (h.dword() && m <= kRFMax) {
    // refined form; its shared memory also holds the eigen-based fallback
    const int mp = m + (m & 1);
    const size_t slot = (((size_t)mp * (mp + 1)) + 3) & ~(size_t)3;
    const size_t fast = (size_t)kRFSlots * slot * sizeof(float);
    const size_t eig = (size_t)(4 * kRRLd * kRRLd + 3 * kRRLd) * sizeof(double) + 3 * kRRLd * sizeof(int);
    allow_dynamic_smem((const void*)k_rayleigh_ritz_refined);
    k_rayleigh_ritz_refined<<<1, kRFThreads, std::max(fast, eig), h.stream>>>(
        m, h.k, G, Hm, h.drop_tol, lam_old, C, lam_new, h.hist, h.hist_rows, hist_row, d_row, h.stop_rule, h.tol,
        h.dstat);
    return (int)cudaGetLastError();
  }
  size_t sm = (size_t)(6 * kRRLd * kRRLd + 3 * kRRLd) * sizeof(double) + 3 * kRRLd * sizeof(int);
  allow_dynamic_smem((const void*)k_rayleigh_ritz_chol);
  k_rayleigh_ritz_chol<<<1, 1024, sm, h.stream>>>(m, h.k, G, Hm, h.drop_tol, lam_old, C, lam_new, h.hist,
                                                 h.hist_rows, hist_row, d_row, h.stop_rule, h.tol, h.dstat,
                                                 h.dword() ? 1 : 0);
  return (int)cudaGetLastError();
}

}  // namespace bpjd
