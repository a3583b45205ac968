// Host-side problem generation: finite-element assembly of the model problems
// (Section 2.1, Section 2.2, Section 6), overlapping box subdomains with their
// colouring (Section 2.3, Assumption 2) and the nodal interpolation V^H -> V^h.
//
// Degrees of freedom are interior grid nodes, lexicographic with x fastest;
// Dirichlet data are imposed by omitting boundary nodes.  The sparsity pattern
// of K and M is the set of node pairs sharing an element (explicit zeros kept).

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bpjd.h"

namespace {

struct CsrBuf {
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int32_t n_rows = 0, n_cols = 0;
  bpjd_csr view() const {
    bpjd_csr c;
    c.n_rows = n_rows;
    c.n_cols = n_cols;
    c.nnz = (int64_t)col.size();
    c.row_ptr = row_ptr.data();
    c.col_idx = col.data();
    c.val = val.data();
    return c;
  }
};

struct ProblemImpl {
  bpjd_problem pub;  // first member: the public pointer is the impl pointer
  CsrBuf K, M, P, P0;
  std::vector<int64_t> sub_ptr;
  std::vector<int32_t> sub_dofs, sub_color;
};

struct Entry {
  int64_t key;  // row * n + col
  double k, m;
};

// Gradients of the barycentric coordinates of a simplex with d+1 vertices
// (rows of J are the edge vectors x_a - x_0); returns the volume.
template <int D>
double simplex_gradients(const double (*x)[D], double (*g)[D]) {
  double J[D][D];
  for (int a = 0; a < D; ++a)
    for (int c = 0; c < D; ++c) J[a][c] = x[a + 1][c] - x[0][c];
  double inv[D][D];
  double det;
  if (D == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    inv[0][0] = J[1][1] / det;
    inv[0][1] = -J[0][1] / det;
    inv[1][0] = -J[1][0] / det;
    inv[1][1] = J[0][0] / det;
  } else {
    const double(*A)[D] = J;
    double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    // inverse = adjugate / det; adj[i][j] = cofactor[j][i]
    double cof[3][3];
    cof[0][0] = c00;
    cof[0][1] = c01;
    cof[0][2] = c02;
    cof[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
    cof[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
    cof[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
    cof[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
    cof[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
    cof[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) inv[i][j] = cof[j][i] / det;
  }
  // x - x0 = J^T lambda  =>  grad lambda_a = column a of J^{-1}
  for (int a = 0; a < D; ++a)
    for (int c = 0; c < D; ++c) g[a + 1][c] = inv[c][a];
  for (int c = 0; c < D; ++c) {
    double s = 0;
    for (int a = 1; a <= D; ++a) s += g[a][c];
    g[0][c] = -s;
  }
  double fact = (D == 2) ? 2.0 : 6.0;
  return std::fabs(det) / fact;
}

template <int D>
void add_simplex(const double (*x)[D], const int64_t* dof, double kappa, std::vector<Entry>& out,
                 int64_t n) {
  double g[D + 1][D];
  double vol = simplex_gradients<D>(x, g);
  const double mscale = vol / double((D + 1) * (D + 2));
  for (int a = 0; a <= D; ++a) {
    if (dof[a] < 0) continue;
    for (int b = 0; b <= D; ++b) {
      if (dof[b] < 0) continue;
      double dot = 0;
      for (int c = 0; c < D; ++c) dot += g[a][c] * g[b][c];
      Entry e;
      e.key = dof[a] * n + dof[b];
      e.k = kappa * vol * dot;
      e.m = mscale * (a == b ? 2.0 : 1.0);
      out.push_back(e);
    }
  }
}

void entries_to_csr(std::vector<Entry>& ent, int64_t n, CsrBuf& K, CsrBuf& M) {
  std::stable_sort(ent.begin(), ent.end(), [](const Entry& a, const Entry& b) { return a.key < b.key; });
  K.n_rows = K.n_cols = M.n_rows = M.n_cols = (int32_t)n;
  K.row_ptr.assign(n + 1, 0);
  M.row_ptr.assign(n + 1, 0);
  size_t i = 0;
  while (i < ent.size()) {
    size_t j = i;
    double ks = 0, ms = 0;
    while (j < ent.size() && ent[j].key == ent[i].key) {
      ks += ent[j].k;
      ms += ent[j].m;
      ++j;
    }
    int64_t r = ent[i].key / n, c = ent[i].key % n;
    K.col.push_back((int32_t)c);
    K.val.push_back(ks);
    M.col.push_back((int32_t)c);
    M.val.push_back(ms);
    K.row_ptr[r + 1]++;
    i = j;
  }
  for (int64_t r = 0; r < n; ++r) K.row_ptr[r + 1] += K.row_ptr[r];
  M.row_ptr = K.row_ptr;
}

int assemble_p1_2d(const bpjd_mesh& m, CsrBuf& K, CsrBuf& M) {
  const int nx = m.n[0], ny = m.n[1];
  const double hx = m.length[0] / nx, hy = m.length[1] / ny;
  const int64_t N = (int64_t)(nx - 1) * (ny - 1);
  auto dof = [&](int i, int j) -> int64_t {
    if (i <= 0 || i >= nx || j <= 0 || j >= ny) return -1;
    return (int64_t)(j - 1) * (nx - 1) + (i - 1);
  };
  std::vector<Entry> ent;
  ent.reserve((size_t)nx * ny * 18);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)
      for (int t = 0; t < 2; ++t) {
        // t = 0: (SW, SE, NE) below the diagonal; t = 1: (SW, NE, NW)
        int vi[3], vj[3];
        vi[0] = i, vj[0] = j;
        if (t == 0) {
          vi[1] = i + 1, vj[1] = j;
          vi[2] = i + 1, vj[2] = j + 1;
        } else {
          vi[1] = i + 1, vj[1] = j + 1;
          vi[2] = i, vj[2] = j + 1;
        }
        double x[3][2];
        int64_t d[3];
        for (int a = 0; a < 3; ++a) {
          x[a][0] = vi[a] * hx;
          x[a][1] = vj[a] * hy;
          d[a] = dof(vi[a], vj[a]);
        }
        double kap = m.kappa ? m.kappa[((size_t)j * nx + i) * 2 + t] : 1.0;
        add_simplex<2>(x, d, kap, ent, N);
      }
  entries_to_csr(ent, N, K, M);
  return BPJD_OK;
}

int assemble_p1_3d(const bpjd_mesh& m, CsrBuf& K, CsrBuf& M) {
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const double h[3] = {m.length[0] / nx, m.length[1] / ny, m.length[2] / nz};
  const int64_t N = (int64_t)(nx - 1) * (ny - 1) * (nz - 1);
  auto dof = [&](int i, int j, int l) -> int64_t {
    if (i <= 0 || i >= nx || j <= 0 || j >= ny || l <= 0 || l >= nz) return -1;
    return ((int64_t)(l - 1) * (ny - 1) + (j - 1)) * (nx - 1) + (i - 1);
  };
  // the six Kuhn tetrahedra: vertex paths 0 -> e_a -> e_a + e_b -> (1,1,1) over the
  // axis permutations (a, b, c) in lexicographic order
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  std::vector<Entry> ent;
  ent.reserve((size_t)nx * ny * nz * 6 * 16);
  for (int l = 0; l < nz; ++l)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double kap = m.kappa ? m.kappa[((size_t)l * ny + j) * nx + i] : 1.0;
        for (int p = 0; p < 6; ++p) {
          int off[4][3] = {{0, 0, 0}};
          for (int s = 1; s <= 3; ++s) {
            for (int c = 0; c < 3; ++c) off[s][c] = off[s - 1][c];
            off[s][perms[p][s - 1]] = 1;
          }
          double x[4][3];
          int64_t d[4];
          for (int a = 0; a < 4; ++a) {
            int gi = i + off[a][0], gj = j + off[a][1], gl = l + off[a][2];
            x[a][0] = gi * h[0];
            x[a][1] = gj * h[1];
            x[a][2] = gl * h[2];
            d[a] = dof(gi, gj, gl);
          }
          add_simplex<3>(x, d, kap, ent, N);
        }
      }
  entries_to_csr(ent, N, K, M);
  return BPJD_OK;
}

// Trilinear bricks, kappa = 1: K = Kz(x)My(x)Mx + Mz(x)Ky(x)Mx + Mz(x)My(x)Kx with the 1-D
// linear-element matrices K1 = (1/h) tridiag(-1, 2, -1), M1 = (h/6) tridiag(1, 4, 1).
int assemble_q1_3d(const bpjd_mesh& m, CsrBuf& K, CsrBuf& M) {
  const int n[3] = {m.n[0], m.n[1], m.n[2]};
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = m.length[d] / n[d];
  const int64_t N = (int64_t)(n[0] - 1) * (n[1] - 1) * (n[2] - 1);
  auto k1 = [&](int d, int o) { return o == 0 ? 2.0 / h[d] : -1.0 / h[d]; };
  auto m1 = [&](int d, int o) { return o == 0 ? 4.0 * (h[d] / 6.0) : 1.0 * (h[d] / 6.0); };
  K.n_rows = K.n_cols = M.n_rows = M.n_cols = (int32_t)N;
  K.row_ptr.assign(N + 1, 0);
  double kap = m.kappa ? m.kappa[0] : 1.0;
  for (int l = 1; l < n[2]; ++l)
    for (int j = 1; j < n[1]; ++j)
      for (int i = 1; i < n[0]; ++i) {
        int64_t r = ((int64_t)(l - 1) * (n[1] - 1) + (j - 1)) * (n[0] - 1) + (i - 1);
        for (int dl = -1; dl <= 1; ++dl)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              int a = i + di, b = j + dj, c = l + dl;
              if (a <= 0 || a >= n[0] || b <= 0 || b >= n[1] || c <= 0 || c >= n[2]) continue;
              int64_t col = ((int64_t)(c - 1) * (n[1] - 1) + (b - 1)) * (n[0] - 1) + (a - 1);
              double mz = m1(2, dl), my = m1(1, dj), mx = m1(0, di);
              double kv = mz * (my * k1(0, di)) + mz * (k1(1, dj) * mx) + k1(2, dl) * (my * mx);
              K.col.push_back((int32_t)col);
              K.val.push_back(kap * kv);
              M.col.push_back((int32_t)col);
              M.val.push_back(mz * (my * mx));
            }
        K.row_ptr[r + 1] = (int64_t)K.col.size();
      }
  M.row_ptr = K.row_ptr;
  return BPJD_OK;
}

// Box partition: along axis d, subdomain s spans the open node-index interval
// (lo, hi), lo = s m - delta (0 for s = 0), hi = (s+1) m + delta (n for the last);
// its dofs are the nodes strictly inside, ascending; colour = sum_d (s_d mod 2) 2^d.
void box_partition(const bpjd_mesh& m, int dim, ProblemImpl& P) {
  int S[3] = {1, 1, 1}, n[3] = {2, 2, 2};
  for (int d = 0; d < dim; ++d) {
    S[d] = m.nsub[d];
    n[d] = m.n[d];
  }
  int64_t inner[3] = {n[0] - 1, n[1] - 1, n[2] - 1};
  P.sub_ptr.assign(1, 0);
  for (int sz = 0; sz < S[2]; ++sz)
    for (int sy = 0; sy < S[1]; ++sy)
      for (int sx = 0; sx < S[0]; ++sx) {
        int s[3] = {sx, sy, sz};
        int a[3], b[3];
        for (int d = 0; d < 3; ++d) {
          if (d >= dim) {
            a[d] = b[d] = 1;
            continue;
          }
          int mm = n[d] / S[d];
          int lo = (s[d] == 0) ? 0 : std::max(s[d] * mm - m.delta, 0);
          int hi = (s[d] == S[d] - 1) ? n[d] : std::min((s[d] + 1) * mm + m.delta, n[d]);
          a[d] = lo + 1;
          b[d] = hi - 1;
        }
        // lexicographic (z, y, x) loops give ascending global dofs
        for (int l = a[2]; l <= b[2]; ++l)
          for (int j = a[1]; j <= b[1]; ++j)
            for (int i = a[0]; i <= b[0]; ++i) {
              int64_t g = (i - 1) + inner[0] * ((j - 1) + (dim == 3 ? inner[1] * (l - 1) : 0));
              P.sub_dofs.push_back((int32_t)g);
            }
        P.sub_ptr.push_back((int64_t)P.sub_dofs.size());
        int col = 0;
        for (int d = 0; d < dim; ++d) col |= (s[d] & 1) << d;
        P.sub_color.push_back(col);
      }
}

// Nodal interpolation of the coarse basis (same element kind on the grid of
// S_d cells per axis, m fine cells per coarse cell on every axis).  A fine node
// at offset r in coarse cell I gets barycentric (P1) or trilinear (Q1)
// coordinates, each an integer numerator over m (or m^3).  Boundary coarse
// nodes and zero values are dropped.
int coarse_interp(const bpjd_mesh& m, int dim, const int32_t* S, CsrBuf& P) {
  int mm = m.n[0] / S[0];
  for (int d = 0; d < dim; ++d)
    if (m.n[d] % S[d] != 0 || m.n[d] / S[d] != mm) return BPJD_ERR_BAD_ARG;
  int64_t inner[3] = {m.n[0] - 1, m.n[1] - 1, dim == 3 ? m.n[2] - 1 : 1};
  int64_t N = inner[0] * inner[1] * inner[2];
  int64_t nH = 1;
  for (int d = 0; d < dim; ++d) nH *= (S[d] - 1);
  if (nH <= 0) return BPJD_ERR_BAD_ARG;
  P.n_rows = (int32_t)N;
  P.n_cols = (int32_t)nH;
  P.row_ptr.assign(N + 1, 0);
  auto coarse_id = [&](const int* C) -> int64_t {
    int64_t idx = 0, stride = 1;
    for (int d = 0; d < dim; ++d) {
      if (C[d] <= 0 || C[d] >= S[d]) return -1;
      idx += (int64_t)(C[d] - 1) * stride;
      stride *= (S[d] - 1);
    }
    return idx;
  };
  const int nz = dim == 3 ? m.n[2] : 2;
  std::vector<std::pair<int64_t, double>> row;
  for (int l = 1; l < nz; ++l)
    for (int j = 1; j < m.n[1]; ++j)
      for (int i = 1; i < m.n[0]; ++i) {
        int node[3] = {i, j, l};
        int cell[3], r[3];
        for (int d = 0; d < dim; ++d) {
          cell[d] = std::min(node[d] / mm, S[d] - 1);
          r[d] = node[d] - cell[d] * mm;
        }
        // (corner offsets, numerator, denominator) triples
        struct W {
          int off[3];
          int64_t num;
          double den;
        } w[8];
        int nw = 0;
        if (m.kind == 0) {
          int rx = r[0], ry = r[1];
          if (rx >= ry) {
            w[0] = {{0, 0, 0}, mm - rx, (double)mm};
            w[1] = {{1, 0, 0}, rx - ry, (double)mm};
            w[2] = {{1, 1, 0}, ry, (double)mm};
          } else {
            w[0] = {{0, 0, 0}, mm - ry, (double)mm};
            w[1] = {{1, 1, 0}, rx, (double)mm};
            w[2] = {{0, 1, 0}, ry - rx, (double)mm};
          }
          nw = 3;
        } else if (m.kind == 1) {
          // sort axes by descending offset (stable for ties)
          int ord[3] = {0, 1, 2};
          for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 3; ++q)
              if (r[ord[q]] > r[ord[p]] || (r[ord[q]] == r[ord[p]] && ord[q] < ord[p])) std::swap(ord[p], ord[q]);
          int a = ord[0], b = ord[1], c = ord[2];
          w[0] = {{0, 0, 0}, mm - r[a], (double)mm};
          w[1] = {{0, 0, 0}, r[a] - r[b], (double)mm};
          w[1].off[a] = 1;
          w[2] = {{0, 0, 0}, r[b] - r[c], (double)mm};
          w[2].off[a] = 1;
          w[2].off[b] = 1;
          w[3] = {{1, 1, 1}, r[c], (double)mm};
          nw = 4;
        } else {
          for (int corner = 0; corner < 8; ++corner) {
            int64_t num = 1;
            W ww;
            for (int d = 0; d < 3; ++d) {
              int bit = (corner >> (2 - d)) & 1;  // z-major corner order, irrelevant after sorting
              ww.off[d] = bit;
              num *= bit ? r[d] : (mm - r[d]);
            }
            ww.num = num;
            ww.den = (double)mm * mm * mm;
            w[nw++] = ww;
          }
        }
        row.clear();
        for (int q = 0; q < nw; ++q) {
          if (w[q].num == 0) continue;
          int C[3];
          for (int d = 0; d < 3; ++d) C[d] = cell[d] + w[q].off[d];
          int64_t c = coarse_id(C);
          if (c < 0) continue;
          row.push_back({c, (double)w[q].num / w[q].den});
        }
        std::sort(row.begin(), row.end());
        int64_t g = (i - 1) + inner[0] * ((j - 1) + inner[1] * (l - 1));
        for (auto& e : row) {
          P.col.push_back((int32_t)e.first);
          P.val.push_back(e.second);
        }
        P.row_ptr[g + 1] = (int64_t)P.col.size();
      }
  return BPJD_OK;
}

}  // namespace

extern "C" int bpjd_problem_create(const bpjd_mesh* mesh, bpjd_problem** out) {
  if (!mesh || !out) return BPJD_ERR_BAD_ARG;
  *out = nullptr;
  const bpjd_mesh& m = *mesh;
  int dim = (m.kind == 0) ? 2 : 3;
  if (m.kind < 0 || m.kind > 2) return BPJD_ERR_BAD_ARG;
  for (int d = 0; d < dim; ++d) {
    if (m.n[d] < 2 || m.nsub[d] < 1 || m.n[d] % m.nsub[d] != 0 || !(m.length[d] > 0)) return BPJD_ERR_BAD_ARG;
  }
  if (m.delta < 0 || m.tau < 0 || m.tau > 6) return BPJD_ERR_BAD_ARG;
  if (m.kind == 2 && m.kappa) {
    size_t ne = (size_t)m.n[0] * m.n[1] * m.n[2];
    for (size_t e = 1; e < ne; ++e)
      if (m.kappa[e] != m.kappa[0]) return BPJD_ERR_UNSUPPORTED;
  }
  ProblemImpl* P = new (std::nothrow) ProblemImpl();
  if (!P) return BPJD_ERR_OOM;
  int rc;
  try {
    if (m.kind == 0)
      rc = assemble_p1_2d(m, P->K, P->M);
    else if (m.kind == 1)
      rc = assemble_p1_3d(m, P->K, P->M);
    else
      rc = assemble_q1_3d(m, P->K, P->M);
    if (rc == BPJD_OK) rc = coarse_interp(m, dim, m.nsub, P->P);
    if (rc == BPJD_OK) {
      if (m.tau == 0) {
        P->P0 = P->P;
      } else {
        int32_t S0[3];
        for (int d = 0; d < 3; ++d) S0[d] = m.nsub[d] << m.tau;
        rc = coarse_interp(m, dim, S0, P->P0);
      }
    }
    if (rc == BPJD_OK) box_partition(m, dim, *P);
  } catch (...) {
    rc = BPJD_ERR_OOM;
  }
  if (rc != BPJD_OK) {
    delete P;
    return rc;
  }
  P->pub.K = P->K.view();
  P->pub.M = P->M.view();
  P->pub.P = P->P.view();
  P->pub.P0 = P->P0.view();
  P->pub.part.n_sub = (int32_t)P->sub_color.size();
  P->pub.part.sub_ptr = P->sub_ptr.data();
  P->pub.part.sub_dofs = P->sub_dofs.data();
  P->pub.part.sub_color = P->sub_color.data();
  P->pub.part.n_colors = 1 << dim;
  *out = &P->pub;
  return BPJD_OK;
}

extern "C" void bpjd_problem_free(bpjd_problem* p) {
  if (!p) return;
  delete reinterpret_cast<ProblemImpl*>(p);
}
