// Host-side problem generation: finite-element assembly of the model problems
// (Section 2.1, Section 2.2, Section 6), overlapping box subdomains with their
// colouring (Section 2.3, Assumption 2) and the nodal interpolation V^H -> V^h
// (for Morley elements, the Morley interpolant of the BFS coarse space).
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
  int32_t n_colors = 0;  // 0: 2^dim (box partitions)
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
void box_partition(const bpjd_mesh& m, int dim, ProblemImpl& P, int dofs_per_node = 1) {
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
              for (int c = 0; c < dofs_per_node; ++c) P.sub_dofs.push_back((int32_t)(dofs_per_node * g + c));
            }
        P.sub_ptr.push_back((int64_t)P.sub_dofs.size());
        int col = 0;
        for (int d = 0; d < dim; ++d) col |= (s[d] & 1) << d;
        P.sub_color.push_back(col);
      }
}

// The partition J_H of Example 6.1 (Section 6) on the P1 grid of kind 0 (n x n
// squares split SW->NE, S x S coarse squares of c = n / S cells): every coarse
// square is cut along its own SW->NE diagonal into two coarse triangles, T = 0
// below it (towards SE) and T = 1 above it, which the fine triangles resolve
// exactly; each is enlarged by `rings` rings of fine triangles (Section 2.3:
// whole elements added layer by layer; one ring adds every fine triangle that
// shares a vertex with the region).  The local dofs are the interior nodes
// whose six surrounding fine triangles all lie in the enlarged region (the
// local functions vanish on its boundary), ascending.  Subdomain id
// 2 (sx + S sy) + T, colour 2 ((sx mod 2) + 2 (sy mod 2)) + T: two coarse
// triangles of one colour are at least c cells apart and each grows by `rings`
// cells, so the colour classes stay disjoint (Assumption 2) while 2 rings < c
// (checked by the caller).
// Fine triangle (i, j, t) of cell (i, j): t = 0 has the vertices (i, j),
// (i+1, j), (i+1, j+1); t = 1 has (i, j), (i+1, j+1), (i, j+1).
void triangle_partition(int n, int S, int rings, ProblemImpl& P) {
  const int c = n / S;
  // cell offsets (di, dj) of the vertices of the two fine triangles of a cell
  static const int vx[2][3] = {{0, 1, 1}, {0, 1, 0}}, vy[2][3] = {{0, 0, 1}, {0, 1, 1}};
  P.sub_ptr.assign(1, 0);
  P.sub_dofs.clear();
  P.sub_color.clear();
  std::vector<uint8_t> tri, node;
  for (int sy = 0; sy < S; ++sy)
    for (int sx = 0; sx < S; ++sx)
      for (int T = 0; T < 2; ++T) {
        // the enlarged region stays within `rings` cells of the coarse square
        const int x0 = std::max(0, sx * c - rings), x1 = std::min(n, (sx + 1) * c + rings);
        const int y0 = std::max(0, sy * c - rings), y1 = std::min(n, (sy + 1) * c + rings);
        const int W = x1 - x0, H = y1 - y0;
        auto at = [&](int t, int i, int j) -> uint8_t& { return tri[((size_t)t * H + (j - y0)) * W + (i - x0)]; };
        auto nd = [&](int i, int j) -> uint8_t& { return node[(size_t)(j - y0) * (W + 1) + (i - x0)]; };
        tri.assign((size_t)2 * W * H, 0);
        for (int j = sy * c; j < (sy + 1) * c; ++j)
          for (int i = sx * c; i < (sx + 1) * c; ++i) {
            const int a = i - sx * c, b = j - sy * c;  // a > b: cell below the diagonal
            at(0, i, j) = (T == 0) ? (a >= b) : (a < b);
            at(1, i, j) = (T == 0) ? (a > b) : (a <= b);
          }
        for (int r = 0; r < rings; ++r) {
          node.assign((size_t)(W + 1) * (H + 1), 0);
          for (int t = 0; t < 2; ++t)
            for (int j = y0; j < y1; ++j)
              for (int i = x0; i < x1; ++i)
                if (at(t, i, j))
                  for (int v = 0; v < 3; ++v) nd(i + vx[t][v], j + vy[t][v]) = 1;
          for (int t = 0; t < 2; ++t)
            for (int j = y0; j < y1; ++j)
              for (int i = x0; i < x1; ++i)
                for (int v = 0; v < 3; ++v)
                  if (nd(i + vx[t][v], j + vy[t][v])) at(t, i, j) = 1;
        }
        // interior node (i, j) is a vertex of t = 0 in the cells (i, j), (i-1, j),
        // (i-1, j-1) and of t = 1 in (i, j), (i-1, j-1), (i, j-1)
        auto in_region = [&](int t, int i, int j) {
          return i >= x0 && i < x1 && j >= y0 && j < y1 && at(t, i, j) != 0;
        };
        for (int j = std::max(1, y0); j <= std::min(n - 1, y1); ++j)
          for (int i = std::max(1, x0); i <= std::min(n - 1, x1); ++i) {
            const bool all = in_region(0, i, j) && in_region(0, i - 1, j) && in_region(0, i - 1, j - 1) &&
                             in_region(1, i, j) && in_region(1, i - 1, j - 1) && in_region(1, i, j - 1);
            if (all) P.sub_dofs.push_back((int32_t)((int64_t)(j - 1) * (n - 1) + (i - 1)));
          }
        P.sub_ptr.push_back((int64_t)P.sub_dofs.size());
        P.sub_color.push_back(2 * ((sx & 1) + 2 * (sy & 1)) + T);
      }
  P.n_colors = 8;
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

// ---------------------------------------------------------------------------
// Morley elements for the clamped plate (Section 2.1 with m = 2; the paper's own
// element for this problem is BFS).  Broken Hessian form sum_T int_T D^2u : D^2v
// and b(u, v) = int u v on the square grid of kind 0 (squares split SW->NE).
// The dofs live on the half-grid (X h/2, Y h/2), X, Y = 0..2n: vertex values at
// (even, even); scaled normal derivatives h du/dy at (odd, even), h du/dx at
// (even, odd) and h (du/dx - du/dy) at (odd, odd) (diagonal edge midpoints).
// Clamped data remove exactly the boundary half-grid points, so the dofs are the
// interior points numbered (Y-1)(2n-1) + (X-1): a subdomain's ascending dofs then
// follow the half-grid rows and its band spans about two cell rows.
// Element quantities are rationals (exact arithmetic below), scaled by h^-2
// (stiffness) or h^2 (mass); the coarse space is BFS on the subdomain grid and the
// transfer matrix entries are rationals rounded once to double.
// ---------------------------------------------------------------------------

int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct Rat {
  int64_t p = 0, q = 1;  // q > 0, gcd(p, q) = 1
  Rat() = default;
  Rat(int64_t a, int64_t b = 1) : p(a), q(b) {
    if (q < 0) {
      p = -p;
      q = -q;
    }
    int64_t g = gcd64(p, q);
    if (g > 1) {
      p /= g;
      q /= g;
    }
  }
  Rat operator+(const Rat& o) const {
    int64_t g = gcd64(q, o.q);
    return Rat(p * (o.q / g) + o.p * (q / g), (q / g) * o.q);
  }
  Rat operator-(const Rat& o) const { return *this + Rat(-o.p, o.q); }
  Rat operator*(const Rat& o) const {
    int64_t g1 = gcd64(p, o.q), g2 = gcd64(o.p, q);
    if (g1 == 0) g1 = 1;
    if (g2 == 0) g2 = 1;
    return Rat((p / g1) * (o.p / g2), (q / g2) * (o.q / g1));
  }
  Rat operator/(const Rat& o) const { return *this * Rat(o.q, o.p); }
  bool zero() const { return p == 0; }
  double to_double() const { return (double)p / (double)q; }
};

enum MorleyFn { MV = 0, MDY = 1, MDX = 2, MDD = 3 };  // value, d/deta, d/dxi, d/dxi - d/deta
const int kMono[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};

Rat rpow(const Rat& x, int e) {
  Rat r(1);
  for (int i = 0; i < e; ++i) r = r * x;
  return r;
}

// functional f applied to xi^p eta^q at (x, y)
Rat morley_functional(int f, int p, int q, const Rat& x, const Rat& y) {
  auto dxi = [&]() { return p > 0 ? Rat(p) * rpow(x, p - 1) * rpow(y, q) : Rat(0); };
  auto deta = [&]() { return q > 0 ? Rat(q) * rpow(x, p) * rpow(y, q - 1) : Rat(0); };
  switch (f) {
    case MV:
      return rpow(x, p) * rpow(y, q);
    case MDY:
      return deta();
    case MDX:
      return dxi();
    default:
      return dxi() - deta();
  }
}

int morley_kind(int X, int Y) { return (X & 1) ? ((Y & 1) ? MDD : MDY) : ((Y & 1) ? MDX : MV); }

struct MorleyRef {
  // local dofs: half-grid offsets within the square and functional
  int off[6][2];
  int fn[6];
  Rat C[6][6];  // C[m][a]: coefficient of monomial m in basis function a
  Rat S[6][6], R[6][6];
};

// shape 0: (SW, SE, NE) below the diagonal, edges bottom / right / diagonal;
// shape 1: (SW, NE, NW) above it, edges diagonal / top / left
MorleyRef morley_reference(int shape) {
  MorleyRef E;
  static const int offs[2][6][2] = {{{0, 0}, {2, 0}, {2, 2}, {1, 0}, {2, 1}, {1, 1}},
                                    {{0, 0}, {2, 2}, {0, 2}, {1, 1}, {1, 2}, {0, 1}}};
  for (int a = 0; a < 6; ++a) {
    E.off[a][0] = offs[shape][a][0];
    E.off[a][1] = offs[shape][a][1];
    E.fn[a] = morley_kind(E.off[a][0], E.off[a][1]);
  }
  // Vandermonde V[r][m] = N_r(monomial m), inverted by Gauss-Jordan
  Rat A[6][12];
  for (int r = 0; r < 6; ++r) {
    Rat x(E.off[r][0], 2), y(E.off[r][1], 2);
    for (int m = 0; m < 6; ++m) A[r][m] = morley_functional(E.fn[r], kMono[m][0], kMono[m][1], x, y);
    for (int m = 0; m < 6; ++m) A[r][6 + m] = Rat(r == m ? 1 : 0);
  }
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    while (A[piv][c].zero()) ++piv;
    for (int j = 0; j < 12; ++j) std::swap(A[c][j], A[piv][j]);
    Rat inv = Rat(1) / A[c][c];
    for (int j = 0; j < 12; ++j) A[c][j] = A[c][j] * inv;
    for (int r = 0; r < 6; ++r) {
      if (r == c || A[r][c].zero()) continue;
      Rat f = A[r][c];
      for (int j = 0; j < 12; ++j) A[r][j] = A[r][j] - f * A[c][j];
    }
  }
  for (int m = 0; m < 6; ++m)
    for (int a = 0; a < 6; ++a) E.C[m][a] = A[m][6 + a];
  // reference-triangle monomial integrals: lower {0 <= eta <= xi <= 1}: 1/((q+1)(p+q+2));
  // upper {0 <= xi <= eta <= 1}: 1/((p+1)(p+q+2))
  auto tri = [&](int p, int q) { return shape == 0 ? Rat(1, (q + 1) * (p + q + 2)) : Rat(1, (p + 1) * (p + q + 2)); };
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      // area 1/2 times the Frobenius product of the Hessians [[2 c_xx, c_xy], [c_xy, 2 c_yy]]
      Rat hh = Rat(4) * E.C[3][a] * E.C[3][b] + Rat(2) * E.C[4][a] * E.C[4][b] + Rat(4) * E.C[5][a] * E.C[5][b];
      E.S[a][b] = Rat(1, 2) * hh;
      Rat acc(0);
      for (int m1 = 0; m1 < 6; ++m1)
        for (int m2 = 0; m2 < 6; ++m2)
          acc = acc + E.C[m1][a] * E.C[m2][b] * tri(kMono[m1][0] + kMono[m2][0], kMono[m1][1] + kMono[m2][1]);
      E.R[a][b] = acc;
    }
  return E;
}

int assemble_morley(const bpjd_mesh& m, CsrBuf& K, CsrBuf& M) {
  const int n = m.n[0];
  const double h = m.length[0] / n;
  const int inner = 2 * n - 1;
  const int64_t N = (int64_t)inner * inner;
  auto dof = [&](int X, int Y) -> int64_t {
    if (X <= 0 || X >= 2 * n || Y <= 0 || Y >= 2 * n) return -1;
    return (int64_t)(Y - 1) * inner + (X - 1);
  };
  std::vector<Entry> ent;
  ent.reserve((size_t)n * n * 2 * 36);
  for (int shape = 0; shape < 2; ++shape) {
    const MorleyRef E = morley_reference(shape);
    double Ke[6][6], Me[6][6];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) {
        Ke[a][b] = E.S[a][b].to_double() / (h * h);
        Me[a][b] = E.R[a][b].to_double() * (h * h);
      }
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        int64_t d[6];
        for (int a = 0; a < 6; ++a) d[a] = dof(2 * i + E.off[a][0], 2 * j + E.off[a][1]);
        for (int a = 0; a < 6; ++a) {
          if (d[a] < 0) continue;
          for (int b = 0; b < 6; ++b) {
            if (d[b] < 0) continue;
            Entry e;
            e.key = d[a] * N + d[b];
            e.k = Ke[a][b];
            e.m = Me[a][b];
            ent.push_back(e);
          }
        }
      }
  }
  entries_to_csr(ent, N, K, M);
  return BPJD_OK;
}

void hermite_basis(Rat C[4][4]);  // cubic Hermite basis on [0, 1] (BFS section below)

// Coarse space for Morley: the conforming BFS space (C^1 bicubic Hermite functions)
// on the S x S subdomain grid, brought into V^h by the Morley interpolant: a fine
// dof takes its value or scaled normal derivative of the coarse function, which is
// C^1, so any coarse cell holding the point gives the same number (the lowest-
// indexed one is used).  Coarse dofs are node-major 4 node + a + 2 b (derivatives
// scaled by H); boundary coarse nodes (clamped) and exact zeros are dropped.
int morley_transfer(const bpjd_mesh& m, int S, CsrBuf& P) {
  const int n = m.n[0];
  if (S < 2 || n % S != 0) return BPJD_ERR_BAD_ARG;
  const int mm = n / S, w = 2 * mm;
  const int inner = 2 * n - 1, mc = S - 1;
  const int64_t N = (int64_t)inner * inner;
  Rat C[4][4];
  hermite_basis(C);
  // 1-D Hermite values (0..3) and derivatives (4..7) at local positions t / w, t = 0..w
  std::vector<std::array<Rat, 8>> H1((size_t)w + 1);
  for (int t = 0; t <= w; ++t) {
    const Rat x(t, w);
    for (int a = 0; a < 4; ++a) {
      Rat v(0), d(0);
      for (int p = 0; p < 4; ++p) {
        v = v + C[p][a] * rpow(x, p);
        if (p) d = d + Rat(p) * C[p][a] * rpow(x, p - 1);
      }
      H1[t][a] = v;
      H1[t][4 + a] = d;
    }
  }
  P.n_rows = (int32_t)N;
  P.n_cols = 4 * mc * mc;
  P.row_ptr.assign(N + 1, 0);
  std::vector<std::pair<int64_t, double>> row;
  for (int Y = 1; Y < 2 * n; ++Y)
    for (int X = 1; X < 2 * n; ++X) {
      const int f = morley_kind(X, Y);
      const int I = std::min(X / w, S - 1), J = std::min(Y / w, S - 1);
      const auto& hx = H1[X - w * I];
      const auto& hy = H1[Y - w * J];
      row.clear();
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          const int In = I + (a >> 1), Jn = J + (b >> 1);
          if (In <= 0 || In >= S || Jn <= 0 || Jn >= S) continue;
          const Rat u = hx[a] * hy[b];
          const Rat ux = hx[4 + a] * hy[b] / Rat(mm);  // fine h d/dx = (h / H) d/ds
          const Rat uy = hx[a] * hy[4 + b] / Rat(mm);
          const Rat v = (f == MV) ? u : (f == MDY) ? uy : (f == MDX) ? ux : ux - uy;
          if (v.zero()) continue;
          row.push_back({4 * ((int64_t)(Jn - 1) * mc + (In - 1)) + (a & 1) + 2 * (b & 1), v.to_double()});
        }
      std::sort(row.begin(), row.end());
      const int64_t g = (int64_t)(Y - 1) * inner + (X - 1);
      for (auto& r : row) {
        P.col.push_back((int32_t)r.first);
        P.val.push_back(r.second);
      }
      P.row_ptr[g + 1] = (int64_t)P.col.size();
    }
  return BPJD_OK;
}

// ---------------------------------------------------------------------------
// Bogner-Fox-Schmit elements for the clamped plate (Section 2.1, Section 2.2,
// m = 2): C^1 bicubics, tensor products of 1-D cubic Hermite functions.  Each
// node carries u, h du/dx, h du/dy, h^2 d^2u/dxdy (node-major dofs
// 4 node + a + 2 b, a / b = x / y derivative order); clamped data remove the
// boundary nodes.  With the 1-D matrices M0 = int phi psi, K1 = int phi' psi',
// K2 = int phi'' psi'' (scaled by h, 1/h, 1/h^3) the stiffness is
// M0 (x) K2 + 2 K1 (x) K1 + K2 (x) M0 (y factor first) and the mass M0 (x) M0;
// on H^2_0 int D^2u : D^2v equals int Delta u Delta v.
// ---------------------------------------------------------------------------

// cubic Hermite basis on [0, 1]: C[p][a] = coefficient of s^p in basis a
// (a = value / derivative at 0, value / derivative at 1)
void hermite_basis(Rat C[4][4]) {
  Rat A[4][8];
  const int V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {1, 1, 1, 1}, {0, 1, 2, 3}};
  for (int r = 0; r < 4; ++r)
    for (int j = 0; j < 8; ++j) A[r][j] = Rat(j < 4 ? V[r][j] : (j - 4 == r ? 1 : 0));
  for (int c = 0; c < 4; ++c) {
    int piv = c;
    while (A[piv][c].zero()) ++piv;
    for (int j = 0; j < 8; ++j) std::swap(A[c][j], A[piv][j]);
    Rat inv = Rat(1) / A[c][c];
    for (int j = 0; j < 8; ++j) A[c][j] = A[c][j] * inv;
    for (int r = 0; r < 4; ++r) {
      if (r == c || A[r][c].zero()) continue;
      Rat f = A[r][c];
      for (int j = 0; j < 8; ++j) A[r][j] = A[r][j] - f * A[c][j];
    }
  }
  for (int p = 0; p < 4; ++p)
    for (int a = 0; a < 4; ++a) C[p][a] = A[p][4 + a];
}

// 1-D element matrices on the unit cell: E[0] = M0, E[1] = K1, E[2] = K2
void hermite_element(Rat E[3][4][4]) {
  Rat C[4][4];
  hermite_basis(C);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int d = 0; d < 3; ++d) {
        // int_0^1 (d-th derivative of basis a)(d-th derivative of basis b)
        Rat acc(0);
        for (int p = d; p < 4; ++p)
          for (int q = d; q < 4; ++q) {
            int64_t fp = 1, fq = 1;
            for (int t = 0; t < d; ++t) {
              fp *= (p - t);
              fq *= (q - t);
            }
            acc = acc + C[p][a] * C[q][b] * Rat(fp * fq, (p - d) + (q - d) + 1);
          }
        E[d][a][b] = acc;
      }
}

int assemble_bfs(const bpjd_mesh& m, CsrBuf& K, CsrBuf& M) {
  const int n = m.n[0];
  const double h = m.length[0] / n;
  const int mi = n - 1;  // interior nodes per axis
  Rat E[3][4][4];
  hermite_element(E);
  const double scale[3] = {h, 1.0 / h, 1.0 / std::pow(h, 3)};
  // assembled 1-D matrices over the interior node dofs (value, h derivative), in the
  // order the cells are visited; entry (r, dr) holds row r, column r + dr - 3
  std::vector<double> G[3];
  const int nd = 2 * mi;
  for (int d = 0; d < 3; ++d) G[d].assign((size_t)nd * 7, 0.0);
  for (int e = 0; e < n; ++e) {
    for (int a = 0; a < 4; ++a) {
      const int ra = 2 * (e - 1) + a;  // interior dof index (node e - 1 + (a >> 1))
      if (ra < 0 || ra >= nd) continue;
      for (int b = 0; b < 4; ++b) {
        const int rb = 2 * (e - 1) + b;
        if (rb < 0 || rb >= nd) continue;
        for (int d = 0; d < 3; ++d) G[d][(size_t)ra * 7 + (rb - ra + 3)] += E[d][a][b].to_double() * scale[d];
      }
    }
  }
  auto g1 = [&](int d, int r, int c) { return G[d][(size_t)r * 7 + (c - r + 3)]; };
  const int64_t N = 4 * (int64_t)mi * mi;
  K.n_rows = K.n_cols = M.n_rows = M.n_cols = (int32_t)N;
  K.row_ptr.assign(N + 1, 0);
  for (int j = 0; j < mi; ++j)
    for (int i = 0; i < mi; ++i)
      for (int c = 0; c < 4; ++c) {
        const int a = c & 1, b = c >> 1;
        const int rx = 2 * i + a, ry = 2 * j + b;
        const int64_t row = 4 * ((int64_t)j * mi + i) + c;
        for (int j2 = std::max(0, j - 1); j2 <= std::min(mi - 1, j + 1); ++j2)
          for (int i2 = std::max(0, i - 1); i2 <= std::min(mi - 1, i + 1); ++i2)
            for (int c2 = 0; c2 < 4; ++c2) {
              const int cx = 2 * i2 + (c2 & 1), cy = 2 * j2 + (c2 >> 1);
              const double My0 = g1(0, ry, cy), Ky1 = g1(1, ry, cy), Ky2 = g1(2, ry, cy);
              const double Mx0 = g1(0, rx, cx), Kx1 = g1(1, rx, cx), Kx2 = g1(2, rx, cx);
              K.col.push_back((int32_t)(4 * ((int64_t)j2 * mi + i2) + c2));
              K.val.push_back((My0 * Kx2 + 2.0 * (Ky1 * Kx1)) + Ky2 * Mx0);
              M.col.push_back(K.col.back());
              M.val.push_back(My0 * Mx0);
            }
        K.row_ptr[row + 1] = (int64_t)K.col.size();
      }
  M.row_ptr = K.row_ptr;
  return BPJD_OK;
}

// Nested coarse interpolation for BFS: fine node dofs of the coarse bicubic Hermite
// functions, a tensor product of the 1-D transfers (exact rationals rounded once).
int bfs_transfer(const bpjd_mesh& m, int S, CsrBuf& P) {
  const int n = m.n[0];
  if (S < 2 || n % S != 0) return BPJD_ERR_BAD_ARG;
  const int mm = n / S;
  Rat C[4][4];
  hermite_basis(C);
  // 1-D: for fine dof fd (node f, order a) the coarse dofs and values
  std::vector<std::vector<std::pair<int, Rat>>> T1((size_t)2 * (n + 1));
  for (int f = 0; f <= n; ++f) {
    const int cell = std::min(f / mm, S - 1);
    const Rat s(f - cell * mm, mm);
    for (int a = 0; a < 4; ++a) {
      const int cdof = 2 * (cell + (a >> 1)) + (a & 1);
      Rat val(0), der(0);
      for (int p = 0; p < 4; ++p) {
        val = val + C[p][a] * rpow(s, p);
        if (p) der = der + Rat(p) * C[p][a] * rpow(s, p - 1);
      }
      der = der / Rat(mm);
      if (!val.zero()) T1[2 * f].push_back({cdof, val});
      if (!der.zero()) T1[2 * f + 1].push_back({cdof, der});
    }
  }
  const int mi = n - 1, mc = S - 1;
  const int64_t N = 4 * (int64_t)mi * mi;
  P.n_rows = (int32_t)N;
  P.n_cols = (int32_t)(4 * (int64_t)mc * mc);
  P.row_ptr.assign(N + 1, 0);
  std::vector<std::pair<int64_t, Rat>> row;
  for (int j = 1; j < n; ++j)
    for (int i = 1; i < n; ++i)
      for (int c = 0; c < 4; ++c) {
        const int a = c & 1, b = c >> 1;
        row.clear();
        for (auto& ty : T1[2 * j + b])
          for (auto& tx : T1[2 * i + a]) {
            const int jc = ty.first >> 1, bc = ty.first & 1, ic = tx.first >> 1, ac = tx.first & 1;
            if (ic <= 0 || ic >= S || jc <= 0 || jc >= S) continue;  // clamped coarse nodes
            const int64_t col = 4 * ((int64_t)(jc - 1) * mc + (ic - 1)) + ac + 2 * bc;
            const Rat v = tx.second * ty.second;
            bool found = false;
            for (auto& r : row)
              if (r.first == col) {
                r.second = r.second + v;
                found = true;
                break;
              }
            if (!found) row.push_back({col, v});
          }
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int64_t, Rat>& u, const std::pair<int64_t, Rat>& v) { return u.first < v.first; });
        const int64_t g = 4 * ((int64_t)(j - 1) * mi + (i - 1)) + c;
        for (auto& r : row) {
          if (r.second.zero()) continue;
          P.col.push_back((int32_t)r.first);
          P.val.push_back(r.second.to_double());
        }
        P.row_ptr[g + 1] = (int64_t)P.col.size();
      }
  return BPJD_OK;
}

// ---------------------------------------------------------------------------
// L-shaped domain of Section 6, Example 6.2: the square grid of kind 0 (n x n
// cells, kappa = 1) minus the quadrant x >= 0, y <= 0 of the centred square.
// Every triangle of that quadrant has its three vertices in the closed quadrant,
// which carries Dirichlet data, so the L-shape's matrices, coarse interpolation
// and subdomain dofs are the square's restricted to the L-shape's interior nodes
// (the square's lexicographic order is kept); the boxes of the domain partition
// are those of the square whose cells lie in the domain.
// ---------------------------------------------------------------------------

// position of every interior node of the square grid (index (j-1)(n-1) + (i-1)) in
// the L-shape's dof list, -1 for the nodes of the closed removed quadrant
std::vector<int64_t> lshape_map(int n) {
  std::vector<int64_t> out((size_t)(n - 1) * (n - 1), -1);
  int64_t next = 0;
  for (int j = 1; j < n; ++j)
    for (int i = 1; i < n; ++i)
      if (!(i >= n / 2 && j <= n / 2)) out[(size_t)(j - 1) * (n - 1) + (i - 1)] = next++;
  return out;
}

void restrict_csr(const CsrBuf& A, const std::vector<int64_t>& rmap, const std::vector<int64_t>& cmap,
                  CsrBuf& out) {
  int64_t nr = 0, nc = 0;
  for (int64_t v : rmap) nr += (v >= 0);
  for (int64_t v : cmap) nc += (v >= 0);
  out.n_rows = (int32_t)nr;
  out.n_cols = (int32_t)nc;
  out.row_ptr.assign(nr + 1, 0);
  out.col.clear();
  out.val.clear();
  for (int64_t r = 0; r < A.n_rows; ++r) {
    if (rmap[r] < 0) continue;
    for (int64_t e = A.row_ptr[r]; e < A.row_ptr[r + 1]; ++e) {
      const int64_t c = cmap[A.col[e]];
      if (c < 0) continue;
      out.col.push_back((int32_t)c);
      out.val.push_back(A.val[e]);
    }
    out.row_ptr[rmap[r] + 1] = (int64_t)out.col.size();
  }
}

int build_lshape(const bpjd_mesh& m, ProblemImpl& P) {
  const int n = m.n[0], S = m.nsub[0];
  bpjd_mesh sq = m;
  sq.kind = 0;
  sq.kappa = nullptr;
  CsrBuf K, M, Pc, P0;
  int rc = assemble_p1_2d(sq, K, M);
  if (rc == BPJD_OK) rc = coarse_interp(sq, 2, m.nsub, Pc);
  int32_t S0[3] = {S << m.tau, S << m.tau, 1};
  if (rc == BPJD_OK && m.tau > 0) rc = coarse_interp(sq, 2, S0, P0);
  if (rc != BPJD_OK) return rc;
  const std::vector<int64_t> fm = lshape_map(n), cm = lshape_map(S);
  restrict_csr(K, fm, fm, P.K);
  restrict_csr(M, fm, fm, P.M);
  restrict_csr(Pc, fm, cm, P.P);
  if (m.tau > 0)
    restrict_csr(P0, fm, lshape_map(S0[0]), P.P0);
  else
    P.P0 = P.P;
  ProblemImpl box;
  box_partition(sq, 2, box);
  P.sub_ptr.assign(1, 0);
  for (int l = 0; l + 1 < (int)box.sub_ptr.size(); ++l) {
    const int sx = l % S, sy = l / S;
    if (sx >= S / 2 && sy < S / 2) continue;  // box of the removed quadrant
    for (int64_t e = box.sub_ptr[l]; e < box.sub_ptr[l + 1]; ++e) {
      const int64_t d = fm[box.sub_dofs[e]];
      if (d >= 0) P.sub_dofs.push_back((int32_t)d);
    }
    P.sub_ptr.push_back((int64_t)P.sub_dofs.size());
    P.sub_color.push_back(box.sub_color[l]);
  }
  return BPJD_OK;
}

// L-shaped prism of Section 6, Example 6.4: the box grid of kind 2 (trilinear
// bricks) minus the prism x >= Lx/2, y >= Ly/2; restricted like the 2-D L-shape.
std::vector<int64_t> lshape3_map(int nx, int ny, int nz) {
  std::vector<int64_t> out((size_t)(nx - 1) * (ny - 1) * (nz - 1), -1);
  int64_t next = 0;
  for (int l = 1; l < nz; ++l)
    for (int j = 1; j < ny; ++j)
      for (int i = 1; i < nx; ++i)
        if (!(i >= nx / 2 && j >= ny / 2)) out[((size_t)(l - 1) * (ny - 1) + (j - 1)) * (nx - 1) + (i - 1)] = next++;
  return out;
}

int build_q1_lshape(const bpjd_mesh& m, ProblemImpl& P) {
  bpjd_mesh bx = m;
  bx.kind = 2;
  bx.kappa = nullptr;
  CsrBuf K, M, Pc, P0;
  int rc = assemble_q1_3d(bx, K, M);
  if (rc == BPJD_OK) rc = coarse_interp(bx, 3, m.nsub, Pc);
  int32_t S0[3];
  for (int d = 0; d < 3; ++d) S0[d] = m.nsub[d] << m.tau;
  if (rc == BPJD_OK && m.tau > 0) rc = coarse_interp(bx, 3, S0, P0);
  if (rc != BPJD_OK) return rc;
  const std::vector<int64_t> fm = lshape3_map(m.n[0], m.n[1], m.n[2]);
  const std::vector<int64_t> cm = lshape3_map(m.nsub[0], m.nsub[1], m.nsub[2]);
  restrict_csr(K, fm, fm, P.K);
  restrict_csr(M, fm, fm, P.M);
  restrict_csr(Pc, fm, cm, P.P);
  if (m.tau > 0)
    restrict_csr(P0, fm, lshape3_map(S0[0], S0[1], S0[2]), P.P0);
  else
    P.P0 = P.P;
  ProblemImpl box;
  box_partition(bx, 3, box);
  const int Sx = m.nsub[0], Sy = m.nsub[1];
  P.sub_ptr.assign(1, 0);
  for (int l = 0; l + 1 < (int)box.sub_ptr.size(); ++l) {
    const int sx = l % Sx, sy = (l / Sx) % Sy;
    if (sx >= Sx / 2 && sy >= Sy / 2) continue;  // box of the removed prism
    for (int64_t e = box.sub_ptr[l]; e < box.sub_ptr[l + 1]; ++e) {
      const int64_t d = fm[box.sub_dofs[e]];
      if (d >= 0) P.sub_dofs.push_back((int32_t)d);
    }
    P.sub_ptr.push_back((int64_t)P.sub_dofs.size());
    P.sub_color.push_back(box.sub_color[l]);
  }
  return BPJD_OK;
}

}  // namespace

extern "C" int bpjd_problem_create(const bpjd_mesh* mesh, bpjd_problem** out) {
  if (!mesh || !out) return BPJD_ERR_BAD_ARG;
  *out = nullptr;
  const bpjd_mesh& m = *mesh;
  int dim = (m.kind == 0 || m.kind == 3 || m.kind == 4 || m.kind == 5) ? 2 : 3;
  if (m.kind < 0 || m.kind > 6) return BPJD_ERR_BAD_ARG;
  for (int d = 0; d < dim; ++d) {
    if (m.n[d] < 2 || m.nsub[d] < 1 || m.n[d] % m.nsub[d] != 0 || !(m.length[d] > 0)) return BPJD_ERR_BAD_ARG;
  }
  if (m.delta < 0 || m.tau < 0 || m.tau > 6) return BPJD_ERR_BAD_ARG;
  if (m.partition != BPJD_PART_BOXES && m.partition != BPJD_PART_TRIANGLES) return BPJD_ERR_BAD_ARG;
  if (m.partition == BPJD_PART_TRIANGLES &&
      (m.kind != 0 || m.n[0] != m.n[1] || m.nsub[0] != m.nsub[1] || !(2 * m.delta < m.n[0] / m.nsub[0])))
    return BPJD_ERR_BAD_ARG;
  if (m.kind == 5 && (m.n[0] % 2 || m.nsub[0] % 2)) return BPJD_ERR_BAD_ARG;
  if (m.kind == 6) {
    if (m.n[0] % 2 || m.n[1] % 2 || m.nsub[0] % 2 || m.nsub[1] % 2) return BPJD_ERR_BAD_ARG;
    if (m.kappa) return BPJD_ERR_UNSUPPORTED;
  }
  if (m.kind == 3 || m.kind == 4 || m.kind == 5) {
    if (m.n[0] != m.n[1] || m.nsub[0] != m.nsub[1] || m.length[0] != m.length[1]) return BPJD_ERR_BAD_ARG;
    if (m.kappa) return BPJD_ERR_UNSUPPORTED;
    if ((m.n[0] / m.nsub[0]) % (1 << m.tau) != 0) return BPJD_ERR_BAD_ARG;
  }
  if (m.kind == 2 && m.kappa) {
    size_t ne = (size_t)m.n[0] * m.n[1] * m.n[2];
    for (size_t e = 1; e < ne; ++e)
      if (m.kappa[e] != m.kappa[0]) return BPJD_ERR_UNSUPPORTED;
  }
  ProblemImpl* P = new (std::nothrow) ProblemImpl();
  if (!P) return BPJD_ERR_OOM;
  int rc;
  try {
    if (m.kind == 6) {
      rc = build_q1_lshape(m, *P);
    } else if (m.kind == 5) {
      rc = build_lshape(m, *P);
    } else if (m.kind == 4) {
      rc = assemble_bfs(m, P->K, P->M);
      if (rc == BPJD_OK) rc = bfs_transfer(m, m.nsub[0], P->P);
      if (rc == BPJD_OK) {
        if (m.tau == 0)
          P->P0 = P->P;
        else
          rc = bfs_transfer(m, m.nsub[0] << m.tau, P->P0);
      }
      if (rc == BPJD_OK) box_partition(m, dim, *P, 4);
    } else if (m.kind == 3) {
      rc = assemble_morley(m, P->K, P->M);
      if (rc == BPJD_OK) rc = morley_transfer(m, m.nsub[0], P->P);
      if (rc == BPJD_OK) {
        if (m.tau == 0)
          P->P0 = P->P;
        else
          rc = morley_transfer(m, m.nsub[0] << m.tau, P->P0);
      }
      if (rc == BPJD_OK) {
        // the box rule on the half-grid carrying the Morley dofs
        bpjd_mesh half = m;
        half.n[0] = 2 * m.n[0];
        half.n[1] = 2 * m.n[1];
        half.delta = 2 * m.delta;
        box_partition(half, dim, *P);
      }
    } else {
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
      if (rc == BPJD_OK) {
        if (m.partition == BPJD_PART_TRIANGLES)
          triangle_partition(m.n[0], m.nsub[0], m.delta, *P);
        else
          box_partition(m, dim, *P);
      }
    }
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
  P->pub.part.n_colors = P->n_colors ? P->n_colors : (1 << dim);
  *out = &P->pub;
  return BPJD_OK;
}

extern "C" void bpjd_problem_free(bpjd_problem* p) {
  if (!p) return;
  delete reinterpret_cast<ProblemImpl*>(p);
}
