"""Finite-element assembly of the discrete eigenproblem K x = lambda M x.

Oracle (test infrastructure only).  Section 2.2: V^h is a conforming space on
a uniform partition; the bilinear forms are a(u, v) = int kappa grad u . grad v
(Eq. (2.1) with a coefficient kappa, constant 1 in the paper's experiments) and
b(u, v) = int u v.  Dirichlet data are imposed by dropping boundary nodes.
Degrees of freedom are interior grid nodes in lexicographic order with x
fastest, then y, then z.

Element kinds
  p1_2d  linear triangles, each grid square split along its SW->NE diagonal
  p1_3d  linear tetrahedra, each cube split into the six Kuhn tetrahedra
  q1_3d  trilinear bricks (Section 6, Example 6.3)

All matrices are scipy CSR, float64, canonical (sorted, summed duplicates).
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def _p1_element_matrices(coords: np.ndarray, kappa: np.ndarray):
    """Element stiffness and mass of linear simplices.

    coords : (E, d+1, d) vertex coordinates;  kappa : (E,) coefficient.
    Stiffness  K_e[a, b] = kappa_e |e| grad(phi_a) . grad(phi_b)
    Mass       M_e[a, b] = |e| (1 + delta_ab) / ((d + 1)(d + 2))
    which is the exact integral of products of barycentric coordinates.
    """
    E, nv, d = coords.shape
    J = coords[:, 1:, :] - coords[:, :1, :]              # rows = edge vectors, (E, d, d)
    det = np.linalg.det(J)
    vol = np.abs(det) / (2.0 if d == 2 else 6.0)
    # gradients of barycentric coordinates 1..d: solve J g = e_a
    Jinv = np.linalg.inv(J)                               # (E, d, d): columns are grads
    g = np.empty((E, nv, d))
    g[:, 1:, :] = np.transpose(Jinv, (0, 2, 1))
    g[:, 0, :] = -g[:, 1:, :].sum(axis=1)
    Ke = (kappa * vol)[:, None, None] * np.einsum("eak,ebk->eab", g, g)
    base = np.full((nv, nv), 1.0) + np.eye(nv)
    Me = (vol / ((d + 1) * (d + 2)))[:, None, None] * base[None, :, :]
    return Ke, Me


def _scatter(conn: np.ndarray, Ke: np.ndarray, Me: np.ndarray, n_nodes: int):
    rows = np.repeat(conn, conn.shape[1], axis=1).ravel()
    cols = np.tile(conn, (1, conn.shape[1])).ravel()
    K = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n_nodes, n_nodes)).tocsr()
    M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(n_nodes, n_nodes)).tocsr()
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def _restrict_interior(Kf, Mf, interior: np.ndarray):
    K = Kf[interior][:, interior].tocsr()
    M = Mf[interior][:, interior].tocsr()
    for A in (K, M):
        A.sum_duplicates()
        A.sort_indices()
    return K, M


def p1_2d_full(nx: int, ny: int, Lx: float, Ly: float, kappa: np.ndarray):
    """P1 stiffness/mass over ALL grid nodes (boundary included), node id = j (nx+1) + i.

    Square (i, j) has triangle 0 = (SW, SE, NE) below the diagonal and
    triangle 1 = (SW, NE, NW) above it; kappa[j, i, t] is the coefficient of
    triangle t.
    """
    hx, hy = Lx / nx, Ly / ny
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")     # (ny, nx)
    node = lambda i, j: j * (nx + 1) + i
    sw, se = node(ii, jj), node(ii + 1, jj)
    ne, nw = node(ii + 1, jj + 1), node(ii, jj + 1)
    conn = np.stack([np.stack([sw, se, ne], -1), np.stack([sw, ne, nw], -1)], axis=2)  # (ny,nx,2,3)
    conn = conn.reshape(-1, 3)
    xy = lambda n_: np.stack([(n_ % (nx + 1)) * hx, (n_ // (nx + 1)) * hy], -1)
    coords = xy(conn)                                                  # (E, 3, 2)
    kap = np.asarray(kappa, dtype=np.float64).reshape(-1)
    Ke, Me = _p1_element_matrices(coords, kap)
    return _scatter(conn, Ke, Me, (nx + 1) * (ny + 1))


def _kuhn_tets():
    """The six Kuhn tetrahedra of the unit cube: vertex paths 0 -> e_a -> e_a+e_b -> (1,1,1)
    over the permutations (a, b, c) of the axes, in lexicographic permutation order."""
    tets = []
    for perm in itertools.permutations(range(3)):
        v = [np.zeros(3, dtype=int)]
        for ax in perm:
            w = v[-1].copy()
            w[ax] = 1
            v.append(w)
        tets.append(np.array(v))
    return tets


def p1_3d_full(nx: int, ny: int, nz: int, Lx: float, Ly: float, Lz: float, kappa: np.ndarray):
    """P1 Kuhn-tetrahedra stiffness/mass over all nodes, node id = (l (ny+1) + j)(nx+1) + i.
    kappa[l, j, i] is the coefficient of cube (i, j, l), shared by its six tetrahedra."""
    h = np.array([Lx / nx, Ly / ny, Lz / nz])
    ci, cj, cl = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, cl = ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(), cl.transpose(2, 1, 0).ravel()
    conns, kaps = [], []
    kap_c = np.asarray(kappa, dtype=np.float64).reshape(-1)          # cube order (l, j, i) C-order
    for tet in _kuhn_tets():
        vs = []
        for off in tet:
            vs.append(((cl + off[2]) * (ny + 1) + (cj + off[1])) * (nx + 1) + (ci + off[0]))
        conns.append(np.stack(vs, -1))
        kaps.append(kap_c)
    conn = np.concatenate(conns, 0)
    kap = np.concatenate(kaps, 0)
    nid = conn
    xyz = np.stack([(nid % (nx + 1)) * h[0], ((nid // (nx + 1)) % (ny + 1)) * h[1],
                    (nid // ((nx + 1) * (ny + 1))) * h[2]], -1)
    Ke, Me = _p1_element_matrices(xyz, kap)
    return _scatter(conn, Ke, Me, (nx + 1) * (ny + 1) * (nz + 1))


def _interior_mask(n):
    grids = np.meshgrid(*[np.arange(m + 1) for m in reversed(n)], indexing="ij")
    # grids are ordered (z, y, x) or (y, x): C-order node id matches x fastest
    mask = np.ones(grids[0].shape, dtype=bool)
    for g, m in zip(grids, reversed(n)):
        mask &= (g > 0) & (g < m)
    return np.flatnonzero(mask.ravel())


def lshape_map(n: int) -> np.ndarray:
    """For the L-shaped domain of Section 6, Example 6.2 (the square grid of n x n cells
    minus the quadrant x >= 0, y <= 0 of the centred square): position of every interior
    node of the square (index (j-1)(n-1) + (i-1)) in the L-shape's dof list, -1 for the
    nodes of the closed removed quadrant (i >= n/2, j <= n/2), which carry Dirichlet data.
    The dofs keep the square's lexicographic order."""
    i, j = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="xy")
    keep = ~((i >= n // 2) & (j <= n // 2)).ravel()
    out = -np.ones(keep.size, dtype=np.int64)
    out[keep] = np.arange(int(keep.sum()))
    return out


def lshape3_map(nx: int, ny: int, nz: int) -> np.ndarray:
    """For the L-shaped prism of Section 6, Example 6.4 (the box grid of nx x ny x nz cells
    minus the prism x >= Lx/2, y >= Ly/2): position of every interior node of the box
    (index ((l-1)(ny-1) + (j-1))(nx-1) + (i-1)) in the domain's dof list, -1 for the nodes
    of the closed removed prism (i >= nx/2, j >= ny/2), which carry Dirichlet data."""
    l, j, i = np.meshgrid(np.arange(1, nz), np.arange(1, ny), np.arange(1, nx), indexing="ij")
    keep = ~((i >= nx // 2) & (j >= ny // 2)).ravel()
    out = -np.ones(keep.size, dtype=np.int64)
    out[keep] = np.arange(int(keep.sum()))
    return out


def assemble(spec):
    """Stiffness K and mass M on interior dofs for a ``workloads.ProblemSpec``
    (only the mesh fields kind, n, length and kappa are used)."""
    if spec.kind == "morley_2d":
        from . import morley
        return morley.assemble(spec.n[0], spec.length[0])
    if spec.kind == "bfs_2d":
        from . import bfs
        return bfs.assemble(spec.n[0], spec.length[0])
    if spec.kind == "q1_lshape":
        # as for the 2-D L-shape: the cells of the removed prism touch only Dirichlet nodes
        K, M = q1_3d_interior(*spec.n, *spec.length)
        keep = np.flatnonzero(lshape3_map(*spec.n) >= 0)
        return _restrict_interior(K, M, keep)
    if spec.kind == "p1_lshape":
        # every triangle of the removed quadrant has its three vertices in the closed
        # quadrant, i.e. on the Dirichlet boundary: the square's matrices restricted to
        # the L-shape's interior nodes are the L-shape's own
        n = spec.n[0]
        Kf, Mf = p1_2d_full(n, n, *spec.length, np.ones((n, n, 2)))
        Ks, Ms = _restrict_interior(Kf, Mf, _interior_mask(spec.n))
        keep = np.flatnonzero(lshape_map(n) >= 0)
        return _restrict_interior(Ks, Ms, keep)
    kap = spec.kappa_array()
    if spec.kind == "p1_2d":
        Kf, Mf = p1_2d_full(*spec.n, *spec.length, kap)
    elif spec.kind == "p1_3d":
        Kf, Mf = p1_3d_full(*spec.n, *spec.length, kap)
    elif spec.kind == "q1_3d":
        if not np.all(kap == kap.flat[0]):
            raise ValueError("q1_3d assembly supports a constant coefficient only")
        K, M = q1_3d_interior(*spec.n, *spec.length)
        return kap.flat[0] * K, M
    else:
        raise ValueError(spec.kind)
    return _restrict_interior(Kf, Mf, _interior_mask(spec.n))


def _q1_1d(m: int, L: float):
    """1-D linear-element matrices on the m-1 interior nodes of [0, L] split into m cells:
    stiffness (1/h) tridiag(-1, 2, -1), mass (h/6) tridiag(1, 4, 1)."""
    h = L / m
    e = np.ones(m - 1)
    K1 = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) / h
    M1 = sp.diags([e[:-1], 4 * e, e[:-1]], [-1, 0, 1]) * (h / 6.0)
    return K1.tocsr(), M1.tocsr()


def q1_3d_interior(nx, ny, nz, Lx, Ly, Lz):
    """Trilinear bricks with kappa = 1: the element matrices are tensor products of the
    1-D linear-element matrices, so the assembled matrices are Kronecker sums
    K = Kz(x)My(x)Mx... (x fastest => x is the last Kronecker factor)."""
    Kx, Mx = _q1_1d(nx, Lx)
    Ky, My = _q1_1d(ny, Ly)
    Kz, Mz = _q1_1d(nz, Lz)
    kr = lambda a, b, c: sp.kron(a, sp.kron(b, c)).tocoo()
    # sum the three terms as COO triplets so that entries cancelling to zero stay in
    # the pattern (node pairs sharing an element), like every other element kind
    terms = [kr(Mz, My, Kx), kr(Mz, Ky, Mx), kr(Kz, My, Mx)]
    K = sp.coo_matrix((np.concatenate([t.data for t in terms]),
                       (np.concatenate([t.row for t in terms]), np.concatenate([t.col for t in terms]))),
                      shape=terms[0].shape).tocsr()
    M = kr(Mz, My, Mx).tocsr()
    for A in (K, M):
        A.sum_duplicates()
        A.sort_indices()
    return K, M
