"""Overlapping box subdomains, local dof lists and colouring.

Oracle (test infrastructure only).  Section 2.3: the coarse partition J_H
into subdomains Omega_l is enlarged layer by layer by whole fine elements into
Omega_l'; delta measures the overlap; the local space V^(l) is the part of V^h
that vanishes outside Omega_l' (zero trace on its boundary).  Assumption 2:
the Omega_l' can be coloured so that same-coloured subdomains are disjoint.

Rule used here (box subdomains on the uniform grid, in fine-node index units):
  * subdomain (s_x, s_y[, s_z]) has id l = s_x + S_x (s_y + S_y s_z);
  * along axis d with m = n_d / S_d elements per subdomain, Omega_l' spans the
    open index interval (lo, hi) with lo = s_d m - delta (0 for s_d = 0) and
    hi = (s_d + 1) m + delta (n_d for the last subdomain), clipped to [0, n_d];
  * the local dofs are the grid nodes strictly inside Omega_l' (so the local
    functions vanish on its boundary), which are interior nodes of Omega;
  * they are listed in ascending global dof order;
  * colour = sum_d (s_d mod 2) 2^d, valid (disjoint colour classes) while
    2 delta <= m.
For Morley elements (morley_2d) the same rule runs on the half-grid that
carries their dofs (2 n points per axis, subdomains of 2 m half-steps grown by
2 delta): the dofs strictly inside Omega_l' are the vertices strictly inside
and the midpoints of the edges not on its boundary, i.e. the Morley functions
with zero values and normal derivatives on the boundary of Omega_l'.
For BFS elements (bfs_2d) the rule picks nodes as for p1_2d, each with its four
dofs (node-major), i.e. the BFS functions in H^2_0(Omega_l').
"""

from __future__ import annotations

import itertools

import numpy as np


def axis_ranges(n: int, S: int, delta: int):
    """Inclusive node-index ranges [a, b] strictly inside each subdomain along one axis."""
    m = n // S
    out = []
    for s in range(S):
        lo = 0 if s == 0 else max(s * m - delta, 0)
        hi = n if s == S - 1 else min((s + 1) * m + delta, n)
        out.append((lo + 1, hi - 1))
    return out


def box_partition(spec):
    """Returns (sub_ptr int64[N+1], sub_dofs int32[sum n_l], sub_color int32[N], n_colors).

    For the L-shaped domain (p1_lshape) the partition J_H of the domain is the boxes of
    the square whose cells lie in the domain (s_x < S/2 or s_y >= S/2); their dofs are
    mapped to the L-shape's numbering (nodes of the removed quadrant dropped); ids follow
    the remaining boxes in order, colours are kept."""
    if spec.kind == "q1_lshape":
        from dataclasses import replace
        from .fem import lshape3_map
        ptr, dofs, col, nc = box_partition(replace(spec, kind="q1_3d"))
        lm = lshape3_map(*spec.n)
        Sx, Sy, _ = spec.nsub
        nptr, ndofs, ncol = [0], [], []
        for l in range(len(ptr) - 1):
            sx, sy = l % Sx, (l // Sx) % Sy
            if sx >= Sx // 2 and sy >= Sy // 2:
                continue                               # box of the removed prism
            d = lm[dofs[ptr[l]:ptr[l + 1]]]
            d = d[d >= 0]
            ndofs.append(d)
            nptr.append(nptr[-1] + len(d))
            ncol.append(col[l])
        return (np.asarray(nptr, dtype=np.int64), np.concatenate(ndofs).astype(np.int32),
                np.asarray(ncol, dtype=np.int32), nc)
    if spec.kind == "p1_lshape":
        from dataclasses import replace
        from .fem import lshape_map
        ptr, dofs, col, nc = box_partition(replace(spec, kind="p1_2d"))
        lm = lshape_map(spec.n[0])
        S = spec.nsub[0]
        nptr, ndofs, ncol = [0], [], []
        for l in range(len(ptr) - 1):
            sx, sy = l % S, l // S
            if sx >= S // 2 and sy < S // 2:
                continue
            d = lm[dofs[ptr[l]:ptr[l + 1]]]
            d = d[d >= 0]
            ndofs.append(d)
            nptr.append(nptr[-1] + len(d))
            ncol.append(col[l])
        return (np.asarray(nptr, dtype=np.int64), np.concatenate(ndofs).astype(np.int32),
                np.asarray(ncol, dtype=np.int32), nc)
    n, S, dim, delta = spec.n, spec.nsub, spec.dim, spec.delta
    if spec.kind == "morley_2d":
        n, delta = tuple(2 * m for m in n), 2 * delta
    ranges = [axis_ranges(n[d], S[d], delta) for d in range(dim)]
    inner = [m - 1 for m in n]                      # interior nodes per axis
    ptr = [0]
    dofs = []
    colors = []
    # subdomain id l = s_x + S_x (s_y + S_y s_z): iterate with x fastest
    for sidx in itertools.product(*[range(S[d]) for d in reversed(range(dim))]):
        s = tuple(reversed(sidx))                   # (s_x, s_y[, s_z])
        axes = [np.arange(ranges[d][s[d]][0], ranges[d][s[d]][1] + 1) for d in range(dim)]
        # global dof of interior node (i, j[, l]) = ((l-1) inner_y + (j-1)) inner_x + (i-1)
        g = np.zeros([len(a) for a in reversed(axes)], dtype=np.int64)
        stride = 1
        for d in range(dim):
            shape = [1] * dim
            shape[dim - 1 - d] = len(axes[d])
            g = g + (axes[d] - 1).reshape(shape) * stride
            stride *= inner[d]
        local = np.sort(g.ravel())
        if spec.kind == "bfs_2d":
            local = (4 * local[:, None] + np.arange(4)[None, :]).ravel()
        dofs.append(local)
        ptr.append(ptr[-1] + len(local))
        colors.append(sum((s[d] % 2) << d for d in range(dim)))
    return (np.asarray(ptr, dtype=np.int64), np.concatenate(dofs).astype(np.int32),
            np.asarray(colors, dtype=np.int32), 1 << dim)


def triangle_partition(n: int, S: int, layers: int):
    """The paper's partition J_H of Section 6, Example 6.1: each of the S x S coarse squares of
    the uniform n x n grid (n a multiple of S) split along its SW->NE diagonal into two
    coarse triangles (N = 2 S^2), each enlarged by `layers` rings of fine triangles (Section
    2.3: whole fine elements added layer by layer; a ring = every fine triangle sharing a
    vertex with the region); the dofs of a subdomain are the interior nodes all of whose fine
    triangles lie in the enlarged region (zero trace on its boundary), ascending.

    Subdomain id = 2 (s_x + S s_y) + t (t = 0 below the diagonal); colour = 2 ((s_x mod 2)
    + 2 (s_y mod 2)) + t.  Two triangles of one colour lie at least one coarse square (n / S fine
    cells) apart, and each grows by `layers` cells towards the other, so same-coloured
    subdomains stay disjoint (Assumption 2) only while 2 layers < n / S; wider enlargements
    are rejected.  Returns (sub_ptr, sub_dofs, sub_color, n_colors = 8)."""
    if S < 1 or n % S != 0:
        raise ValueError(f"the fine grid ({n}) must refine the coarse grid ({S}) evenly")
    if not 0 <= 2 * layers < n // S:
        raise ValueError(f"{layers} rings on coarse squares of {n // S} cells would overlap same-coloured "
                         "subdomains (Assumption 2 needs 2 layers < n / S)")
    m = n // S
    # fine triangle (i, j, t) of square (i, j): t = 0 (SW, SE, NE), t = 1 (SW, NE, NW)
    vert = {0: ((0, 0), (1, 0), (1, 1)), 1: ((0, 0), (1, 1), (0, 1))}
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")      # [j, i]
    ptr, dofs, colors = [0], [], []
    for sy in range(S):
        for sx in range(S):
            for T in (0, 1):
                li, lj = ii - sx * m, jj - sy * m
                inside = (li >= 0) & (li < m) & (lj >= 0) & (lj < m)
                reg = np.zeros((2, n, n), dtype=bool)                     # [t, j, i]
                if T == 0:
                    reg[0] = inside & (li >= lj)
                    reg[1] = inside & (li > lj)
                else:
                    reg[0] = inside & (li < lj)
                    reg[1] = inside & (li <= lj)
                for _ in range(layers):
                    node = np.zeros((n + 1, n + 1), dtype=bool)           # [j, i]
                    for t in (0, 1):
                        for (di, dj) in vert[t]:
                            node[dj:dj + n, di:di + n] |= reg[t]
                    for t in (0, 1):
                        touch = np.zeros((n, n), dtype=bool)
                        for (di, dj) in vert[t]:
                            touch |= node[dj:dj + n, di:di + n]
                        reg[t] |= touch
                # a node is a dof when every fine triangle around it is in the region
                ok = np.ones((n + 1, n + 1), dtype=bool)
                cover = np.zeros((n + 1, n + 1), dtype=np.int32)
                for t in (0, 1):
                    for (di, dj) in vert[t]:
                        pad = np.zeros((n + 1, n + 1), dtype=bool)
                        pad[dj:dj + n, di:di + n] = reg[t]
                        cnt = np.zeros((n + 1, n + 1), dtype=np.int32)
                        cnt[dj:dj + n, di:di + n] = 1
                        cover += pad.astype(np.int32)
                        ok &= ~((cnt == 1) & ~pad)
                jn, in_ = np.nonzero(ok & (cover > 0))
                keep = (in_ > 0) & (in_ < n) & (jn > 0) & (jn < n)
                local = np.sort((jn[keep] - 1) * (n - 1) + (in_[keep] - 1))
                dofs.append(local)
                ptr.append(ptr[-1] + len(local))
                colors.append(2 * ((sx % 2) + 2 * (sy % 2)) + T)
    return (np.asarray(ptr, dtype=np.int64), np.concatenate(dofs).astype(np.int32),
            np.asarray(colors, dtype=np.int32), 8)
