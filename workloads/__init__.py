"""Seeded synthetic workload generators for the two-level BPJD eigensolver.

This package only *describes* eigenproblems: mesh resolution, domain size,
the coefficient field kappa sampled per element, the subdomain grid, the
overlap width and the number k of wanted eigenpairs, plus the seeded request
stream of the serving workload.  It holds none of the solver's arithmetic:
no finite-element assembly, no partition rule, no coarse interpolation and no
eigensolver step.  Both the CPU oracle (``oracle/``) and the CUDA library
(``paper_2203_06327_gb300``) consume these descriptions and build everything
else independently.

Problem classes follow the model problems of the paper (Section 2.1, the
Laplacian eigenproblem with Dirichlet data) discretised as in Section 2.2 and
the experiments of Section 6:

* ``p1_2d``   -- P1 Lagrange elements on a uniform grid of nx x ny squares,
  each split along its SW->NE diagonal (Section 6, Example 6.1 uses a uniform
  triangle partition).
* ``p1_3d``   -- P1 Lagrange elements on the Kuhn (Freudenthal) split of a
  uniform nx x ny x nz cube grid into six tetrahedra per cube.
* ``q1_3d``   -- trilinear elements on a uniform cube grid (Section 6,
  Example 6.3).
* ``morley_2d`` -- the clamped plate Delta^2 u = lambda u (Section 2.1, m = 2)
  with Morley's nonconforming quadratic triangles on the same square grid as
  ``p1_2d`` (the paper itself uses BFS elements for this problem); no
  coefficient, square domain.
* ``p1_lshape`` -- P1 (as ``p1_2d``) on the L-shaped domain of Section 6,
  Example 6.2: the square [-L/2, L/2]^2 minus the quadrant [0, L/2) x (-L/2, 0],
  i.e. the square's grid with the cells of that quadrant removed; no coefficient.
* ``q1_lshape`` -- trilinear elements (as ``q1_3d``) on the L-shaped prism of
  Section 6, Example 6.4: the box [0, Lx] x [0, Ly] x [0, Lz] minus
  [Lx/2, Lx) x [Ly/2, Ly) x (0, Lz); no coefficient.
* ``bfs_2d`` -- the clamped plate with the paper's conforming Bogner-Fox-Schmit
  element (bicubic Hermite: value, two first and the mixed derivative per node);
  no coefficient, square domain.

Layout of the per-element coefficient array ``kappa`` (float64, C order):

* p1_2d: shape (ny, nx, 2); [j, i, 0] is the triangle of square (i, j) below
  the SW->NE diagonal (vertices SW, SE, NE), [j, i, 1] the one above it
  (vertices SW, NE, NW).  The value is kappa at the triangle's centroid.
* p1_3d / q1_3d: shape (nz, ny, nx); one value per cube (kappa at the cube
  centre), shared by the cube's tetrahedra.
"""

from .specs import (
    ProblemSpec,
    kappa_field_2d,
    config_c1,
    config_c2,
    config_c2_scaled,
    config_c3,
    config_c4,
    config_c4_bfs,
    config_small_2d,
    config_small_3d,
    config_small_bfs,
    config_small_lshape,
    config_small_morley,
    config_table1_col1,
    config_table3_col1,
    config_table5,
    config_table7_col1,
    serving_stream,
)

__all__ = [
    "ProblemSpec",
    "kappa_field_2d",
    "config_c1",
    "config_c2",
    "config_c2_scaled",
    "config_c3",
    "config_c4",
    "config_c4_bfs",
    "config_small_2d",
    "config_small_3d",
    "config_small_bfs",
    "config_small_lshape",
    "config_small_morley",
    "config_table1_col1",
    "config_table3_col1",
    "config_table5",
    "config_table7_col1",
    "serving_stream",
]
