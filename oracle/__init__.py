"""Plain FP64 CPU oracle of the two-level BPJD eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only the test-suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` use it.  It shares
no code with the CUDA library: it has its own finite-element assembly, its own
subdomain partition and coarse interpolation, and its own BPJD iteration,
written in NumPy/SciPy double precision for readability rather than speed.

Modules
  fem        finite-element stiffness/mass assembly (Section 2.2, Section 6)
  morley     Morley elements for the clamped plate (Section 2.1, m = 2): assembly,
             intergrid transfer V^H -> V^h, half-grid dof numbering
  bfs        Bogner-Fox-Schmit elements for the clamped plate (Section 2.2, m = 2):
             tensor-product assembly and the nested coarse interpolation
  partition  overlapping box subdomains and colouring (Section 2.3, Assumption 2)
  coarse     nodal interpolation from the coarse space V^H (Section 2.3)
  bpjd       the two-level BPJD method (Section 3, Algorithm 3.1, Eq. (3.3))
  metrics    gap between subspaces (Definition 2.1), residuals, clusters

Every function cites the passage it follows.  Functions without an external
pin are marked "parity unpinned" in their docstrings.  Pins by module:
fem, coarse, partition -> tests/test_oracle_fem.py,
tests/test_oracle_partition_coarse.py, tests/test_oracle_lshape.py (paper
tables, closed forms, brute force); morley -> tests/test_oracle_morley.py;
bfs -> tests/test_oracle_bfs.py; bpjd -> tests/test_oracle_bpjd.py (dense
eigensolves, textbook reductions, paper iteration counts); metrics ->
tests/test_oracle_metrics.py (hand-computed angles and residuals, principal
angles of scipy on the Cholesky-transformed spans, hand-made clusters).
"""
