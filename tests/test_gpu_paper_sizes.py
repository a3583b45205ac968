"""The paper's experiments at its larger mesh sizes, on the GPU (Section 6).

Every printed eigenvalue of the larger columns of Tables 1, 3, 5 and 7 is reproduced
to 8 decimals by the library's own assembly of the same discretisation, solved with
the paper's stop rule sum_i |lambda_i^{k+1} - lambda_i^k| < 1e-10 (Algorithm 3.1
Step 4) with FP32 local solves and every other step in FP64 (BPJD_MIXED_LOCAL): the
rule is absolute, summed over 19 or 20 eigenvalues, and with the double-word products
of BPJD_MIXED it was not met within 300 iterations on the million-dof mesh of Table 1
(the relative-residual rule of the other tests is met there as everywhere).  The
printed eigenvalues do not depend on the subdomain
decomposition; the boxes used here keep each local band within the library's
kernel tiers (the paper's N = 512 triangles with delta / H = 1/4 would give local
problems of 10^4..10^5 dofs at these sizes).  The iteration counts are printed beside
the paper's (they depend on the decomposition: Tables 2, 4 and 6 show them falling
with N).  Tolerance: 6e-9 absolute (half a unit in the 8th decimal plus the solve's
eigenvalue error).
"""

from dataclasses import replace

import numpy as np
import pytest

from conftest import golden
from workloads import config_table1_col1, config_table3_col1, config_table5, config_table7_col1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2203_06327_gb300.binding")


def _solve_paper_rule(spec, scratch_gib, precision=None):
    pb = B.problem_from_spec(spec)
    sv = B.Solver.from_problem(pb, spec.k, device="cuda", precision=precision or B.MIXED_LOCAL, subspace=B.W_3K,
                               stop_rule=B.STOP_DLAMBDA, tol=1e-10, max_iter=300,
                               local_scratch_bytes=int(scratch_gib * (1 << 30)))
    lam, X, st = sv.solve(eigvecs=None)
    sv.close()
    del pb
    torch.cuda.empty_cache()
    return lam, st


# Table 1 (Example 6.1, P1 on (0, pi)^2, s = 19): columns 3-5 (261121, 1046529 and
# 4190209 dofs), boxes of 32 x 32 elements with delta = 8 layers (delta / H = 1/4 as in
# the paper); the paper prints 22 iterations for each with N = 512.
@pytest.mark.parametrize("col,n", [(2, 512), (3, 1024), (4, 2048)])
def test_table1_larger_columns(col, n):
    spec = replace(config_table1_col1(), n=(n, n), nsub=(n // 32, n // 32), delta=8, name=f"table1_n{n}")
    lam, st = _solve_paper_rule(spec, 64)
    want = np.array([r[col] for r in golden("table1.txt")])
    print(f"Table 1 column {col + 1}: {spec.n_dofs} dofs, {st['iters']} iterations (paper: 22)")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


# Table 3 (Example 6.2, P1 on the L-shaped domain, s = 20): columns 3-4 (195585 and
# 784385 dofs), boxes of 32 x 32 elements, delta = 8 (delta / H = 1/4); the paper prints
# 21 iterations for each with N = 384.
@pytest.mark.parametrize("col,n", [(2, 512), (3, 1024)])
def test_table3_larger_columns(col, n):
    spec = replace(config_table3_col1(), n=(n, n), nsub=(n // 32, n // 32), delta=8, name=f"table3_n{n}")
    lam, st = _solve_paper_rule(spec, 32)
    want = np.array([r[col] for r in golden("table3.txt")])
    print(f"Table 3 column {col + 1}: {spec.n_dofs} dofs, {st['iters']} iterations (paper: 21)")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


# Table 5 (Example 6.3, trilinear elements on (0, pi)^3, s = 20): columns 3-4 (250047 and
# 2048383 dofs), boxes of 8^3 elements with delta = 1 layer; the paper prints 16 and 17
# iterations with N = 512 and delta / H = 1/2.
@pytest.mark.parametrize("col,n", [(2, 64), (3, 128)])
def test_table5_larger_columns(col, n):
    spec = replace(config_table5(n), nsub=(n // 8,) * 3, delta=1, name=f"table5_n{n}")
    lam, st = _solve_paper_rule(spec, 32)
    want = np.array([r[col] for r in golden("table5.txt")])
    print(f"Table 5 column {col + 1}: {spec.n_dofs} dofs, {st['iters']} iterations (paper: {[16, 17][col - 2]})")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


# Table 7 (Example 6.4, trilinear elements on the L-shaped prism, s = 20): columns 2-3
# (91295 and 758079 dofs) on the paper's N = 1536 subdomain boxes, delta = 2 and 1 layers
# (delta / H = 1/2 and 1/8); the paper prints 17 and 18 iterations with delta / H = 1/2.
@pytest.mark.parametrize("col,scale,delta", [(1, 2, 2), (2, 4, 1)])
def test_table7_larger_columns(col, scale, delta):
    base = config_table7_col1()
    spec = replace(base, n=tuple(m * scale for m in base.n), delta=delta, name=f"table7_x{scale}")
    lam, st = _solve_paper_rule(spec, 32)
    want = np.array([r[col] for r in golden("table7.txt")])
    print(f"Table 7 column {col + 1}: {spec.n_dofs} dofs, {st['iters']} iterations (paper: {[15, 17, 18][col]})")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


# ---- the paper's own partition of Example 6.1 (N = 2 S^2 coarse triangles) ----------
# delta / H = 1/4 with H the diameter sqrt(2) pi / S of a coarse triangle and h = pi / n
# is sqrt(2) n / (4 S) fine steps; the enlargement by whole rings of fine triangles takes
# the nearest integer.

def _rings(n, S):
    return int(round(2 ** 0.5 * n / (4 * S)))


@pytest.mark.parametrize("rings,its_oracle", [(2, 22), (3, 20)])
def test_table1_first_column_on_the_paper_partition(rings, its_oracle):
    """Table 1, first column (16129 dofs) on the paper's 512 coarse triangles, in FP64: the
    iteration count under the paper's stop rule equals the oracle's on the same partition
    (22 with 2 rings, 20 with 3; delta / H = 1/4 is 2.83 fine steps, so the two bracket the
    printed 21), and every printed eigenvalue is reproduced to 8 decimals."""
    spec = replace(config_table1_col1(), nsub=(16, 16), delta=rings, partition="triangles",
                   name=f"table1_tri_r{rings}")
    lam, st = _solve_paper_rule(spec, 4, precision=B.FP64)
    want = np.array([r[0] for r in golden("table1.txt")])
    print(f"Table 1 column 1, 512 triangles, {rings} rings: {st['iters']} iterations (paper: 21)")
    assert st["converged"] == 1
    assert st["iters"] == its_oracle
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


# Table 1, columns 2-4 (65025, 261121 and 1046529 dofs) on the paper's N = 512 triangles with
# delta / H = 1/4 (6, 11 and 23 rings); the paper prints 22 iterations for each.
@pytest.mark.parametrize("col,n", [(1, 256), (2, 512), (3, 1024)])
def test_table1_columns_on_the_paper_partition(col, n):
    spec = replace(config_table1_col1(), n=(n, n), nsub=(16, 16), delta=_rings(n, 16), partition="triangles",
                   name=f"table1_tri_n{n}")
    lam, st = _solve_paper_rule(spec, 64)
    want = np.array([r[col] for r in golden("table1.txt")])
    print(f"Table 1 column {col + 1}, 512 triangles, {spec.delta} rings: {spec.n_dofs} dofs, "
          f"{st['iters']} iterations (paper: 22)")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


def test_iterations_fall_with_the_number_of_subdomains():
    """Table 2's experiment (iterations against N with delta / H = 1/4 fixed) on Table 1's
    1046529-dof mesh: N = 512, 2048 and 8192 coarse triangles (23, 11 and 6 rings).  The
    paper prints 22 / 18 / 16 at 16769025 dofs; here the counts must not grow with N, and the
    eigenvalues are Table 1's fourth column to 8 decimals."""
    want = np.array([r[3] for r in golden("table1.txt")])
    its = []
    for S in (16, 32, 64):
        spec = replace(config_table1_col1(), n=(1024, 1024), nsub=(S, S), delta=_rings(1024, S),
                       partition="triangles", name=f"table2_tri_S{S}")
        lam, st = _solve_paper_rule(spec, 64)
        print(f"N = {2 * S * S} triangles, {spec.delta} rings: {st['iters']} iterations")
        assert st["converged"] == 1
        np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)
        its.append(st["iters"])
    print(f"iterations for N = 512 / 2048 / 8192: {its} (paper, 16769025 dofs: 22 / 18 / 16)")
    assert its[0] >= its[1] >= its[2], its


def test_table1_sixth_column_on_the_paper_partition():
    """Table 1's sixth column (16769025 dofs) on the paper's partition with N = 8192 coarse
    triangles (23 rings, delta / H = 1/4), the last entry of Table 2 (16 iterations in the
    paper): every printed eigenvalue to 8 decimals.  The local factors of all 8192 x 19
    (subdomain, shift) pairs exceed the 32 GiB scratch bound, so the local solves run in
    chunks and factorise at every application."""
    n, S = 4096, 64
    spec = replace(config_table1_col1(), n=(n, n), nsub=(S, S), delta=_rings(n, S), partition="triangles",
                   name="table1_tri_n4096")
    lam, st = _solve_paper_rule(spec, 32)
    want = np.array([r[5] for r in golden("table1.txt")])
    print(f"Table 1 column 6, N = 8192 triangles, {spec.delta} rings: {spec.n_dofs} dofs, "
          f"{st['iters']} iterations (paper, Table 2: 16)")
    assert st["converged"] == 1
    np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)


def test_iterations_fall_with_the_number_of_subdomains_lshape():
    """Table 4's experiment (iterations against N at delta / H = 1/4 fixed) on the L-shaped
    domain, on Table 3's 784385-dof mesh: the boxes of the 16 x 16, 32 x 32 and 64 x 64 grids
    over the square that lie in the domain (192, 768 and 3072 subdomains; the paper's N = 384,
    1536 and 6144 triangles are the halves of such squares), delta = 16, 8 and 4 layers.  The
    paper prints 21 / 18 / 16 at 12574721 dofs; here the counts must not grow with N, and the
    eigenvalues are Table 3's fourth column to 8 decimals."""
    want = np.array([r[3] for r in golden("table3.txt")])
    its = []
    for S in (16, 32, 64):
        spec = replace(config_table3_col1(), n=(1024, 1024), nsub=(S, S), delta=1024 // (4 * S),
                       name=f"table4_S{S}")
        lam, st = _solve_paper_rule(spec, 32)
        print(f"{S} x {S} boxes over the square, delta = {spec.delta}: {st['iters']} iterations")
        assert st["converged"] == 1
        np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)
        its.append(st["iters"])
    print(f"iterations for 192 / 768 / 3072 boxes: {its} (paper, 12574721 dofs, N = 384 / 1536 / 6144: 21 / 18 / 16)")
    assert its[0] >= its[1] >= its[2], its


def test_iterations_fall_with_the_number_of_subdomains_prism():
    """Table 8's experiment (iterations against N) on the L-shaped prism, on Table 7's
    758079-dof mesh: the paper's N = 1536 and 12288 cubes of sides pi/8 and pi/16, with
    delta / H = 1/4 for both (2 and 1 layers; the paper's 1/2 would give the 1536 cubes local
    bands beyond the kernel tiers).  The paper prints 18 / 15 at 6177407 dofs; here the count
    must not grow with N, and the eigenvalues are Table 7's third column to 8 decimals."""
    base = config_table7_col1()
    want = np.array([r[2] for r in golden("table7.txt")])
    its = []
    for f, delta in ((1, 2), (2, 1)):
        spec = replace(base, n=tuple(m * 4 for m in base.n), nsub=tuple(m * f for m in base.nsub), delta=delta,
                       name=f"table8_N{1536 * f ** 3}")
        lam, st = _solve_paper_rule(spec, 32)
        print(f"N = {1536 * f ** 3} cubes, delta = {delta}: {st['iters']} iterations")
        assert st["converged"] == 1
        np.testing.assert_allclose(lam, want, rtol=0, atol=6e-9)
        its.append(st["iters"])
    print(f"iterations for N = 1536 / 12288: {its} (paper, 6177407 dofs, delta / H = 1/2: 18 / 15)")
    assert its[0] >= its[1], its
