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


def _solve_paper_rule(spec, scratch_gib):
    pb = B.problem_from_spec(spec)
    sv = B.Solver.from_problem(pb, spec.k, device="cuda", precision=B.MIXED_LOCAL, subspace=B.W_3K,
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
