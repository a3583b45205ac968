"""Host-side checks of the CUDA library (no GPU needed): it loads, exports every
entry point declared in include/bpjd.h, its problem generators agree with the
oracle's (bit-exact patterns and index maps, values to 1e-15), and argument
validation in bpjd_setup rejects bad inputs before any device work."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import problem as oracle_problem
from workloads import (config_c1, config_small_2d, config_small_3d, config_small_bfs, config_small_lshape,
                       config_small_morley, config_table1_col1, config_table3_col1, config_table7_col1,
                       ProblemSpec)

B = pytest.importorskip("paper_2203_06327_gb300.binding")


def test_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "bpjd.h")) as f:
        text = f.read()
    declared = set(re.findall(r"\b(bpjd_[a-z_0-9]+)\s*\(", text))
    assert declared, "no declarations found"
    lib = C.CDLL(B.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(B.EXPORTED) <= declared


def _cmp_csr(lib_csr, ora, rel=2e-15):
    ora = ora.tocsr()
    ora.sort_indices()
    np.testing.assert_array_equal(lib_csr.row_ptr, ora.indptr)
    np.testing.assert_array_equal(lib_csr.col_idx, ora.indices)
    scale = np.abs(ora.data).max()
    np.testing.assert_allclose(lib_csr.val, ora.data, rtol=0, atol=rel * scale)


@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_3d(),
                                  config_small_3d(kind="q1_3d"), config_small_3d(n=16, ns=4, delta=2),
                                  config_small_morley(), config_small_morley(n=24, ns=4, delta=2, k=4, tau=1),
                                  config_small_morley(n=32, ns=8, delta=1, k=8),
                                  config_small_bfs(), config_small_bfs(n=24, ns=4, delta=2, k=4, tau=1),
                                  config_small_lshape(), config_table3_col1(), config_table7_col1()],
                         ids=lambda s: s.name + f"_tau{s.tau}")
def test_generators_match_oracle(spec):
    lp = B.problem_from_spec(spec)
    op = oracle_problem.build(spec)
    _cmp_csr(lp.K, op.K)
    _cmp_csr(lp.M, op.M)
    _cmp_csr(lp.P, op.P)
    _cmp_csr(lp.P0, op.P0)
    np.testing.assert_array_equal(lp.part.sub_ptr, op.sub_ptr)
    np.testing.assert_array_equal(lp.part.sub_dofs, op.sub_dofs)
    np.testing.assert_array_equal(lp.part.sub_color, op.sub_color)
    assert lp.part.n_colors == op.n_colors


def test_c2_generators_match_oracle_full_size():
    """The 261121-dof C2 workload: patterns and maps bit-exact at full size."""
    from workloads import config_c2
    spec = config_c2()
    lp = B.problem_from_spec(spec)
    from oracle import fem, partition
    K, M = fem.assemble(spec)
    _cmp_csr(lp.K, K)
    _cmp_csr(lp.M, M)
    ptr, dofs, col, nc = partition.box_partition(spec)
    np.testing.assert_array_equal(lp.part.sub_ptr, ptr)
    np.testing.assert_array_equal(lp.part.sub_dofs, dofs)


def test_c3_generators_match_oracle_full_size():
    """The 250047-dof C3 workload (P1 Kuhn tetrahedra on 64^3 cubes, 8^3 boxes, delta = 1):
    patterns, coarse interpolation and partition bit-exact, values to 4e-15."""
    from workloads import config_c3
    spec = config_c3()
    lp = B.problem_from_spec(spec)
    op = oracle_problem.build(spec)
    # a diagonal entry sums the contributions of 24 tetrahedra, added in different
    # orders by the two assemblies: up to 24 half-ulps (2.7e-15) relative
    _cmp_csr(lp.K, op.K, rel=4e-15)
    _cmp_csr(lp.M, op.M, rel=4e-15)
    P = op.P.tocsr()
    P.sort_indices()
    np.testing.assert_array_equal(lp.P.row_ptr, P.indptr)
    np.testing.assert_array_equal(lp.P.col_idx, P.indices)
    np.testing.assert_array_equal(lp.P.val, P.data)
    np.testing.assert_array_equal(lp.part.sub_ptr, op.sub_ptr)
    np.testing.assert_array_equal(lp.part.sub_dofs, op.sub_dofs)
    np.testing.assert_array_equal(lp.part.sub_color, op.sub_color)


def test_c4_generators_match_oracle_full_size():
    """The 261121-dof clamped plate (Morley): matrices, transfer and partition bit-exact."""
    from workloads import config_c4
    spec = config_c4()
    lp = B.problem_from_spec(spec)
    op = oracle_problem.build(spec)
    for a, b in ((lp.K, op.K), (lp.M, op.M), (lp.P, op.P)):
        b = b.tocsr()
        b.sort_indices()
        np.testing.assert_array_equal(a.row_ptr, b.indptr)
        np.testing.assert_array_equal(a.col_idx, b.indices)
        np.testing.assert_array_equal(a.val, b.data)
    np.testing.assert_array_equal(lp.part.sub_ptr, op.sub_ptr)
    np.testing.assert_array_equal(lp.part.sub_dofs, op.sub_dofs)
    np.testing.assert_array_equal(lp.part.sub_color, op.sub_color)


@pytest.mark.parametrize("n,S,rings", [(128, 16, 2), (128, 16, 3), (64, 8, 1), (96, 4, 5), (256, 16, 6),
                                        (48, 3, 0), (32, 2, 7)])
def test_triangle_partition_matches_oracle(n, S, rings):
    """Example 6.1's partition J_H (coarse squares cut along the SW->NE diagonal, each
    coarse triangle grown by rings of fine triangles): the library's generator and the
    oracle's, written independently from the same definition, agree bit for bit; the
    matrices and the coarse interpolation are those of the box partition."""
    from dataclasses import replace
    spec = replace(config_table1_col1(), n=(n, n), nsub=(S, S), delta=rings, k=min(4, (S - 1) ** 2 - 1),
                   partition="triangles")
    lp = B.problem_from_spec(spec)
    op = oracle_problem.build(spec)
    np.testing.assert_array_equal(lp.part.sub_ptr, op.sub_ptr)
    np.testing.assert_array_equal(lp.part.sub_dofs, op.sub_dofs)
    np.testing.assert_array_equal(lp.part.sub_color, op.sub_color)
    assert lp.part.n_colors == op.n_colors == 8
    assert len(lp.part.sub_ptr) - 1 == 2 * S * S
    box = B.problem_from_spec(replace(spec, partition="boxes"))
    for a, b in ((lp.K, box.K), (lp.M, box.M), (lp.P, box.P)):
        np.testing.assert_array_equal(a.col_idx, b.col_idx)
        np.testing.assert_array_equal(a.val, b.val)


def test_triangle_partition_rejects_bad_meshes():
    for args in [dict(kind="p1_2d", n=(64, 64), nsub=(8, 8), delta=4),      # 2 delta = n / nsub
                 dict(kind="p1_2d", n=(64, 32), nsub=(8, 4), delta=1),      # unequal axes
                 dict(kind="p1_3d", n=(8, 8, 8), nsub=(2, 2, 2), delta=1),  # not the P1 square grid
                 dict(kind="morley_2d", n=(16, 16), nsub=(4, 4), delta=1)]:
        L = (1.0,) * len(args["n"])
        with pytest.raises(B.BpjdError) as e:
            B.problem_create(args["kind"], args["n"], L, args["nsub"], args["delta"], partition="triangles")
        assert e.value.code == B.ERR_BAD_ARG


def test_problem_create_rejects_bad_mesh():
    with pytest.raises(B.BpjdError) as e:
        B.problem_create("p1_2d", (10, 10), (1.0, 1.0), (3, 3), 1)      # 10 not a multiple of 3
    with pytest.raises(B.BpjdError):
        B.problem_create("morley_2d", (16, 12), (1.0, 1.0), (4, 4), 1)  # Morley needs square cells
    with pytest.raises(B.BpjdError):
        B.problem_create("morley_2d", (16, 16), (1.0, 1.0), (4, 4), 1, kappa=np.ones((16, 16, 2)))
    with pytest.raises(B.BpjdError):
        B.problem_create("bfs_2d", (16, 16), (1.0, 2.0), (4, 4), 1)       # BFS needs square cells
    assert e.value.code == B.ERR_BAD_ARG


def _c1_arrays():
    return B.problem_from_spec(config_c1())


def test_setup_rejects_invalid_csr():
    pb = _c1_arrays()
    bad = B.CsrArrays(pb.K.n_rows, pb.K.n_cols, pb.K.row_ptr.copy(), pb.K.col_idx.copy(), pb.K.val)
    bad.col_idx[1], bad.col_idx[2] = bad.col_idx[2], bad.col_idx[1]           # unsorted row
    with pytest.raises(B.BpjdError) as e:
        B.Solver(bad, pb.M, pb.P, pb.P0, pb.part, 6)
    assert e.value.code == B.ERR_CSR_INVALID
    bad2 = B.CsrArrays(pb.K.n_rows, pb.K.n_cols, pb.K.row_ptr, pb.K.col_idx.copy(), pb.K.val)
    bad2.col_idx[5] = pb.K.n_cols                                              # out of range
    with pytest.raises(B.BpjdError) as e:
        B.Solver(bad2, pb.M, pb.P, pb.P0, pb.part, 6)
    assert e.value.code == B.ERR_CSR_INVALID


def test_setup_rejects_invalid_csr_in_any_row_range():
    """Host matrices with millions of entries are validated in row ranges on several threads:
    a defect in the first, a middle or the last row is found, whichever range holds it."""
    from workloads import config_c2
    pb = B.problem_from_spec(config_c2())
    K = pb.K
    n = K.n_rows
    for row in (0, n // 2 + 17, n - 1):
        ci = K.col_idx.copy()
        e = int(K.row_ptr[row])
        ci[e] = K.n_cols if row != n // 2 + 17 else ci[e + 1]      # out of range, or a repeated column
        bad = B.CsrArrays(n, K.n_cols, K.row_ptr, ci, K.val)
        with pytest.raises(B.BpjdError) as err:
            B.Solver(bad, pb.M, pb.P, pb.P0, pb.part, 12)
        assert err.value.code == B.ERR_CSR_INVALID, row


def test_setup_rejects_invalid_map_and_k():
    pb = _c1_arrays()
    dofs = pb.part.sub_dofs.copy()
    dofs[3], dofs[4] = dofs[4], dofs[3]
    part = B.PartitionArrays(pb.part.sub_ptr, dofs, pb.part.sub_color, 4)
    with pytest.raises(B.BpjdError) as e:
        B.Solver(pb.K, pb.M, pb.P, pb.P0, part, 6)
    assert e.value.code == B.ERR_MAP_INVALID
    with pytest.raises(B.BpjdError) as e:
        B.Solver(pb.K, pb.M, pb.P, None, pb.part, 9)                          # n_H = 9
    assert e.value.code == B.ERR_K_TOO_LARGE
    with pytest.raises(B.BpjdError) as e:
        B.Solver(pb.K, pb.M, pb.P, None, pb.part, 0)
    assert e.value.code == B.ERR_BAD_ARG


def test_setup_rejects_unknown_precision_and_subspace():
    """Precision must be FP64, MIXED or MIXED_LOCAL, the search space 2k or 3k; both are
    checked before any device work."""
    pb = _c1_arrays()
    for kw in ({"precision": 3}, {"precision": -1}, {"subspace": 2}):
        with pytest.raises(B.BpjdError) as e:
            B.Solver(pb.K, pb.M, pb.P, pb.P0, pb.part, 6, **kw)
        assert e.value.code == B.ERR_UNSUPPORTED
    assert (B.FP64, B.MIXED, B.MIXED_LOCAL) == (0, 1, 2)


def test_noalloc_gram_refuses_oversize_rows_before_any_launch():
    """The allocation-free block inner product indexes rows with 32-bit integers, so
    n > 2^31 - 1 is refused on the host (no device work: the fake pointers below are
    never dereferenced), as are the other size limits."""
    fn = B.lib.bpjd_block_gram_noalloc
    fn.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    fake = (C.c_void_p * 2)(0x1000, 0x2000)
    out = C.c_void_p(0x3000)
    assert fn(1 << 31, 4, 2, fake, 2, fake, 1, out, None) == B.ERR_TOO_LARGE
    assert fn((1 << 40) + 5, 1, 1, fake, 1, fake, 0, out, None) == B.ERR_TOO_LARGE
    # bad arguments come back as BAD_ARG, also before any launch
    assert fn(0, 4, 2, fake, 2, fake, 1, out, None) == B.ERR_BAD_ARG
    assert fn(100, 40, 2, fake, 2, fake, 1, out, None) == B.ERR_BAD_ARG      # 80 columns > 64
    assert fn(100, 4, 2, fake, 1, fake, 1, out, None) == B.ERR_BAD_ARG       # symmetric needs nu == nv
