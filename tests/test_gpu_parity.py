"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (derived from the arithmetic, see the design notes):
  * SpMM (FP64, <= 27 terms per entry): 1e-13 relative to the row-wise scale.
  * Preconditioner FP64: 1e-10 relative to max |z| (banded vs dense Cholesky of
    local matrices with condition ~ (H/h)^2 ~ 1e3..1e4).  MIXED (FP32 local
    solves): 2e-3 relative to max |z| (eps_32 times the local condition number).
  * Eigenvalues: 1e-10 relative (FP64 path), 1e-9 (mixed path); cluster
    subspace gap theta_b <= 1e-6; relative residual <= 1e-8.
"""

from dataclasses import replace

import numpy as np
import pytest
import scipy.linalg as la

from oracle import bpjd as obpjd
from oracle import metrics, problem as oproblem
from workloads import (config_c1, config_small_2d, config_small_3d, config_small_bfs, config_small_lshape,
                       config_small_morley, ProblemSpec)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2203_06327_gb300.binding")

DEV = "cuda"


def _solver(spec, device_inputs=True, **kw):
    pb = B.problem_from_spec(spec)
    return pb, B.Solver.from_problem(pb, spec.k, device=DEV if device_inputs else None, **kw)


@pytest.fixture(scope="module")
def c1_oracle():
    op = oproblem.build(config_c1())
    S = op.setup()
    return op, S


@pytest.mark.parametrize("ncols", [1, 6, 12, 16, 24])
def test_spmm_matches_oracle(c1_oracle, ncols):
    op, S = c1_oracle
    pb, sv = _solver(config_c1())
    X = np.random.default_rng(ncols).standard_normal((sv.n, ncols))
    Xd = torch.tensor(X, device=DEV)
    YA = torch.empty_like(Xd)
    YM = torch.empty_like(Xd)
    sv.spmm(Xd, YA, YM)
    torch.cuda.synchronize()
    for Y, A in ((YA, op.K), (YM, op.M)):
        ref = A @ X
        scale = abs(A) @ np.abs(X)
        assert np.all(np.abs(Y.cpu().numpy() - ref) <= 1e-13 * scale + 1e-300)


# band windows 14, 17, 31, 37, 43 (blocked tensor-core kernel, tiers 16..48), 58 and 92 (the
# several-warp blocked kernel, tiers 64 and 96), 111 (one CTA per pair, tier 128); Morley
# (clamped plate) windows 25, 49 and 145 (the last above every tier: shared-memory kernel)
@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_2d(nx=112, ny=112, nsx=4, nsy=4, delta=1),
                                  config_small_2d(nx=128, ny=128, nsx=4, nsy=4, delta=2), config_small_3d(),
                                  config_small_3d(kind="q1_3d"), config_small_3d(n=24, ns=4),
                                  config_small_3d(n=32, ns=4), config_small_3d(n=36, ns=4),
                                  config_small_morley(n=32, ns=8, delta=1, k=8),
                                  config_small_morley(n=32, ns=4, delta=2, k=6, tau=1),
                                  config_small_morley(n=128, ns=4, delta=2, k=2),
                                  config_small_bfs(), config_small_bfs(n=32, ns=8, delta=1, k=8)],
                         ids=lambda s: s.name)
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED], ids=["fp64", "mixed"])
def test_preconditioner_matches_oracle(spec, precision):
    op = oproblem.build(spec)
    S = op.setup()
    pb, sv = _solver(spec, precision=precision)
    k = spec.k
    rng = np.random.default_rng(7)
    rho = rng.standard_normal((sv.n, k))
    lam = np.sort(S.lam0H[:k]) * rng.uniform(0.9, 1.0, k)       # shifts below the initial Ritz values
    Z_ref = obpjd.apply_preconditioner(S, rho, lam)
    Zd = torch.empty((sv.n, k), dtype=torch.float64, device=DEV)
    sv.apply_preconditioner(torch.tensor(rho, device=DEV), torch.tensor(lam, device=DEV), Zd)
    Z = Zd.cpu().numpy()
    # FP32 local factorisations: forward error ~ sqrt(B) kappa eps_32 with kappa the (diagonally
    # scaled) condition number of K_l - lambda M_l: a few hundred for the second-order windows
    # here; about 4.3e4 for clamped-plate windows of 36 cells (fourth order: kappa ~ (H/h)^4),
    # i.e. sqrt(145) 4.3e4 6e-8 = 3e-2 at window 145 (Morley and BFS alike)
    if precision == B.FP64:
        tol = 1e-10
    elif spec.kind in ("morley_2d", "bfs_2d"):
        tol = 5e-2
    else:
        tol = 2e-3
    assert np.abs(Z - Z_ref).max() <= tol * np.abs(Z_ref).max()


@pytest.mark.parametrize("spec", [config_c1(), config_small_3d(n=32, ns=4),
                                  config_small_morley(n=128, ns=4, delta=2, k=8, tau=1)], ids=lambda s: s.name)
def test_mixed_local_preconditioner_equals_mixed(spec):
    """BPJD_MIXED_LOCAL runs the same FP32 local kernels and FP64 coarse term as BPJD_MIXED.
    The clamped-plate case has C4's local window (145, tier 152) on 128 (subdomain, shift)
    pairs with 373 MB of band records, and serves as the profiling case of that kernel."""
    op = oproblem.build(spec)
    S = op.setup()
    k = spec.k
    rng = np.random.default_rng(11)
    rho = torch.tensor(rng.standard_normal((op.K.shape[0], k)), device=DEV)
    lam = torch.tensor(np.sort(S.lam0H[:k]) * rng.uniform(0.9, 1.0, k), device=DEV)
    out = []
    for precision in (B.MIXED, B.MIXED_LOCAL):
        pb, sv = _solver(spec, precision=precision)
        Zd = torch.empty((sv.n, k), dtype=torch.float64, device=DEV)
        sv.apply_preconditioner(rho, lam, Zd)
        out.append(Zd.cpu().numpy())
        sv.close()
    np.testing.assert_array_equal(out[0], out[1])


def _check_solution(op, lam, X, lam_ref, V_ref, rtol):
    k = len(lam)
    np.testing.assert_allclose(lam, lam_ref[:k], rtol=rtol)
    assert metrics.rel_residuals(op.K, op.M, lam, X).max() <= 1e-8
    for a, b in metrics.clusters(lam_ref[:k]):
        assert metrics.gap_b(X[:, a:b], V_ref[:, a:b], op.M) <= 1e-6
    np.testing.assert_allclose(X.T @ (op.M @ X), np.eye(k), atol=1e-10)


@pytest.mark.parametrize("subspace", [B.W_2K, B.W_3K], ids=["W2k", "W3k"])
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED], ids=["fp64", "mixed"])
def test_c1_solve_matches_oracle(c1_oracle, subspace, precision):
    op, S = c1_oracle
    spec = config_c1()
    pb, sv = _solver(spec, precision=precision, subspace=subspace)
    lam, X, st = sv.solve()
    assert st["converged"] == 1
    w, V = la.eigh(op.K.toarray(), op.M.toarray())
    _check_solution(op, lam, X, w, V, 1e-10 if precision == B.FP64 else 1e-9)
    ref = obpjd.solve(S, tol=1e-8, subspace="2s" if subspace == B.W_2K else "3s")
    if precision == B.FP64:
        # same trajectory: iteration count and per-step Ritz values
        assert st["iters"] == ref.iterations
        H = sv.history()
        Hr = np.array(ref.history_lam)
        n = min(len(H), len(Hr))
        np.testing.assert_allclose(H[:n], Hr[:n], rtol=1e-9)
    else:
        assert abs(st["iters"] - ref.iterations) <= max(3, ref.iterations // 5)


@pytest.mark.parametrize("spec", [config_small_2d(), config_small_3d(), config_small_3d(kind="q1_3d"),
                                  config_small_2d(nx=40, ny=40, nsx=5, nsy=5, delta=1, k=1, kappa="random"),
                                  config_small_morley(n=32, ns=8, delta=1, k=8),
                                  config_small_morley(n=32, ns=4, delta=2, k=6, tau=1),
                                  config_small_bfs(), config_small_bfs(n=32, ns=8, delta=1, k=8),
                                  config_small_lshape()],
                         ids=lambda s: s.name)
def test_other_problems_solve(spec):
    op = oproblem.build(spec)
    w, V = la.eigh(op.K.toarray(), op.M.toarray())
    for precision in (B.FP64, B.MIXED, B.MIXED_LOCAL):
        pb, sv = _solver(spec, precision=precision, subspace=B.W_3K)
        lam, X, st = sv.solve()
        assert st["converged"] == 1
        _check_solution(op, lam, X, w, V, 1e-10 if precision == B.FP64 else 1e-9)


def test_host_inputs_and_device_eigvecs_agree():
    spec = config_small_2d()
    pb = B.problem_from_spec(spec)
    s_host = B.Solver.from_problem(pb, spec.k, device=None)
    s_dev = B.Solver.from_problem(pb, spec.k, device=DEV)
    l1, X1, _ = s_host.solve()
    l2, X2, _ = s_dev.solve(eigvecs="device")
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(X1, X2.cpu().numpy())
    # repeated solves restart from the initial guess and are bit-reproducible
    l3, X3, _ = s_host.solve()
    np.testing.assert_array_equal(l1, l3)
    np.testing.assert_array_equal(X1, X3)


def test_local_indefinite_reported():
    spec = replace(config_c1(), tau=0)
    pb, sv = _solver(spec)
    with pytest.raises(B.BpjdError) as e:
        sv.solve()
    assert e.value.code == B.ERR_LOCAL_INDEFINITE


def test_coarse_gap_reported():
    """Trilinear elements on a cube keep the exact multiplicities of the Laplacian (Table 5):
    the 2nd to 4th coarse eigenvalues coincide, so k = 2 violates Assumption 1 on V^H."""
    spec = replace(config_small_3d(kind="q1_3d"), k=2)
    pb = B.problem_from_spec(spec)
    with pytest.raises(B.BpjdError) as e:
        B.Solver.from_problem(pb, 2, device=DEV)
    assert e.value.code == B.ERR_GAP
    op = oproblem.build(spec)
    with pytest.raises(obpjd.CoarseGap):
        op.setup()


def test_paper_stop_rule():
    op = oproblem.build(config_c1())
    ref = obpjd.solve(op.setup(), tol=1e-10, stop="dlambda", subspace="3s")
    pb, sv = _solver(config_c1(), subspace=B.W_3K, stop_rule=B.STOP_DLAMBDA, tol=1e-10)
    lam, X, st = sv.solve()
    assert st["converged"] == 1 and st["sum_abs_dlambda"] < 1e-10
    assert st["iters"] == ref.iterations
    np.testing.assert_allclose(lam, ref.lam, rtol=1e-10)


def test_block_gram_matches_oracle_products():
    """bpjd_block_gram (double-word Dot2 products) against FP64 NumPy products."""
    spec = config_small_2d()
    pb, sv = _solver(spec, precision=B.MIXED)
    rng = np.random.default_rng(11)
    k = spec.k
    blocks = [rng.standard_normal((sv.n, k)) * 10.0 ** rng.integers(-3, 3) for _ in range(3)]
    U = [torch.tensor(b, device=DEV) for b in blocks]
    out = torch.empty((3 * k, 3 * k), dtype=torch.float64, device=DEV)
    sv.block_gram(U, U, out, symmetric=True)
    Wn = np.hstack(blocks)
    ref = Wn.T @ Wn
    scale = np.abs(Wn).T @ np.abs(Wn)
    assert np.all(np.abs(out.cpu().numpy() - ref) <= 1e-14 * scale)
    out2 = torch.empty((k, 2 * k), dtype=torch.float64, device=DEV)
    sv.block_gram(U[:1], U[1:], out2, symmetric=False)
    ref2 = blocks[0].T @ np.hstack(blocks[1:])
    scale2 = np.abs(blocks[0]).T @ np.abs(np.hstack(blocks[1:]))
    assert np.all(np.abs(out2.cpu().numpy() - ref2) <= 1e-14 * scale2)


@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_3d(n=24, ns=4),
                                  config_small_morley(n=32, ns=4, delta=2, k=6, tau=1)], ids=lambda s: s.name)
@pytest.mark.parametrize("precision", [B.FP64, B.MIXED], ids=["fp64", "mixed"])
def test_chunked_local_solves_bit_identical(spec, precision):
    """Local solves taken chunk by chunk of subdomains (a scratch bound of one byte:
    one subdomain per chunk) give exactly the results of one chunk: every (subdomain,
    shift) pair is factorised and solved independently of which pairs share a launch.
    (Exact shifts on both sides: factors are only reused when they are all resident.)"""
    pb = B.problem_from_spec(spec)
    ref = B.Solver.from_problem(pb, spec.k, device=DEV, precision=precision, subspace=B.W_3K,
                                local_refactor_tol=-1.0)
    one = B.Solver.from_problem(pb, spec.k, device=DEV, precision=precision, subspace=B.W_3K,
                                local_scratch_bytes=1, local_refactor_tol=-1.0)
    assert one.device_bytes() < ref.device_bytes()
    l0, X0, st0 = ref.solve()
    l1, X1, st1 = one.solve()
    assert st0["iters"] == st1["iters"]
    np.testing.assert_array_equal(l0, l1)
    np.testing.assert_array_equal(X0, X1)
    ref.close()
    one.close()


@pytest.mark.parametrize("spec", [config_c1(), config_small_2d(), config_small_3d(n=24, ns=4),
                                  config_small_morley(n=32, ns=4, delta=2, k=6, tau=1)], ids=lambda s: s.name)
def test_factor_reuse_gives_the_exact_shift_eigenpairs(spec):
    """Reusing the local factors while the shifts stay within 3e-4 (the default with FP32
    local solves), and even reusing the first factors for every later application
    (tolerance 1e30: the forward sweep on stored factors runs at every step), converge
    to the eigenpairs of the exact-shift solve (Eq. (3.3) at every application)."""
    pb = B.problem_from_spec(spec)
    op = oproblem.build(spec)
    res = {}
    for name, tol in (("exact", -1.0), ("default", 0.0), ("first", 1e30)):
        sv = B.Solver.from_problem(pb, spec.k, device=DEV, precision=B.MIXED, subspace=B.W_3K,
                                   local_refactor_tol=tol, max_iter=2000)
        res[name] = sv.solve()
        sv.close()
    l0, X0, st0 = res["exact"]
    for name in ("default", "first"):
        lam, X, st = res[name]
        assert st["converged"] == 1, name
        np.testing.assert_allclose(lam, l0, rtol=1e-9, err_msg=name)
        assert metrics.rel_residuals(op.K, op.M, lam, X).max() <= 1e-8, name
        for a, b in metrics.clusters(l0):
            if b < spec.k:
                assert metrics.gap_b(X[:, a:b], X0[:, a:b], op.M) <= 1e-6, (name, a, b)
    assert abs(res["default"][2]["iters"] - st0["iters"]) <= 2


@pytest.mark.parametrize("spec,precision,subspace,extra", [
    (config_c1(), B.MIXED, B.W_3K, {}),                                   # window tier 16: factor-reuse IF/ELSE
    (config_c1(), B.FP64, B.W_3K, {}),                                    # exact shifts, native FP64
    (config_c1(), B.MIXED, B.W_2K, {}),                                   # 2k space: the graph runs from step 0
    (config_small_3d(n=24, ns=4), B.MIXED, B.W_3K, {}),                   # wide tier 64
    (config_small_morley(n=32, ns=4, delta=2, k=6, tau=1), B.MIXED, B.W_3K, {}),   # shared-memory kernel
    (config_small_2d(), B.MIXED, B.W_3K, {"local_scratch_bytes": 1}),     # chunked local solves
    (config_c1(), B.MIXED, B.W_3K, {"stop_rule": B.STOP_DLAMBDA, "tol": 1e-10}),
    (config_c1(), B.MIXED, B.W_3K, {"max_iter": 5}),                      # step limit
], ids=["c1-mixed", "c1-fp64", "c1-2k", "cube24", "morley", "chunked", "dlambda", "maxiter"])
def test_graph_loop_equals_host_loop(spec, precision, subspace, extra, monkeypatch):
    """The iteration loop captured as one CUDA graph (stop test, step limit and factor-reuse
    decision taken on the device by kernels that set conditional nodes) runs the same
    kernels in the same order as the host-driven loop: bit-identical eigenpairs, Ritz-value
    history and iteration count; a second solve on the same handle reuses the graph."""
    pb = B.problem_from_spec(spec)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("BPJD_GRAPH", mode)
        sv = B.Solver.from_problem(pb, spec.k, device=DEV, precision=precision, subspace=subspace, **extra)
        lam, X, st = sv.solve(raise_on_noconv=False)
        hist = sv.history()
        lam2, X2, st2 = sv.solve(raise_on_noconv=False)
        np.testing.assert_array_equal(lam2, lam)
        np.testing.assert_array_equal(X2, X)
        assert st2["iters"] == st["iters"] and st2["status"] == st["status"]
        out[mode] = (lam, X, st, hist)
        sv.close()
    (lg, Xg, sg, hg), (le, Xe, se, he) = out["1"], out["0"]
    assert sg["iters"] == se["iters"] and sg["status"] == se["status"] and sg["converged"] == se["converged"]
    np.testing.assert_array_equal(lg, le)
    np.testing.assert_array_equal(Xg, Xe)
    np.testing.assert_array_equal(hg, he)
    if "max_iter" in extra:
        assert sg["status"] == B.ERR_NOCONV and sg["iters"] == extra["max_iter"]
