"""The serving entry points (bpjd_server_*): independent requests solved concurrently
on worker streams give exactly the results of the same requests solved one at a
time, errors stay with their request, and the memory budget is enforced."""

from dataclasses import replace

import numpy as np
import pytest

from workloads import config_c1, config_small_2d, config_small_3d, serving_stream

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2203_06327_gb300.binding")


def _alone(pb, k):
    sv = B.Solver.from_problem(pb, k, device=None, precision=B.MIXED, subspace=B.W_3K)
    lam, X, st = sv.solve()
    sv.close()
    return lam, X


def test_mixed_requests_match_solves_alone():
    specs = [config_c1(), config_small_2d(), config_small_3d(), config_small_3d(kind="q1_3d"),
             config_small_2d(nx=64, ny=64, nsx=4, nsy=4, delta=2, k=7),
             config_small_2d(nx=40, ny=40, nsx=5, nsy=5, delta=1, k=1, kappa="random")]
    pbs = [B.problem_from_spec(s) for s in specs]
    srv = B.Server(workers=3)
    try:
        tickets = [srv.submit(pb, s.k) for pb, s in zip(pbs, specs)]
        results = [srv.poll(t) for t in tickets]
    finally:
        srv.close()
    for pb, s, (rc, lam, X, st, times) in zip(pbs, specs, results):
        assert rc == B.OK, (s.name, rc)
        assert st["converged"] == 1
        assert times[0] >= 0 and times[1] > 0 and times[2] >= times[1]
        lam1, X1 = _alone(pb, s.k)
        np.testing.assert_array_equal(lam, lam1)
        np.testing.assert_array_equal(X, X1)


def test_serving_stream_requests_solve():
    """The first requests of the seeded serving stream (mixed sizes and k)."""
    reqs = serving_stream(6, seed=0)
    srv = B.Server(workers=4)
    try:
        tickets = [(r, srv.submit(B.problem_from_spec(r.spec), r.spec.k)) for r in reqs]
        for r, t in tickets:
            rc, lam, X, st, times = srv.poll(t)
            assert rc == B.OK, r.spec.name
            assert st["max_rel_resid"] <= 1e-8
            assert np.all(np.diff(lam) >= 0)
    finally:
        srv.close()


def test_serving_stream_requests_match_reference_eigenpairs():
    """The first 8 requests of the seeded serving stream (P1 on 64..512 squares, random
    smooth kappa, k in 4..16) solved by the server, each checked against the k lowest
    generalised eigenpairs of the oracle's own assembly of the same request (dense eigh
    below 4000 dofs, shift-invert eigsh above): eigenvalues to 1e-9 relative, cluster
    subspace gaps <= 1e-6, relative residuals <= 1e-8, X^T M X = I."""
    import scipy.linalg as la
    import scipy.sparse.linalg as sla
    from oracle import metrics, problem as oproblem
    reqs = serving_stream(8, seed=0)
    srv = B.Server(workers=4)
    try:
        tickets = [(r, srv.submit(B.problem_from_spec(r.spec), r.spec.k)) for r in reqs]
        results = [(r, srv.poll(t)) for r, t in tickets]
    finally:
        srv.close()
    for r, (rc, lam, X, st, times) in results:
        assert rc == B.OK, r.spec.name
        k = r.spec.k
        op = oproblem.build(r.spec)
        K, M = op.K.tocsr(), op.M.tocsr()
        if K.shape[0] < 4000:
            w, V = la.eigh(K.toarray(), M.toarray(), subset_by_index=[0, k])
        else:
            w, V = sla.eigsh(K.tocsc(), k + 4, M.tocsc(), sigma=0.0, which="LM", tol=1e-13,
                             v0=np.random.default_rng(0).standard_normal(K.shape[0]))
            order = np.argsort(w)
            w, V = w[order], V[:, order]
        np.testing.assert_allclose(lam, w[:k], rtol=1e-9, err_msg=r.spec.name)
        assert metrics.rel_residuals(K, M, lam, X).max() <= 1e-8, r.spec.name
        for a, b in metrics.clusters(w[: k + 1]):
            if b <= k:
                assert metrics.gap_b(X[:, a:b], V[:, a:b], M) <= 1e-6, (r.spec.name, a, b)
        np.testing.assert_allclose(X.T @ (M @ X), np.eye(k), atol=1e-10)


def test_errors_stay_with_their_request():
    bad = replace(config_c1(), tau=0)   # first local shifted matrices indefinite
    good = config_small_2d()
    srv = B.Server(workers=2)
    try:
        t_bad = srv.submit(B.problem_from_spec(bad), bad.k)
        t_good = srv.submit(B.problem_from_spec(good), good.k)
        assert srv.poll(t_bad)[0] == B.ERR_LOCAL_INDEFINITE
        assert srv.poll(t_good)[0] == B.OK
        with pytest.raises(KeyError):
            srv.poll(t_bad)
    finally:
        srv.close()


def test_budget_rejects_oversize_request():
    srv = B.Server(workers=1, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(B.BpjdError) as e:
            srv.submit(B.problem_from_spec(config_c1()), 6)
        assert e.value.code == B.ERR_TOO_LARGE
    finally:
        srv.close()


def test_local_solves_share_launches_across_requests():
    """With batch_local (the default) the local solves of the requests in flight run in
    shared grouped launches, one per kernel kind and window tier (here tiers 16, 24 and the
    wide tier 64), so there are fewer launch groups than preconditioner applications; every
    request's result is bitwise that of the same request served with packing off and of the
    request solved alone."""
    specs = [config_c1(), replace(config_c1(), k=5), config_small_2d(),
             config_small_2d(nx=64, ny=64, nsx=4, nsy=4, delta=2, k=7),
             config_small_2d(nx=64, ny=64, nsx=8, nsy=8, delta=2, k=4), config_small_3d(n=24, ns=4)]
    pbs = [B.problem_from_spec(s) for s in specs]
    out = {}
    for batch in (True, False):
        srv = B.Server(workers=len(specs), batch_local=batch, batch_wait_us=2000)
        try:
            tickets = [srv.submit(pb, s.k) for pb, s in zip(pbs, specs)]
            results = [srv.poll(t) for t in tickets]
            out[batch] = (results, srv.batch_stats())
        finally:
            srv.close()
    (packed, (groups, apps)), (plain, stats_off) = out[True], out[False]
    assert stats_off == (0, 0)
    assert 0 < groups < apps, (groups, apps)
    for pb, s, r1, r0 in zip(pbs, specs, packed, plain):
        assert r1[0] == B.OK and r0[0] == B.OK, s.name
        np.testing.assert_array_equal(r1[1], r0[1])
        np.testing.assert_array_equal(r1[2], r0[2])
        assert r1[3]["iters"] == r0[3]["iters"]
        lam1, X1 = _alone(pb, s.k)
        np.testing.assert_array_equal(r1[1], lam1)
        np.testing.assert_array_equal(r1[2], X1)
