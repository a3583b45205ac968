"""Bounded device-side waits report BPJD_ERR_TIMEOUT and leave the context usable.

The local-solve kernels spin on an mbarrier until a bulk copy into shared memory
completes.  With the wait limit set to 0 attempts every such wait gives up at once:
the kernel flags the timeout, waits (with a fixed bound of its own) for its copies
still in flight, and returns, so nothing hangs and nothing faults.  The call reports
ERR_TIMEOUT; with the default limit restored the same handle solves again and
reproduces its earlier result bit for bit.
"""

import numpy as np
import pytest

from workloads import config_c1, config_small_3d

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2203_06327_gb300.binding")


# C1: band window 12 (tier 16: the several-shift tensor-core factorisation and the
# staged backward substitution, both with bulk copies); 24^3 P1 tetrahedra on 4^3
# subdomains: window 58 (tier 64: the wide factorisation, staged backward substitution)
@pytest.mark.parametrize("spec", [config_c1(), config_small_3d(n=24, ns=4)], ids=lambda s: s.name)
def test_wait_timeout_reported_and_context_usable(spec):
    pb = B.problem_from_spec(spec)
    sv = B.Solver.from_problem(pb, spec.k, device="cuda", precision=B.MIXED, subspace=B.W_3K)
    lay = sv.layout()
    assert lay["band_window"] <= 64
    lam0, X0, st0 = sv.solve()
    assert st0["converged"] == 1

    sv.set_wait_limit(0)
    with pytest.raises(B.BpjdError) as e:
        sv.solve()
    assert e.value.code == B.ERR_TIMEOUT
    k = spec.k
    rng = np.random.default_rng(3)
    rho = torch.tensor(rng.standard_normal((sv.n, k)), device="cuda")
    lam = torch.tensor(lam0 * 0.95, device="cuda")
    Z = torch.empty((sv.n, k), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BpjdError) as e:
        sv.apply_preconditioner(rho, lam, Z)
    assert e.value.code == B.ERR_TIMEOUT
    torch.cuda.synchronize()

    sv.set_wait_limit(1 << 22)
    lam1, X1, st1 = sv.solve()
    assert st1["converged"] == 1 and st1["iters"] == st0["iters"]
    np.testing.assert_array_equal(lam1, lam0)
    np.testing.assert_array_equal(X1, X0)
    sv.apply_preconditioner(rho, lam, Z)
    assert torch.isfinite(Z).all()
    with pytest.raises(B.BpjdError) as e:
        sv.set_wait_limit(-1)
    assert e.value.code == B.ERR_BAD_ARG
    sv.close()
