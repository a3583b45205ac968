"""The allocation-free block inner product, bpjd_block_gram_noalloc.

It is meant for callers that cannot call cudaMalloc (their device memory is
owned by their own pool or arena, or an allocation's implicit synchronisation
is not acceptable where they call): it takes device inputs and output from the
caller and keeps its partial sums in a static device array.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
B = pytest.importorskip("paper_2203_06327_gb300.binding")

from workloads import config_small_2d  # noqa: E402


def _noalloc(n, k, U, V, out, symmetric):
    fn = B.lib.bpjd_block_gram_noalloc
    fn.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                   C.c_void_p]
    fn.restype = C.c_int
    pu = (C.c_void_p * len(U))(*[u.data_ptr() for u in U])
    pv = (C.c_void_p * len(V))(*[v.data_ptr() for v in V])
    stream = torch.cuda.current_stream().cuda_stream
    return fn(n, k, len(U), pu, len(V), pv, 1 if symmetric else 0, out.data_ptr(), stream)


def test_noalloc_gram_matches_block_gram_twice():
    spec = config_small_2d()
    pb = B.problem_from_spec(spec)
    sv = B.Solver.from_problem(pb, spec.k, device="cuda", precision=B.MIXED)
    n, k = sv.n, spec.k
    rng = np.random.default_rng(5)
    for call, (nu, sym) in enumerate([(3, True), (2, False)]):
        U = [torch.tensor(rng.standard_normal((n, k)), device="cuda") for _ in range(nu)]
        V = U if sym else [torch.tensor(rng.standard_normal((n, k)), device="cuda") for _ in range(3)]
        ref = torch.empty((nu * k, len(V) * k), dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        sv.block_gram(U, V, ref, symmetric=sym)
        assert _noalloc(n, k, U, V, got, sym) == B.OK
        torch.cuda.synchronize()
        Un = np.hstack([u.cpu().numpy() for u in U])
        Vn = np.hstack([v.cpu().numpy() for v in V])
        scale = np.abs(Un).T @ np.abs(Vn)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.abs(g - r) <= 1e-14 * scale), f"call {call}"
        assert np.all(np.abs(g - Un.T @ Vn) <= 1e-14 * scale), f"call {call}"


def test_noalloc_gram_rejects_oversize():
    """Four n x k blocks with n = 2^20, k = 16 (64 columns, the full tile set) need more
    partial sums than the static array holds.  The blocks are real (one 128 MiB tensor
    behind all four pointers) and so is the output, so that a broken size guard makes
    the assertion fail instead of reading past an allocation."""
    n, k = 1 << 20, 16
    block = torch.zeros((n, k), dtype=torch.float64, device="cuda")
    out = torch.zeros((4 * k, 4 * k), dtype=torch.float64, device="cuda")
    U = [block] * 4
    assert _noalloc(n, k, U, U, out, False) == B.ERR_TOO_LARGE
    del block
