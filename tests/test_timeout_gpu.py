"""The bounded device wait of the persistent Alg. 2 kernel, made to expire.

Every grid barrier of the persistent solver kernels gives up after
aln_options.wait_limit_us: the kernel stops every block (no copies or
tensor-core work are in flight in these kernels) and aln_solve reports
ALN_ERR_TIMEOUT instead of hanging.  The test knob test_barrier_skew makes
each barrier wait for arrivals that never come, so the limit (1 ms here)
runs out on the first barrier — no fault, no trap, no endless loop.  Then the
same context, with the knob back at 0, must solve the problem to the oracle's
answer.
"""
import time

import numpy as np
import pytest

from oracle import nnls as O
from paper_1502_01645_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aln():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_01645_gb300 import build_lib, aln as binding
    build_lib.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def problem():
    p = W.lopsided_single(d=1200, n=300, seed=31)
    A64, b64 = p.A.astype(np.float64), p.B[0].astype(np.float64)
    x_star = O.reference_solution(A64, b64)[0]
    return p, A64, b64, x_star


@pytest.mark.parametrize("prec,kernel", [("split_bf16", 2), ("fp64", 2), ("split_bf16", 1)])
def test_expired_barrier_wait_returns_timeout_then_context_solves(aln, problem, prec, kernel):
    p, A64, b64, x_star = problem
    A = p.A if prec == "split_bf16" else A64
    b = p.B[0] if prec == "split_bf16" else b64
    with aln.Solver(prec, iter_kernel=kernel) as s:
        s.prepare(A, b)
        s.set_wait_limit(1000, 1)          # 1 ms, one arrival that never comes
        t0 = time.perf_counter()
        with pytest.raises(aln.AlnError) as e:
            s.solve(tol=1e-9)
        assert e.value.code == aln.ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0   # gave up, did not hang
        s.set_wait_limit(0, 0)             # back to normal on the same context
        X, info = s.solve(tol=1e-9)
    rel, _ = O.kkt_residual(A64, b64, X[0])
    assert info[0].status == aln.RHS_CONVERGED
    assert rel <= 1e-9
    assert np.linalg.norm(X[0] - x_star) <= 1e-5 * np.linalg.norm(x_star)


def test_timeout_option_at_create(aln, problem):
    p, A64, b64, _ = problem
    with aln.Solver("split_bf16", wait_limit_us=2000, test_barrier_skew=3) as s:
        s.prepare(p.A, p.B[0])
        with pytest.raises(aln.AlnError) as e:
            s.solve(tol=1e-6)
        assert e.value.code == aln.ERR_TIMEOUT
        s.set_wait_limit(0, 0)
        X, info = s.solve(tol=1e-6)
    assert O.kkt_residual(A64, b64, X[0])[0] <= 1e-6
