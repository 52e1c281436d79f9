"""The paper's test-case design (§5, Table 1) through the C ABI: every kind
T1…T6 at reduced size and at the paper's n = 4000, d = 6000, checked by the
FP64 oracle's KKT residual from A (relative ≤ tol), the reported residual
against the oracle's, and the objective against the convexity bound
F(x) − F* ≤ ∇F(x)ᵀ(x − x*) with x* the oracle's polished optimum."""
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


def _check(A, b, x, info, tol, polish=True):
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    rel, F = O.kkt_residual(A64, b64, x)
    assert rel <= tol, (rel, info)
    assert np.all(x >= 0.0)
    np.testing.assert_allclose(info.rel_kkt, rel, rtol=1e-4, atol=1e-15)
    if polish:
        xs, _, _, _ = O.reference_solution(A64, b64)
        Fs = O.nnls_objective(A64, b64, xs)
        gF = A64.T @ (A64 @ x - b64)
        assert F <= Fs + max(gF @ (x - xs), 0.0) + 1e-9 * max(Fs, 1e-300) + 1e-12


@pytest.mark.parametrize("kind", sorted(W.TCASES))
@pytest.mark.parametrize("sub", [0, 4])
def test_reduced_size_split(aln, kind, sub):
    P = W.tcase(kind, sub, n=400, d=600)
    with aln.Solver("split_bf16") as s:
        s.prepare(P.A, P.B)
        X, info = s.solve(tol=1e-6, max_iter=400000)
    _check(P.A, P.B[0], X[0], info[0], 1e-6)


@pytest.mark.parametrize("kind", ["T1", "T4", "T6"])
def test_reduced_size_fp64(aln, kind):
    P = W.tcase(kind, 2, n=300, d=450, dtype=np.float64)
    with aln.Solver("fp64") as s:
        s.prepare(P.A, P.B)
        X, info = s.solve(tol=1e-10, max_iter=400000)
    _check(P.A, P.B[0], X[0], info[0], 1e-10)


@pytest.mark.parametrize("kind", sorted(W.TCASES))
def test_paper_size(aln, kind):
    """n = 4000, d = 6000 (the paper's size), the 20%-sparse sub-test, in the
    launch configuration bench.py's paper_tcases workload times."""
    P = W.tcase(kind, 2)
    with aln.Solver("split_bf16") as s:
        s.prepare(P.A, P.B)
        X, info = s.solve(tol=1e-6, max_iter=400000)
    _check(P.A, P.B[0], X[0], info[0], 1e-6, polish=False)
