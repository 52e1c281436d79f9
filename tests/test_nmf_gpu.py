"""NMF by alternating NNLS (aln_nmf) through the C ABI against the FP64
oracle in oracle/nmf.py.

Tolerances: every sub-problem is solved to relative KKT 1e-7 on the GPU and
1e-10 by the oracle, so each half-step's solution differs by about the GPU
tolerance relative to the data; over four outer iterations the objectives
agree to 1e-5 relative and the factors to 1e-3 (relative Frobenius norm).
The block-minimisation property (a non-increasing objective) holds up to the
same inexactness, 1e-6 relative per step."""
import numpy as np
import pytest

from oracle import nmf as N
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


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,r", [(120, 90, 6), (70, 130, 9), (40, 6, 3)])
def test_matches_oracle(aln, m, n, r):
    """Batched H- and W-steps (m, n ≥ batch_min), and a case with n below
    batch_min (the W-step's 40 rows batched, the H-step's 6 columns one by
    one)."""
    V, W0, H0 = W.nmf_matrix(m, n, r, seed=m + n)
    with aln.Solver("split_bf16") as s:
        Wg, Hg, obj = s.nmf(V, W0, H0, outer=4, tol=1e-7)
    Wo, Ho, objo = N.anls(V.astype(np.float64), W0, H0, outer=4, tol=1e-10)
    np.testing.assert_allclose(obj, objo, rtol=1e-5)
    assert _rel(Wg @ Hg, Wo @ Ho) <= 1e-3
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    # the reported objective is ½‖V − WH‖² of the returned factors
    assert obj[-1] == pytest.approx(N.objective(V.astype(np.float64), Wg, Hg), rel=1e-6)
    assert all(b <= a * (1 + 1e-6) for a, b in zip(obj, obj[1:])), obj


def test_final_w_step_is_optimal(aln):
    V, W0, H0 = W.nmf_matrix(150, 110, 8, seed=3)
    with aln.Solver("split_bf16") as s:
        Wg, Hg, obj = s.nmf(V, W0, H0, outer=3, tol=1e-7)
    V64 = V.astype(np.float64)
    for i in range(0, 150, 7):
        rel, _ = O.kkt_residual(Hg.T, V64[i, :], Wg[i, :])
        assert rel <= 1e-7 * 1.01, (i, rel)


def test_exact_factorisation_is_recovered(aln):
    g = np.random.default_rng(12)
    Ws = g.random((60, 4)) * (g.random((60, 4)) < 0.7)
    Hs = g.random((4, 50)) * (g.random((4, 50)) < 0.7)
    V = np.asfortranarray((Ws @ Hs).astype(np.float32))
    W0 = np.asfortranarray(Ws + 0.05 * g.random(Ws.shape))
    with aln.Solver("split_bf16") as s:
        Wg, Hg, obj = s.nmf(V, W0, np.ones((4, 50), order="F"), outer=30, tol=1e-9)
    assert obj[-1] <= 1e-6 * 0.5 * float(np.sum(V.astype(np.float64) ** 2)), obj[-1]


def test_device_inputs_match_host(aln):
    import torch
    V, W0, H0 = W.nmf_matrix(100, 80, 5, seed=21)
    with aln.Solver("split_bf16") as s:
        Wh, Hh, oh = s.nmf(V, W0, H0, outer=2, tol=1e-7)
    Vd = torch.from_numpy(np.ascontiguousarray(V.T)).cuda().t()
    Wd = torch.from_numpy(np.ascontiguousarray(W0.T)).cuda().t()
    Hd = torch.from_numpy(np.ascontiguousarray(H0.T)).cuda().t()
    with aln.Solver("split_bf16") as s:
        Wg, Hg, og = s.nmf(Vd, Wd, Hd, outer=2, tol=1e-7)
    np.testing.assert_array_equal(og, oh)
    np.testing.assert_array_equal(Wg.cpu().numpy(), Wh)
    np.testing.assert_array_equal(Hg.cpu().numpy(), Hh)


def test_errors(aln):
    V, W0, H0 = W.nmf_matrix(20, 16, 4, seed=2)
    with aln.Solver("split_bf16") as s:
        with pytest.raises(aln.AlnError) as e:       # r > min(m, n)
            s.nmf(V[:, :3].copy(order="F"), W0, H0[:, :3].copy(order="F"))
        assert e.value.code == aln.ERR_INVALID_ARG
        Vb = V.copy(order="F")
        Vb[3, 4] = np.nan
        with pytest.raises(aln.AlnError) as e:
            s.nmf(Vb, W0, H0)
        assert e.value.code == aln.ERR_NONFINITE


def test_full_size(aln):
    """The bench's 4096×4096, r = 64 matrix, 2 outer iterations: the objective
    falls, and sampled rows of the final W-step meet the KKT tolerance."""
    V, W0, H0 = W.nmf_matrix()
    with aln.Solver("split_bf16") as s:
        Wg, Hg, obj = s.nmf(V, W0, H0, outer=2, tol=1e-6)
    V64 = V.astype(np.float64)
    assert obj[1] <= obj[0] * (1 + 1e-6) and obj[0] < N.objective(V64, W0, H0)
    for i in range(0, 4096, 512):
        rel, _ = O.kkt_residual(Hg.T, V64[i, :], Wg[i, :])
        assert rel <= 1e-6 * 1.01, (i, rel)


def test_rank_one_and_fp64_context(aln):
    """r = 1 (scalar sub-problems), and a context in FP64 precision (each
    sub-problem by the FP64 method, one right-hand side at a time)."""
    V, W0, H0 = W.nmf_matrix(40, 30, 1, seed=31)
    Wo, Ho, objo = N.anls(V.astype(np.float64), W0, H0, outer=3, tol=1e-10)
    with aln.Solver("split_bf16") as s:
        Wg, Hg, obj = s.nmf(V, W0, H0, outer=3, tol=1e-8)
    np.testing.assert_allclose(obj, objo, rtol=1e-6)
    V2, W2, H2 = W.nmf_matrix(30, 20, 3, seed=32)
    Wo2, Ho2, objo2 = N.anls(V2.astype(np.float64), W2, H2, outer=2, tol=1e-11)
    with aln.Solver("fp64") as s:
        Wg2, Hg2, obj2 = s.nmf(V2, W2, H2, outer=2, tol=1e-11)
    # each half-step's matrix is the other factor rounded to FP32 (the input
    # type of V), so the sub-problems differ from the oracle's by ~6e-8
    np.testing.assert_allclose(obj2, objo2, rtol=1e-6)
