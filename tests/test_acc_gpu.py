"""Anti+Acc (§5) through the C ABI against the FP64 oracle in oracle/acc.py.

Tolerances (written here; the arithmetic behind them is in the design notes):
  * L = λ_max(Q): the power iteration stops when two quotients agree to 1e-7
    (FP64) or 1e-6 (FP32 products), so the CUDA and oracle estimates agree to
    about that; compared at 2e-6 (FP64) and 2e-5 (split-BF16, whose Q differs
    from the oracle's by the split bound).
  * FP64 trajectory: the first K iterates with each side's own L; the two L
    differ by ≤ 2e-6 relative and the accelerated map amplifies it slowly, so
    x_K is compared at 1e-5 relative.
  * Solutions: FP64 relative KKT from A at the requested tol; the objective
    within the convexity bound F(x) − F* ≤ ∇F(x)ᵀ(x − x*) of the oracle's
    polished optimum; at tol 1e-9 also x to 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import acc as AC
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


def _lopsided(d, n, seed, zero_frac=0.6, dtype=np.float32):
    r = np.random.default_rng(seed)
    A = r.random((d, n)) * np.exp(r.uniform(-2, 2, n))
    x = np.where(r.random(n) < zero_frac, 0.0, r.exponential(1.0, n))
    b = A @ x + 0.01 * np.linalg.norm(A @ x) / np.sqrt(d) * r.standard_normal(d)
    return np.asfortranarray(A.astype(dtype)), b.astype(dtype)


def _oracle_L(A, b):
    H, h = O.nqp_from_nnls(A.astype(np.float64), b.astype(np.float64))
    Q, q, s = O.antilopsided_scaling(H, h)
    rho, _ = AC.power_iteration(Q)
    return AC.step_constant(rho), Q, q, s


@pytest.mark.parametrize("prec,d,n,rtol", [("fp64", 400, 130, 2e-6), ("fp64", 90, 1, 2e-6),
                                            ("split_bf16", 900, 300, 2e-5),
                                            ("split_bf16", 3000, 1029, 2e-5)])
def test_lipschitz_matches_oracle(aln, prec, d, n, rtol):
    dt = np.float64 if prec == "fp64" else np.float32
    A, b = _lopsided(d, n, seed=d + n, dtype=dt)
    L, Q, q, s = _oracle_L(A, b)
    with aln.Solver(prec, algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, b)
        sv.solve(tol=1e-6)
        st = sv.stats()
    assert st.power_products >= 2
    assert abs(st.lipschitz - L) <= rtol * L, (st.lipschitz, L)
    assert st.lipschitz <= np.linalg.eigvalsh(Q).max() * (1 + 10 * rtol)


@pytest.mark.parametrize("K", [1, 2, 3, 25])
def test_fp64_trajectory_matches_oracle(aln, K):
    """The first K steps (no stop before K): x_K of the CUDA kernel against
    the oracle's x_K, each with its own L."""
    A, b = _lopsided(500, 200, seed=21, dtype=np.float64)
    L, Q, q, s = _oracle_L(A, b)
    with aln.Solver("fp64", algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, b)
        X, info = sv.solve(tol=1e-300, max_iter=K)
    assert info[0].iters == K and info[0].status == aln.RHS_MAXITER
    r = AC.solve_nqp_acc(Q, q, L, eps=0.0, max_iter=K)
    xo = O.unscale(r.y, s)
    np.testing.assert_allclose(X[0], xo, rtol=0, atol=1e-5 * np.abs(xo).max())


@pytest.mark.parametrize("prec,d,n,tol", [("split_bf16", 2000, 500, 1e-6),
                                           ("split_bf16", 700, 257, 1e-9),
                                           ("split_bf16", 130, 129, 1e-6),
                                           ("fp64", 600, 200, 1e-10)])
def test_solutions_meet_tolerance(aln, prec, d, n, tol):
    dt = np.float64 if prec == "fp64" else np.float32
    A, b = _lopsided(d, n, seed=3 * d + n, dtype=dt)
    with aln.Solver(prec, algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, b)
        X, info = sv.solve(tol=tol, max_iter=400000)
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    rel, F = O.kkt_residual(A64, b64, X[0])
    assert rel <= tol, (rel, info[0])
    assert info[0].status in (aln.RHS_CONVERGED, aln.RHS_EMPTY_PASSIVE)
    np.testing.assert_allclose(info[0].rel_kkt, rel, rtol=1e-4, atol=1e-15)
    xs, _, _, _ = O.reference_solution(A64, b64)
    Fs = O.nnls_objective(A64, b64, xs)
    # convexity: F(x) − F* ≤ ∇F(x)ᵀ(x − x*), ∇F = Aᵀ(Ax − b); and F ≥ F*
    gF = A64.T @ (A64 @ X[0] - b64)
    assert Fs * (1 - 1e-12) <= F <= Fs + max(gF @ (X[0] - xs), 0.0) + 1e-9 * Fs
    if tol < 1e-6:
        assert np.linalg.norm(X[0] - xs) <= 1e-6 * np.linalg.norm(xs)


def test_agrees_with_alg2_and_multi_rhs(aln):
    """Several right-hand sides (fewer than batch_min: both solvers take them
    one after another) reach the optimum Alg. 2 reaches."""
    A, _ = _lopsided(1200, 300, seed=5)
    r = np.random.default_rng(6)
    X0 = np.where(r.random((6, 300)) < 0.7, 0.0, r.exponential(1.0, (6, 300)))
    B = (X0 @ A.T.astype(np.float64)).astype(np.float32)
    with aln.Solver("split_bf16", algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, B)
        Xa, ia = sv.solve(tol=1e-9, max_iter=400000)
    with aln.Solver("split_bf16") as sv:
        sv.prepare(A, B)
        Xg, ig = sv.solve(tol=1e-9)
    for c in range(6):
        assert ia[c].rel_kkt <= 1e-9 and ig[c].rel_kkt <= 1e-9
        np.testing.assert_allclose(Xa[c], Xg[c], rtol=0, atol=1e-5 * np.abs(Xg[c]).max())


def test_edge_cases(aln):
    A, b = _lopsided(80, 30, seed=9)
    with aln.Solver("split_bf16", algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, np.zeros_like(b))                  # b = 0: x = 0, nothing passive
        X, info = sv.solve(tol=1e-8)
        assert np.all(X[0] == 0.0) and info[0].iters == 0
        assert info[0].status == aln.RHS_EMPTY_PASSIVE
        A1 = A[:, :1].copy(order="F")                   # n = 1
        sv.prepare(A1, b)
        X, info = sv.solve(tol=1e-10)
        xs = max(0.0, float(A1[:, 0].astype(np.float64) @ b.astype(np.float64)) /
                 float(A1[:, 0].astype(np.float64) @ A1[:, 0].astype(np.float64)))
        assert abs(X[0][0] - xs) <= 1e-7 * max(xs, 1e-30)
        Az = A.copy(order="F")                          # a zero column
        Az[:, 4] = 0.0
        sv.prepare(Az, b)
        X, info = sv.solve(tol=1e-8, max_iter=400000)
        rel, _ = O.kkt_residual(Az.astype(np.float64), b.astype(np.float64), X[0])
        assert rel <= 1e-8 and X[0][4] == 0.0
        # warm start at the solution: no step is needed
        sv.prepare(A, b)
        X, info = sv.solve(tol=1e-6, max_iter=400000)
        X2, info2 = sv.solve(tol=1e-6, X0=X)
        assert info2[0].iters == 0


def test_unsupported_combinations(aln):
    A, b = _lopsided(80, 30, seed=9)
    with aln.Solver("split_bf16", algorithm=aln.ALG_ANTI_ACC) as sv:
        with pytest.raises(aln.AlnError) as e:
            sv.prepare_grouped([(A, b), (A, b)])
        assert e.value.code == aln.ERR_UNSUPPORTED


def test_full_size_lopsided_single(aln):
    """The 20000×5000 lopsided problem in the launch configuration bench.py
    times with --algorithm anti_acc: FP64 KKT ≤ 1e-6 from A by the oracle,
    x ⪰ 0, and the reported residual matches the oracle's."""
    P = W.lopsided_single()
    A, b = P.A, P.B[0]
    with aln.Solver("split_bf16", algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, b)
        X, info = sv.solve(tol=1e-6, max_iter=400000)
        st = sv.stats()
    assert info[0].status == aln.RHS_CONVERGED and info[0].rel_kkt <= 1e-6
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    rel, F = O.kkt_residual(A64, b64, X[0])
    assert rel <= 1e-6 and np.all(X[0] >= 0.0)
    np.testing.assert_allclose(info[0].rel_kkt, rel, rtol=1e-4)
    assert st.lipschitz > 0.0 and st.power_products >= 2


def test_fp64_warm_start_and_several_rhs(aln):
    """FP64 Anti+Acc with three right-hand sides solved in turn, then
    restarted from the solutions (no step needed)."""
    A, _ = _lopsided(300, 90, seed=17, dtype=np.float64)
    r = np.random.default_rng(18)
    Xt = np.where(r.random((3, 90)) < 0.6, 0.0, r.random((3, 90)))
    B = Xt @ A.T
    with aln.Solver("fp64", algorithm=aln.ALG_ANTI_ACC) as sv:
        sv.prepare(A, B)
        X, info = sv.solve(tol=1e-10, max_iter=400000)
        X2, info2 = sv.solve(tol=1e-10, X0=X)
    for c in range(3):
        rel, _ = O.kkt_residual(A, B[c], X[c])
        assert rel <= 1e-10, (c, rel)
        assert info2[c].iters == 0
