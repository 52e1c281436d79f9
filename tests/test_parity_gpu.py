"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (written here, derived in the design notes):
  * FP64 path: Q, q, s to 1e-12 relative; solutions |ΔF|/F* ≤ 1e-10 and
    ‖Δx‖∞/‖x*‖∞ ≤ 1e-8 against the oracle's polished optimum.
  * Split-BF16 Gram (exact three-term split a = h + m + l, six products):
    |ΔQ_ij| ≤ 2⁻²² (dropped m·l, l·m, l·l terms) + 3·d·2⁻²⁴ (FP32
    accumulation bound) + 2⁻²³ (scaling), mean |ΔQ| ≤ 1e-6; q and s are FP64
    (1e-12).
  * Mixed-precision solutions: FP64 relative KKT ≤ 1e-6 and
    ‖Δx‖₂/‖x*‖₂ ≤ 1e-5.
"""
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


def _oracle_scaled(A, b):
    H, h = O.nqp_from_nnls(A, b)
    return O.antilopsided_scaling(H, h)


def _split_bound(d):
    return 2.0 ** -22 + 3 * d * 2.0 ** -24 + 2.0 ** -23


# ----------------------------------------------------------------- Alg. 1 rows
@pytest.mark.parametrize("d,n", [(300, 200), (129, 65), (50, 1), (40, 257)])
def test_fp64_scaled_problem_matches_oracle(aln, d, n):
    r = np.random.default_rng(d * 1000 + n)
    A = np.asfortranarray(r.random((d, n)))
    b = r.standard_normal(d)
    with aln.Solver("fp64") as s:
        s.prepare(A, b)
        Q, q, sc = s.export()
    Qo, qo, so = _oracle_scaled(A, b)
    np.testing.assert_allclose(sc, so, rtol=1e-13)
    np.testing.assert_allclose(Q, Qo, atol=1e-12)
    np.testing.assert_allclose(q[0], qo, atol=1e-12 * np.abs(qo).max())
    np.testing.assert_array_equal(np.diag(Q), 1.0)


@pytest.mark.parametrize("d,n", [(700, 300), (64, 128), (1000, 129), (130, 1), (257, 400),
                                 (1500, 2304)])
def test_split_bf16_gram_matches_oracle(aln, d, n):
    """tcgen05 Gram: several 128-tiles plus a ragged tail in n and in d;
    n = 2304 has 171 tile pairs, more than one wave, so the pairs past the
    last full wave run as stream-K (pairs split over several CTAs and summed
    from partial tiles)."""
    r = np.random.default_rng(7 * d + n)
    A64 = r.random((d, n)) * np.exp(r.uniform(np.log(1e-2), np.log(1e2), n))[None, :]
    A = np.asfortranarray(A64.astype(np.float32))
    b = (A.astype(np.float64) @ r.random(n)).astype(np.float32)
    with aln.Solver("split_bf16") as s:
        s.prepare(A, b)
        Q, q, sc = s.export()
    Qo, qo, so = _oracle_scaled(A, b)
    np.testing.assert_allclose(sc, so, rtol=1e-13)
    np.testing.assert_allclose(q[0], qo, atol=1e-12 * np.abs(qo).max())
    err = np.abs(Q - Qo)
    assert err.max() <= _split_bound(d), err.max()
    assert err.mean() <= 5e-6
    np.testing.assert_array_equal(Q, Q.T)
    np.testing.assert_array_equal(np.diag(Q), 1.0)


@pytest.mark.parametrize("device_a", [False, True])
def test_split_bf16_gram_tall_narrow_split_k(aln, device_a):
    """d = 20000, n = 300: 6 tile pairs for ~150 SMs, so each pair's 313 K
    blocks run as 19 chunks on separate CTAs whose partial tiles the pair's
    last CTA adds in a fixed order.  Host A takes the chunked-copy prepare,
    device A the single launch; Q within the split-Gram bound of the oracle's,
    the same bits on a second prepare, and a solve to FP64 KKT 1e-9."""
    import torch
    r = np.random.default_rng(31)
    d, n = 20000, 300
    A64 = r.random((d, n)) * np.exp(r.uniform(np.log(1e-2), np.log(1e2), n))[None, :]
    A = np.asfortranarray(A64.astype(np.float32))
    xt = np.where(r.random(n) < 0.5, 0.0, r.random(n))
    b = (A.astype(np.float64) @ xt + 0.01 * r.standard_normal(d)).astype(np.float32)
    A_in, b_in = A, b
    if device_a:
        A_in = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
        b_in = torch.from_numpy(b).cuda()
    with aln.Solver("split_bf16") as s:
        s.prepare(A_in, b_in)
        Q, q, sc = s.export()
        X, info = s.solve(tol=1e-9)
        s.prepare(A_in, b_in)
        Q2, _, _ = s.export()
    np.testing.assert_array_equal(Q2, Q)
    np.testing.assert_array_equal(Q, Q.T)
    Qo, qo, so = _oracle_scaled(A, b)
    assert np.abs(Q - Qo).max() <= _split_bound(d)
    np.testing.assert_allclose(q[0], qo, atol=1e-12 * np.abs(qo).max())
    rel, _ = O.kkt_residual(A.astype(np.float64), b.astype(np.float64), X[0])
    assert rel <= 1e-9, rel


@pytest.mark.parametrize("d,n", [(3000, 2300), (20000, 300), (40000, 1300), (5000, 4224)])
def test_host_and_device_input_give_the_same_result(aln, d, n):
    """Host A is copied in 512-column chunks, and the Gram's tile pairs run
    in whole waves as the chunks land (the rest with the last chunk); device
    A takes one launch.  Each pair's K chunking (split K for tall, narrow A;
    stream-K for the pairs past the last full wave) is fixed by the whole
    matrix, so both give the same Q bits, the same iterations and the same
    solution: n = 2300 (5 chunks, pairs deferred to whole waves, 19
    stream-K pairs), n = 300 and 1300 with split K (every chunk launches
    what it completes), n = 4224 (9 chunks, 105 stream-K pairs)."""
    import torch
    r = np.random.default_rng(d + n)
    A64 = r.random((d, n)) * np.exp(r.uniform(np.log(1e-2), np.log(1e2), n))[None, :]
    A = np.asfortranarray(A64.astype(np.float32))
    xt = np.where(r.random(n) < 0.6, 0.0, r.random(n))
    b = (A.astype(np.float64) @ xt + 0.01 * r.standard_normal(d)).astype(np.float32)
    out = []
    for dev in (False, True):
        A_in = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t() if dev else A
        b_in = torch.from_numpy(b).cuda() if dev else b
        with aln.Solver("split_bf16") as s:
            s.prepare(A_in, b_in)
            Q, q, sc = s.export()
            X, info = s.solve(tol=1e-7)
        out.append((Q, q, X, info[0].iters))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][3] == out[1][3]
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_split_gram_zero_column(aln):
    r = np.random.default_rng(5)
    A = np.asfortranarray(r.random((200, 150)).astype(np.float32))
    A[:, 17] = 0.0
    b = r.random(200).astype(np.float32)
    with aln.Solver("split_bf16") as s:
        s.prepare(A, b)
        Q, q, sc = s.export()
    assert sc[17] == 1.0 and q[0, 17] == 0.0
    assert np.all(Q[17] == 0.0) and np.all(Q[:, 17] == 0.0)


# ----------------------------------------------------------------- Alg. 2 rows
def _parity_fp64(x, A, b, x_star):
    F = O.nnls_objective(A, b, x)
    Fs = O.nnls_objective(A, b, x_star)
    assert abs(F - Fs) / Fs <= 1e-10
    if np.all(x_star == 0.0):          # optimum at the origin: exact zeros expected
        assert np.all(x == 0.0)
    else:
        assert np.abs(x - x_star).max() / np.abs(x_star).max() <= 1e-8


def test_fp64_solve_uniform_small(aln):
    """The plain FP64 configuration: A 1000×200 U[0,1], half of x_true zero
    (n = 200: the loop runs on one thread-block cluster)."""
    p = W.uniform_small()
    A, b = p.A, p.B[0]
    x_star, _, _, _ = O.reference_solution(A, b)
    with aln.Solver("fp64") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-12)
        assert s.stats().iter_kernel == 3
    assert info[0].status == aln.RHS_CONVERGED
    assert info[0].rel_kkt <= 1e-12
    _parity_fp64(X[0], A, b, x_star)
    rel, F = O.kkt_residual(A, b, X[0])
    assert rel <= 1e-12
    np.testing.assert_allclose(info[0].objective, F, rtol=1e-12)


@pytest.mark.parametrize("d,n", [(40, 1), (60, 2), (90, 31), (100, 33), (300, 129), (600, 257)])
def test_fp64_solve_ragged_sizes(aln, d, n):
    r = np.random.default_rng(d + 17 * n)
    A = np.asfortranarray(r.random((d, n)))
    xt = np.where(r.random(n) < 0.5, 0.0, r.random(n))
    b = A @ xt + 0.01 * r.standard_normal(d)
    x_star, _, _, _ = O.reference_solution(A, b)
    with aln.Solver("fp64") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-12)
    assert info[0].rel_kkt <= 1e-12
    _parity_fp64(X[0], A, b, x_star)


def _mixed_gate(A, b, x, x_star):
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    rel, _ = O.kkt_residual(A64, b64, x)
    assert rel <= 1e-6, rel
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) <= 1e-5


@pytest.mark.parametrize("d,n", [(3000, 800), (900, 300)])
def test_single_rhs_tight_tolerance(aln, d, n):
    """The replicated kernel keeps y as a float pair, so the FP64 refinement
    reaches relative KKT 1e-11, far below the FP32 rounding of y."""
    p = W.lopsided_single(d=d, n=n, seed=40 + n)
    A, b = p.A, p.B[0]
    with aln.Solver("split_bf16") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-11)
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    rel, _ = O.kkt_residual(A64, b64, X[0])
    assert rel <= 1e-11, (rel, info[0])
    assert info[0].status == aln.RHS_CONVERGED
    x_star, _, _, _ = O.reference_solution(A64, b64)
    assert np.linalg.norm(X[0] - x_star) <= 1e-7 * np.linalg.norm(x_star)


def test_mixed_solve_lopsided(aln):
    """Lopsided single-RHS configuration at reduced size (4000×1000)."""
    p = W.lopsided_single(d=4000, n=1000)
    A, b = p.A, p.B[0]
    x_star, _, _, _ = O.reference_solution(A.astype(np.float64), b.astype(np.float64))
    with aln.Solver("split_bf16") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-10)
        Xb, infob = s.solve(tol=1e-6)
    assert infob[0].rel_kkt <= 1e-6
    rel_b, _ = O.kkt_residual(A.astype(np.float64), b.astype(np.float64), Xb[0])
    assert rel_b <= 1e-6
    _mixed_gate(A, b, X[0], x_star)


@pytest.mark.parametrize("d,n", [(70, 1), (80, 3), (150, 65), (500, 129), (900, 300)])
def test_mixed_solve_ragged_sizes(aln, d, n):
    r = np.random.default_rng(3 * d + n)
    A = np.asfortranarray(r.random((d, n)).astype(np.float32))
    xt = np.where(r.random(n) < 0.6, 0.0, r.random(n))
    b = (A.astype(np.float64) @ xt + 0.01 * r.standard_normal(d)).astype(np.float32)
    x_star, _, _, _ = O.reference_solution(A.astype(np.float64), b.astype(np.float64))
    with aln.Solver("split_bf16") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-10)
    _mixed_gate(A, b, X[0], x_star)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_zero_solution_when_Atb_nonpositive(aln, prec):
    r = np.random.default_rng(12)
    A = np.asfortranarray(r.random((30, 8)))
    b = -r.random(30)
    if prec == "split_bf16":
        A, b = np.asfortranarray(A.astype(np.float32)), b.astype(np.float32)
    with aln.Solver(prec) as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-10)
    assert info[0].iters == 0 and info[0].status == aln.RHS_EMPTY_PASSIVE
    assert np.all(X[0] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_zero_column_solution(aln, prec):
    r = np.random.default_rng(13)
    A = r.random((120, 40))
    A[:, 3] = 0.0
    b = A @ r.random(40) + 0.01 * r.standard_normal(120)
    dt = np.float64 if prec == "fp64" else np.float32
    A, b = np.asfortranarray(A.astype(dt)), b.astype(dt)
    x_star, _, _, _ = O.reference_solution(A.astype(np.float64), b.astype(np.float64))
    with aln.Solver(prec) as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-10)
    assert X[0, 3] == 0.0
    assert np.linalg.norm(X[0] - x_star) / np.linalg.norm(x_star) <= 1e-5


def test_warm_start_at_optimum_takes_no_iterations(aln):
    p = W.uniform_small(d=300, n=60, seed=77)
    A, b = p.A, p.B[0]
    x_star, _, _, _ = O.reference_solution(A, b)
    with aln.Solver("fp64") as s:
        s.prepare(A, b)
        X, info = s.solve(tol=1e-9, X0=x_star[None, :].copy())
    assert info[0].iters <= 2
    _parity_fp64(X[0], A, b, x_star)


def test_max_iter_is_reported_not_raised(aln):
    p = W.uniform_small()
    with aln.Solver("fp64", max_refine=0) as s:
        s.prepare(p.A, p.B[0])
        X, info = s.solve(tol=1e-14, max_iter=5)
    assert info[0].status == aln.RHS_MAXITER
    assert info[0].iters == 5
    assert np.all(X[0] >= 0.0)


def test_device_and_host_pointers_agree(aln):
    import torch
    p = W.uniform_small(d=400, n=100, seed=9)
    with aln.Solver("fp64") as s:
        s.prepare(p.A, p.B[0])
        Xh, ih = s.solve(tol=1e-12)
    At = torch.from_numpy(np.ascontiguousarray(p.A.T)).cuda().t()   # column-major view
    Bt = torch.from_numpy(p.B).cuda()
    Xd = torch.zeros((1, 100), dtype=torch.float64, device="cuda")
    with aln.Solver("fp64") as s:
        s.prepare(At, Bt)
        s.solve(tol=1e-12, X=Xd)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(Xd.cpu().numpy(), Xh)


def test_errors(aln):
    r = np.random.default_rng(1)
    A = np.asfortranarray(r.random((20, 5)))
    b = r.random(20)
    with aln.Solver("fp64") as s:
        with pytest.raises(aln.AlnError) as e:
            s.solve()
        assert e.value.code == aln.ERR_NOT_PREPARED
        A2 = A.copy(order="F")
        A2[3, 2] = np.nan
        with pytest.raises(aln.AlnError) as e:
            s.prepare(A2, b)
        assert e.value.code == aln.ERR_NONFINITE
        b2 = b.copy()
        b2[0] = np.inf
        with pytest.raises(aln.AlnError) as e:
            s.prepare(A, b2)
        assert e.value.code == aln.ERR_NONFINITE
        s.prepare(A, b)
        with pytest.raises(aln.AlnError) as e:
            s.solve(tol=-1.0)
        assert e.value.code == aln.ERR_INVALID_ARG
        X0 = np.full((1, 5), np.nan)
        with pytest.raises(aln.AlnError) as e:
            s.solve(X0=X0)
        assert e.value.code == aln.ERR_NONFINITE


def test_kkt_entry_point_matches_oracle(aln):
    p = W.lopsided_single(d=2000, n=500, seed=4)
    A, b = p.A, p.B[0]
    r = np.random.default_rng(2)
    X = np.where(r.random((3, 500)) < 0.5, 0.0, r.random((3, 500)))
    X[2] = 0.0
    B = np.stack([b, b * 0.5, b]).astype(np.float32)
    with aln.Solver("split_bf16") as s:
        s.prepare(A, B)
        rel, F = s.kkt(X)
    for c in range(3):
        ro, Fo = O.kkt_residual(A.astype(np.float64), B[c].astype(np.float64), X[c])
        np.testing.assert_allclose(rel[c], ro, rtol=1e-10)
        np.testing.assert_allclose(F[c], Fo, rtol=1e-10)
    np.testing.assert_allclose(rel[2], 1.0, rtol=1e-12)


def test_multiple_rhs_each_match_oracle(aln):
    p = W.shared_multi_rhs(d=1500, n=300, k=6, seed=33)
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, p.B)
        X, info = s.solve(tol=1e-10)
    A64 = p.A.astype(np.float64)
    for c in range(p.k):
        b64 = p.B[c].astype(np.float64)
        x_star, _, _, _ = O.reference_solution(A64, b64)
        _mixed_gate(p.A, p.B[c], X[c], x_star)


# ------------------------------------------------------------- batched solver
def test_batched_prepare_matches_oracle(aln):
    """Batched prepare: q from exact BF16 digit products on the tensor cores
    and the scaled matrix from FP32-pipe Dot2 products (both FP64-level
    accuracy); q and s to 1e-12, Q (kept in FP32 for the iteration) to FP32
    rounding."""
    p = W.shared_multi_rhs(d=1300, n=257, k=70, seed=37)
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, p.B)
        Q, q, sc = s.export()
    A64 = p.A.astype(np.float64)
    H, h = O.nqp_from_nnls(A64, p.B.astype(np.float64))
    Qo, qo, so = O.antilopsided_scaling(H, h)
    np.testing.assert_allclose(sc, so, rtol=1e-13)
    np.testing.assert_allclose(q, qo, rtol=0, atol=1e-12 * np.abs(qo).max())
    np.testing.assert_allclose(Q, Qo, rtol=0, atol=2.0 ** -23)
    np.testing.assert_array_equal(Q, Q.T)


@pytest.mark.parametrize("signed,d,n,k", [(False, 997, 130, 70), (True, 997, 130, 70),
                                          (True, 700, 60, 300)])
def test_batched_q_from_digit_products(aln, signed, d, n, k):
    """q = −D⁻¹Aᵀb of the batched prepare (exact 7-bit digit products on the
    tensor cores, 49 bits per value, pairs of order ≤ 8) against FP64, entry
    by entry, relative to Σ_t |a_ti b_t| / s_i (the natural scale of a
    compensated product): columns six decades apart, a zero column, mixed
    signs, d, n and k ragged against the 64 × 128 × 64 tiles; n = 60 < 128
    with k = 300 runs the product transposed (the wide side on the 128-row
    tiles)."""
    r = np.random.default_rng(91 + signed + n)
    A = r.random((d, n)) * np.exp(r.uniform(np.log(1e-3), np.log(1e3), n))[None, :]
    B = r.standard_normal((k, d)) if signed else r.random((k, d))
    if signed:
        A *= r.choice([-1.0, 1.0], size=A.shape)
    A[:, 5] = 0.0
    A = np.asfortranarray(A.astype(np.float32))
    B = np.ascontiguousarray(B.astype(np.float32))
    with aln.Solver("split_bf16") as s:
        s.prepare(A, B)
        _, q, sc = s.export()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    norms = np.sqrt((A64 * A64).sum(axis=0))
    safe = np.where(norms > 0, norms, 1.0)
    qo = -(B64 @ A64) / safe[None, :]
    scale = (np.abs(B64) @ np.abs(A64)) / safe[None, :]
    assert np.all(np.abs(q - qo) <= 1e-13 * scale + 1e-300)
    assert np.all(q[:, 5] == 0.0)


def test_batched_multi_rhs_matches_oracle(aln):
    """Many RHS sharing A (NMF inner-solve shape): the batched tensor-core
    solver meets the mixed-precision gates on every column."""
    p = W.shared_multi_rhs(d=1500, n=300, k=40, seed=34)
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, p.B)
        X, info = s.solve(tol=1e-9)
        Xb, infob = s.solve(tol=1e-6)
    A64 = p.A.astype(np.float64)
    for c in range(p.k):
        b64 = p.B[c].astype(np.float64)
        x_star, _, _, _ = O.reference_solution(A64, b64)
        _mixed_gate(p.A, p.B[c], X[c], x_star)
        rel, F = O.kkt_residual(A64, b64, Xb[c])
        assert rel <= 1e-6
        np.testing.assert_allclose(infob[c].rel_kkt, rel, rtol=1e-8, atol=1e-14)
        np.testing.assert_allclose(infob[c].objective, F, rtol=1e-9)


def test_batched_phase_then_tail(aln):
    """More columns than the tail threshold (2 per SM): the tcgen05 batched
    phase runs first and hands the last columns to the tail (one CTA per
    column, then thread-block clusters as columns finish, in budgeted
    launches); every column meets the FP64 KKT gate and agrees with the
    single right-hand-side path."""
    p = W.shared_multi_rhs(d=1200, n=180, k=420, seed=38)
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, p.B)
        X, info = s.solve(tol=1e-8)
    A64 = p.A.astype(np.float64)
    for c in range(0, p.k, 7):
        rel, _ = O.kkt_residual(A64, p.B[c].astype(np.float64), X[c])
        assert rel <= 1e-8, (c, rel, info[c])
    with aln.Solver("split_bf16", batch_min=10 ** 6) as s:
        s.prepare(p.A, p.B[:20])
        Xs, _ = s.solve(tol=1e-8)
    for c in range(20):
        assert np.linalg.norm(X[c] - Xs[c]) <= 1e-4 * max(np.linalg.norm(Xs[c]), 1e-30)


def test_batched_agrees_with_single_rhs_path(aln):
    p = W.shared_multi_rhs(d=800, n=200, k=12, seed=35)
    with aln.Solver("split_bf16") as s:
        s.prepare(p.A, p.B)
        Xb, ib = s.solve(tol=1e-9)
    with aln.Solver("split_bf16", batch_min=10 ** 6) as s:
        s.prepare(p.A, p.B)
        Xs, is_ = s.solve(tol=1e-9)
    for c in range(p.k):
        assert np.linalg.norm(Xb[c] - Xs[c]) <= 2e-5 * np.linalg.norm(Xs[c])


@pytest.mark.parametrize("d,n,k", [(600, 100, 40), (300, 33, 24), (200, 7, 16), (500, 128, 20),
                                   (90, 32, 9), (260, 64, 12), (270, 65, 12)])
def test_batched_small_n_matches_oracle(aln, d, n, k):
    """n ≤ 128: the warp-per-column kernel runs each column's Alg. 2 loop
    (VPL = 1, 2, 4 entries per lane, ragged n); every column meets the FP64
    KKT gate from A and the x-gate against the oracle's optimum at tol 1e-9,
    a zero right-hand side stops at once, and a start point at the solution
    needs (almost) no iteration."""
    r = np.random.default_rng(d + n + k)
    A = np.asfortranarray((r.random((d, n)) * np.exp(r.uniform(-1, 1, n))).astype(np.float32))
    X_true = np.where(r.random((k, n)) < 0.6, 0.0, r.random((k, n)))
    B = (X_true @ A.astype(np.float64).T + 0.01 * r.standard_normal((k, d))).astype(np.float32)
    B[1] = -np.abs(B[1]) if n > 1 else B[1]
    with aln.Solver("split_bf16") as s:
        s.prepare(A, B)
        X, info = s.solve(tol=1e-9)
        X2, info2 = s.solve(tol=1e-9, X0=X.copy())
    A64 = A.astype(np.float64)
    for c in range(k):
        b64 = B[c].astype(np.float64)
        rel, F = O.kkt_residual(A64, b64, X[c])
        assert rel <= 1e-9, (c, rel, info[c])
        # the batched FP64 check forms g64 = Q64·y + q as Dot2 products on FP32
        # pairs (≈ 2⁻⁴⁸ per entry): about 1e-14 absolute in the relative residual
        np.testing.assert_allclose(info[c].rel_kkt, rel, rtol=1e-6, atol=5e-14)
        if c != 1:                       # column 1 has the optimum x = 0
            x_star, _, _, _ = O.reference_solution(A64, b64)
            _mixed_gate(A, B[c], X[c], x_star)
        assert info2[c].iters <= max(3, info[c].iters // 4)
    assert info[1].iters == 0 and info[1].status == aln.RHS_EMPTY_PASSIVE
    assert np.all(X[1] == 0.0)


def test_batched_edge_columns(aln):
    """Zero RHS (x = 0 at once), ragged n across tiles, a start point."""
    r = np.random.default_rng(36)
    d, n, k = 500, 131, 20
    A = np.asfortranarray(r.random((d, n)).astype(np.float32))
    X_true = np.where(r.random((k, n)) < 0.7, 0.0, r.random((k, n)))
    B = (X_true @ A.astype(np.float64).T + 0.01 * r.standard_normal((k, d))).astype(np.float32)
    B[3] = -np.abs(B[3])            # Aᵀb ≤ 0: optimum 0, empty passive set
    with aln.Solver("split_bf16") as s:
        s.prepare(A, B)
        X, info = s.solve(tol=1e-8)
        assert info[3].iters == 0 and info[3].status == aln.RHS_EMPTY_PASSIVE
        assert np.all(X[3] == 0.0)
        X2, info2 = s.solve(tol=1e-8, X0=X.copy())
    A64 = A.astype(np.float64)
    for c in range(k):
        rel, _ = O.kkt_residual(A64, B[c].astype(np.float64), X[c])
        assert rel <= 1e-8
        assert info2[c].iters <= max(3, info[c].iters // 4)


# ------------------------------------------------------- full-size configurations
def test_full_size_lopsided_single(aln):
    """The default workload at full size (20000×5000) in the launch
    configuration bench.py times (device inputs, tol 1e-6): 64 sampled Q
    entries and 32 q entries against the oracle's single-entry definitions
    (FP64 products of two columns), the solution's FP64 KKT residual and
    objective by the oracle from A, and x ⪰ 0."""
    import torch
    p = W.lopsided_single()
    A, b = p.A, p.B[0]
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    Bt = torch.from_numpy(np.ascontiguousarray(p.B)).cuda()
    with aln.Solver("split_bf16") as s:
        s.prepare(At, Bt)
        Q, q, sc = s.export()
        X, info = s.solve(tol=1e-6)
    A64, b64 = A.astype(np.float64), b.astype(np.float64)
    norms = np.sqrt(np.einsum("ij,ij->j", A64, A64))
    r = np.random.default_rng(51)
    for i, j in list(r.integers(0, p.n, (62, 2))) + [(0, 4999), (4999, 4999)]:
        qo = 1.0 if i == j else A64[:, i] @ A64[:, j] / (norms[i] * norms[j])
        assert abs(Q[i, j] - qo) <= _split_bound(p.d), (i, j)
    for j in r.integers(0, p.n, 32):
        qo = -(A64[:, j] @ b64) / norms[j]
        assert abs(q[0, j] - qo) <= 1e-12 * max(1.0, abs(qo))
    np.testing.assert_allclose(sc, norms, rtol=1e-13)
    assert info[0].status == aln.RHS_CONVERGED
    rel, F = O.kkt_residual(A64, b64, X[0])
    assert rel <= 1e-6 and np.all(X[0] >= 0.0)
    np.testing.assert_allclose(info[0].rel_kkt, rel, rtol=1e-6)
    np.testing.assert_allclose(info[0].objective, F, rtol=1e-9)


def test_full_size_shared_multi_rhs(aln):
    """The multi-RHS configuration at full size (10000×1000, k = 4096) in the
    launch configuration bench.py times: every column's reported FP64 KKT
    residual ≤ 1e-6; 24 sampled columns' residual and objective by the
    oracle from A, matching the reported ones; X ⪰ 0."""
    import torch
    p = W.shared_multi_rhs()
    At = torch.from_numpy(np.ascontiguousarray(p.A.T)).cuda().t()
    Bt = torch.from_numpy(np.ascontiguousarray(p.B)).cuda()
    with aln.Solver("split_bf16") as s:
        s.prepare(At, Bt)
        X, info = s.solve(tol=1e-6)
    assert max(i.rel_kkt for i in info) <= 1e-6
    assert np.all(X >= 0.0)
    A64 = p.A.astype(np.float64)
    for c in np.random.default_rng(52).choice(p.k, 24, replace=False):
        b64 = p.B[c].astype(np.float64)
        rel, F = O.kkt_residual(A64, b64, X[c])
        assert rel <= 1e-6, (c, rel)
        np.testing.assert_allclose(info[c].rel_kkt, rel, rtol=1e-6, atol=1e-13)
        np.testing.assert_allclose(info[c].objective, F, rtol=1e-9)
