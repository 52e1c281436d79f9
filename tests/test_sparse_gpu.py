"""Parity of the CSC prepare (aln_prepare_csc, block-sparse tensor-core Gram)
against the FP64 CPU oracle and against the dense prepare on the same matrix.

Tolerances (written here): Q from the block-sparse Gram meets the same bound
as the dense split-BF16 Gram (|ΔQ_ij| ≤ 2⁻²² + 3·d·2⁻²⁴ + 2⁻²³, the dropped
split terms plus FP32 accumulation and scaling); q and s are FP64 (1e-12
relative).  A block that is zero in either operand adds exactly zero to H, so
Q from the CSC form equals Q from the dense form except where the two
prepares' FP64 scale factors (different summation orders) round to different
FP32 values: at most one FP32 ulp, and in almost no entry.  Solutions: FP64
relative KKT ≤ the requested tolerance and ‖Δx‖₂/‖x*‖₂ ≤ 1e-5 against the
oracle's optimum (as for the dense mixed-precision path).
"""
import numpy as np
import pytest

from oracle import nnls as O
from oracle import sparse as S
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


def _split_bound(d):
    return 2.0 ** -22 + 3 * d * 2.0 ** -24 + 2.0 ** -23


def _oracle(p):
    return S.scaled_problem_csc(p.d, p.n, p.col_ptr, p.row_idx, p.vals, p.B[0])


def _export_csc(aln, p, precision="split_bf16", **opts):
    with aln.Solver(precision, **opts) as s:
        s.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals, p.B)
        return s.export()


def _export_dense(aln, A, B, precision="split_bf16", **opts):
    with aln.Solver(precision, **opts) as s:
        s.prepare(A, B)
        return s.export()


# (d, n, band, density): several column tiles with a ragged last tile, d not a
# multiple of 64, and tile pairs whose row windows never meet (skipped whole)
BANDED = [(3000, 700, 400, 0.2), (5000, 300, 200, 0.5), (130, 129, 40, 0.5), (64, 1, 64, 1.0)]


@pytest.mark.parametrize("d,n,band,density", BANDED)
def test_csc_scaled_problem_matches_oracle(aln, d, n, band, density):
    p = W.banded_tall(d=d, n=n, band=band, density=density, seed=d + n)
    Q, q, s = _export_csc(aln, p)
    Qo, qo, so = _oracle(p)
    np.testing.assert_allclose(s, so, rtol=1e-13)
    np.testing.assert_allclose(q[0], qo, atol=1e-12 * np.abs(qo).max())
    err = np.abs(Q - Qo)
    assert err.max() <= _split_bound(d), err.max()
    np.testing.assert_array_equal(Q, Q.T)
    # entries whose columns share no stored row are exactly zero
    np.testing.assert_array_equal(Q[Qo == 0.0], 0.0)


# (d, n, band, density): tile pairs whose common blocks exceed the chunk size
# run as several CTAs whose partial tiles are added at the end (split K); the
# dense Gram splits K too when it has fewer tile pairs than SMs
DENSE_CMP = [(3000, 700, 400, 0.2), (5000, 300, 200, 0.5), (20000, 256, 20000, 0.05)]


@pytest.mark.parametrize("d,n,band,density", DENSE_CMP)
def test_csc_gram_equals_dense_gram(aln, d, n, band, density):
    """Both Grams add the same block products (a skipped block adds exact
    zeros); they differ only in how the FP32 sums are grouped (each chunk
    sums its blocks, the chunks are added in order).  Each is an FP32
    summation of at most ⌈d/64⌉ block terms whose scaled magnitudes add up to
    at most 1 (Cauchy–Schwarz), so |ΔQ| ≤ 2·⌈d/64⌉·2⁻²⁴, plus one FP32
    rounding of each scale factor."""
    p = W.banded_tall(d=d, n=n, band=band, density=density, seed=7 * d + n)
    Qc, qc, sc = _export_csc(aln, p)
    Qd, qd, sd = _export_dense(aln, p.dense(), p.B)
    np.testing.assert_allclose(sc, sd, rtol=1e-14)
    np.testing.assert_allclose(qc, qd, rtol=1e-13, atol=1e-300)
    np.testing.assert_array_equal(Qc, Qc.T)
    bound = (2 * -(-d // 64) + 2) * 2.0 ** -24
    assert np.abs(Qc - Qd).max() <= bound, np.abs(Qc - Qd).max()
    Qo, _, _ = _oracle(p)
    assert np.abs(Qc - Qo).max() <= _split_bound(d)
    # deterministic: a second prepare gives the same bits
    Qc2, _, _ = _export_csc(aln, p)
    np.testing.assert_array_equal(Qc2, Qc)


@pytest.mark.parametrize("sub", [2, 4])
def test_csc_elementwise_sparse_tcase(aln, sub):
    """The paper's sparse sub-tests (§5, up to 40% zero entries) through the
    CSC form: every block is occupied, so the Gram does the dense work."""
    p = W.tcase("T2", sub=sub, n=600, d=900)
    cp, ri, v = W.to_csc(p.A)
    sp = W.SparseProblem(900, 600, cp, ri, v, p.B, p.x_true, 1e-6)
    Q, q, s = _export_csc(aln, sp)
    Qo, qo, so = _oracle(sp)
    assert np.abs(Q - Qo).max() <= _split_bound(900)
    np.testing.assert_allclose(s, so, rtol=1e-13)
    with aln.Solver("split_bf16") as sv:
        sv.prepare_csc(900, cp, ri, v, p.B)
        X, info = sv.solve(tol=1e-8)
    A64 = p.A.astype(np.float64)
    b64 = p.B[0].astype(np.float64)
    rel, _ = O.kkt_residual(A64, b64, X[0])
    assert rel <= 1e-8, rel
    x_star, _, _, _ = O.reference_solution(A64, b64)
    assert np.linalg.norm(X[0] - x_star) <= 1e-5 * np.linalg.norm(x_star)


@pytest.mark.parametrize("d,n,band,density", BANDED[:3])
def test_csc_solve_matches_oracle(aln, d, n, band, density):
    p = W.banded_tall(d=d, n=n, band=band, density=density, seed=3 * d + n)
    A64 = S.csc_to_dense(p.d, p.n, p.col_ptr, p.row_idx, p.vals)
    b64 = p.B[0].astype(np.float64)
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals, p.B)
        X, info = s.solve(tol=1e-9)
    assert info[0].rel_kkt <= 1e-9
    rel, F = O.kkt_residual(A64, b64, X[0])
    assert rel <= 1e-9, rel
    np.testing.assert_allclose(info[0].objective, F, rtol=1e-9)
    x_star, _, _, _ = O.reference_solution(A64, b64)
    assert np.linalg.norm(X[0] - x_star) <= 1e-5 * np.linalg.norm(x_star)


def test_csc_fp64_and_many_rhs_paths(aln):
    """FP64 precision (FP64 Gram of the scattered matrix) and the
    many-right-hand-side solver behind the same entry point."""
    p = W.banded_tall(d=2000, n=300, band=300, density=0.3, seed=5, dtype=np.float64)
    Q, q, s = _export_csc(aln, p, "fp64")
    Qo, qo, so = _oracle(p)
    np.testing.assert_allclose(Q, Qo, atol=1e-12)
    np.testing.assert_allclose(q[0], qo, atol=1e-12 * np.abs(qo).max())
    r = np.random.default_rng(6)
    A64 = p.dense().astype(np.float64)
    B = np.ascontiguousarray((r.random((40, 300)) * (r.random((40, 300)) < 0.3)) @ A64.T)
    B32 = B.astype(np.float32)
    with aln.Solver("split_bf16", batch_min=32) as sv:
        sv.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals.astype(np.float32), B32)
        X, info = sv.solve(tol=1e-7)
    A32 = p.dense().astype(np.float32).astype(np.float64)
    for c in (0, 17, 39):
        rel, _ = O.kkt_residual(A32, B32[c].astype(np.float64), X[c])
        assert rel <= 1e-7, (c, rel)


def test_csc_empty_columns_and_tiles(aln):
    """Columns with no entries (s = 1, Q_ii = 0, x_i = 0), a whole column tile
    with none, and an A with no entries at all."""
    d, n = 500, 300
    r = np.random.default_rng(8)
    A = np.zeros((d, n), np.float32, order="F")
    keep = [j for j in range(n) if not (128 <= j < 256) and j % 7 != 3]
    for j in keep:
        rows = r.choice(d, 40, replace=False)
        A[rows, j] = r.random(40).astype(np.float32) + 0.1
    b = (A.astype(np.float64) @ r.random(n)).astype(np.float32)
    cp, ri, v = W.to_csc(A)
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(d, cp, ri, v, b)
        Q, q, sc = s.export()
        X, info = s.solve(tol=1e-8)
    empty = np.setdiff1d(np.arange(n), keep)
    assert np.all(sc[empty] == 1.0) and np.all(q[0, empty] == 0.0)
    assert np.all(Q[empty] == 0.0) and np.all(np.diag(Q)[keep] == 1.0)
    assert np.all(X[0, empty] == 0.0)
    rel, _ = O.kkt_residual(A.astype(np.float64), b.astype(np.float64), X[0])
    assert rel <= 1e-8
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(d, np.zeros(n + 1, np.int64), np.zeros(0, np.int32),
                      np.zeros(0, np.float32), b)
        Q, q, sc = s.export()
        X, info = s.solve(tol=1e-8)
    assert np.all(Q == 0.0) and np.all(sc == 1.0) and np.all(X == 0.0)


def test_csc_device_inputs(aln):
    import torch
    p = W.banded_tall(d=2500, n=400, band=300, density=0.2, seed=9)
    Qh, qh, sh = _export_csc(aln, p)
    dev = torch.device("cuda")
    cp = torch.from_numpy(p.col_ptr).to(dev)
    ri = torch.from_numpy(p.row_idx).to(dev)
    v = torch.from_numpy(p.vals).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(p.d, cp, ri, v, B)
        Qd, qd, sd = s.export()
        torch.cuda.synchronize()
    np.testing.assert_array_equal(Qd, Qh)
    np.testing.assert_array_equal(qd, qh)
    with aln.Solver("split_bf16") as s:  # arrays on different sides
        with pytest.raises(aln.AlnError):
            s.prepare_csc(p.d, p.col_ptr, ri, p.vals, p.B)


@pytest.mark.parametrize("what", ["unsorted", "duplicate", "row_range", "col_ptr", "nan"])
def test_csc_malformed_inputs_are_rejected(aln, what):
    p = W.banded_tall(d=400, n=50, band=100, density=0.3, seed=10)
    cp, ri, v = p.col_ptr.copy(), p.row_idx.copy(), p.vals.copy()
    t = int(cp[20]) + 3
    if what == "unsorted":
        ri[t], ri[t + 1] = ri[t + 1], ri[t]
    elif what == "duplicate":
        ri[t + 1] = ri[t]
    elif what == "row_range":
        ri[int(cp[50]) - 1] = 400
    elif what == "col_ptr":
        cp[30] = cp[31] + 1
    else:
        v[t] = np.nan
    code = aln.ERR_NONFINITE if what == "nan" else aln.ERR_INVALID_ARG
    with aln.Solver("split_bf16") as s:
        with pytest.raises(aln.AlnError) as e:
            s.prepare_csc(p.d, cp, ri, v, p.B)
        assert e.value.code == code
        # the context stays usable
        s.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals, p.B)
        X, info = s.solve(tol=1e-6)
        assert info[0].rel_kkt <= 1e-6


def test_csc_full_size_sampled(aln):
    """The tall workload at full size (200000×5000, 3·10⁶ entries): sampled
    entries of Q and q against the oracle's single-entry products, and the
    library's FP64 KKT residual of the solution."""
    p = W.banded_tall()
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals, p.B)
        Q, q, sc = s.export()
        X, info = s.solve(tol=p.tol)
    assert info[0].rel_kkt <= p.tol
    r = np.random.default_rng(11)
    pairs = [(int(i), int(min(p.n - 1, max(0, i + r.integers(-200, 201)))))
             for i in r.integers(0, p.n, 60)] + [(0, 4999), (2500, 2500)]
    for i, j in pairs:
        h_ii = S.gram_entry(p.col_ptr, p.row_idx, p.vals, i, i)
        h_jj = S.gram_entry(p.col_ptr, p.row_idx, p.vals, j, j)
        h_ij = S.gram_entry(p.col_ptr, p.row_idx, p.vals, i, j)
        qo = h_ij / np.sqrt(h_ii * h_jj) if i != j else 1.0
        assert abs(Q[i, j] - qo) <= _split_bound(p.d), (i, j, Q[i, j], qo)
    b = p.B[0]
    for j in r.integers(0, p.n, 40):
        h_jj = S.gram_entry(p.col_ptr, p.row_idx, p.vals, int(j), int(j))
        qo = -S.atb_entry(p.col_ptr, p.row_idx, p.vals, b, int(j)) / np.sqrt(h_jj)
        assert abs(q[0, j] - qo) <= 1e-12 * max(1.0, abs(qo))
    assert np.all(X[0] >= 0.0)
    rel, F = S.kkt_residual_csc(p.d, p.n, p.col_ptr, p.row_idx, p.vals, b, X[0])
    assert rel <= p.tol, rel
    assert rel == pytest.approx(info[0].rel_kkt, rel=1e-6)
    assert F == pytest.approx(info[0].objective, rel=1e-10)


def test_csc_extreme_tall(aln):
    """20 000 000 × 300 with 40 entries per column (8·10⁹ elements dense,
    12 000 stored): row indices beyond 2²⁴ and 312 500 K blocks.  The columns
    draw their rows from a pool of 2000 rows spread over the whole range, so
    they overlap and every tile pair has ~2000 common blocks (split K over
    ~25 CTAs per pair).  Sampled Q and q entries against the oracle's
    single-entry products; the solution's KKT residual and objective by the
    oracle, evaluated from the CSC arrays."""
    d, n, per = 20_000_000, 300, 40
    g = np.random.default_rng(41)
    pool = np.sort(g.choice(d, 2000, replace=False))
    cp = np.arange(n + 1, dtype=np.int64) * per
    ri = np.concatenate([np.sort(g.choice(pool, per, replace=False)) for _ in range(n)])
    ri = ri.astype(np.int32)
    v = (1.0 - g.random(n * per)).astype(np.float32)
    cols = np.repeat(np.arange(n), per)
    x_true = np.where(g.random(n) < 0.5, 0.0, g.random(n))
    b = np.bincount(ri, weights=v.astype(np.float64) * x_true[cols], minlength=d)
    b[pool] += 0.01 * g.standard_normal(pool.size)
    b = b.astype(np.float32)
    tol = 1e-8
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(d, cp, ri, v, b)
        Q, q, sc = s.export()
        X, info = s.solve(tol=tol)
    assert info[0].rel_kkt <= tol
    for i, j in [(0, 0), (0, 1), (5, 299), (150, 151), (299, 299)] + \
            [(int(a), int(c)) for a, c in g.integers(0, n, (40, 2))]:
        h_ii = S.gram_entry(cp, ri, v, i, i)
        h_jj = S.gram_entry(cp, ri, v, j, j)
        qo = 1.0 if i == j else S.gram_entry(cp, ri, v, i, j) / np.sqrt(h_ii * h_jj)
        assert abs(Q[i, j] - qo) <= 2.0 ** -22 + 3 * 2000 * 2.0 ** -24, (i, j, Q[i, j], qo)
    for j in (0, 77, 299):
        qo = -S.atb_entry(cp, ri, v, b, j) / np.sqrt(S.gram_entry(cp, ri, v, j, j))
        assert abs(q[0, j] - qo) <= 1e-12 * max(1.0, abs(qo))
    rel, F = S.kkt_residual_csc(d, n, cp, ri, v, b, X[0])
    assert rel <= tol, rel
    assert F == pytest.approx(info[0].objective, rel=1e-10)


@pytest.mark.parametrize("d,n,band,density", [(3000, 700, 400, 0.2), (130, 129, 40, 0.5)])
def test_csc_kkt_pass_matches_oracle(aln, d, n, band, density):
    """The FP64 KKT pass of a CSC context with FP32 values reads the CSC
    arrays and the packed blocks (no dense copy): residual and objective of
    arbitrary non-negative points against the oracle's, computed from the
    dense matrix, and against the dense context's pass."""
    p = W.banded_tall(d=d, n=n, band=band, density=density, seed=d - n)
    A64 = S.csc_to_dense(p.d, p.n, p.col_ptr, p.row_idx, p.vals)
    b64 = p.B[0].astype(np.float64)
    r = np.random.default_rng(d)
    X = np.where(r.random((3, n)) < 0.5, 0.0, r.exponential(1.0, (3, n)))
    X[2] = 0.0                                   # the origin: ḡ = min(q, 0)
    with aln.Solver("split_bf16") as s:
        s.prepare_csc(p.d, p.col_ptr, p.row_idx, p.vals, p.B)
        got = [s.kkt(np.ascontiguousarray(X[c:c + 1])) for c in range(3)]
    with aln.Solver("split_bf16") as s:
        s.prepare(p.dense(), p.B)
        ref = [s.kkt(np.ascontiguousarray(X[c:c + 1])) for c in range(3)]
    for c in range(3):
        rel_o, F_o = O.kkt_residual(A64, b64, X[c])
        assert got[c][0][0] == pytest.approx(rel_o, rel=1e-10), c
        assert got[c][1][0] == pytest.approx(F_o, rel=1e-12), c
        assert got[c][0][0] == pytest.approx(ref[c][0][0], rel=1e-10), c
        assert got[c][1][0] == pytest.approx(ref[c][1][0], rel=1e-12), c
    assert got[2][0][0] == pytest.approx(1.0, rel=1e-12)


def _rule_tiles(p):
    """Tile pairs (I, J) of 128 columns whose columns share an occupied 64-row
    block: the only tiles the block-sparse Gram multiplies, and the tiles the
    Alg. 2 products read on a CSC context (the rule of the bench's
    q_tile_fraction)."""
    cols = np.repeat(np.arange(p.n), np.diff(p.col_ptr))
    tiles = (p.n + 127) // 128
    occ = np.zeros((tiles, (p.d + 63) // 64), dtype=np.int64)
    occ[cols // 128, p.row_idx // 64] = 1
    return (occ @ occ.T) > 0


@pytest.mark.parametrize("d,n,band,density", [(3000, 700, 400, 0.2), (6000, 1000, 300, 0.3)])
def test_csc_nonzero_tiles_lie_in_the_skip_rule(aln, d, n, band, density):
    """Every 128×128 tile of Q with a non-zero entry belongs to a pair of
    column tiles that share an occupied 64-row block, and every tile outside
    that set is exactly zero — so the products that skip those tiles skip
    only exact zeros.  The problem has several tile pairs whose row windows
    never meet."""
    p = W.banded_tall(d=d, n=n, band=band, density=density, seed=41)
    Q, _, _ = _export_csc(aln, p)
    rule = _rule_tiles(p)
    T = rule.shape[0]
    assert not rule.all(), "the case must have zero tile pairs"
    nz = np.zeros((T, T), dtype=bool)
    for I in range(T):
        for J in range(T):
            blk = Q[I * 128:(I + 1) * 128, J * 128:(J + 1) * 128]
            nz[I, J] = bool(np.any(blk != 0.0))
    assert not np.any(nz & ~rule), "a non-zero tile outside the skip rule"
    # the oracle's dense Q is zero exactly outside the rule too (up to pairs
    # whose shared blocks hold no common row: those are zero in both)
    Qo, _, _ = _oracle(p)
    for I in range(T):
        for J in range(T):
            if not rule[I, J]:
                assert np.all(Qo[I * 128:(I + 1) * 128, J * 128:(J + 1) * 128] == 0.0)
