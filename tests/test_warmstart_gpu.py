"""Learned start point (tcgen05 BF16 network, FP32 accumulation) against the
FP64 oracle in oracle/mlp.py, through the C ABI.

Tolerance: the products take BF16 operands (8 significant bits, relative
rounding 2⁻⁹) and accumulate in FP32, so loss and gradients are compared per
tensor in relative norm to 2e-2; start points to 3e-2."""
import numpy as np
import pytest

from oracle import mlp as MO
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _prepared(aln, d, n, k, seed):
    r = np.random.default_rng(seed)
    A = np.asfortranarray((r.random((d, n)) * np.exp(r.uniform(-2, 2, n))).astype(np.float32))
    X = np.where(r.random((k, n)) < 0.8, 0.0, r.exponential(1.0, (k, n)))
    B = (X @ A.T.astype(np.float64)).astype(np.float32)
    s = aln.Solver("split_bf16")
    s.prepare(A, B)
    return s, A, B


@pytest.mark.parametrize("n,hidden,batch", [(100, 192, 150), (64, 128, 128), (300, 256, 37)])
def test_gradients_match_oracle(aln, n, hidden, batch):
    """One forward/backward pass: ragged M (batch), N and K (2n, hidden) over
    several 128×128 tiles."""
    s, A, B = _prepared(aln, 3 * n, n, 4, seed=n + hidden)
    with s:
        _, q, sc = s.export()
        r = np.random.default_rng(7)
        p = MO.init_params(2 * n, hidden, 2 * n, seed=3)
        for k in ("b1", "b2", "b3"):
            p[k] = r.normal(0, 0.05, p[k].shape)
        s.warmstart_init(hidden, 1)
        s.warmstart_set({k: v.astype(np.float32) for k, v in p.items()})
        got = s.warmstart_get()
        for k in p:
            np.testing.assert_array_equal(got[k], p[k].astype(np.float32))
        Qb = r.normal(size=(batch, n)) * 3.0
        Yb = np.maximum(r.normal(size=(batch, n)), 0.0) * 2.0
        loss, g = s.warmstart_grad(Qb, Yb)
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    U, qn = MO.features(Qb, sc)
    T, C = MO.targets(Yb, qn)
    L, go = MO.loss_and_grad(p32, U, T, C)
    assert abs(loss - L) <= 2e-2 * abs(L), (loss, L)
    for k in MO.PARAM_NAMES:
        assert _rel(g[k].astype(np.float64), go[k]) <= 2e-2, (k, _rel(g[k], go[k]))


def test_training_and_warm_start(aln):
    """Train on solved right-hand sides of one A, then start held-out solves
    from the prediction: the loss falls, the start points match the oracle's
    prediction with the same weights, and the warm solves need fewer
    iterations than cold ones while meeting the same tolerance."""
    d, n = 800, 200
    train = W.warmstart_family(d=d, n=n, k=8192, support=(5, 40), seed=11)
    held = W.warmstart_family(d=d, n=n, k=256, support=(5, 40), seed=11, rhs_seed=12)
    np.testing.assert_array_equal(train.A, held.A)
    with aln.Solver("split_bf16") as s:
        s.prepare(train.A, train.B)
        X, info = s.solve(tol=1e-8)
        _, q, sc = s.export()
        Ys = X * sc[None, :]
        hist = s.warmstart_train(q, Ys, epochs=40, batch=256, hidden=512, lr=1e-3, seed=5)
        assert hist[-1] < 0.5 * hist[0], hist
        params = s.warmstart_get()
        # the normalisation statistics are those of the training set
        st = MO.stats(q, Ys)
        np.testing.assert_allclose(params["mu"], st["mu"], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(params["sd"], st["sd"], rtol=1e-5)
        assert abs(params["tau"] - st["tau"]) <= 1e-5 * st["tau"]
        # held-out right-hand sides of the same A
        s.prepare(held.A, held.B)
        Qh, qh, sh = s.export()
        X0, kept = s.warmstart_predict()
        Xc, ic = s.solve(tol=1e-6)
        Xw, iw = s.solve(tol=1e-6, X0=X0)
    assert kept.mean() > 0.9
    cold = np.mean([i.iters for i in ic])
    warm = np.mean([i.iters for i in iw])
    assert warm < 0.85 * cold, (warm, cold)
    A64 = held.A.astype(np.float64)
    for c in range(held.k):
        rel, _ = O.kkt_residual(A64, held.B[c].astype(np.float64), Xw[c])
        assert rel <= 1e-6
    # start points against the oracle's prediction with the same weights
    p64 = {k: params[k].astype(np.float64) for k in MO.PARAM_NAMES}
    st64 = {"mu": params["mu"].astype(np.float64), "sd": params["sd"].astype(np.float64),
            "tau": params["tau"]}
    y0o = MO.predict(p64, qh, sh, Qh, st64)
    y0 = X0 * sh[None, :]
    both = (np.abs(y0o).sum(axis=1) > 0) & (kept == 1)
    assert both.sum() >= 0.5 * held.k
    assert _rel(y0[both], y0o[both]) <= 3e-2


def test_warmstart_errors(aln):
    s, A, B = _prepared(aln, 60, 20, 2, seed=1)
    with s:
        with pytest.raises(aln.AlnError) as e:
            s.warmstart_predict()
        assert e.value.code == aln.ERR_INVALID_ARG
        with pytest.raises(aln.AlnError) as e:
            aln.aln_warmstart_init(s.ctx, 0, 0)
        assert e.value.code == aln.ERR_INVALID_ARG


def test_full_size_warm_start_configuration(aln):
    """The warm-start configuration's A (8000×2000, lopsided column scales)
    and the bench's network width (4096), trained on 16384 solved right-hand
    sides: every one of 256 held-out warm solves meets FP64 KKT ≤ 1e-6 (8 of
    them by the oracle from A), every start point is feasible and no worse
    than the origin (the start is Alg. 2's exact line search along the
    prediction), and the start points match the oracle's prediction with the
    same weights."""
    d, n = 8000, 2000
    train = W.warmstart_family(d=d, n=n, k=16384, seed=1005)
    held = W.warmstart_family(d=d, n=n, k=256, seed=1005, rhs_seed=1005 + 7919)
    with aln.Solver("split_bf16") as s:
        s.prepare(train.A, train.B)
        X, info = s.solve(tol=1e-6)
        _, q, sc = s.export()
        s.warmstart_train(q, X * sc[None, :], epochs=20, batch=256, hidden=4096, lr=1e-3,
                          seed=7)
        params = s.warmstart_get()
        s.prepare(held.A, held.B)
        Qh, qh, sh = s.export()
        X0, kept = s.warmstart_predict()
        Xw, iw = s.solve(tol=1e-6, X0=X0)
    assert max(i.rel_kkt for i in iw) <= 1e-6
    assert np.all(X0 >= 0.0)
    A64 = held.A.astype(np.float64)
    for c in np.random.default_rng(53).choice(held.k, 8, replace=False):
        b64 = held.B[c].astype(np.float64)
        rel, _ = O.kkt_residual(A64, b64, Xw[c])
        assert rel <= 1e-6, (c, rel)
        f0 = O.nnls_objective(A64, b64, np.zeros(n))
        assert O.nnls_objective(A64, b64, X0[c]) <= f0 * (1 + 1e-6), c
    p64 = {k: params[k].astype(np.float64) for k in MO.PARAM_NAMES}
    st64 = {"mu": params["mu"].astype(np.float64), "sd": params["sd"].astype(np.float64),
            "tau": params["tau"]}
    cols = np.arange(16)
    y0o = MO.predict(p64, qh[cols], sh, Qh, st64)
    y0 = (X0 * sh[None, :])[cols]
    both = (np.abs(y0o).sum(axis=1) > 0) & (kept[cols] == 1)
    assert both.sum() >= 8
    assert _rel(y0[both], y0o[both]) <= 3e-2
