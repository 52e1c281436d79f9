"""Learned start point (tcgen05 BF16 network, FP32 accumulation, direction
feature z = −Q⁻¹q from an FP32 Newton–Schulz inverse) against the FP64 oracle
in oracle/mlp.py (exact inverse), through the C ABI.

Tolerance: the layer products take BF16 operands (8 significant bits, relative
rounding 2⁻⁹) and accumulate in FP32.  Each backward product adds the rounding
of its BF16 operands (dO, W3, dZ2, W2, dZ1, u), so the gradients are compared
with the exact FP64 oracle per tensor in relative norm to 2e-2 for the output
layer and the skips, 5e-2 for layer 2 and 1e-1 for layer 1 (a CPU emulation of
the same BF16 roundings reaches 2.5-6.2e-2 on the layer-1 cases here), and with
that emulation (the oracle's formulas with every product operand rounded to
BF16 where the kernels round it) to 1e-2 per tensor; start points to 3e-2.
The FP32 inverse carries about cond(Q)·2⁻²⁴ relative error, far below those."""
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


def _bf16(x):
    """Round to the nearest BF16 (ties to even), returned in FP64."""
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bf16_gradients(p, U, zt, T, C):
    """The oracle's backward pass with every layer product's operands rounded
    to BF16 where the kernels round them (u, weights, h1, h2, dO, dZ2, dZ1);
    sums in FP64."""
    n = T.shape[1]
    W = {k: _bf16(p[k]) for k in ("W1", "W2", "W3")}
    Ub = _bf16(U)
    Z1 = Ub @ W["W1"].T + p["b1"]
    H1 = _bf16(np.maximum(Z1, 0.0))
    Z2 = H1 @ W["W2"].T + p["b2"]
    H2 = _bf16(np.maximum(Z2, 0.0))
    O = H2 @ W["W3"].T + p["b3"]
    O = np.hstack([O[:, :n] + p["e"] * zt, O[:, n:] + p["f"] * zt])
    m = T.size
    dy = 2.0 * (O[:, :n] - T) / m
    dl = (1.0 / (1.0 + np.exp(-O[:, n:])) - C) / m
    dO = _bf16(np.hstack([dy, dl]))
    g = {"W3": dO.T @ H2, "b3": dO.sum(0), "e": (dy * zt).sum(0), "f": (dl * zt).sum(0)}
    dZ2 = _bf16((dO @ W["W3"]) * (Z2 > 0))
    g["W2"], g["b2"] = dZ2.T @ H1, dZ2.sum(0)
    dZ1 = _bf16((dZ2 @ W["W2"]) * (Z1 > 0))
    g["W1"], g["b1"] = dZ1.T @ Ub, dZ1.sum(0)
    return g


TOL_EXACT = {"W3": 2e-2, "b3": 2e-2, "e": 2e-2, "f": 2e-2, "W2": 5e-2, "b2": 5e-2,
             "W1": 1e-1, "b1": 1e-1}


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
    several 128×128 tiles; every parameter, the skips included."""
    s, A, B = _prepared(aln, 3 * n, n, 4, seed=n + hidden)
    with s:
        Q, q, sc = s.export()
        Qinv = np.linalg.inv(Q)
        r = np.random.default_rng(7)
        p = MO.init_params(2 * n, hidden, 2 * n, seed=3)
        for k in ("b1", "b2", "b3"):
            p[k] = r.normal(0, 0.05, p[k].shape)
        p["e"] = r.normal(1.0, 0.2, n)
        p["f"] = r.normal(3.0, 0.5, n)
        s.warmstart_init(hidden, 1)
        s.warmstart_set({k: v.astype(np.float32) for k, v in p.items()})
        got = s.warmstart_get()
        for k in p:
            np.testing.assert_array_equal(got[k], p[k].astype(np.float32))
        Qb = r.normal(size=(batch, n)) * 3.0
        Yb = np.maximum(r.normal(size=(batch, n)), 0.0) * 2.0
        loss, g = s.warmstart_grad(Qb, Yb)
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    U, qn, zt = MO.features(Qb, Qinv)
    T, C = MO.targets(Yb, qn)
    L, go = MO.loss_and_grad(p32, U, zt, T, C)
    assert abs(loss - L) <= 2e-2 * abs(L), (loss, L)
    ge = _bf16_gradients(p32, U, zt, T, C)
    for k in MO.PARAM_NAMES:
        gk = g[k].astype(np.float64)
        assert _rel(gk, go[k]) <= TOL_EXACT[k], (k, _rel(gk, go[k]))
        assert _rel(gk, ge[k]) <= 1e-2, (k, _rel(gk, ge[k]))


def _oracle_stats(params):
    return {k: (params[k].astype(np.float64) if k != "tau" else params[k])
            for k in ("mu", "sd", "muz", "sdz", "tau")}


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
        Qtr, _, _ = s.export()
        Qinv = np.linalg.inv(Qtr)
        st = MO.stats(q, Ys, Qinv)
        np.testing.assert_allclose(params["mu"], st["mu"], rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(params["sd"], st["sd"], rtol=1e-5)
        assert abs(params["tau"] - st["tau"]) <= 1e-5 * st["tau"]
        # the direction statistics come from the FP32 inverse: 1e-3
        np.testing.assert_allclose(params["muz"], st["muz"], rtol=1e-3,
                                   atol=1e-3 * np.abs(st["muz"]).max())
        np.testing.assert_allclose(params["sdz"], st["sdz"], rtol=1e-3)
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
    y0o = MO.predict(p64, qh, np.linalg.inv(Qh), Qh, _oracle_stats(params))
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


def test_named_warm_start_configuration(aln):
    """The warm-start configuration as named: A 8000×2000 with lopsided column
    scales, a network of two hidden layers of 1024, trained on 200 000 solved
    right-hand sides and evaluated on 16 384 held-out ones of the same A.
    Warm starts need fewer than 0.85× the cold iterations; every held-out warm
    solve meets FP64 KKT ≤ 1e-6 (reported for all, by the oracle from A for
    8); every start point is feasible and no worse than the origin; the start
    points match the oracle's prediction with the same weights."""
    torch = pytest.importorskip("torch")
    d, n, k_train, k_held = 8000, 2000, 200000, 16384
    A, Btr = W.warmstart_family_device(d=d, n=n, k=k_train, seed=1005)
    _, Bh = W.warmstart_family_device(d=d, n=n, k=k_held, seed=1005, rhs_seed=1005 + 7919)
    At = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
    with aln.Solver("split_bf16") as s:
        s.prepare(At, Btr)
        Xtr = torch.zeros((k_train, n), dtype=torch.float64, device="cuda")
        _, info = s.solve(tol=1e-6, X=Xtr)
        assert max(i.rel_kkt for i in info) <= 1e-6
        qd = torch.zeros((k_train, n), dtype=torch.float64, device="cuda")
        sd = torch.zeros(n, dtype=torch.float64, device="cuda")
        aln.aln_export_scaled(s.ctx, None, n, qd, n, sd)
        Yd = Xtr * sd[None, :]
        del Btr, Xtr
        hist = s.warmstart_train(qd, Yd, epochs=20, batch=1024, hidden=1024, lr=1e-3, seed=7)
        assert hist[-1] < hist[0], hist
        params = s.warmstart_get()
        del qd, Yd
        s.prepare(At, Bh)
        Xc, ic = s.solve(tol=1e-6)
        X0, kept = s.warmstart_predict()
        Xw, iw = s.solve(tol=1e-6, X0=X0)
        Qh, qh, sh = s.export()
    cold = np.mean([i.iters for i in ic])
    warm = np.mean([i.iters for i in iw])
    assert warm < 0.85 * cold, (warm, cold)
    assert max(i.rel_kkt for i in iw) <= 1e-6
    assert np.all(X0 >= 0.0)
    A64 = A.astype(np.float64)
    Bh64 = Bh.cpu().numpy().astype(np.float64)
    for c in np.random.default_rng(53).choice(k_held, 8, replace=False):
        rel, _ = O.kkt_residual(A64, Bh64[c], Xw[c])
        assert rel <= 1e-6, (c, rel)
        f0 = O.nnls_objective(A64, Bh64[c], np.zeros(n))
        assert O.nnls_objective(A64, Bh64[c], X0[c]) <= f0 * (1 + 1e-6), c
    p64 = {k: params[k].astype(np.float64) for k in MO.PARAM_NAMES}
    cols = np.arange(16)
    y0o = MO.predict(p64, qh[cols], np.linalg.inv(Qh), Qh, _oracle_stats(params))
    y0 = (X0 * sh[None, :])[cols]
    both = (np.abs(y0o).sum(axis=1) > 0) & (kept[cols] == 1)
    assert both.sum() >= 8
    assert _rel(y0[both], y0o[both]) <= 3e-2
