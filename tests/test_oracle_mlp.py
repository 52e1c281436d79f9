"""Pins of the warm-start MLP oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: central finite differences of the loss, the
closed form of Adam's first steps, limits of the loss terms, the feature
normalisation, and the fallback rule of the start point."""
import numpy as np
import pytest

from oracle import mlp as M


def _tiny(seed=0, n=3, hidden=5, B=4):
    r = np.random.default_rng(seed)
    p = M.init_params(2 * n, hidden, 2 * n, seed=seed)
    for k in ("b1", "b2", "b3"):
        p[k] = r.normal(0, 0.1, p[k].shape)
    q = r.normal(size=(B, n))
    s = np.exp(r.uniform(-2, 2, n))
    U, qn = M.features(q, s)
    Y = np.maximum(r.normal(size=(B, n)), 0.0)
    T, C = M.targets(Y, qn)
    return p, U, T, C


def _fd_check(p, U, T, C, h=1e-6, per_tensor=6, seed=1):
    """Relative error of the analytic gradient against central differences on
    random entries of every parameter tensor."""
    _, g = M.loss_and_grad(p, U, T, C)
    r = np.random.default_rng(seed)
    worst = 0.0
    for k in M.PARAM_NAMES:
        flat = p[k].reshape(-1)
        for idx in r.choice(flat.size, size=min(per_tensor, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, U, T, C)
            flat[idx] = old - h
            lm = M.loss(p, U, T, C)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            worst = max(worst, abs(fd - an) / max(abs(fd), abs(an), 1e-8))
    return worst


def test_gradient_matches_central_differences():
    p, U, T, C = _tiny()
    _, (_, Z1, _, Z2, _) = M.forward(p, U)
    # keep every pre-activation away from the ReLU kink by more than h
    assert np.abs(Z1).min() > 1e-4 and np.abs(Z2).min() > 1e-4
    assert _fd_check(p, U, T, C) <= 1e-6


def test_gradient_check_catches_a_dropped_relu_mask(monkeypatch):
    p, U, T, C = _tiny()
    real = M.loss_and_grad

    def wrong(p_, U_, T_, C_):
        # the same backward pass with the first ReLU mask dropped
        O, (U_, Z1, H1, Z2, H2) = M.forward(p_, U_)
        B, n = T_.shape
        m = B * n
        dO = np.hstack([2.0 * (O[:, :n] - T_) / m,
                        (1.0 / (1.0 + np.exp(-O[:, n:])) - C_) / m])
        g = {"W3": dO.T @ H2, "b3": dO.sum(0)}
        dZ2 = (dO @ p_["W3"]) * (Z2 > 0)
        g["W2"], g["b2"] = dZ2.T @ H1, dZ2.sum(0)
        dZ1 = dZ2 @ p_["W2"]
        g["W1"], g["b1"] = dZ1.T @ U_, dZ1.sum(0)
        return real(p_, U_, T_, C_)[0], g

    monkeypatch.setattr(M, "loss_and_grad", wrong)
    p, U, T, C = _tiny(seed=3, hidden=8)
    _, (_, Z1, _, _, _) = M.forward(p, U)
    assert (Z1 < 0).any()
    assert _fd_check(p, U, T, C, per_tensor=40) > 1e-3


def test_loss_limits():
    # BCE at ℓ = 0 is log 2 whatever the class; huge logits do not overflow
    assert M.bce(np.array(0.0), 1.0) == pytest.approx(np.log(2.0))
    assert M.bce(np.array(0.0), 0.0) == pytest.approx(np.log(2.0))
    big = M.bce(np.array([1000.0, -1000.0]), np.array([1.0, 0.0]))
    assert np.all(np.isfinite(big)) and np.all(big < 1e-300 + 1e-12)
    assert M.bce(np.array(-1000.0), 1.0) == pytest.approx(1000.0)
    # a network that outputs the targets exactly and confident logits: L → 0
    n, B = 3, 2
    T = np.array([[0.2, 0.0, 0.5], [0.0, 0.1, 0.0]])
    C = (T > 0).astype(float)
    p = {"W1": np.zeros((4, 2 * n)), "b1": np.ones(4), "W2": np.eye(4), "b2": np.zeros(4),
         "W3": np.zeros((2 * n, 4)), "b3": np.zeros(2 * n)}
    U = np.zeros((B, 2 * n))
    # constant output: row-independent, so use one row of targets
    p["b3"] = np.concatenate([T[0], np.where(C[0] > 0, 60.0, -60.0)])
    L = M.loss(p, U[:1], T[:1], C[:1])
    assert L < 1e-25


def test_adam_first_steps_closed_form():
    # with m = v = 0, bias correction makes the first step −lr·g/(|g| + ε)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    st = M.adam_init(p)
    M.adam_step(p, g, st, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p["w"], [1.0, -2.0, 3.0] - 0.1 * g["w"] / (np.abs(g["w"]) + 1e-8))
    # a constant gradient keeps the same step size in later steps
    before = p["w"].copy()
    M.adam_step(p, g, st, lr=0.1, eps=1e-8)
    np.testing.assert_allclose(p["w"] - before, -0.1 * g["w"] / (np.abs(g["w"]) + 1e-8),
                               rtol=1e-12)


def test_features_normalisation():
    r = np.random.default_rng(4)
    n = 7
    q = r.normal(size=(3, n))
    s = np.exp(r.uniform(-3, 3, n))
    U, qn = M.features(q, s)
    np.testing.assert_allclose(qn, np.linalg.norm(q, axis=1))
    np.testing.assert_allclose(np.linalg.norm(U[:, :n], axis=1), 1.0)
    z = U[0, n:]
    assert abs(z.mean()) < 1e-14 and abs(z.std() - 1.0) < 1e-14
    # scale invariance of the q-part, and constant s gives z = 0
    U2, _ = M.features(5.0 * q, s)
    np.testing.assert_allclose(U2[:, :n], U[:, :n])
    U3, _ = M.features(q, np.full(n, 2.0))
    assert np.all(U3[:, n:] == 0.0)
    # q = 0: zero q-part and zero target
    U4, qn4 = M.features(np.zeros((1, n)), s)
    assert qn4[0] == 0.0 and np.all(U4[0, :n] == 0.0)


def _identity_net(n, sign):
    """h1 = relu(sign·q/‖q‖) on the first n units, ŷ = h1[:n], logits 5."""
    hidden = 2 * n
    p = {"W1": np.zeros((2 * n, 2 * n)), "b1": np.zeros(2 * n),
         "W2": np.eye(2 * n), "b2": np.zeros(2 * n),
         "W3": np.zeros((2 * n, hidden)), "b3": np.zeros(2 * n)}
    p["W1"][:n, :n] = sign * np.eye(n)
    p["W3"][:n, :n] = np.eye(n)
    p["b3"][n:] = 5.0
    return p


def test_predict_line_search_rule():
    n = 4
    Q = np.eye(n)
    s = np.ones(n)
    q = -np.array([[1.0, 2.0, 0.5, 3.0]])
    # direction −q/‖q‖ with Q = I: the exact line search lands on y* = −q
    p = _identity_net(n, -1.0)
    np.testing.assert_allclose(M.predict(p, q, s, Q)[0], -q[0])
    # the start does not depend on the predicted magnitude
    p10 = dict(p, W3=10.0 * p["W3"])
    np.testing.assert_allclose(M.predict(p10, q, s, Q), M.predict(p, q, s, Q))
    # a direction that does not descend (qᵀd ≥ 0) gives y⁰ = 0
    assert np.all(M.predict(_identity_net(n, 1.0), -q, s, Q) == 0.0)
    # logits ≤ 0 switch every entry off
    p["b3"][n:] = -5.0
    assert np.all(M.predict(p, q, s, Q) == 0.0)


def test_predict_is_the_best_point_on_its_ray():
    """f(y⁰) ≤ f(α·d) for every α ≥ 0 on a grid, and f(y⁰) ≤ 0 = f(0)."""
    r = np.random.default_rng(8)
    n = 12
    A = np.abs(r.normal(size=(40, n)))
    H = A.T @ A
    sc = np.sqrt(np.diag(H))
    Q = H / np.outer(sc, sc)
    q = -(r.random((16, n)) @ A.T @ A) / sc + 0.3 * r.normal(size=(16, n))
    p = M.init_params(2 * n, 32, 2 * n, seed=9)
    p["b3"][n:] = 2.0
    y0 = M.predict(p, q, sc, Q)
    U, _ = M.features(q, sc)
    O, _ = M.forward(p, U)
    d = np.maximum(O[:, :n], 0.0) * (O[:, n:] > 0)

    def f(y, qq):
        return 0.5 * y @ Q @ y + qq @ y

    for b in range(len(q)):
        fy = f(y0[b], q[b])
        assert fy <= 1e-14
        for a in np.linspace(0.0, 3.0, 61) * max(np.abs(y0[b]).max(), 1e-3) / max(
                np.abs(d[b]).max(), 1e-12):
            assert fy <= f(a * d[b], q[b]) + 1e-12


def test_normalisation_statistics():
    r = np.random.default_rng(10)
    n, m = 5, 300
    q = r.normal(size=(m, n)) + np.array([3.0, 0, 0, 0, -1.0])
    Y = np.maximum(r.normal(size=(m, n)), 0.0) * 7.0
    st = M.stats(q, Y)
    U, qn = M.features(q, np.ones(n), st)
    np.testing.assert_allclose(U[:, :n].mean(axis=0), 0.0, atol=1e-12)
    np.testing.assert_allclose(U[:, :n].std(axis=0), 1.0, rtol=1e-12)
    T, _ = M.targets(Y, qn, st["tau"])
    assert abs(np.sqrt(np.mean(T ** 2)) - 1.0) < 1e-12


def test_training_lowers_the_loss():
    r = np.random.default_rng(5)
    n, m = 6, 256
    A = np.abs(r.normal(size=(30, n)))
    s = np.linalg.norm(A, axis=0)
    X = np.maximum(r.normal(size=(m, n)), 0.0)
    Ys = X * s
    Qs = -(X @ A.T @ A) / s     # q = −D⁻¹Aᵀb with b = A x (noise-free)
    p = M.init_params(2 * n, 32, 2 * n, seed=1)
    hist = M.train(p, Qs, Ys, s, epochs=100, batch=32, lr=3e-3)
    assert hist[-1] < 0.45 * hist[0]
    assert hist[-1] < hist[len(hist) // 3]
